// Run-time dispatch of the Wilson-clover operator: the hop (the dslash), the clover
// multiply, the fused even-odd operator M-hat = A_ee - kappa^2 H_eo A_oo^{-1} H_oe and
// K = M-hat^dag M-hat, on the stencil instantiations of dslash_<prec>_<dag>.cu.
#include "dslash.h"
#include "hop.cuh"

namespace pfmp {

PFMP_DSLASH_DECLARE(PFMP_F64, false)
PFMP_DSLASH_DECLARE(PFMP_F64, true)
PFMP_DSLASH_DECLARE(PFMP_F32, false)
PFMP_DSLASH_DECLARE(PFMP_F32, true)
PFMP_DSLASH_DECLARE(PREC_DF, false)
PFMP_DSLASH_DECLARE(PREC_DF, true)
PFMP_DSLASH_DECLARE(PFMP_H16, false)
PFMP_DSLASH_DECLARE(PFMP_H16, true)

template <int PREC>
__global__ void k_clover_mul(Geom g, typename Prec<PREC>::vec* out, const typename Prec<PREC>::vec* in,
                             const typename Prec<PREC>::vec* clov) {
  using T = typename Prec<PREC>::real;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  HermBlock<T> B[2];
  load_clover(B, clov, cb, g.Vh);
  Spinor<T> x;
  load_spinor(x, in, cb, g.Vh);
  store_spinor(out, clover_apply(B, x), cb, g.Vh);
}

static void require_clover_built(pfmp_op* op) {
  PFMP_REQUIRE(op->built_version == op->ctx->gauge_version, PFMP_E_INVALID,
               "gauge field changed since the clover term was built: call pfmp_op_update");
}

void hop(pfmp_op* op, int prec, void* out, const void* in, int out_parity, bool dagger) {
  if (prec == PFMP_F64)
    dagger ? hop_plain_t<PFMP_F64, true>(op, out, in, out_parity) : hop_plain_t<PFMP_F64, false>(op, out, in, out_parity);
  else if (prec == PFMP_H16)
    dagger ? hop_plain_t<PFMP_H16, true>(op, out, in, out_parity) : hop_plain_t<PFMP_H16, false>(op, out, in, out_parity);
  else
    dagger ? hop_plain_t<PFMP_F32, true>(op, out, in, out_parity) : hop_plain_t<PFMP_F32, false>(op, out, in, out_parity);
}

void clover_mul(pfmp_op* op, int prec, void* out, const void* in, int parity) {
  require_clover_built(op);
  const Geom& g = op->ctx->g;
  if (prec == PFMP_F64)
    k_clover_mul<PFMP_F64><<<nblocks(g.Vh), kBlock, 0, op->ctx->stream>>>(g, (double2*)out, (const double2*)in,
                                                                            op->clov64[parity]);
  else
    k_clover_mul<PFMP_F32><<<nblocks(g.Vh), kBlock, 0, op->ctx->stream>>>(g, (float4*)out, (const float4*)in,
                                                                            op->clov32[parity]);
  PFMP_CHECK_LAUNCH();
}

template <int PREC>
static void mhat_p(pfmp_op* op, void* out, const void* in, bool dagger, double* norm_out, CGScalars* scal, void* t) {
  if (dagger)
    mhat_t<PREC, true>(op, out, in, norm_out, scal, t);
  else
    mhat_t<PREC, false>(op, out, in, norm_out, scal, t);
}

// M-hat with a caller-supplied odd-site temporary (the allocation-free entry point); the
// same two launches as mhat() below, and the operator's own temporaries are untouched
void mhat_with_temp(pfmp_op* op, int prec, void* out, const void* in, bool dagger, void* temp) {
  require_clover_built(op);
  if (prec == PFMP_F64)
    mhat_p<PFMP_F64>(op, out, in, dagger, nullptr, nullptr, temp);
  else
    mhat_p<PFMP_F32>(op, out, in, dagger, nullptr, nullptr, temp);
}

void mhat(pfmp_op* op, int prec, void* out, const void* in, bool dagger, double* norm_out, CGScalars* scal) {
  require_clover_built(op);
  if (prec == PFMP_F64)
    mhat_p<PFMP_F64>(op, out, in, dagger, norm_out, scal, op->t64);
  else if (prec == PFMP_H16)
    mhat_p<PFMP_H16>(op, out, in, dagger, norm_out, scal, op->t16);
  else
    mhat_p<PFMP_F32>(op, out, in, dagger, norm_out, scal, op->t32);
}

// K in double-float: in/out are df even fields ([12][Vh] float4), FP32-pipe arithmetic
void kop_df(pfmp_op* op, void* out, const void* in) {
  require_clover_built(op);
  op->kapply += 1;
  mhat_p<PREC_DF>(op, op->edf, in, false, nullptr, nullptr, op->tdf);
  mhat_p<PREC_DF>(op, out, op->edf, true, nullptr, nullptr, op->tdf);
}

// out (odd) = A_oo^{-1} H_oe in (or the adjoint hop), FP64 or FP32: the first half of
// M-hat, used by the force terms
void hop_clov_odd(pfmp_op* op, int prec, void* out, const void* in, bool dagger) {
  require_clover_built(op);
  if (prec == PFMP_F64)
    dagger ? hop_clov_odd_t<PFMP_F64, true>(op, out, in, nullptr) : hop_clov_odd_t<PFMP_F64, false>(op, out, in, nullptr);
  else
    dagger ? hop_clov_odd_t<PFMP_F32, true>(op, out, in, nullptr) : hop_clov_odd_t<PFMP_F32, false>(op, out, in, nullptr);
}

// out = K in; <in, K in> = ||M-hat in||^2 is reduced in the second kernel of M-hat
void kop(pfmp_op* op, int prec, void* out, const void* in, double* pKp_dev, CGScalars* scal) {
  op->kapply += 1;
  void* e = prec == PFMP_F64 ? (void*)op->e64 : (prec == PFMP_H16 ? (void*)op->e16 : (void*)op->e32);
  mhat(op, prec, e, in, false, pKp_dev, scal);
  mhat(op, prec, out, e, true, nullptr, scal);
}

}  // namespace pfmp
