// Wilson hop (the dslash), clover multiply, and the fused even-odd operator
// M-hat = A_ee - kappa^2 H_eo A_oo^{-1} H_oe and K = M-hat^dag M-hat.
//
// One thread per output site.  Each thread spin-projects its 8 neighbours to
// two-component half spinors (the projectors (1 -+ g_mu) have rank 2), multiplies by
// the link (FP32: 12-real links, third row rebuilt in registers), and rebuilds the
// four-component result.  Two fused epilogues make M-hat a two-kernel operation:
//   EPI_CLOV  out = C (H in)            (odd sites: C = A_oo^{-1})
//   EPI_XPAY  out = C x + coef (H in)   (even sites: C = A_ee, x the local input), with
//             an optional grid reduction of ||out||^2 feeding the CG scalars.
// M-hat^dag uses the adjoint hop (projector signs swapped): A is Hermitian, so
// M-hat^dag = A_ee - kappa^2 H^dag_eo A_oo^{-1} H^dag_oe.
#include "dfloat.cuh"
#include "hop.cuh"

#ifndef HOP_MINB_F32
#define HOP_MINB_F32 7
#endif
#ifndef HOP_MINB_H16
#define HOP_MINB_H16 7
#endif

namespace pfmp {

// Resident 128-thread blocks per SM that the register allocation must allow.  The
// stencil is bound by memory latency, so more warps in flight pay even at the cost of a
// few spilled registers (FP32, 32^3x64: 0.85 -> 0.89 of the copy bandwidth at 7 blocks);
// FP64 and double-float keep the compiler's choice (a bound of 3 blocks made the rolled
// double-float stencil 7-18% slower).
template <int PREC>
constexpr int hop_min_blocks() {
  return PREC == PFMP_F32 ? HOP_MINB_F32 : PREC == PFMP_H16 ? HOP_MINB_H16 : 1;
}

// Double-float arithmetic takes the rolled stencil: unrolled, its ~18k instructions per
// thread stall on instruction fetch (ncu at 16^3x32: ~10 "no instruction" stall cycles
// per issue, 13% of the FP32 pipe); rolled, a K application is 2.5-2.9x faster.  FP64 is
// bound by GB300's FP64 rate and runs slower rolled (+28%), so it stays unrolled.
template <int PREC>
__host__ __device__ constexpr bool hop_rolled() {
  return PREC == PREC_DF;
}

template <int PREC, bool DAG, int EPI, bool REDUCE>
__global__ void __launch_bounds__(128, hop_min_blocks<PREC>()) k_hop(HopParams<PREC> a) {
  if (a.scal && a.scal->done) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  double nrm[1] = {0.0};
  if (cb < a.g.Vh) {
    Spinor<typename Prec<PREC>::real> out;
    if constexpr (hop_rolled<PREC>())
      out = hop_site_rolled<PREC, DAG, EPI>(a, cb);
    else
      out = hop_site<PREC, DAG, EPI>(a, cb);
    store_spinor(a.out, out, cb, a.g.Vh);
    if (REDUCE) nrm[0] = spinor_norm2(out);
  }
  if (REDUCE) {
    double tot[1];
    if (grid_sum<1>(nrm, a.rb, tot)) {
      *a.norm_out = tot[0];
      if (a.scal) a.scal->alpha = a.scal->rr / tot[0];
    }
  }
}

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

// ---------------------------------------------------------------- host drivers
constexpr int kHopBlock = 128;

template <int PREC>
static HopParams<PREC> params(pfmp_op* op, int p, void* out, const void* in) {
  using vec = typename Prec<PREC>::vec;
  HopParams<PREC> a;
  a.g = op->ctx->g;
  a.p = p;
  a.out = (vec*)out;
  a.in = (const vec*)in;
  a.gauge = PREC == PFMP_F64   ? (const vec*)(const void*)op->ctx->U64c
            : PREC == PREC_DF  ? (const vec*)(const void*)op->ctx->Udf
            : PREC == PFMP_H16 ? (const vec*)(const void*)op->ctx->U16
                               : (const vec*)(const void*)op->ctx->U32;
  a.clov = nullptr;
  a.x = nullptr;
  a.coef = 1.0;
  a.rb = op->ctx->rb;
  a.norm_out = nullptr;
  a.scal = nullptr;
  return a;
}

// algorithmic bytes of one launch: per output site 8 links (12 reals), one input spinor
// (each neighbour read once with ideal reuse), the output spinor, plus the clover
// blocks (72 reals) and for EPI_XPAY the local input spinor
template <int PREC>
static double hop_bytes(int epi, int Vh) {
  if (PREC == PFMP_H16) {  // FP16 reals, plus the FP32 scale of every spinor read or written
    const double b = 8 * 12 * 2 + 52 + 52 + (epi >= EPI_CLOV ? 72 * 2 : 0) + (epi == EPI_XPAY ? 52 : 0);
    return b * (double)Vh;
  }
  const double link = PREC == PREC_DF ? 18 : 12;
  const double reals = 8 * link + 24 + 24 + (epi >= EPI_CLOV ? 72 : 0) + (epi == EPI_XPAY ? 24 : 0);
  return reals * (PREC == PFMP_F32 ? 4 : 8) * (double)Vh;
}

template <int PREC>
static int split_of(const pfmp_op* op) {
  return op->nsplit[PREC == PFMP_F64 ? 0 : (PREC == PFMP_F32 ? 1 : 2)];
}

template <int PREC, bool DAG, int EPI, bool RED>
static void launch(const HopParams<PREC>& a, pfmp_op* op) {
  pfmp_ctx* c = op->ctx;
  cudaEvent_t ev;
  prof_start(c, &ev);
  const int bs = op->hop_block;
  if constexpr (PREC == PFMP_H16) {  // one thread per site only
    k_hop<PREC, DAG, EPI, RED><<<nblocks(a.g.Vh, bs), bs, 0, c->stream>>>(a);
  } else {
    const int ns = split_of<PREC>(op);
    const long n = (long)a.g.Vh * ns;
    switch (ns) {
      case 2: k_hop_split<PREC, DAG, EPI, RED, 2><<<nblocks(n, bs), bs, 0, c->stream>>>(a); break;
      case 4: k_hop_split<PREC, DAG, EPI, RED, 4><<<nblocks(n, bs), bs, 0, c->stream>>>(a); break;
      case 8: k_hop_split<PREC, DAG, EPI, RED, 8><<<nblocks(n, bs), bs, 0, c->stream>>>(a); break;
      default: k_hop<PREC, DAG, EPI, RED><<<nblocks(a.g.Vh, bs), bs, 0, c->stream>>>(a); break;
    }
  }
  PFMP_CHECK_LAUNCH();
  prof_stop(c,
            PREC == PFMP_F64   ? PFMP_KERNEL_HOP_F64
            : PREC == PREC_DF  ? PFMP_KERNEL_HOP_DF
            : PREC == PFMP_H16 ? PFMP_KERNEL_HOP_H16
                               : PFMP_KERNEL_HOP_F32,
            hop_bytes<PREC>(EPI, a.g.Vh), ev);
}

template <int PREC>
static const typename Prec<PREC>::vec* clov_ptr(pfmp_op* op, int parity) {
  if (PREC == PFMP_F64) return (const typename Prec<PREC>::vec*)(const void*)op->clov64[parity];
  if (PREC == PREC_DF) return (const typename Prec<PREC>::vec*)(const void*)op->clovdf[parity];
  if (PREC == PFMP_H16) return (const typename Prec<PREC>::vec*)(const void*)op->clov16[parity];
  return (const typename Prec<PREC>::vec*)(const void*)op->clov32[parity];
}

static void require_clover(pfmp_op* op) {
  PFMP_REQUIRE(op->built_version == op->ctx->gauge_version, PFMP_E_INVALID,
               "gauge field changed since the clover term was built: call pfmp_op_update");
}

template <int PREC>
static void hop_t(pfmp_op* op, void* out, const void* in, int p, bool dagger) {
  auto a = params<PREC>(op, p, out, in);
  if (dagger)
    launch<PREC, true, EPI_PLAIN, false>(a, op);
  else
    launch<PREC, false, EPI_PLAIN, false>(a, op);
}

void hop(pfmp_op* op, int prec, void* out, const void* in, int out_parity, bool dagger) {
  if (prec == PFMP_F64)
    hop_t<PFMP_F64>(op, out, in, out_parity, dagger);
  else if (prec == PFMP_H16)
    hop_t<PFMP_H16>(op, out, in, out_parity, dagger);
  else
    hop_t<PFMP_F32>(op, out, in, out_parity, dagger);
}

void clover_mul(pfmp_op* op, int prec, void* out, const void* in, int parity) {
  require_clover(op);
  const Geom& g = op->ctx->g;
  if (prec == PFMP_F64)
    k_clover_mul<PFMP_F64><<<nblocks(g.Vh), kBlock, 0, op->ctx->stream>>>(g, (double2*)out, (const double2*)in,
                                                                            clov_ptr<PFMP_F64>(op, parity));
  else
    k_clover_mul<PFMP_F32><<<nblocks(g.Vh), kBlock, 0, op->ctx->stream>>>(g, (float4*)out, (const float4*)in,
                                                                            clov_ptr<PFMP_F32>(op, parity));
  PFMP_CHECK_LAUNCH();
}

template <int PREC>
static void mhat_t(pfmp_op* op, void* out, const void* in, bool dagger, double* norm_out, CGScalars* scal) {
  void* t = PREC == PFMP_F64   ? (void*)op->t64
            : PREC == PREC_DF  ? (void*)op->tdf
            : PREC == PFMP_H16 ? (void*)op->t16
                               : (void*)op->t32;
  pfmp_op* s = op;
  // t = A_oo^{-1} H_oe in
  auto a1 = params<PREC>(op, 1, t, in);
  a1.clov = clov_ptr<PREC>(op, 1);
  a1.scal = scal;
  // out = A_ee in - kappa^2 H_eo t
  auto a2 = params<PREC>(op, 0, out, t);
  a2.clov = clov_ptr<PREC>(op, 0);
  a2.x = (const typename Prec<PREC>::vec*)in;
  a2.coef = -op->kappa * op->kappa;
  a2.norm_out = norm_out;
  a2.scal = scal;
  if (dagger) {
    launch<PREC, true, EPI_CLOV, false>(a1, s);
    if (norm_out)
      launch<PREC, true, EPI_XPAY, true>(a2, s);
    else
      launch<PREC, true, EPI_XPAY, false>(a2, s);
  } else {
    launch<PREC, false, EPI_CLOV, false>(a1, s);
    if (norm_out)
      launch<PREC, false, EPI_XPAY, true>(a2, s);
    else
      launch<PREC, false, EPI_XPAY, false>(a2, s);
  }
}

// M-hat with a caller-supplied odd-site temporary (used by the allocation-free entry
// point); the same two launches as mhat() below
void mhat_with_temp(pfmp_op* op, int prec, void* out, const void* in, bool dagger, void* temp) {
  require_clover(op);
  if (prec == PFMP_F64) {
    double2* keep = op->t64;
    op->t64 = (double2*)temp;
    try {
      mhat_t<PFMP_F64>(op, out, in, dagger, nullptr, nullptr);
    } catch (...) {
      op->t64 = keep;
      throw;
    }
    op->t64 = keep;
  } else {
    float4* keep = op->t32;
    op->t32 = (float4*)temp;
    try {
      mhat_t<PFMP_F32>(op, out, in, dagger, nullptr, nullptr);
    } catch (...) {
      op->t32 = keep;
      throw;
    }
    op->t32 = keep;
  }
}

void mhat(pfmp_op* op, int prec, void* out, const void* in, bool dagger, double* norm_out, CGScalars* scal) {
  require_clover(op);
  if (prec == PFMP_F64)
    mhat_t<PFMP_F64>(op, out, in, dagger, norm_out, scal);
  else if (prec == PFMP_H16)
    mhat_t<PFMP_H16>(op, out, in, dagger, norm_out, scal);
  else
    mhat_t<PFMP_F32>(op, out, in, dagger, norm_out, scal);
}

// K in double-float: in/out are df even fields ([12][Vh] float4), FP32-pipe arithmetic
void kop_df(pfmp_op* op, void* out, const void* in) {
  require_clover(op);
  op->kapply += 1;
  mhat_t<PREC_DF>(op, op->edf, in, false, nullptr, nullptr);
  mhat_t<PREC_DF>(op, out, op->edf, true, nullptr, nullptr);
}

// out (odd) = A_oo^{-1} H_oe in (or the adjoint hop), FP64: the first half of M-hat,
// used by the force terms
void hop_clov_odd(pfmp_op* op, void* out, const void* in, bool dagger) {
  require_clover(op);
  auto a = params<PFMP_F64>(op, 1, out, in);
  a.clov = clov_ptr<PFMP_F64>(op, 1);
  if (dagger)
    launch<PFMP_F64, true, EPI_CLOV, false>(a, op);
  else
    launch<PFMP_F64, false, EPI_CLOV, false>(a, op);
}

// out = K in; <in, K in> = ||M-hat in||^2 is reduced in the second kernel of M-hat
void kop(pfmp_op* op, int prec, void* out, const void* in, double* pKp_dev, CGScalars* scal) {
  op->kapply += 1;
  void* e = prec == PFMP_F64 ? (void*)op->e64 : (prec == PFMP_H16 ? (void*)op->e16 : (void*)op->e32);
  mhat(op, prec, e, in, false, pKp_dev, scal);
  mhat(op, prec, out, e, true, nullptr, scal);
}

}  // namespace pfmp
