// Stencil kernels of the Wilson-clover operator and their launch drivers, templated on
// the arithmetic (FP64, FP32, double-float, FP16 storage) and on the adjoint.  Included
// only by the dslash_<prec>_<dag>.cu files, each of which instantiates one (precision,
// adjoint) pair, so that the heavy template instantiations compile in parallel;
// dslash.h declares what they export and dslash.cu dispatches on run-time arguments.
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
#pragma once
#include "dslash.h"
#include "dfloat.cuh"
#include "hop.cuh"

#ifndef HOP_MINB_F32
#define HOP_MINB_F32 7
#endif
#ifndef HOP_MINB_H16
#define HOP_MINB_H16 6
#endif
#ifndef HOP_MINB_F64
#define HOP_MINB_F64 1
#endif

namespace pfmp {

// Resident 128-thread blocks per SM that the register allocation must allow.  The
// stencil is bound by memory latency, so more warps in flight pay even at the cost of a
// few spilled registers (FP32, 32^3x64: 0.85 -> 0.89 of the copy bandwidth at 7 blocks).
// The FP16-storage stencil does more arithmetic per byte and runs best with a few more
// registers (K at 32^3x64: 97.4 us per launch at 7 blocks, 93.1 at 6 or 5, 103 at 8);
// FP64 and double-float keep the compiler's choice (a bound of 3 blocks made the rolled
// double-float stencil 7-18% slower).
template <int PREC>
constexpr int hop_min_blocks() {
  return PREC == PFMP_F32 ? HOP_MINB_F32 : PREC == PFMP_H16 ? HOP_MINB_H16 : PREC == PFMP_F64 ? HOP_MINB_F64 : 1;
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
    else if constexpr (PREC == PFMP_H16)
      out = hop_site_h16<DAG, EPI>(a, cb);
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

// ---------------------------------------------------------------- host drivers
constexpr int kHopBlock = 128;

template <int PREC>
HopParams<PREC> params(pfmp_op* op, int p, void* out, const void* in) {
  using vec = typename Prec<PREC>::vec;
  HopParams<PREC> a;
  a.g = op->ctx->g;
  a.p = p;
  a.out = (vec*)out;
  a.in = (const vec*)in;
  a.gauge = PREC == PFMP_F64   ? (const vec*)(const void*)op->ctx->U64
            : PREC == PREC_DF  ? (const vec*)(const void*)op->ctx->Udf
            : PREC == PFMP_H16 ? (const vec*)(const void*)op->ctx->U16
                               : (const vec*)(const void*)op->ctx->U32;
  a.clov = nullptr;
  a.x = nullptr;
  a.in2 = nullptr;
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
double hop_bytes(int epi, int Vh) {
  if (PREC == PFMP_H16) {  // FP16 reals, plus the FP32 scale of every spinor read or written
    const double b = 8 * 12 * 2 + 52 + 52 + (epi >= EPI_CLOV ? 72 * 2 : 0) + (epi == EPI_XPAY ? 52 : 0);
    return b * (double)Vh;
  }
  const double link = (PREC == PREC_DF || PREC == PFMP_F64) ? 18 : 12;
  const double reals = 8 * link + 24 + 24 + (epi >= EPI_CLOV ? 72 : 0) + (epi == EPI_XPAY ? 24 : 0);
  return reals * (PREC == PFMP_F32 ? 4 : 8) * (double)Vh;
}

template <int PREC>
int split_of(const pfmp_op* op) {
  return op->nsplit[PREC == PFMP_F64 ? 0 : (PREC == PFMP_F32 ? 1 : 2)];
}

template <int PREC, bool DAG, int EPI, bool RED>
void launch(const HopParams<PREC>& a, pfmp_op* op) {
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
const typename Prec<PREC>::vec* clov_ptr(pfmp_op* op, int parity) {
  if (PREC == PFMP_F64) return (const typename Prec<PREC>::vec*)(const void*)op->clov64[parity];
  if (PREC == PREC_DF) return (const typename Prec<PREC>::vec*)(const void*)op->clovdf[parity];
  if (PREC == PFMP_H16) return (const typename Prec<PREC>::vec*)(const void*)op->clov16[parity];
  return (const typename Prec<PREC>::vec*)(const void*)op->clov32[parity];
}

// out (parity p) = coef H in, plain epilogue
template <int PREC, bool DAG>
void hop_plain_t(pfmp_op* op, void* out, const void* in, int p) {
  auto a = params<PREC>(op, p, out, in);
  launch<PREC, DAG, EPI_PLAIN, false>(a, op);
}

// out (odd) = A_oo^{-1} H_oe in: the first half of M-hat (and of its adjoint)
template <int PREC, bool DAG>
void hop_clov_odd_t(pfmp_op* op, void* out, const void* in, CGScalars* scal) {
  auto a = params<PREC>(op, 1, out, in);
  a.clov = clov_ptr<PREC>(op, 1);
  a.scal = scal;
  launch<PREC, DAG, EPI_CLOV, false>(a, op);
}

// out = M-hat in (or M-hat^dag in) through the odd temporary t: t = A_oo^{-1} H_oe in,
// then out = A_ee in - kappa^2 H_eo t (with ||out||^2 -> *norm_out when asked)
template <int PREC, bool DAG>
void mhat_t(pfmp_op* op, void* out, const void* in, double* norm_out, CGScalars* scal, void* t) {
  hop_clov_odd_t<PREC, DAG>(op, t, in, scal);
  auto a2 = params<PREC>(op, 0, out, t);
  a2.clov = clov_ptr<PREC>(op, 0);
  a2.x = (const typename Prec<PREC>::vec*)in;
  a2.coef = -op->kappa * op->kappa;
  a2.norm_out = norm_out;
  a2.scal = scal;
  if (norm_out)
    launch<PREC, DAG, EPI_XPAY, true>(a2, op);
  else
    launch<PREC, DAG, EPI_XPAY, false>(a2, op);
}

#define PFMP_DSLASH_INSTANTIATE(PREC, DAG)                                                              \
  template void hop_plain_t<PREC, DAG>(pfmp_op*, void*, const void*, int);                              \
  template void hop_clov_odd_t<PREC, DAG>(pfmp_op*, void*, const void*, CGScalars*);                    \
  template void mhat_t<PREC, DAG>(pfmp_op*, void*, const void*, double*, CGScalars*, void*);

}  // namespace pfmp
