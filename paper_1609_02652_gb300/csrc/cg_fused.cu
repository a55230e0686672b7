// One FP32 CG iteration of the mixed solver as four stencil kernels: the CG vector
// updates ride in the stencil kernels instead of running as kernels of their own.
//
//   phase 1  t = A_oo^{-1} H_oe p,  p = r + beta p_old formed where the stencil reads it
//   phase 2  e = A_ee p - kappa^2 H_eo t with the local p formed the same way and stored;
//            ||e||^2 = <p, K p> -> alpha = rr / <p, K p>
//   phase 3  t = A_oo^{-1} H^dag_oe e
//   phase 4  K p = A_ee e - kappa^2 H^dag_eo t (not stored): x += alpha p, r -= alpha K p;
//            ||r||^2 -> beta = ||r||^2 / rr, rr, iteration count, done
//
// (K = M-hat^dag M-hat; the same recurrences as the six-kernel iteration, with the p
// update of iteration k carried out by iteration k + 1's first two phases.)  The
// scalars live on the device; every kernel returns at once when done is set, so a
// CUDA-graph chunk of iterations stops where the CG converged.  The first iteration
// starts from p_old = r, beta = 0.
#include "context.h"
#include "hop.cuh"

namespace pfmp {

namespace {

// resident 128-thread blocks per SM: 7 as the FP32 stencil; 6 for the two kernels that
// also carry CG vectors (at 7 they spill 0.1-0.6 KB per thread)
constexpr int kMinBlocks = 7;
constexpr int kMinBlocksVec = 6;

__device__ __forceinline__ float4 f4(const cplx<float>& a, const cplx<float>& b) { return make_float4(a.re, a.im, b.re, b.im); }

__global__ void __launch_bounds__(128, kMinBlocks) k_cgf_1(HopParams<PFMP_F32> a) {
  if (a.scal->done) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= a.g.Vh) return;
  const float beta = (float)a.scal->beta;
  const Spinor<float> out = hop_site<PFMP_F32, false, EPI_CLOV, false, true>(a, cb, beta);
  store_spinor(a.out, out, cb, a.g.Vh);
}

__global__ void __launch_bounds__(128, kMinBlocksVec) k_cgf_2(HopParams<PFMP_F32> a, const float4* __restrict__ r,
                                                           float4* __restrict__ p) {
  CGScalars* sc = a.scal;
  if (sc->done) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  double nrm[1] = {0.0};
  if (cb < a.g.Vh) {
    // the hop first (coef H t), then the local direction and the A_ee epilogue, so that
    // the local spinor is not live across the stencil
    Spinor<float> out = hop_site<PFMP_F32, false, EPI_PLAIN>(a, cb);
    const float beta = (float)sc->beta;
    Spinor<float> pl, q;
    load_spinor(pl, r, cb, a.g.Vh);
    load_spinor(q, p, cb, a.g.Vh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) pl.s[s][c] = pl.s[s][c] + beta * q.s[s][c];
    store_spinor(p, pl, cb, a.g.Vh);
    HermBlock<float> B[2];
    load_clover(B, a.clov, cb, a.g.Vh);
    const Spinor<float> ap = clover_apply(B, pl);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = out.s[s][c] + ap.s[s][c];
    store_spinor(a.out, out, cb, a.g.Vh);
    nrm[0] = spinor_norm2(out);
  }
  double tot[1];
  if (grid_sum<1>(nrm, a.rb, tot)) {
    sc->pAp = tot[0];
    sc->alpha = sc->rr / tot[0];
  }
}

__global__ void __launch_bounds__(128, kMinBlocks) k_cgf_3(HopParams<PFMP_F32> a) {
  if (a.scal->done) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= a.g.Vh) return;
  store_spinor(a.out, hop_site<PFMP_F32, true, EPI_CLOV>(a, cb), cb, a.g.Vh);
}

__global__ void __launch_bounds__(128, kMinBlocksVec) k_cgf_4(HopParams<PFMP_F32> a, float4* __restrict__ x,
                                                           float4* __restrict__ r, const float4* __restrict__ p) {
  CGScalars* sc = a.scal;
  if (sc->done) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int Vh = a.g.Vh;
  double v[1] = {0.0};
  if (cb < Vh) {
    const float al = (float)sc->alpha;
    const Spinor<float> kp = hop_site<PFMP_F32, true, EPI_XPAY>(a, cb);
    float acc = 0.f;  // the site's |r|^2 in FP32, across sites in FP64
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const size_t i = (size_t)k * Vh + cb;
      const float4 kv = f4(kp.s[(2 * k) / 3][(2 * k) % 3], kp.s[(2 * k + 1) / 3][(2 * k + 1) % 3]);
      float4 xx = x[i], rr = r[i];
      const float4 pp = p[i];
      xx.x += al * pp.x;
      xx.y += al * pp.y;
      xx.z += al * pp.z;
      xx.w += al * pp.w;
      rr.x -= al * kv.x;
      rr.y -= al * kv.y;
      rr.z -= al * kv.z;
      rr.w -= al * kv.w;
      x[i] = xx;
      r[i] = rr;
      acc += rr.x * rr.x + rr.y * rr.y + rr.z * rr.z + rr.w * rr.w;
    }
    v[0] = acc;
  }
  double t[1];
  if (grid_sum<1>(v, a.rb, t)) {
    sc->rr_new = t[0];
    sc->beta = t[0] / sc->rr;
    sc->rr = t[0];
    sc->iter += 1;
    if (t[0] < sc->stop_rr || !(t[0] == t[0])) {
      sc->done_next = 1;
      sc->done = 1;
    }
  }
}

// per output site: the plain stencil's algorithmic reals (8 links of 12, input and output
// spinors, clover blocks, local input) plus the CG vectors each phase reads or writes
double reals_per_site(int phase) {
  const double hop = 8 * 12 + 24 + 24 + 72;
  switch (phase) {
    case 1: return hop + 24;            // + p_old beside r
    case 2: return hop + 24 + 24 + 24;  // + r, p_old read, p stored (the local input read is r)
    case 3: return hop;
    default: return hop + 24 + 72 + 48 - 24;  // + local e; x, r, p read; x, r stored; K p not stored
  }
}

}  // namespace

// one fused FP32 CG iteration on the context's stream; x, r, p: FP32 even fields (p holds
// the previous direction, r the current residual, beta in op->scal the pending step)
void cg_fused_iteration(pfmp_op* op, float4* x, float4* r, float4* p) {
  pfmp_ctx* c = op->ctx;
  const Geom& g = c->g;
  const int bs = op->hop_block;
  const dim3 grid(nblocks(g.Vh, bs));
  HopParams<PFMP_F32> a{};
  a.g = g;
  a.gauge = c->U32;
  a.rb = c->rb;
  a.scal = op->scal;
  cudaEvent_t ev;
  // phase 1
  a.p = 1;
  a.in = r;
  a.in2 = p;
  a.out = op->t32;
  a.clov = op->clov32[1];
  a.coef = 1.0;
  prof_start(c, &ev);
  k_cgf_1<<<grid, bs, 0, c->stream>>>(a);
  PFMP_CHECK_LAUNCH();
  prof_stop(c, PFMP_KERNEL_CG_F32, reals_per_site(1) * 4.0 * g.Vh, ev);
  // phase 2
  a.p = 0;
  a.in = op->t32;
  a.in2 = nullptr;
  a.out = op->e32;
  a.clov = op->clov32[0];
  a.coef = -op->kappa * op->kappa;
  prof_start(c, &ev);
  k_cgf_2<<<grid, bs, 0, c->stream>>>(a, r, p);
  PFMP_CHECK_LAUNCH();
  prof_stop(c, PFMP_KERNEL_CG_F32, reals_per_site(2) * 4.0 * g.Vh, ev);
  // phase 3
  a.p = 1;
  a.in = op->e32;
  a.out = op->t32;
  a.clov = op->clov32[1];
  a.coef = 1.0;
  prof_start(c, &ev);
  k_cgf_3<<<grid, bs, 0, c->stream>>>(a);
  PFMP_CHECK_LAUNCH();
  prof_stop(c, PFMP_KERNEL_CG_F32, reals_per_site(3) * 4.0 * g.Vh, ev);
  // phase 4
  a.p = 0;
  a.in = op->t32;
  a.x = op->e32;
  a.out = nullptr;
  a.clov = op->clov32[0];
  a.coef = -op->kappa * op->kappa;
  prof_start(c, &ev);
  k_cgf_4<<<grid, bs, 0, c->stream>>>(a, x, r, p);
  PFMP_CHECK_LAUNCH();
  prof_stop(c, PFMP_KERNEL_CG_F32, reals_per_site(4) * 4.0 * g.Vh, ev);
  op->kapply += 1;
}

}  // namespace pfmp
