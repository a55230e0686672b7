// The Wilson-clover stencil at one site, shared by the single-system kernels
// (dslash.cu) and the grouped multi-system kernels (batch.cu).  One thread per output
// site: the 8 neighbours are spin-projected to half spinors (the projectors
// (1 -+ g_mu) have rank 2), multiplied by the link (12-real links, third row rebuilt in
// registers) and rebuilt; the epilogue then applies the clover blocks:
//   EPI_PLAIN  out = coef (H in)
//   EPI_CLOV   out = coef C (H in)            (odd sites: C = A_oo^{-1})
//   EPI_XPAY   out = C x + coef (H in)        (even sites: C = A_ee, x the local input)
#pragma once
#include "context.h"
#include "fields.cuh"
#include "spin.cuh"

namespace pfmp {

enum { EPI_PLAIN = 0, EPI_CLOV = 1, EPI_XPAY = 2 };

template <int PREC>
struct HopParams {
  using vec = typename Prec<PREC>::vec;
  Geom g;
  int p;  // output parity
  vec* out;
  const vec* in;     // parity 1 - p
  const vec* gauge;  // [2][4][link_vecs][Vh]
  const vec* clov;   // clover blocks of parity p (EPI_CLOV, EPI_XPAY)
  const vec* x;      // local input of parity p (EPI_XPAY)
  double coef;
  ReduceBuf rb;
  double* norm_out;  // ||out||^2 (device) when reducing
  CGScalars* scal;   // optional: alpha = rr / ||out||^2; skip all work once done
};

// forward (x+mu, projector 1 + SF g) and backward (x-mu, projector 1 - SF g) terms
template <int PREC, int MU, int SF>
__device__ __forceinline__ void hop_dir(Spinor<typename Prec<PREC>::real>& acc, const HopParams<PREC>& a,
                                        const int x[4], int cb) {
  using T = typename Prec<PREC>::real;
  constexpr int LV = Prec<PREC>::link_vecs;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  {
    const int n = nbr_cb(g, x, MU, +1);
    Spinor<T> psi;
    load_spinor(psi, a.in, n, Vh);
    Half<T> h = project<MU, SF>(psi);
    Mat3<T> U;
    load_link(U, a.gauge + (size_t)((a.p * 4 + MU) * LV) * Vh, cb, Vh);
    Half<T> r = mul_half(U, h);
    if (MU == 3 && x[3] == g.L[3] - 1) scale_half(r, (T)g.bc_t);
    accumulate<MU, SF>(acc, r);
  }
  {
    const int n = nbr_cb(g, x, MU, -1);
    Spinor<T> psi;
    load_spinor(psi, a.in, n, Vh);
    Half<T> h = project<MU, -SF>(psi);
    Mat3<T> U;
    load_link(U, a.gauge + (size_t)(((1 - a.p) * 4 + MU) * LV) * Vh, n, Vh);
    Half<T> r = mul_half_dag(U, h);
    if (MU == 3 && x[3] == 0) scale_half(r, (T)g.bc_t);
    accumulate<MU, -SF>(acc, r);
  }
}

// the stencil at one output site cb: hop, spin projection and the fused epilogue
template <int PREC, bool DAG, int EPI>
__device__ __forceinline__ Spinor<typename Prec<PREC>::real> hop_site(const HopParams<PREC>& a, int cb) {
  using T = typename Prec<PREC>::real;
  int x[4];
  cb_coords(a.g, cb, a.p, x);
  Spinor<T> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.s[s][c] = mk<T>(0, 0);
  constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF g_mu
  hop_dir<PREC, 0, SF>(acc, a, x, cb);
  hop_dir<PREC, 1, SF>(acc, a, x, cb);
  hop_dir<PREC, 2, SF>(acc, a, x, cb);
  hop_dir<PREC, 3, SF>(acc, a, x, cb);
  Spinor<T> out;
  const T cf = (T)a.coef;
  if (EPI == EPI_PLAIN) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = cf * acc.s[s][c];
  } else if (EPI == EPI_CLOV) {
    HermBlock<T> B[2];
    load_clover(B, a.clov, cb, a.g.Vh);
    out = clover_apply(B, acc);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = cf * out.s[s][c];
  } else {
    HermBlock<T> B[2];
    load_clover(B, a.clov, cb, a.g.Vh);
    Spinor<T> xl;
    load_spinor(xl, a.x, cb, a.g.Vh);
    out = clover_apply(B, xl);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = out.s[s][c] + cf * acc.s[s][c];
  }
  return out;
}

template <typename T>
__device__ __forceinline__ double spinor_norm2(const Spinor<T>& v) {
  double t = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) t += (double)norm2(v.s[s][c]);
  return t;
}

}  // namespace pfmp
