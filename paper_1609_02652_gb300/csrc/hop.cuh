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
  const vec* gauge;  // per (parity, mu) link planes, located by link_plane
  const vec* clov;   // clover blocks of parity p (EPI_CLOV, EPI_XPAY)
  const vec* x;      // local input of parity p (EPI_XPAY)
  const vec* in2;    // second input (XPY stencils: the input is in + beta in2)
  double coef;
  ReduceBuf rb;
  double* norm_out;  // ||out||^2 (device) when reducing
  CGScalars* scal;   // optional: alpha = rr / ||out||^2; skip all work once done
};

// the stencil's input at site n: a.in, or with XPY a.in + beta a.in2 (a CG direction
// p = r + beta p_old formed where the stencil reads it)
template <int PREC, bool CG, bool XPY>
__device__ __forceinline__ void load_in(Spinor<typename Prec<PREC>::real>& psi, const HopParams<PREC>& a, int n, int Vh,
                                        typename Prec<PREC>::real beta) {
  load_spinor<CG>(psi, a.in, n, Vh);
  if constexpr (XPY) {
    Spinor<typename Prec<PREC>::real> q;
    load_spinor<CG>(q, a.in2, n, Vh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) psi.s[s][c] = psi.s[s][c] + beta * q.s[s][c];
  }
}

// forward (x+mu, projector 1 + SF g) and backward (x-mu, projector 1 - SF g) terms
template <int PREC, int MU, int SF, bool CG = false, bool XPY = false>
__device__ __forceinline__ void hop_dir(Spinor<typename Prec<PREC>::real>& acc, const HopParams<PREC>& a,
                                        const int x[4], int cb,
                                        typename Prec<PREC>::real beta = typename Prec<PREC>::real(0)) {
  using T = typename Prec<PREC>::real;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  {
    const int n = nbr_cb(g, x, MU, +1);
    Spinor<T> psi;
    load_in<PREC, CG, XPY>(psi, a, n, Vh, beta);
    Half<T> h = project<MU, SF>(psi);
    Mat3<T> U;
    load_link(U, link_plane<PREC>(a.gauge, a.p * 4 + MU, Vh), cb, Vh);
    Half<T> r = mul_half(U, h);
    if (MU == 3 && x[3] == g.L[3] - 1) scale_half(r, (T)g.bc_t);
    accumulate<MU, SF>(acc, r);
  }
  {
    const int n = nbr_cb(g, x, MU, -1);
    Spinor<T> psi;
    load_in<PREC, CG, XPY>(psi, a, n, Vh, beta);
    Half<T> h = project<MU, -SF>(psi);
    Mat3<T> U;
    load_link(U, link_plane<PREC>(a.gauge, (1 - a.p) * 4 + MU, Vh), n, Vh);
    Half<T> r = mul_half_dag(U, h);
    if (MU == 3 && x[3] == 0) scale_half(r, (T)g.bc_t);
    accumulate<MU, -SF>(acc, r);
  }
}

// the stencil at one output site cb: hop, spin projection and the fused epilogue.  XPY:
// the input is a.in + beta a.in2; xl: the local input of EPI_XPAY given by the caller
// instead of loaded from a.x
template <int PREC, bool DAG, int EPI, bool CG = false, bool XPY = false>
__device__ __forceinline__ Spinor<typename Prec<PREC>::real> hop_site(
    const HopParams<PREC>& a, int cb, typename Prec<PREC>::real beta = typename Prec<PREC>::real(0),
    const Spinor<typename Prec<PREC>::real>* xl_given = nullptr) {
  using T = typename Prec<PREC>::real;
  int x[4];
  cb_coords(a.g, cb, a.p, x);
  Spinor<T> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.s[s][c] = mk<T>(0, 0);
  constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF g_mu
  hop_dir<PREC, 0, SF, CG, XPY>(acc, a, x, cb, beta);
  hop_dir<PREC, 1, SF, CG, XPY>(acc, a, x, cb, beta);
  hop_dir<PREC, 2, SF, CG, XPY>(acc, a, x, cb, beta);
  hop_dir<PREC, 3, SF, CG, XPY>(acc, a, x, cb, beta);
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
    if (xl_given)
      xl = *xl_given;
    else
      load_spinor<CG>(xl, a.x, cb, a.g.Vh);
    out = clover_apply(B, xl);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = out.s[s][c] + cf * acc.s[s][c];
  }
  return out;
}

// ---------------------------------------------------------------- FP16 storage, half2 arithmetic
// The stencil on FP16 storage converts few values to FP32: each neighbour spinor
// (stored as value / scale, |entries| <= 1) is spin-projected in packed half2 adds, the
// FP16 link (never converted; its third row rebuilt in half2) multiplies the half
// spinor with half2 FMAs, and only the 12 reals of each direction's product are
// converted, multiplied by the neighbour's scale (and the boundary factor) and summed in
// FP32, where the four-component rebuild and the clover epilogue happen.  Conversions per
// site: 8 x 12 + 72 (clover) instead of 8 x (24 + 12) + 72.  Complex numbers are half2
// (re, im); a x b = hi(a) (i b) + lo(a) b with lo, hi the broadcast real and imaginary
// parts, and conj(a) x b = lo(a) b - hi(a) (i b).
__device__ __forceinline__ __half2 u2h2(uint32_t u) {
  __half2 h;
  memcpy(&h, &u, 4);
  return h;
}
__device__ __forceinline__ __half2 h2_times_i(__half2 v) {  // i v = (-im, re)
  return __hmul2(__lowhigh2highlow(v), __floats2half2_rn(-1.f, 1.f));
}
__device__ __forceinline__ __half2 h2_cmul(__half2 a, __half2 b, __half2 ib) {  // a b
  return __hfma2(__high2half2(a), ib, __hmul2(__low2half2(a), b));
}
__device__ __forceinline__ __half2 h2_cfma(__half2 a, __half2 b, __half2 ib, __half2 acc) {  // acc + a b
  return __hfma2(__high2half2(a), ib, __hfma2(__low2half2(a), b, acc));
}
__device__ __forceinline__ __half2 h2_cjfma(__half2 a, __half2 b, __half2 ib, __half2 acc) {  // acc + conj(a) b
  return __hfma2(__hneg2(__high2half2(a)), ib, __hfma2(__low2half2(a), b, acc));
}
__device__ __forceinline__ __half2 h2_conj(__half2 v) { return __hmul2(v, __floats2half2_rn(1.f, -1.f)); }

// FP16 link as half2 [3][3], third row conj(row0 x row1) rebuilt in half2
__device__ __forceinline__ void load_link_h2(__half2 U[3][3], const uint4* __restrict__ f, int cb, int Vh) {
  const uint4 v0 = __ldg(f + cb);
  const uint2 v1 = __ldg(reinterpret_cast<const uint2*>(f + Vh) + cb);
  U[0][0] = u2h2(v0.x);
  U[0][1] = u2h2(v0.y);
  U[0][2] = u2h2(v0.z);
  U[1][0] = u2h2(v0.w);
  U[1][1] = u2h2(v1.x);
  U[1][2] = u2h2(v1.y);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3, l = (j + 2) % 3;
    const __half2 b1 = U[1][l], b2 = U[1][k];
    const __half2 t = h2_cmul(U[0][k], b1, h2_times_i(b1));
    U[2][j] = h2_conj(__hsub2(t, h2_cmul(U[0][l], b2, h2_times_i(b2))));
  }
}

// (1 + S g_MU) psi of a half2 spinor p[spin][colour]: the two components h[2][3]
template <int MU, int S>
__device__ __forceinline__ void project_h2(const __half2 p[4][3], __half2 h[2][3]) {
  const __half2 pi = __floats2half2_rn(-1.f, 1.f), mi = __floats2half2_rn(1.f, -1.f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {  // p0 +- i p3, p1 +- i p2
      h[0][c] = __hfma2(__lowhigh2highlow(p[3][c]), S > 0 ? pi : mi, p[0][c]);
      h[1][c] = __hfma2(__lowhigh2highlow(p[2][c]), S > 0 ? pi : mi, p[1][c]);
    } else if (MU == 1) {  // p0 -+ p3, p1 +- p2
      h[0][c] = S > 0 ? __hsub2(p[0][c], p[3][c]) : __hadd2(p[0][c], p[3][c]);
      h[1][c] = S > 0 ? __hadd2(p[1][c], p[2][c]) : __hsub2(p[1][c], p[2][c]);
    } else if (MU == 2) {  // p0 +- i p2, p1 -+ i p3
      h[0][c] = __hfma2(__lowhigh2highlow(p[2][c]), S > 0 ? pi : mi, p[0][c]);
      h[1][c] = __hfma2(__lowhigh2highlow(p[3][c]), S > 0 ? mi : pi, p[1][c]);
    } else {  // p0 +- p2, p1 +- p3
      h[0][c] = S > 0 ? __hadd2(p[0][c], p[2][c]) : __hsub2(p[0][c], p[2][c]);
      h[1][c] = S > 0 ? __hadd2(p[1][c], p[3][c]) : __hsub2(p[1][c], p[3][c]);
    }
  }
}

// one hop term on FP16 storage: load, project, transport in half2; the product times
// `scale` (the neighbour's spinor scale and boundary factor) summed into acc in FP32
template <int MU, int S, bool DAGU>
__device__ __forceinline__ void hop_term_h16(Spinor<float>& acc, const uint4* __restrict__ in, const uint4* lf, int n,
                                             int lcb, int Vh, float bcf) {
  __half2 p[4][3];
  const float sc = bcf * __ldg(reinterpret_cast<const float*>(in + (size_t)3 * Vh) + n);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 v = __ldg(in + (size_t)k * Vh + n);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) p[(4 * k + j) / 3][(4 * k + j) % 3] = u2h2(w[j]);
  }
  __half2 h[2][3], ih[2][3];
  project_h2<MU, S>(p, h);
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) ih[k][c] = h2_times_i(h[k][c]);
  __half2 U[3][3];
  load_link_h2(U, lf, lcb, Vh);
  Half<float> r;
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      __half2 t;
      if (DAGU) {  // sum_j conj(U[j][i]) h[k][j]
        t = h2_cjfma(U[0][i], h[k][0], ih[k][0], __float2half2_rn(0.f));
        t = h2_cjfma(U[1][i], h[k][1], ih[k][1], t);
        t = h2_cjfma(U[2][i], h[k][2], ih[k][2], t);
      } else {  // sum_j U[i][j] h[k][j]
        t = h2_cmul(U[i][0], h[k][0], ih[k][0]);
        t = h2_cfma(U[i][1], h[k][1], ih[k][1], t);
        t = h2_cfma(U[i][2], h[k][2], ih[k][2], t);
      }
      const float2 f = __half22float2(t);
      r.h[k][i] = mk(sc * f.x, sc * f.y);
    }
  accumulate<MU, S>(acc, r);
}

template <int MU, int SF>
__device__ __forceinline__ void hop_dir_h16(Spinor<float>& acc, const HopParams<PFMP_H16>& a, const int x[4],
                                            int cb) {
  const Geom& g = a.g;
  const int Vh = g.Vh;
  {
    const int n = nbr_cb(g, x, MU, +1);
    const float f = (MU == 3 && x[3] == g.L[3] - 1) ? (float)g.bc_t : 1.0f;
    hop_term_h16<MU, SF, false>(acc, a.in, link_plane<PFMP_H16>(a.gauge, a.p * 4 + MU, Vh), n, cb, Vh, f);
  }
  {
    const int n = nbr_cb(g, x, MU, -1);
    const float f = (MU == 3 && x[3] == 0) ? (float)g.bc_t : 1.0f;
    hop_term_h16<MU, -SF, true>(acc, a.in, link_plane<PFMP_H16>(a.gauge, (1 - a.p) * 4 + MU, Vh), n, n, Vh, f);
  }
}

template <bool DAG, int EPI>
__device__ __forceinline__ Spinor<float> hop_site_h16(const HopParams<PFMP_H16>& a, int cb) {
  int x[4];
  cb_coords(a.g, cb, a.p, x);
  Spinor<float> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.s[s][c] = mk(0.f, 0.f);
  constexpr int SF = DAG ? +1 : -1;
  hop_dir_h16<0, SF>(acc, a, x, cb);
  hop_dir_h16<1, SF>(acc, a, x, cb);
  hop_dir_h16<2, SF>(acc, a, x, cb);
  hop_dir_h16<3, SF>(acc, a, x, cb);
  Spinor<float> out;
  const float cf = (float)a.coef;
  if (EPI == EPI_PLAIN) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = cf * acc.s[s][c];
  } else if (EPI == EPI_CLOV) {
    HermBlock<float> B[2];
    load_clover(B, a.clov, cb, a.g.Vh);
    out = clover_apply(B, acc);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = cf * out.s[s][c];
  } else {
    HermBlock<float> B[2];
    load_clover(B, a.clov, cb, a.g.Vh);
    Spinor<float> xl;
    load_spinor(xl, a.x, cb, a.g.Vh);
    out = clover_apply(B, xl);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) out.s[s][c] = out.s[s][c] + cf * acc.s[s][c];
  }
  return out;
}

// ---------------------------------------------------------------- rolled stencil
// The same stencil with the 8 hop terms in a run-time loop and the two clover blocks in
// another, so that the colour multiply and the 6x6 block product exist once in the code
// instead of eight and two times.  The projector and rebuild of direction mu with sign S
// are written as unit phases c in {+-1, +-i}:
//   h0 = psi0 + c0 psi_A,  h1 = psi1 + c1 psi_B      (A, B = 3, 2 for mu < 2; 2, 3 else)
//   out0 += r0, out1 += r1, out2 += c2 r_P, out3 += c3 r_Q  (P, Q = 1, 0 for mu < 2; 0, 1 else)
// with c imaginary for mu = 0, 2 and, for s = sign(S),
//   c0 = -s (mu = 1) else s;  c1 = -s (mu = 2) else s;  c2 = -s (mu even) else s;
//   c3 = -s (mu < 2) else s
// (the chiral-basis projectors of spin.cuh; parity tests compare both forms).  Backward
// terms multiply by U^dag, formed in registers by selects.

// v times (isI ? i : 1) times (neg ? -1 : 1)
template <typename T>
__device__ __forceinline__ cplx<T> unit_phase(const cplx<T>& v, bool isI, bool neg) {
  const cplx<T> w = isI ? mk(-v.im, v.re) : v;
  return neg ? -w : w;
}

template <typename T>
__device__ __forceinline__ void dagger_if(Mat3<T>& U, bool dag) {
  Mat3<T> V;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V.m[i][j] = dag ? conj(U.m[j][i]) : U.m[i][j];
  U = V;
}

// checkerboard index of x + dir mu for a run-time mu (static indexing only)
__device__ __forceinline__ int nbr_cb_rt(const Geom& g, const int x[4], int mu, int dir) {
  int y[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int v = x[m] + (m == mu ? dir : 0);
    y[m] = v == g.L[m] ? 0 : (v < 0 ? g.L[m] - 1 : v);
  }
  return cb_index(g, y);
}

template <int PREC, bool DAG, int EPI, bool CG = false>
__device__ __forceinline__ Spinor<typename Prec<PREC>::real> hop_site_rolled(const HopParams<PREC>& a, int cb) {
  using T = typename Prec<PREC>::real;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  int x[4];
  cb_coords(g, cb, a.p, x);
  Spinor<T> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.s[s][c] = mk<T>(0, 0);
  constexpr bool SF_POS = DAG;  // forward projector 1 + SF g_mu, SF = +1 for the adjoint
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const bool sp = fwd ? SF_POS : !SF_POS;  // sign of this term's projector
    const int n = nbr_cb_rt(g, x, mu, fwd ? +1 : -1);
    Spinor<T> psi;
    load_spinor<CG>(psi, a.in, n, Vh);
    const bool low = mu < 2, isI = (mu & 1) == 0;
    const bool n0 = (mu == 1) == sp, n1 = (mu == 2) == sp, n2 = isI == sp, n3 = low == sp;
    Half<T> h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> pa = low ? psi.s[3][c] : psi.s[2][c];
      const cplx<T> pb = low ? psi.s[2][c] : psi.s[3][c];
      h.h[0][c] = psi.s[0][c] + unit_phase(pa, isI, n0);
      h.h[1][c] = psi.s[1][c] + unit_phase(pb, isI, n1);
    }
    Mat3<T> U;
    load_link(U, link_plane<PREC>(a.gauge, (fwd ? a.p : 1 - a.p) * 4 + mu, Vh), fwd ? cb : n, Vh);
    dagger_if(U, !fwd);
    Half<T> r = mul_half(U, h);
    const bool edge = mu == 3 && (fwd ? x[3] == g.L[3] - 1 : x[3] == 0);
    const bool flip = edge && g.bc_t < 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> r0 = flip ? -r.h[0][c] : r.h[0][c];
      const cplx<T> r1 = flip ? -r.h[1][c] : r.h[1][c];
      acc.s[0][c] = acc.s[0][c] + r0;
      acc.s[1][c] = acc.s[1][c] + r1;
      acc.s[2][c] = acc.s[2][c] + unit_phase(low ? r1 : r0, isI, n2);
      acc.s[3][c] = acc.s[3][c] + unit_phase(low ? r0 : r1, isI, n3);
    }
  }
  const T cf = (T)a.coef;
  if (EPI == EPI_PLAIN) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc.s[s][c] = cf * acc.s[s][c];
    return acc;
  }
  // clover: out = cf C acc (EPI_CLOV) or C x + cf acc (EPI_XPAY), one 6x6 block at a time
  Spinor<T> src;
  if (EPI == EPI_XPAY)
    load_spinor<CG>(src, a.x, cb, Vh);
  else
    src = acc;
  Spinor<T> out;
#pragma unroll 1
  for (int blk = 0; blk < 2; ++blk) {
    HermBlock<T> B;
    load_clover_block(B, a.clov, blk, cb, Vh);
    cplx<T> v[6], y[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = blk ? src.s[2 + k / 3][k % 3] : src.s[k / 3][k % 3];
    herm_apply(B, v, y);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int s = k / 3, c = k % 3;
      if (EPI == EPI_CLOV) {
        y[k] = cf * y[k];
      } else {
        y[k] = y[k] + cf * (blk ? acc.s[2 + s][c] : acc.s[s][c]);
      }
      if (blk)
        out.s[2 + s][c] = y[k];
      else
        out.s[s][c] = y[k];
    }
  }
  return out;
}

// ---------------------------------------------------------------- split-site kernel
// NS threads per output site: thread t takes the hop terms t, t + NS, ... (term =
// 2 mu + {0 forward, 1 backward}), the partial spinors are summed by a butterfly of
// warp shuffles, and the first thread of the site applies the epilogue.  Measured on
// GB300 this is slower than one thread per site at every lattice size from 8^3x16 to
// 32^3x64, in FP32, FP64 and double-float; it is kept as an option (pfmp_op_set_split)
// with parity tests, and the default is one thread per site.
template <int PREC, int MU, int FWD, int SF>
__device__ __forceinline__ void hop_term(Spinor<typename Prec<PREC>::real>& acc, const HopParams<PREC>& a,
                                         const int x[4], int cb) {
  using T = typename Prec<PREC>::real;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int n = nbr_cb(g, x, MU, FWD ? +1 : -1);
  Spinor<T> psi;
  load_spinor(psi, a.in, n, Vh);
  Mat3<T> U;
  if (FWD) {
    Half<T> h = project<MU, SF>(psi);
    load_link(U, link_plane<PREC>(a.gauge, a.p * 4 + MU, Vh), cb, Vh);
    Half<T> r = mul_half(U, h);
    if (MU == 3 && x[3] == g.L[3] - 1) scale_half(r, (T)g.bc_t);
    accumulate<MU, SF>(acc, r);
  } else {
    Half<T> h = project<MU, -SF>(psi);
    load_link(U, link_plane<PREC>(a.gauge, (1 - a.p) * 4 + MU, Vh), n, Vh);
    Half<T> r = mul_half_dag(U, h);
    if (MU == 3 && x[3] == 0) scale_half(r, (T)g.bc_t);
    accumulate<MU, -SF>(acc, r);
  }
}

template <int PREC, int SF>
__device__ __forceinline__ void hop_term_rt(int term, Spinor<typename Prec<PREC>::real>& acc,
                                            const HopParams<PREC>& a, const int x[4], int cb) {
  switch (term) {
    case 0: hop_term<PREC, 0, 1, SF>(acc, a, x, cb); break;
    case 1: hop_term<PREC, 0, 0, SF>(acc, a, x, cb); break;
    case 2: hop_term<PREC, 1, 1, SF>(acc, a, x, cb); break;
    case 3: hop_term<PREC, 1, 0, SF>(acc, a, x, cb); break;
    case 4: hop_term<PREC, 2, 1, SF>(acc, a, x, cb); break;
    case 5: hop_term<PREC, 2, 0, SF>(acc, a, x, cb); break;
    case 6: hop_term<PREC, 3, 1, SF>(acc, a, x, cb); break;
    default: hop_term<PREC, 3, 0, SF>(acc, a, x, cb); break;
  }
}

__device__ __forceinline__ float shfl_x(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_x(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <typename T>
__device__ __forceinline__ T shfl_x(T v, int m) {  // double-float and other pair types
  return T(shfl_x(v.hi, m), shfl_x(v.lo, m));
}

template <int PREC, bool DAG, int EPI, bool REDUCE, int NS>
__global__ void __launch_bounds__(128) k_hop_split(HopParams<PREC> a) {
  using T = typename Prec<PREC>::real;
  if (a.scal && a.scal->done) return;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int t = (int)(tid % NS);
  const int cb0 = (int)(tid / NS);
  const bool live = cb0 < a.g.Vh;
  const int cb = live ? cb0 : a.g.Vh - 1;  // idle lanes still join the shuffles
  int x[4];
  cb_coords(a.g, cb, a.p, x);
  Spinor<T> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.s[s][c] = mk<T>(0, 0);
  constexpr int SF = DAG ? +1 : -1;
#pragma unroll
  for (int k = 0; k < 8 / NS; ++k) hop_term_rt<PREC, SF>(t + k * NS, acc, a, x, cb);
#pragma unroll
  for (int m = 1; m < NS; m <<= 1)
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc.s[s][c].re = acc.s[s][c].re + shfl_x(acc.s[s][c].re, m);
        acc.s[s][c].im = acc.s[s][c].im + shfl_x(acc.s[s][c].im, m);
      }
  // the first thread of the site applies the epilogue to the summed hop, as in k_hop
  const T cf = (T)a.coef;
  double nrm[1] = {0.0};
  if (t == 0 && live) {
    Spinor<T> out;
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
    store_spinor(a.out, out, cb, a.g.Vh);
    if (REDUCE) {
      double tt = 0;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) tt += (double)norm2(out.s[s][c]);
      nrm[0] = tt;
    }
  }
  if (REDUCE) {
    double tot[1];
    if (grid_sum<1>(nrm, a.rb, tot)) {
      *a.norm_out = tot[0];
      if (a.scal) a.scal->alpha = a.scal->rr / tot[0];
    }
  }
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
