// Spin projection in the chiral gamma basis: the two independent components of
// (1 + S g_mu) psi and the rebuild of the four-component spinor from them, plus colour
// multiplication of half spinors.  Shared by the stencil and the force kernels.
#pragma once
#include "pfmp_internal.cuh"

namespace pfmp {

// half spinor of (1 + S g_MU) psi, and the rebuild of the full result from it
template <int MU, int S, typename T>
__device__ __forceinline__ Half<T> project(const Spinor<T>& p) {
  Half<T> h;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {
      h.h[0][c] = S > 0 ? p.s[0][c] + times_i(p.s[3][c]) : p.s[0][c] - times_i(p.s[3][c]);
      h.h[1][c] = S > 0 ? p.s[1][c] + times_i(p.s[2][c]) : p.s[1][c] - times_i(p.s[2][c]);
    } else if (MU == 1) {
      h.h[0][c] = S > 0 ? p.s[0][c] - p.s[3][c] : p.s[0][c] + p.s[3][c];
      h.h[1][c] = S > 0 ? p.s[1][c] + p.s[2][c] : p.s[1][c] - p.s[2][c];
    } else if (MU == 2) {
      h.h[0][c] = S > 0 ? p.s[0][c] + times_i(p.s[2][c]) : p.s[0][c] - times_i(p.s[2][c]);
      h.h[1][c] = S > 0 ? p.s[1][c] - times_i(p.s[3][c]) : p.s[1][c] + times_i(p.s[3][c]);
    } else {
      h.h[0][c] = S > 0 ? p.s[0][c] + p.s[2][c] : p.s[0][c] - p.s[2][c];
      h.h[1][c] = S > 0 ? p.s[1][c] + p.s[3][c] : p.s[1][c] - p.s[3][c];
    }
  }
  return h;
}

template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(Spinor<T>& a, const Half<T>& h) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.s[0][c] = a.s[0][c] + h.h[0][c];
    a.s[1][c] = a.s[1][c] + h.h[1][c];
    if (MU == 0) {  // r2 = -S i h1, r3 = -S i h0
      a.s[2][c] = S > 0 ? a.s[2][c] + times_mi(h.h[1][c]) : a.s[2][c] + times_i(h.h[1][c]);
      a.s[3][c] = S > 0 ? a.s[3][c] + times_mi(h.h[0][c]) : a.s[3][c] + times_i(h.h[0][c]);
    } else if (MU == 1) {  // r2 = S h1, r3 = -S h0
      a.s[2][c] = S > 0 ? a.s[2][c] + h.h[1][c] : a.s[2][c] - h.h[1][c];
      a.s[3][c] = S > 0 ? a.s[3][c] - h.h[0][c] : a.s[3][c] + h.h[0][c];
    } else if (MU == 2) {  // r2 = -S i h0, r3 = S i h1
      a.s[2][c] = S > 0 ? a.s[2][c] + times_mi(h.h[0][c]) : a.s[2][c] + times_i(h.h[0][c]);
      a.s[3][c] = S > 0 ? a.s[3][c] + times_i(h.h[1][c]) : a.s[3][c] + times_mi(h.h[1][c]);
    } else {  // r2 = S h0, r3 = S h1
      a.s[2][c] = S > 0 ? a.s[2][c] + h.h[0][c] : a.s[2][c] - h.h[0][c];
      a.s[3][c] = S > 0 ? a.s[3][c] + h.h[1][c] : a.s[3][c] - h.h[1][c];
    }
  }
}

template <typename T>
__device__ __forceinline__ Half<T> mul_half(const Mat3<T>& U, const Half<T>& h) {
  Half<T> r;
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) r.h[k][i] = U.m[i][0] * h.h[k][0] + U.m[i][1] * h.h[k][1] + U.m[i][2] * h.h[k][2];
  return r;
}
template <typename T>
__device__ __forceinline__ Half<T> mul_half_dag(const Mat3<T>& U, const Half<T>& h) {
  Half<T> r;
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      r.h[k][i] = cj_mul(U.m[0][i], h.h[k][0]) + cj_mul(U.m[1][i], h.h[k][1]) + cj_mul(U.m[2][i], h.h[k][2]);
  return r;
}
template <typename T>
__device__ __forceinline__ void scale_half(Half<T>& h, T s) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) h.h[k][i] = s * h.h[k][i];
}

}  // namespace pfmp
