// Double-float ("df") arithmetic: a value is hi + lo with two FP32 numbers, |lo| <=
// ulp(hi)/2, about 48 significant bits.  GB300's FP64 pipe is a small fraction of its
// FP32 pipe, so the FP64-accurate true residual of the mixed solvers runs the stencil in
// df on the FP32 pipe instead of in FP64.
//
// Published error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2):  s = a + b, e = (a - (s - (s - a))) + (b - (s - a))
//   FastTwoSum (Dekker 1971, |a| >= |b|):  s = a + b, e = b - (s - a)
//   TwoProd with a fused multiply-add:  p = a b, e = fma(a, b, -p)
// Addition is the "sloppy" df add (TwoSum of the high parts, low parts added, one
// renormalisation): its error is bounded by a few df ulps of |x| + |y|, which is what a
// stencil sum of many terms needs.  Multiplication is TwoProd of the high parts plus the
// cross terms, renormalised.
#pragma once
#include "fields.cuh"

namespace pfmp {

struct df {
  float hi, lo;
  __host__ __device__ df() : hi(0.f), lo(0.f) {}
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df(int v) : hi((float)v), lo(0.f) {}
  // exact split of a double into two floats (the low part rounds the remainder)
  __host__ __device__ explicit df(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df(s, e);
}
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
__device__ __forceinline__ df operator+(df x, df y) {
  df s = df_two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}

template <>
struct Prec<2> {  // double-float, used only inside the library (the true residual)
  using real = df;
  using vec = float4;                  // one complex df: (re.hi, re.lo, im.hi, im.lo)
  static constexpr int spinor_vecs = 12;
  static constexpr int link_vecs = 9;  // full 3x3, no reconstruction
  static constexpr int clover_vecs = 36;
};
constexpr int PREC_DF = 2;

__device__ __forceinline__ cplx<df> c_of(float4 v) { return mk(df(v.x, v.y), df(v.z, v.w)); }
__device__ __forceinline__ float4 v_of(cplx<df> c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }

template <bool CG = false>
__device__ __forceinline__ void load_spinor(Spinor<df>& s, const float4* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 12; ++k) s.s[k / 3][k % 3] = c_of(ldf<CG>(f + (size_t)k * Vh + cb));
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ f, const Spinor<df>& s, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 12; ++k) f[(size_t)k * Vh + cb] = v_of(s.s[k / 3][k % 3]);
}
__device__ __forceinline__ void load_link(Mat3<df>& U, const float4* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 9; ++k) U.m[k / 3][k % 3] = c_of(__ldg(f + (size_t)k * Vh + cb));
}
// clover blocks in the FP64 layout, each double2 (a, b) stored as float4 (a.hi, a.lo, b.hi, b.lo)
__device__ __forceinline__ void load_clover_block(HermBlock<df>& b, const float4* __restrict__ f, int blk, int cb, int Vh) {
  const float4* g = f + (size_t)(18 * blk) * Vh;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float4 v = __ldg(g + (size_t)k * Vh + cb);
    b.d[2 * k] = df(v.x, v.y);
    b.d[2 * k + 1] = df(v.z, v.w);
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) b.o[k] = c_of(__ldg(g + (size_t)(3 + k) * Vh + cb));
}
__device__ __forceinline__ void load_clover(HermBlock<df> b[2], const float4* __restrict__ f, int cb, int Vh) {
  load_clover_block(b[0], f, 0, cb, Vh);
  load_clover_block(b[1], f, 1, cb, Vh);
}

template <>
__device__ __forceinline__ void store_chunk<2>(float4* f, int k, int cb, int Vh, const cplx<df>* v) {
  f[(size_t)k * Vh + cb] = v_of(v[0]);
}

__device__ __forceinline__ float4 split2(double2 v) {
  const float a = (float)v.x, b = (float)v.y;
  return make_float4(a, (float)(v.x - (double)a), b, (float)(v.y - (double)b));
}

}  // namespace pfmp
