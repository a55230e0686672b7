// Load/store of spinors, links and clover blocks in the device layouts (see
// pfmp_internal.cuh), templated on the storage precision.
#pragma once
#include <cuda_fp16.h>

#include "pfmp_internal.cuh"

namespace pfmp {

template <int PREC>
struct Prec;
template <>
struct Prec<PFMP_F64> {
  using real = double;
  using vec = double2;
  static constexpr int spinor_vecs = 12;
  static constexpr int link_vecs = 9;  // 18 reals (the master field)
  static constexpr int clover_vecs = 36;
};
template <>
struct Prec<PFMP_F32> {
  using real = float;
  using vec = float4;
  static constexpr int spinor_vecs = 6;
  static constexpr int link_vecs = 3;
  static constexpr int clover_vecs = 18;
};

template <>
struct Prec<PFMP_H16> {  // FP16 storage, FP32 arithmetic
  using real = float;
  using vec = uint4;  // four complex FP16
  static constexpr int spinor_vecs = 3;  // followed by one FP32 scale per site
  static constexpr int link_vecs = 0;    // 24 bytes per link: see link_plane
  static constexpr int clover_vecs = 9;
};

__device__ __forceinline__ float2 h2_to_f2(uint32_t u) {
  __half2 h;
  memcpy(&h, &u, 4);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2_to_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// ---------------------------------------------------------------- spinors
// A field read with CG = true goes through L2 only (ld.global.cg): a persistent kernel
// reads fields that other blocks rewrote earlier in the same launch, and L1 is not
// coherent across SMs.  The default is the read-only path (ld.global.nc).
template <bool CG, typename V>
__device__ __forceinline__ V ldf(const V* p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return __ldg(p);
}

template <bool CG = false>
__device__ __forceinline__ void load_spinor(Spinor<double>& s, const double2* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 v = ldf<CG>(f + (size_t)k * Vh + cb);
    s.s[k / 3][k % 3] = mk(v.x, v.y);
  }
}
__device__ __forceinline__ void store_spinor(double2* __restrict__ f, const Spinor<double>& s, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 12; ++k) f[(size_t)k * Vh + cb] = make_double2(s.s[k / 3][k % 3].re, s.s[k / 3][k % 3].im);
}
template <bool CG = false>
__device__ __forceinline__ void load_spinor(Spinor<float>& s, const float4* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float4 v = ldf<CG>(f + (size_t)k * Vh + cb);
    s.s[(2 * k) / 3][(2 * k) % 3] = mk(v.x, v.y);
    s.s[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(v.z, v.w);
  }
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ f, const Spinor<float>& s, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    cplx<float> a = s.s[(2 * k) / 3][(2 * k) % 3], b = s.s[(2 * k + 1) / 3][(2 * k + 1) % 3];
    f[(size_t)k * Vh + cb] = make_float4(a.re, a.im, b.re, b.im);
  }
}

// FP16: [3][Vh] uint4 (complex 4k .. 4k+3 in word k) then FP32 scale[Vh]; value = scale * h
template <bool CG = false>
__device__ __forceinline__ void load_spinor(Spinor<float>& s, const uint4* __restrict__ f, int cb, int Vh) {
  const float sc = __ldg(reinterpret_cast<const float*>(f + (size_t)3 * Vh) + cb);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 v = __ldg(f + (size_t)k * Vh + cb);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 a = h2_to_f2(w[j]);
      s.s[(4 * k + j) / 3][(4 * k + j) % 3] = mk(sc * a.x, sc * a.y);
    }
  }
}
__device__ __forceinline__ void store_spinor(uint4* __restrict__ f, const Spinor<float>& s, int cb, int Vh) {
  float m = 0.f;
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) m = fmaxf(m, fmaxf(fabsf(s.s[sp][c].re), fabsf(s.s[sp][c].im)));
  const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const cplx<float> a = s.s[(4 * k + j) / 3][(4 * k + j) % 3];
      w[j] = f2_to_h2(inv * a.re, inv * a.im);
    }
    f[(size_t)k * Vh + cb] = make_uint4(w[0], w[1], w[2], w[3]);
  }
  reinterpret_cast<float*>(f + (size_t)3 * Vh)[cb] = m;
}

// ---------------------------------------------------------------- links
// link field of one (parity, mu): base pointer at [parity][mu], vectors strided by Vh.
// FP64: the full 18-real link of the master field (the FP64 stencil is bound by the FP64
// pipe, not by bytes, so it reads the third row instead of rebuilding it); FP32 and FP16:
// 12 reals, the third row rebuilt as conj(row0 x row1)
__device__ __forceinline__ void load_link(Mat3<double>& U, const double2* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = __ldg(f + (size_t)k * Vh + cb);
    U.m[k / 3][k % 3] = mk(v.x, v.y);
  }
}
__device__ __forceinline__ void load_link(Mat3<float>& U, const float4* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float4 v = __ldg(f + (size_t)k * Vh + cb);
    U.m[(2 * k) / 3][(2 * k) % 3] = mk(v.x, v.y);
    U.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(v.z, v.w);
  }
  reconstruct_row2(U);
}

// FP16 12-real link: per (parity, mu) a plane of Vh uint4 (complex 0..3) followed by a
// plane of Vh uint2 (complex 4 and 5), 24 bytes per link; planes start at multiples of
// 1.5 Vh uint4 (Vh is a multiple of 8, so every plane is 16-byte aligned)
__device__ __forceinline__ void load_link(Mat3<float>& U, const uint4* __restrict__ f, int cb, int Vh) {
  const uint4 v0 = __ldg(f + cb);
  const uint2 v1 = __ldg(reinterpret_cast<const uint2*>(f + Vh) + cb);
  const uint32_t w[6] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y};
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float2 a = h2_to_f2(w[j]);
    U.m[j / 3][j % 3] = mk(a.x, a.y);
  }
  reconstruct_row2(U);
}

// start of the links of parity-direction index pm = 4 parity + mu
template <int PREC>
__host__ __device__ __forceinline__ const typename Prec<PREC>::vec* link_plane(const typename Prec<PREC>::vec* g,
                                                                               int pm, int Vh) {
  if constexpr (PREC == PFMP_H16)
    return g + (size_t)pm * 3 * (Vh / 2);
  else
    return g + (size_t)pm * Prec<PREC>::link_vecs * Vh;
}

// master gauge field: double2 [2][4][9][Vh], full 3x3
__device__ __forceinline__ void load_link18(Mat3<double>& U, const double2* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = f[(size_t)k * Vh + cb];
    U.m[k / 3][k % 3] = mk(v.x, v.y);
  }
}
__device__ __forceinline__ void store_link18(double2* __restrict__ f, const Mat3<double>& U, int cb, int Vh) {
#pragma unroll
  for (int k = 0; k < 9; ++k) f[(size_t)k * Vh + cb] = make_double2(U.m[k / 3][k % 3].re, U.m[k / 3][k % 3].im);
}

// ---------------------------------------------------------------- clover blocks
// one chiral block: 6 diagonal reals, 15 lower-triangle complex entries
template <typename T>
struct HermBlock {
  T d[6];
  cplx<T> o[15];  // (1,0),(2,0),(2,1),(3,0),(3,1),(3,2),(4,0),...,(5,4)
};
__host__ __device__ __forceinline__ int tri_index(int i, int j) { return i * (i - 1) / 2 + j; }  // i > j

// one Hermitian block (blk = 0: spins 0, 1; blk = 1: spins 2, 3)
__device__ __forceinline__ void load_clover_block(HermBlock<double>& b, const double2* __restrict__ f, int blk, int cb,
                                                  int Vh) {
  const double2* g = f + (size_t)(18 * blk) * Vh;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double2 v = __ldg(g + (size_t)k * Vh + cb);
    b.d[2 * k] = v.x;
    b.d[2 * k + 1] = v.y;
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    double2 v = __ldg(g + (size_t)(3 + k) * Vh + cb);
    b.o[k] = mk(v.x, v.y);
  }
}
__device__ __forceinline__ void load_clover(HermBlock<double> b[2], const double2* __restrict__ f, int cb, int Vh) {
  load_clover_block(b[0], f, 0, cb, Vh);
  load_clover_block(b[1], f, 1, cb, Vh);
}
__device__ __forceinline__ void store_clover(double2* __restrict__ f, const HermBlock<double> b[2], int cb, int Vh) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    double2* g = f + (size_t)(18 * blk) * Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) g[(size_t)k * Vh + cb] = make_double2(b[blk].d[2 * k], b[blk].d[2 * k + 1]);
#pragma unroll
    for (int k = 0; k < 15; ++k) g[(size_t)(3 + k) * Vh + cb] = make_double2(b[blk].o[k].re, b[blk].o[k].im);
  }
}
__device__ __forceinline__ void load_clover(HermBlock<float> b[2], const float4* __restrict__ f, int cb, int Vh) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    const float4* g = f + (size_t)(9 * blk) * Vh;
    float4 v0 = __ldg(g + cb), v1 = __ldg(g + (size_t)Vh + cb);
    b[blk].d[0] = v0.x;
    b[blk].d[1] = v0.y;
    b[blk].d[2] = v0.z;
    b[blk].d[3] = v0.w;
    b[blk].d[4] = v1.x;
    b[blk].d[5] = v1.y;
    b[blk].o[0] = mk(v1.z, v1.w);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      float4 v = __ldg(g + (size_t)(2 + k) * Vh + cb);
      b[blk].o[1 + 2 * k] = mk(v.x, v.y);
      b[blk].o[2 + 2 * k] = mk(v.z, v.w);
    }
  }
}

// FP16 clover: [9][Vh] uint4, word j = reals 8j .. 8j+7 of the 72-real sequence of the
// FP32 layout (per block: 6 diagonal reals, then the 15 lower-triangle complex entries)
__device__ __forceinline__ void load_clover(HermBlock<float> b[2], const uint4* __restrict__ f, int cb, int Vh) {
  float r[72];
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const uint4 v = __ldg(f + (size_t)j * Vh + cb);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 a = h2_to_f2(w[q]);
      r[8 * j + 2 * q] = a.x;
      r[8 * j + 2 * q + 1] = a.y;
    }
  }
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
#pragma unroll
    for (int i = 0; i < 6; ++i) b[blk].d[i] = r[36 * blk + i];
#pragma unroll
    for (int k = 0; k < 15; ++k) b[blk].o[k] = mk(r[36 * blk + 6 + 2 * k], r[36 * blk + 7 + 2 * k]);
  }
}

// y = B x for one Hermitian 6x6 block (x, y indexed 3*(spin - 2*blk) + colour)
template <typename T>
__device__ __forceinline__ void herm_apply(const HermBlock<T>& B, const cplx<T> x[6], cplx<T> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = B.d[i] * x[i];
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      cplx<T> a = B.o[tri_index(i, j)];
      y[i] = y[i] + a * x[j];
      y[j] = y[j] + cj_mul(a, x[i]);
    }
}

template <typename T>
__device__ __forceinline__ Spinor<T> clover_apply(const HermBlock<T> B[2], const Spinor<T>& in) {
  Spinor<T> out;
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    cplx<T> x[6], y[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) x[k] = in.s[2 * blk + k / 3][k % 3];
    herm_apply(B[blk], x, y);
#pragma unroll
    for (int k = 0; k < 6; ++k) out.s[2 * blk + k / 3][k % 3] = y[k];
  }
  return out;
}

// complex entries per storage chunk: 2 for FP32 (float4), 1 for FP64 and double-float
template <int PREC>
struct ChunkInfo {
  static constexpr int per = PREC == PFMP_F32 ? 2 : 1;
  static constexpr int n = 12 / per;
};

template <int PREC>
__device__ __forceinline__ void store_chunk(typename Prec<PREC>::vec* f, int k, int cb, int Vh,
                                            const cplx<typename Prec<PREC>::real>* v);
template <>
__device__ __forceinline__ void store_chunk<PFMP_F32>(float4* f, int k, int cb, int Vh, const cplx<float>* v) {
  f[(size_t)k * Vh + cb] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
}
template <>
__device__ __forceinline__ void store_chunk<PFMP_F64>(double2* f, int k, int cb, int Vh, const cplx<double>* v) {
  f[(size_t)k * Vh + cb] = make_double2(v[0].re, v[0].im);
}

}  // namespace pfmp
