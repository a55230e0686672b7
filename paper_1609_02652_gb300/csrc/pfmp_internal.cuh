// Internal definitions of the PF-MP GB300 library: field layouts, complex arithmetic,
// lattice geometry and error plumbing.  Nothing here is part of the C-ABI.
//
// Device layouts (all parity-split, "chunk-major" so that consecutive threads read
// consecutive 16-byte words; Vh = V/2 sites per parity, cb = lexicographic index / 2):
//   spinor  F64: double2 [12][Vh]   (24 reals: (spin*3 + colour)*2 + re/im)
//           F32: float4  [6][Vh]
//   link    F64: double2 [2 parity][4 mu][9][Vh]   (18 reals, row-major 3x3)
//           F32: float4  [2][4][3][Vh]             (12 reals: rows 0 and 1; row 2
//                                                    rebuilt as conj(row0 x row1))
//   clover  F64: double2 [36][Vh] per parity, F32: float4 [18][Vh]  (two 6x6 Hermitian
//           chiral blocks, 36 reals each: 6 diagonal reals then the 15 lower-triangle
//           complex entries (1,0),(2,0),(2,1),(3,0),...,(5,4))
//   momentum / force: double [2][4][8][Vh] algebra coefficients p_a of P = sum p_a T_a
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>

#include "../../include/pfmp.h"

namespace pfmp {

// ------------------------------------------------------------------ error plumbing
struct Err {
  int code;
};
#define PFMP_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      pfmp::set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));      \
      throw pfmp::Err{PFMP_E_CUDA};                                                  \
    }                                                                                \
  } while (0)
#define PFMP_CHECK_LAUNCH()   \
  do {                        \
    pfmp::count_launch();     \
    PFMP_CUDA(cudaGetLastError()); \
  } while (0)
#define PFMP_REQUIRE(cond, code_, msg)                                               \
  do {                                                                               \
    if (!(cond)) {                                                                   \
      pfmp::set_last_error(msg);                                                     \
      throw pfmp::Err{code_};                                                        \
    }                                                                                \
  } while (0)

void set_last_error(const std::string& s);
void count_launch();
void count_launches(long long n);
long long launch_count();

// ------------------------------------------------------------------ complex
template <typename T>
struct cplx {
  T re, im;
};
template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T r, T i) {
  cplx<T> c;
  c.re = r;
  c.im = i;
  return c;
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a) { return mk(-a.re, -a.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.re, -a.im); }
// a * conj(b)
template <typename T>
__host__ __device__ __forceinline__ cplx<T> mul_cj(cplx<T> a, cplx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cplx<T> cj_mul(cplx<T> a, cplx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> times_i(cplx<T> a) { return mk(-a.im, a.re); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> times_mi(cplx<T> a) { return mk(a.im, -a.re); }
template <typename T>
__host__ __device__ __forceinline__ T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

template <typename T>
struct Spinor {
  cplx<T> s[4][3];
};
template <typename T>
struct Mat3 {
  cplx<T> m[3][3];
};
template <typename T>
struct Half {  // a spin-projected (two-component) spinor
  cplx<T> h[2][3];
};

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];     // x, y, z, t
  int Vh;       // sites per parity
  int V;
  double bc_t;  // fermion time boundary factor (+1 or -1)
};

// full coordinates of checkerboard site cb of parity p
__host__ __device__ __forceinline__ void cb_coords(const Geom& g, int cb, int p, int x[4]) {
  int r = cb * 2;
  int x0 = r % g.L[0];
  r /= g.L[0];
  x[1] = r % g.L[1];
  r /= g.L[1];
  x[2] = r % g.L[2];
  x[3] = r / g.L[2];
  x[0] = x0 + ((p + x[1] + x[2] + x[3]) & 1);
}
__host__ __device__ __forceinline__ int lex_index(const Geom& g, const int x[4]) {
  return x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
}
__host__ __device__ __forceinline__ int cb_index(const Geom& g, const int x[4]) { return lex_index(g, x) >> 1; }
// checkerboard index of x +- mu (the neighbour has the other parity)
__host__ __device__ __forceinline__ int nbr_cb(const Geom& g, const int x[4], int mu, int dir) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] += dir;
  if (y[mu] == g.L[mu]) y[mu] = 0;
  if (y[mu] < 0) y[mu] = g.L[mu] - 1;
  return cb_index(g, y);
}

// ------------------------------------------------------------------ SU(3)
template <typename T>
__host__ __device__ __forceinline__ void reconstruct_row2(Mat3<T>& U) {
  // row2 = conj(row0 x row1) for a special unitary matrix
  U.m[2][0] = conj(U.m[0][1] * U.m[1][2] - U.m[0][2] * U.m[1][1]);
  U.m[2][1] = conj(U.m[0][2] * U.m[1][0] - U.m[0][0] * U.m[1][2]);
  U.m[2][2] = conj(U.m[0][0] * U.m[1][1] - U.m[0][1] * U.m[1][0]);
}

template <typename T>
__host__ __device__ __forceinline__ Mat3<T> matmul(const Mat3<T>& A, const Mat3<T>& B) {
  Mat3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<T> s = A.m[i][0] * B.m[0][j];
      s = s + A.m[i][1] * B.m[1][j];
      s = s + A.m[i][2] * B.m[2][j];
      C.m[i][j] = s;
    }
  return C;
}
// A * B^dag
template <typename T>
__host__ __device__ __forceinline__ Mat3<T> matmul_nd(const Mat3<T>& A, const Mat3<T>& B) {
  Mat3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<T> s = mul_cj(A.m[i][0], B.m[j][0]);
      s = s + mul_cj(A.m[i][1], B.m[j][1]);
      s = s + mul_cj(A.m[i][2], B.m[j][2]);
      C.m[i][j] = s;
    }
  return C;
}
// A^dag * B
template <typename T>
__host__ __device__ __forceinline__ Mat3<T> matmul_dn(const Mat3<T>& A, const Mat3<T>& B) {
  Mat3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<T> s = cj_mul(A.m[0][i], B.m[0][j]);
      s = s + cj_mul(A.m[1][i], B.m[1][j]);
      s = s + cj_mul(A.m[2][i], B.m[2][j]);
      C.m[i][j] = s;
    }
  return C;
}
template <typename T>
__host__ __device__ __forceinline__ Mat3<T> dagger(const Mat3<T>& A) {
  Mat3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.m[i][j] = conj(A.m[j][i]);
  return C;
}
template <typename T>
__host__ __device__ __forceinline__ Mat3<T> mat_add(const Mat3<T>& A, const Mat3<T>& B) {
  Mat3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.m[i][j] = A.m[i][j] + B.m[i][j];
  return C;
}
template <typename T>
__host__ __device__ __forceinline__ Mat3<T> mat_zero() {
  Mat3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.m[i][j] = mk<T>(0, 0);
  return C;
}

// ------------------------------------------------------------------ launch helpers
constexpr int kBlock = 256;
inline int nblocks(long n, int block = kBlock) { return (int)((n + block - 1) / block); }

}  // namespace pfmp
