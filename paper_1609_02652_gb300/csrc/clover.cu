// Clover term: field strength from the four plaquette leaves, the two chiral 6x6
// blocks of A = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}, and on odd sites
// A^{-1} with log det A by Cholesky.  FP64 throughout; the FP32 copy is rounded last.
// F_{mu nu} depends on the gauge field only: it is computed once per gauge-field version
// (one thread per site and plane) and shared by every operator (kappa) of the context.
//
// In the chiral gamma basis sigma_{mu nu} = diag(s+, s-) with 2x2 Pauli blocks, so
//   sum_{mu<nu} sigma F = sum_k s_k (x) X_k,
//   upper (spins 0,1): X1 = F12 - F03, X2 = F02 + F13, X3 = F01 - F23,
//   lower (spins 2,3): X1 = F12 + F03, X2 = F02 - F13, X3 = F01 + F23,
// and each block is 1 - kappa c_sw [[X3, X1 - i X2], [X1 + i X2, -X3]].
#include <cstring>

#include "context.h"
#include "dfloat.cuh"
#include "fields.cuh"

namespace pfmp {

__device__ __forceinline__ Mat3<double> mlink(const double2* U, const Geom& g, const int x[4], int mu) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  Mat3<double> M;
  load_link18(M, U + (size_t)((p * 4 + mu) * 9) * g.Vh, cb_index(g, x), g.Vh);
  return M;
}
__device__ __forceinline__ void shift(const Geom& g, const int x[4], int mu, int d, int y[4]) {
  for (int k = 0; k < 4; ++k) y[k] = x[k];
  y[mu] = (y[mu] + d + g.L[mu]) % g.L[mu];
}

// the link U_mu(x): FP64 from the master field, FP32 from the 12-real compressed copy
template <typename T>
__device__ __forceinline__ Mat3<T> clink(const void* U, const Geom& g, const int x[4], int mu);
template <>
__device__ __forceinline__ Mat3<double> clink<double>(const void* U, const Geom& g, const int x[4], int mu) {
  return mlink((const double2*)U, g, x, mu);
}
template <>
__device__ __forceinline__ Mat3<float> clink<float>(const void* U, const Geom& g, const int x[4], int mu) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  Mat3<float> M;
  load_link(M, link_plane<PFMP_F32>((const float4*)U, p * 4 + mu, g.Vh), cb_index(g, x), g.Vh);
  return M;
}

// F_{mu nu}(x): traceless part of (Q - Q^dag)/(8i), Q = sum of the four leaves at x
template <typename T>
__device__ Mat3<T> field_strength(const void* U, const Geom& g, const int x[4], int mu, int nu) {
  int xpm[4], xpn[4], xmm[4], xmn[4], xmmpn[4], xmmmn[4], xpmmn[4];
  shift(g, x, mu, 1, xpm);
  shift(g, x, nu, 1, xpn);
  shift(g, x, mu, -1, xmm);
  shift(g, x, nu, -1, xmn);
  shift(g, xmm, nu, 1, xmmpn);
  shift(g, xmm, nu, -1, xmmmn);
  shift(g, xpm, nu, -1, xpmmn);
  const Mat3<T> Um = clink<T>(U, g, x, mu), Un = clink<T>(U, g, x, nu);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  Mat3<T> Q = matmul_nd(matmul_nd(matmul(Um, clink<T>(U, g, xpm, nu)), clink<T>(U, g, xpn, mu)), Un);
  // leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  const Mat3<T> Um_xmm = clink<T>(U, g, xmm, mu);
  Mat3<T> L = matmul(matmul_nd(matmul_nd(Un, clink<T>(U, g, xmmpn, mu)), clink<T>(U, g, xmm, nu)), Um_xmm);
  Q = mat_add(Q, L);
  // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  {
    Mat3<T> A = dagger(Um_xmm);
    A = matmul_nd(A, clink<T>(U, g, xmmmn, nu));
    A = matmul(A, clink<T>(U, g, xmmmn, mu));
    A = matmul(A, clink<T>(U, g, xmn, nu));
    L = A;
  }
  Q = mat_add(Q, L);
  // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
  {
    Mat3<T> A = dagger(clink<T>(U, g, xmn, nu));
    A = matmul(A, clink<T>(U, g, xmn, mu));
    A = matmul(A, clink<T>(U, g, xpmmn, nu));
    A = matmul_nd(A, Um);
    L = A;
  }
  Q = mat_add(Q, L);
  Mat3<T> F;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx<T> d = Q.m[i][j] - conj(Q.m[j][i]);
      F.m[i][j] = (T)0.125 * times_mi(d);
    }
  const T tr = (F.m[0][0].re + F.m[1][1].re + F.m[2][2].re) / (T)3;
  for (int i = 0; i < 3; ++i) {
    F.m[i][i].re -= tr;
    F.m[i][i].im = 0;
  }
  return F;
}

struct CloverOut {
  double2* A64;   // even: A
  double2* Ai64;  // odd: A^{-1}
  float4* A32;
  float4* Ai32;
  float4* Adf;    // double-float copies of A64 / Ai64
  float4* Aidf;
  int* bad;
};

template <typename T>
__device__ __forceinline__ void store_block32(float4* f, const HermBlock<T>& b, int blk, int cb, int Vh) {
  float4* g = f + (size_t)(9 * blk) * Vh;
  g[cb] = make_float4((float)b.d[0], (float)b.d[1], (float)b.d[2], (float)b.d[3]);
  g[(size_t)Vh + cb] = make_float4((float)b.d[4], (float)b.d[5], (float)b.o[0].re, (float)b.o[0].im);
#pragma unroll
  for (int k = 0; k < 7; ++k)
    g[(size_t)(2 + k) * Vh + cb] =
        make_float4((float)b.o[1 + 2 * k].re, (float)b.o[1 + 2 * k].im, (float)b.o[2 + 2 * k].re, (float)b.o[2 + 2 * k].im);
}

// F_{mu nu} of every site and plane, one thread per (site, plane): the Hermitian matrix as
// its three diagonal reals and the upper triangle (0,1), (0,2), (1,2), 9 reals per plane,
// [2 parity][6 plane][9][Vh]
template <typename T>
__global__ void k_field_strength(Geom g, const void* __restrict__ U, double* __restrict__ Fout) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y / 6, pl = blockIdx.y % 6;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, p, x);
  const int mu = pl < 3 ? 0 : (pl < 5 ? 1 : 2);
  const int nu = pl < 3 ? pl + 1 : (pl < 5 ? pl - 1 : 3);
  const Mat3<T> F = field_strength<T>(U, g, x, mu, nu);
  double* o = Fout + (size_t)((p * 6 + pl) * 9) * g.Vh + cb;
  o[0] = F.m[0][0].re;
  o[(size_t)g.Vh] = F.m[1][1].re;
  o[2 * (size_t)g.Vh] = F.m[2][2].re;
  o[3 * (size_t)g.Vh] = F.m[0][1].re;
  o[4 * (size_t)g.Vh] = F.m[0][1].im;
  o[5 * (size_t)g.Vh] = F.m[0][2].re;
  o[6 * (size_t)g.Vh] = F.m[0][2].im;
  o[7 * (size_t)g.Vh] = F.m[1][2].re;
  o[8 * (size_t)g.Vh] = F.m[1][2].im;
}

template <typename T>
__device__ __forceinline__ Mat3<T> load_fmunu(const double* __restrict__ Fin, const Geom& g, int p, int pl, int cb) {
  const double* f = Fin + (size_t)((p * 6 + pl) * 9) * g.Vh + cb;
  T v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = (T)__ldg(f + (size_t)k * g.Vh);
  Mat3<T> F;
  F.m[0][0] = mk(v[0], T(0));
  F.m[1][1] = mk(v[1], T(0));
  F.m[2][2] = mk(v[2], T(0));
  F.m[0][1] = mk(v[3], v[4]);
  F.m[1][0] = mk(v[3], -v[4]);
  F.m[0][2] = mk(v[5], v[6]);
  F.m[2][0] = mk(v[5], -v[6]);
  F.m[1][2] = mk(v[7], v[8]);
  F.m[2][1] = mk(v[7], -v[8]);
  return F;
}

template <typename T>
__device__ __forceinline__ void store_block64(double2* f, const HermBlock<T>& b, int blk, int cb, int Vh) {
  double2* g = f + (size_t)(18 * blk) * Vh;
#pragma unroll
  for (int k = 0; k < 3; ++k) g[(size_t)k * Vh + cb] = make_double2(b.d[2 * k], b.d[2 * k + 1]);
#pragma unroll
  for (int k = 0; k < 15; ++k) g[(size_t)(3 + k) * Vh + cb] = make_double2(b.o[k].re, b.o[k].im);
}
template <typename T>
__device__ __forceinline__ void store_block_df(float4* f, const HermBlock<T>& b, int blk, int cb, int Vh) {
  float4* g = f + (size_t)(18 * blk) * Vh;
#pragma unroll
  for (int k = 0; k < 3; ++k) g[(size_t)k * Vh + cb] = split2(make_double2(b.d[2 * k], b.d[2 * k + 1]));
#pragma unroll
  for (int k = 0; k < 15; ++k) g[(size_t)(3 + k) * Vh + cb] = split2(make_double2(b.o[k].re, b.o[k].im));
}

// In place on a packed Hermitian block: the Cholesky factor L (A = L L^dag, lower
// triangle, real diagonal), then L^{-1} (lower triangular), then A^{-1} = L^{-dag} L^{-1}.
// Every loop runs over the full 0..5 range with the triangle selected by a condition, so
// that after unrolling every index is a constant and the block stays in registers.
// Returns false (and the identity) if A is not positive definite; logdet = log det A.
template <typename T>
__device__ __forceinline__ bool invert_block(HermBlock<T>& B, double& logdet) {
  bool ok = true;
  logdet = 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    T d = B.d[j];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < j) d -= norm2(B.o[tri_index(j, k)]);
    if (!(d > T(0))) {
      ok = false;
      d = T(1);
    }
    const T ljj = sqrt(d);
    B.d[j] = ljj;
    logdet += 2.0 * (double)log(ljj);
    const T r = T(1) / ljj;
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i > j) {
        cplx<T> s = B.o[tri_index(i, j)];
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (k < j) s = s - mul_cj(B.o[tri_index(i, k)], B.o[tri_index(j, k)]);
        B.o[tri_index(i, j)] = r * s;
      }
  }
  if (!ok) {
#pragma unroll
    for (int i = 0; i < 6; ++i) B.d[i] = T(1);
#pragma unroll
    for (int k = 0; k < 15; ++k) B.o[k] = mk(T(0), T(0));
    logdet = 0.0;
    return false;
  }
  // L^{-1}: diagonal 1 / L_ii; column by column, (L^{-1})_ij = -(1 / L_ii) sum_{j<=k<i} L_ik (L^{-1})_kj.
  // Row i of column j reads L_ik for k >= j (not yet overwritten) and (L^{-1})_kj for k < i.
#pragma unroll
  for (int i = 0; i < 6; ++i) B.d[i] = T(1) / B.d[i];
#pragma unroll
  for (int j = 0; j < 6; ++j)
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i > j) {
        cplx<T> s = B.d[j] * B.o[tri_index(i, j)];
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (k > j && k < i) s = s + B.o[tri_index(i, k)] * B.o[tri_index(k, j)];
        B.o[tri_index(i, j)] = (-B.d[i]) * s;
      }
  // A^{-1}_ij = sum_{k >= max(i, j)} conj(Li_ki) Li_kj (lower triangle, i >= j)
  HermBlock<T> R;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j <= i) {
        cplx<T> s = i == j ? mk(B.d[i] * B.d[i], T(0)) : B.d[i] * B.o[tri_index(i, j)];
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (k > i) s = s + cj_mul(B.o[tri_index(k, i)], B.o[tri_index(k, j)]);
        if (i == j)
          R.d[i] = s.re;
        else
          R.o[tri_index(i, j)] = s;
      }
  B = R;
  return true;
}

// One thread per (site, chiral block): lanes 2n and 2n + 1 take the two blocks of a site.
// Block blk (spins 2 blk, 2 blk + 1) of A = 1 - kappa c_sw sigma.F / 2 from the six planes
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): with s = -1 (blk 0) or +1 (blk 1),
// X1 = F_12 + s F_03, X2 = F_02 - s F_13, X3 = F_01 + s F_23 and
// A = [[1 - kc X3, -kc (X1 - i X2)], [-kc (X1 + i X2), 1 + kc X3]].
// Even sites store A_ee, odd sites A_oo^{-1} and their log det (grid-stride, so the grid
// and the reduction's block count stay bounded at any volume).  T is the arithmetic:
// double, or float for the clover terms built from an FP32 field strength inside an MD
// with FP32 forces (FP32 is all the accuracy such a field strength carries).
template <typename T>
__global__ void __launch_bounds__(128, 3) k_clover_build(Geom g, const double* __restrict__ Fin, double kc_d,
                                                         CloverOut out, ReduceBuf rb, double* logdet_out) {
  const T kc = (T)kc_d;
  const int p = blockIdx.y;
  double ld[1] = {0.0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < 2L * g.Vh; t += (long)gridDim.x * blockDim.x) {
    const int cb = (int)(t >> 1), blk = (int)(t & 1);
    const T s = blk == 0 ? T(-1) : T(1);
    Mat3<T> X1, X2, X3;
    {
      const Mat3<T> F01 = load_fmunu<T>(Fin, g, p, 0, cb), F23 = load_fmunu<T>(Fin, g, p, 5, cb);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X3.m[i][j] = F01.m[i][j] + s * F23.m[i][j];
    }
    {
      const Mat3<T> F12 = load_fmunu<T>(Fin, g, p, 3, cb), F03 = load_fmunu<T>(Fin, g, p, 2, cb);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X1.m[i][j] = F12.m[i][j] + s * F03.m[i][j];
    }
    {
      const Mat3<T> F02 = load_fmunu<T>(Fin, g, p, 1, cb), F13 = load_fmunu<T>(Fin, g, p, 4, cb);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X2.m[i][j] = F02.m[i][j] - s * F13.m[i][j];
    }
    HermBlock<T> B;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      B.d[i] = T(1) - kc * X3.m[i][i].re;
      B.d[i + 3] = T(1) + kc * X3.m[i][i].re;
#pragma unroll
      for (int j = 0; j < i; ++j) {
        B.o[tri_index(i, j)] = -kc * X3.m[i][j];
        B.o[tri_index(i + 3, j + 3)] = kc * X3.m[i][j];
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) B.o[tri_index(i + 3, j)] = -kc * (X1.m[i][j] + times_i(X2.m[i][j]));
    }
    if (p == 0) {
      store_block64(out.A64, B, blk, cb, g.Vh);
      store_block_df(out.Adf, B, blk, cb, g.Vh);
      store_block32(out.A32, B, blk, cb, g.Vh);
    } else {
      double l;
      if (!invert_block(B, l)) atomicExch(out.bad, 1);
      ld[0] += l;
      store_block64(out.Ai64, B, blk, cb, g.Vh);
      store_block_df(out.Aidf, B, blk, cb, g.Vh);
      store_block32(out.Ai32, B, blk, cb, g.Vh);
    }
  }
  double tot[1];
  if (grid_sum<1>(ld, rb, tot)) *logdet_out = tot[0];
}

// FP16 copy of the FP32 clover blocks: word j of the FP16 layout holds FP32 words 2j
// and 2j + 1 (8 reals)
__global__ void k_clover_h16(const float4* __restrict__ src, uint4* __restrict__ dst, int Vh) {
  const long n = 9L * Vh;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long j = i / Vh, cb = i - j * Vh;
    const float4 a = src[(size_t)(2 * j) * Vh + cb], b = src[(size_t)(2 * j + 1) * Vh + cb];
    dst[i] = make_uint4(f2_to_h2(a.x, a.y), f2_to_h2(a.z, a.w), f2_to_h2(b.x, b.y), f2_to_h2(b.z, b.w));
  }
}

// prec = PFMP_F64: from the FP64 master links; PFMP_F32: FP32 arithmetic on the
// compressed links (the clover terms an MD with FP32 forces uses between the trajectory
// ends).  An FP64 result also serves an FP32 request.
void field_strength_update(pfmp_ctx* c, int prec) {
  if (c->fmunu && c->fmunu_version == c->gauge_version && (c->fmunu_prec == PFMP_F64 || prec == PFMP_F32)) return;
  if (!c->fmunu) c->fmunu = (double*)dev_alloc((size_t)c->g.Vh * 2 * 6 * 9 * sizeof(double));
  dim3 grid(nblocks(c->g.Vh, 128), 12);
  if (prec == PFMP_F64)
    k_field_strength<double><<<grid, 128, 0, c->stream>>>(c->g, c->U64, c->fmunu);
  else
    k_field_strength<float><<<grid, 128, 0, c->stream>>>(c->g, c->U32, c->fmunu);
  PFMP_CHECK_LAUNCH();
  c->fmunu_version = c->gauge_version;
  c->fmunu_prec = prec;
}

void clover_build(pfmp_op* op, int fprec) {
  pfmp_ctx* c = op->ctx;
  field_strength_update(c, fprec);
  CloverOut o;
  o.A64 = op->clov64[0];
  o.Ai64 = op->clov64[1];
  o.A32 = op->clov32[0];
  o.Ai32 = op->clov32[1];
  o.Adf = op->clovdf[0];
  o.Aidf = op->clovdf[1];
  o.bad = (int*)(c->d_sums + 8);
  PFMP_CUDA(cudaMemsetAsync(o.bad, 0, sizeof(int), c->stream));
  dim3 grid(std::min(nblocks(2L * c->g.Vh, 128), 152 * 24), 2);
  if (fprec == PFMP_F64)
    k_clover_build<double><<<grid, 128, 0, c->stream>>>(c->g, c->fmunu, op->kappa * op->csw, o, c->rb, c->d_sums);
  else
    k_clover_build<float><<<grid, 128, 0, c->stream>>>(c->g, c->fmunu, op->kappa * op->csw, o, c->rb, c->d_sums);
  PFMP_CHECK_LAUNCH();
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  int bad;
  memcpy(&bad, c->h_sums + 8, sizeof(int));
  PFMP_REQUIRE(bad == 0, PFMP_E_NAN, "clover block not positive definite (A has a non-positive eigenvalue)");
  op->logdet_oo = c->h_sums[0];
  for (int p = 0; p < 2; ++p) {
    k_clover_h16<<<nblocks(9L * c->g.Vh), kBlock, 0, c->stream>>>(op->clov32[p], op->clov16[p], c->g.Vh);
    PFMP_CHECK_LAUNCH();
  }
  op->built_version = c->gauge_version;
  op->built_prec = fprec;
}

}  // namespace pfmp
