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

__device__ void store_clover_df(float4* f, const HermBlock<double> b[2], int cb, int Vh) {
  for (int blk = 0; blk < 2; ++blk) {
    float4* g = f + (size_t)(18 * blk) * Vh;
    for (int k = 0; k < 3; ++k) g[(size_t)k * Vh + cb] = split2(make_double2(b[blk].d[2 * k], b[blk].d[2 * k + 1]));
    for (int k = 0; k < 15; ++k) g[(size_t)(3 + k) * Vh + cb] = split2(make_double2(b[blk].o[k].re, b[blk].o[k].im));
  }
}

__device__ void store_block32(float4* f, const HermBlock<double>& b, int blk, int cb, int Vh) {
  float4* g = f + (size_t)(9 * blk) * Vh;
  g[cb] = make_float4((float)b.d[0], (float)b.d[1], (float)b.d[2], (float)b.d[3]);
  g[(size_t)Vh + cb] = make_float4((float)b.d[4], (float)b.d[5], (float)b.o[0].re, (float)b.o[0].im);
  for (int k = 0; k < 7; ++k)
    g[(size_t)(2 + k) * Vh + cb] =
        make_float4((float)b.o[1 + 2 * k].re, (float)b.o[1 + 2 * k].im, (float)b.o[2 + 2 * k].re, (float)b.o[2 + 2 * k].im);
}

// Cholesky A = L L^dag (6x6 Hermitian positive definite); returns false if not PD.
__device__ bool cholesky6(const cplx<double> A[6][6], cplx<double> L[6][6], double& logdet) {
  logdet = 0.0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = mk(0.0, 0.0);
  for (int j = 0; j < 6; ++j) {
    double d = A[j][j].re;
    for (int k = 0; k < j; ++k) d -= norm2(L[j][k]);
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    L[j][j] = mk(ljj, 0.0);
    logdet += 2.0 * log(ljj);
    for (int i = j + 1; i < 6; ++i) {
      cplx<double> s = A[i][j];
      for (int k = 0; k < j; ++k) s = s - mul_cj(L[i][k], L[j][k]);
      L[i][j] = (1.0 / ljj) * s;
    }
  }
  return true;
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

__device__ __forceinline__ Mat3<double> load_fmunu(const double* __restrict__ Fin, const Geom& g, int p, int pl,
                                                   int cb) {
  const double* f = Fin + (size_t)((p * 6 + pl) * 9) * g.Vh + cb;
  double v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = __ldg(f + (size_t)k * g.Vh);
  Mat3<double> F;
  F.m[0][0] = mk(v[0], 0.0);
  F.m[1][1] = mk(v[1], 0.0);
  F.m[2][2] = mk(v[2], 0.0);
  F.m[0][1] = mk(v[3], v[4]);
  F.m[1][0] = mk(v[3], -v[4]);
  F.m[0][2] = mk(v[5], v[6]);
  F.m[2][0] = mk(v[5], -v[6]);
  F.m[1][2] = mk(v[7], v[8]);
  F.m[2][1] = mk(v[7], -v[8]);
  return F;
}

__global__ void k_clover_build(Geom g, const double* __restrict__ Fin, double kc, CloverOut out, ReduceBuf rb,
                               double* logdet_out) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  double ld[1] = {0.0};
  if (cb < g.Vh) {
    Mat3<double> F[6];
    for (int k = 0; k < 6; ++k) F[k] = load_fmunu(Fin, g, p, k, cb);
    // F index: 0:(0,1) 1:(0,2) 2:(0,3) 3:(1,2) 4:(1,3) 5:(2,3)
    HermBlock<double> B[2];
    for (int blk = 0; blk < 2; ++blk) {
      const double s = blk == 0 ? -1.0 : 1.0;
      cplx<double> A[6][6];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cplx<double> X1 = F[3].m[i][j] + s * F[2].m[i][j];
          cplx<double> X2 = F[1].m[i][j] - s * F[4].m[i][j];
          cplx<double> X3 = F[0].m[i][j] + s * F[5].m[i][j];
          const double one = (i == j) ? 1.0 : 0.0;
          A[i][j] = mk(one, 0.0) - kc * X3;
          A[i + 3][j + 3] = mk(one, 0.0) + kc * X3;
          A[i][j + 3] = -kc * (X1 - times_i(X2));
          A[i + 3][j] = -kc * (X1 + times_i(X2));
        }
      if (p == 0) {
        for (int i = 0; i < 6; ++i) B[blk].d[i] = A[i][i].re;
        for (int i = 1; i < 6; ++i)
          for (int j = 0; j < i; ++j) B[blk].o[tri_index(i, j)] = A[i][j];
      } else {
        cplx<double> L[6][6];
        double l;
        if (!cholesky6(A, L, l)) {
          atomicExch(out.bad, 1);
          l = 0.0;
          for (int i = 0; i < 6; ++i) L[i][i] = mk(1.0, 0.0);
        }
        ld[0] += l;
        // Linv = L^{-1} (lower triangular), A^{-1} = Linv^dag Linv
        cplx<double> Li[6][6];
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) Li[i][j] = mk(0.0, 0.0);
        for (int j = 0; j < 6; ++j) {
          Li[j][j] = mk(1.0 / L[j][j].re, 0.0);
          for (int i = j + 1; i < 6; ++i) {
            cplx<double> s2 = mk(0.0, 0.0);
            for (int kk = j; kk < i; ++kk) s2 = s2 + L[i][kk] * Li[kk][j];
            Li[i][j] = (-1.0 / L[i][i].re) * s2;
          }
        }
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j <= i; ++j) {
            cplx<double> s2 = mk(0.0, 0.0);
            for (int kk = i; kk < 6; ++kk) s2 = s2 + cj_mul(Li[kk][i], Li[kk][j]);
            if (i == j)
              B[blk].d[i] = s2.re;
            else
              B[blk].o[tri_index(i, j)] = s2;
          }
      }
    }
    if (p == 0) {
      store_clover(out.A64, B, cb, g.Vh);
      store_clover_df(out.Adf, B, cb, g.Vh);
      store_block32(out.A32, B[0], 0, cb, g.Vh);
      store_block32(out.A32, B[1], 1, cb, g.Vh);
    } else {
      store_clover(out.Ai64, B, cb, g.Vh);
      store_clover_df(out.Aidf, B, cb, g.Vh);
      store_block32(out.Ai32, B[0], 0, cb, g.Vh);
      store_block32(out.Ai32, B[1], 1, cb, g.Vh);
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
  dim3 grid(nblocks(c->g.Vh, 128), 2);
  k_clover_build<<<grid, 128, 0, c->stream>>>(c->g, c->fmunu, op->kappa * op->csw, o, c->rb, c->d_sums);
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
