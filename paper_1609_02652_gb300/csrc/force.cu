// Fermion, clover and gauge forces (App. C), accumulated in FP64 as algebra coefficients
// f[p][mu][a][cb] = dS/d omega_a for U_mu(x) -> exp(i omega_a T_a) U_mu(x).
//
// The fermion forces of App. C are sums of contractions Re[eta^dag (dK/dU) chi].  With
// K = M-hat^dag M-hat:
//   Re eta^dag dK chi = Re (M-hat chi)^dag dM-hat eta + Re (M-hat eta)^dag dM-hat chi,
// and with M-hat = A_ee - kappa^2 H_eo A_oo^{-1} H_oe,
//   a^dag dM-hat b = a^dag dA_ee b - kappa^2 [a^dag dH_eo y + w^dag dH_oe b - w^dag dA_oo y],
//   y = A_oo^{-1} H_oe b,  w = A_oo^{-1} H^dag_oe a.
// Hop terms: for a link U_mu(z) the forward term a(z)^dag (1 - g_mu) dU b(z+mu) and the
// backward term a(z+mu)^dag (1 + g_mu) dU^dag b(z) give, with dU = i w T U,
//   d/dw_a = i tr(T_a Z),  Z = sum_s (U R_f)_s ((1 - g_mu) L_f)_s^dag - sum_s R_b,s (U (1 + g_mu) L_b)_s^dag.
// Clover terms: a^dag (sigma (x) dF) b = tr_c(dF G), G = sum_{s s'} sigma_{s s'} b_s' a_s^dag;
// with F = traceless part of (Q - Q^dag)/(8i),
//   Re tr(dF G) = (1/8) Im tr(dQ H),  H = G~ + G~^dag (G~ traceless),
// so each site keeps one Hermitian traceless H per plane (8 reals) summed over every
// term, and one final kernel differentiates the clover leaves: for U_mu(z) in the plane
// (mu, nu) with corners z, z+mu, z+mu+nu, z+nu (above) and z-nu, z-nu+mu (below),
//   d/dw_a = (1/8) Re tr(T_a [U X_above - Y_below U^dag]),
//   X_above = H(z+mu) V1 V2 V3 + V1 H(z+mu+nu) V2 V3 + V1 V2 H(z+nu) V3 + V1 V2 V3 H(z),
//   Y_below = H(z) W1 W2 W3 + W1 H(z-nu) W2 W3 + W1 W2 H(z-nu+mu) W3 + W1 W2 W3 H(z+mu),
//   V1 = U_nu(z+mu), V2 = U_mu(z+nu)^dag, V3 = U_nu(z)^dag,
//   W1 = U_nu(z-nu)^dag, W2 = U_mu(z-nu), W3 = U_nu(z-nu+mu).
// Gauge force (Wilson action, beta/3 normalisation): d/dw_a = (beta/3) Im tr(T_a U S),
// S the sum of the six staples.
#include <algorithm>
#include <cmath>

#include "context.h"
#include "fields.cuh"
#include "spin.cuh"

namespace pfmp {

constexpr double kInvSqrt3 = 0.57735026918962576451;

// c_a = tr(lambda_a M), a = 1..8 (complex)
template <typename T>
__device__ __forceinline__ void tr_lambda(const Mat3<T>& M, cplx<T> t[8]) {
  t[0] = M.m[1][0] + M.m[0][1];
  t[1] = times_i(M.m[0][1] - M.m[1][0]);
  t[2] = M.m[0][0] - M.m[1][1];
  t[3] = M.m[2][0] + M.m[0][2];
  t[4] = times_i(M.m[0][2] - M.m[2][0]);
  t[5] = M.m[2][1] + M.m[1][2];
  t[6] = times_i(M.m[1][2] - M.m[2][1]);
  t[7] = (T)kInvSqrt3 * (M.m[0][0] + M.m[1][1] - (T)2 * M.m[2][2]);
}

// H = sum_a h_a T_a (Hermitian traceless), in the arithmetic of T
template <typename T>
__device__ __forceinline__ Mat3<T> from_algebra(const T h[8]) {
  Mat3<T> H;
  const T s = (T)0.5, r3 = (T)kInvSqrt3;
  H.m[0][0] = mk<T>(s * (h[2] + r3 * h[7]), 0);
  H.m[1][1] = mk<T>(s * (-h[2] + r3 * h[7]), 0);
  H.m[2][2] = mk<T>(s * ((T)-2 * r3 * h[7]), 0);
  H.m[0][1] = mk<T>(s * h[0], -s * h[1]);
  H.m[1][0] = mk<T>(s * h[0], s * h[1]);
  H.m[0][2] = mk<T>(s * h[3], -s * h[4]);
  H.m[2][0] = mk<T>(s * h[3], s * h[4]);
  H.m[1][2] = mk<T>(s * h[5], -s * h[6]);
  H.m[2][1] = mk<T>(s * h[5], s * h[6]);
  return H;
}

// the link U_mu(x) at full coordinates: FP64 from the master field, FP32 from the
// 12-real compressed copy (third row rebuilt)
template <typename T>
__device__ __forceinline__ Mat3<T> glink(const void* gauge, const Geom& g, const int x[4], int mu);

__device__ __forceinline__ Mat3<double> mlink(const double2* U, const Geom& g, const int x[4], int mu) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  Mat3<double> M;
  load_link18(M, U + (size_t)((p * 4 + mu) * 9) * g.Vh, cb_index(g, x), g.Vh);
  return M;
}
template <>
__device__ __forceinline__ Mat3<double> glink<double>(const void* gauge, const Geom& g, const int x[4], int mu) {
  return mlink((const double2*)gauge, g, x, mu);
}
template <>
__device__ __forceinline__ Mat3<float> glink<float>(const void* gauge, const Geom& g, const int x[4], int mu) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  Mat3<float> M;
  load_link(M, link_plane<PFMP_F32>((const float4*)gauge, p * 4 + mu, g.Vh), cb_index(g, x), g.Vh);
  return M;
}
// y = x + d mu-hat (d = +-1), periodic
__device__ __forceinline__ void shift(const Geom& g, const int x[4], int mu, int d, int y[4]) {
  for (int k = 0; k < 4; ++k) y[k] = x[k];
  int v = y[mu] + d;
  if (v >= g.L[mu]) v -= g.L[mu];
  if (v < 0) v += g.L[mu];
  y[mu] = v;
}

__device__ __forceinline__ double* fptr(double* F, const Geom& g, int p, int mu, int a) {
  return F + (size_t)((p * 4 + mu) * 8 + a) * g.Vh;
}

// outer product sum_s u_s v_s^dag over 4 spins
template <typename T>
__device__ __forceinline__ Mat3<T> outer(const Spinor<T>& u, const Spinor<T>& v) {
  Mat3<T> M;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx<T> s = mk<T>(0, 0);
      for (int k = 0; k < 4; ++k) s = s + mul_cj(u.s[k][i], v.s[k][j]);
      M.m[i][j] = s;
    }
  return M;
}

// (1 + S g_MU) psi as a full spinor
template <int MU, int S, typename T>
__device__ __forceinline__ Spinor<T> proj_full(const Spinor<T>& p) {
  Spinor<T> r;
  for (int s = 0; s < 4; ++s)
    for (int c = 0; c < 3; ++c) r.s[s][c] = mk<T>(0, 0);
  accumulate<MU, S>(r, project<MU, S>(p));
  return r;
}

template <typename T>
__device__ __forceinline__ Spinor<T> umul(const Mat3<T>& U, const Spinor<T>& v) {
  Spinor<T> r;
  for (int s = 0; s < 4; ++s)
    for (int i = 0; i < 3; ++i) r.s[s][i] = U.m[i][0] * v.s[s][0] + U.m[i][1] * v.s[s][1] + U.m[i][2] * v.s[s][2];
  return r;
}

// the link U_MU(z) of the force kernels: FP64 from the master field, FP32 from the
// 12-real compressed copy (third row rebuilt)
template <int PREC>
__device__ __forceinline__ Mat3<typename Prec<PREC>::real> force_link(const void* gauge, const Geom& g, int pz, int cb,
                                                                      const int z[4], int mu) {
  if constexpr (PREC == PFMP_F64) {
    return mlink((const double2*)gauge, g, z, mu);
  } else {
    Mat3<float> U;
    load_link(U, link_plane<PFMP_F32>((const float4*)gauge, pz * 4 + mu, g.Vh), cb, g.Vh);
    return U;
  }
}

// Spinor products in the arithmetic of PREC (FP64, or FP32 for the MD forces, whose
// value only has to be a deterministic function of the gauge field).  On the sites of
// parity pz the forward and backward fields of a contraction (a, b, y, w) are
// (L_f, R_f, L_b, R_b) = (a, y, w, b) for pz = 0 and (w, b, a, y) for pz = 1.  The link
// factors out of the batch's sum:
//   sum_k c_k Z_k = U X_f - X_b U^dag,  X_f = sum_k c_k sum_s R_f,s ((1 - g) L_f)_s^dag,
//                                       X_b = sum_k c_k sum_s R_b,s ((1 + g) L_b)_s^dag,
// so each contraction costs two spin-summed outer products, accumulated in PREC, and the
// FP64 force is read and written once per batch.
template <int PREC, int MU>
__device__ void hop_force_dir(double* F, const void* gauge, const Geom& g, int pz, int cb, const int z[4],
                              const DerivBatch& B) {
  using T = typename Prec<PREC>::real;
  using V = typename Prec<PREC>::vec;
  const int n = nbr_cb(g, z, MU, +1);
  Mat3<T> Xf = mat_zero<T>(), Xb = mat_zero<T>();
#pragma unroll 1
  for (int k = 0; k < B.n; ++k) {
    {
      const DerivSet& d = B.s[k];
      const V* Lf = (const V*)(pz == 0 ? d.a : d.w);
      const V* Rf = (const V*)(pz == 0 ? d.y : d.b);
      const V* Lb = (const V*)(pz == 0 ? d.w : d.a);
      const V* Rb = (const V*)(pz == 0 ? d.b : d.y);
      Spinor<T> lf, rf, lb, rb;
      load_spinor(lf, Lf, cb, g.Vh);
      load_spinor(rf, Rf, n, g.Vh);
      load_spinor(lb, Lb, n, g.Vh);
      load_spinor(rb, Rb, cb, g.Vh);
      const T c = (T)d.c_hop;
      const Mat3<T> Of = outer(rf, proj_full<MU, -1>(lf));
      const Mat3<T> Ob = outer(rb, proj_full<MU, +1>(lb));
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          Xf.m[i][j] = Xf.m[i][j] + c * Of.m[i][j];
          Xb.m[i][j] = Xb.m[i][j] + c * Ob.m[i][j];
        }
    }
  }
  const Mat3<T> U = force_link<PREC>(gauge, g, pz, cb, z, MU);
  const Mat3<T> A = matmul(U, Xf), Bm = matmul_nd(Xb, U);
  Mat3<T> Z;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Z.m[i][j] = A.m[i][j] - Bm.m[i][j];
  cplx<T> t[8];
  tr_lambda(Z, t);
  // Re(i tr(T_a Z)) = -Im tr(T_a Z) = -(1/2) Im tr(lambda_a Z)
  const double c = (MU == 3 && z[3] == g.L[3] - 1) ? -0.5 * g.bc_t : -0.5;
#pragma unroll
  for (int a = 0; a < 8; ++a) fptr(F, g, pz, MU, a)[cb] += c * (double)t[a].im;
}

// A block takes 32 sites of parity blockIdx.y; warp mu of the block takes direction mu,
// so the four warps read the same local spinors close together (from L1 after the first)
template <int PREC>
__global__ void __launch_bounds__(128) k_force_hop(double* F, const void* gauge, Geom g, DerivBatch B) {
  const int cb = blockIdx.x * 32 + (threadIdx.x & 31);
  const int mu = threadIdx.x >> 5;
  const int pz = blockIdx.y;
  if (cb >= g.Vh) return;
  int z[4];
  cb_coords(g, cb, pz, z);
  switch (mu) {
    case 0: hop_force_dir<PREC, 0>(F, gauge, g, pz, cb, z, B); break;
    case 1: hop_force_dir<PREC, 1>(F, gauge, g, pz, cb, z, B); break;
    case 2: hop_force_dir<PREC, 2>(F, gauge, g, pz, cb, z, B); break;
    default: hop_force_dir<PREC, 3>(F, gauge, g, pz, cb, z, B); break;
  }
}

__device__ __forceinline__ double* hptr(double* Hc, const Geom& g, int p, int plane, int a) {
  return Hc + (size_t)((p * 6 + plane) * 8 + a) * g.Vh;
}

// P_K of chiral block B (spins 2B, 2B + 1) from O_ij = b_{2B+j} a_{2B+i}^dag:
// P_0 = O01 + O10, P_1 = -i O01 + i O10, P_2 = O00 - O11
template <int K, typename T>
__device__ __forceinline__ Mat3<T> pauli_P(const Spinor<T>& a, const Spinor<T>& b, int B) {
  Mat3<T> P;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if constexpr (K == 0)
        P.m[c][d] = mul_cj(b.s[2 * B + 1][c], a.s[2 * B][d]) + mul_cj(b.s[2 * B][c], a.s[2 * B + 1][d]);
      else if constexpr (K == 1)
        P.m[c][d] = times_i(mul_cj(b.s[2 * B][c], a.s[2 * B + 1][d]) - mul_cj(b.s[2 * B + 1][c], a.s[2 * B][d]));
      else
        P.m[c][d] = mul_cj(b.s[2 * B][c], a.s[2 * B][d]) - mul_cj(b.s[2 * B + 1][c], a.s[2 * B + 1][d]);
    }
  return P;
}

// The two planes built from the Pauli component K, summed over the contractions of a
// batch: (planes, G) = K 2: (01, P+ + P-), (23, -P+ + P-); K 1: (02, P+ + P-),
// (13, P+ - P-); K 0: (03, -P+ + P-), (12, P+ + P-), with P+ / P- the blocks 0 / 1.
// P is linear in the contraction's fields: the batch's P+ and P- are accumulated in
// PREC and reduced to algebra components once.
template <int PREC, int K>
__device__ __forceinline__ void clover_insert_pair(double* Hc, const Geom& g, int p, int cb, const DerivBatch& B) {
  using T = typename Prec<PREC>::real;
  using V = typename Prec<PREC>::vec;
  Mat3<T> P[2] = {mat_zero<T>(), mat_zero<T>()};
#pragma unroll 1
  for (int s = 0; s < B.n; ++s) {
    {
      const DerivSet& d = B.s[s];
      const T coef = (T)(2.0 * (p == 0 ? d.c_even : d.c_odd));
      Spinor<T> a, b;
      load_spinor(a, (const V*)(p == 0 ? d.a : d.w), cb, g.Vh);
      load_spinor(b, (const V*)(p == 0 ? d.b : d.y), cb, g.Vh);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const Mat3<T> Pq = pauli_P<K>(a, b, q);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) P[q].m[i][j] = P[q].m[i][j] + coef * Pq.m[i][j];
      }
    }
  }
  double r[2][8];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    cplx<T> t[8];
    tr_lambda(P[q], t);
#pragma unroll
    for (int k = 0; k < 8; ++k) r[q][k] = (double)t[k].re;
  }
  // plane index (0,1)=0 (0,2)=1 (0,3)=2 (1,2)=3 (1,3)=4 (2,3)=5
  constexpr int plA = K == 2 ? 0 : (K == 1 ? 1 : 2);
  constexpr int plB = K == 2 ? 5 : (K == 1 ? 4 : 3);
  constexpr double sA = K == 0 ? -1.0 : 1.0;  // sign of P+ in plane plA
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    hptr(Hc, g, p, plA, k)[cb] += sA * r[0][k] + r[1][k];
    if constexpr (K == 1)
      hptr(Hc, g, p, plB, k)[cb] += r[0][k] - r[1][k];
    else if constexpr (K == 2)
      hptr(Hc, g, p, plB, k)[cb] += -r[0][k] + r[1][k];
    else
      hptr(Hc, g, p, plB, k)[cb] += r[0][k] + r[1][k];
  }
}

// Hc[p] += coef (G~ + G~^dag) for G(a, b): h_a += 4 coef Re tr(T_a G) = 2 coef Re tr(lambda_a G),
// summed over the contractions of a batch: on the even sites G(a, b) with c_even, on the
// odd sites G(w, y) with c_odd.  A block takes 32 sites of parity blockIdx.y and warp K
// the Pauli component K (two of the six planes), so the three warps read the same
// spinors close together and each thread keeps 16 accumulators live instead of 48.
template <int PREC>
__global__ void __launch_bounds__(96) k_clover_insert(double* Hc, Geom g, DerivBatch B) {
  const int cb = blockIdx.x * 32 + (threadIdx.x & 31);
  const int K = threadIdx.x >> 5;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  switch (K) {
    case 0: clover_insert_pair<PREC, 0>(Hc, g, p, cb, B); break;
    case 1: clover_insert_pair<PREC, 1>(Hc, g, p, cb, B); break;
    default: clover_insert_pair<PREC, 2>(Hc, g, p, cb, B); break;
  }
}

// Hc[odd] += coef (G~ + G~^dag) with G = sum_{ij} sigma_{ji} Ainv_block(i, j) (det force)
__global__ void k_clover_insert_det(double* Hc, Geom g, const double2* Ainv, double coef) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  HermBlock<double> B[2];
  load_clover(B, Ainv, cb, g.Vh);
  // full 6x6 blocks
  Mat3<double> P[2][3];
  for (int blk = 0; blk < 2; ++blk) {
    cplx<double> M[6][6];
    for (int i = 0; i < 6; ++i) M[i][i] = mk(B[blk].d[i], 0.0);
    for (int i = 1; i < 6; ++i)
      for (int j = 0; j < i; ++j) {
        M[i][j] = B[blk].o[tri_index(i, j)];
        M[j][i] = conj(M[i][j]);
      }
    // colour block (i, j) of spins (2 blk + i, 2 blk + j): M[3i + c][3j + d]
    // G = sum_{ij} sigma_{ji} X_ij; sigma_k blocks: s1 -> X01 + X10, s2 -> i X01 - i X10, s3 -> X00 - X11
    // (sigma_{ji}: s2_{10} = i multiplies X_01, s2_{01} = -i multiplies X_10)
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        cplx<double> x00 = M[c][d], x01 = M[c][3 + d], x10 = M[3 + c][d], x11 = M[3 + c][3 + d];
        P[blk][0].m[c][d] = x01 + x10;
        P[blk][1].m[c][d] = times_i(x01 - x10);
        P[blk][2].m[c][d] = x00 - x11;
      }
  }
  Mat3<double> G[6];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      G[0].m[c][d] = P[0][2].m[c][d] + P[1][2].m[c][d];
      G[1].m[c][d] = P[0][1].m[c][d] + P[1][1].m[c][d];
      G[2].m[c][d] = P[1][0].m[c][d] - P[0][0].m[c][d];
      G[3].m[c][d] = P[0][0].m[c][d] + P[1][0].m[c][d];
      G[4].m[c][d] = P[0][1].m[c][d] - P[1][1].m[c][d];
      G[5].m[c][d] = P[1][2].m[c][d] - P[0][2].m[c][d];
    }
  for (int pl = 0; pl < 6; ++pl) {
    cplx<double> t[8];
    tr_lambda(G[pl], t);
    for (int k = 0; k < 8; ++k) hptr(Hc, g, 1, pl, k)[cb] += 2.0 * coef * t[k].re;
  }
}

// the insertion H of a plane at full coordinates x, times sgn, from a copy of Hc in T
template <typename T>
__device__ __forceinline__ Mat3<T> load_H(const T* Hc, const Geom& g, const int x[4], int plane, T sgn) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(g, x);
  T h[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) h[a] = sgn * __ldg(Hc + (size_t)((p * 6 + plane) * 8 + a) * g.Vh + cb);
  return from_algebra<T>(h);
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

__device__ __forceinline__ int plane_index(int mu, int nu) {
  // (0,1)=0 (0,2)=1 (0,3)=2 (1,2)=3 (1,3)=4 (2,3)=5
  const int a = mu < nu ? mu : nu, b = mu < nu ? nu : mu;
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// F[p] += (1/8) Re tr(T_a [U X_above - Y_below U^dag]) summed over the three planes,
// one thread per (site, mu).  With V1 = U_nu(z+mu), V2 = U_mu(z+nu)^dag, V3 = U_nu(z)^dag,
// W1 = U_nu(z-nu)^dag, W2 = U_mu(z-nu), W3 = U_nu(z-nu+mu) and H_y the clover insertion
// at site y:
//   U X = U H_{z+mu} V1 V2 V3 + U V1 H_{z+mu+nu} V2 V3 + U V1 V2 H_{z+nu} V3 + U V1 V2 V3 H_z
//   Y U^dag = H_z W1 W2 W3 U^dag + W1 H_{z-nu} W2 W3 U^dag + W1 W2 H_{z-nu+mu} W3 U^dag
//             + W1 W2 W3 H_{z+mu} U^dag
// both summed Horner-fashion (U X from the left with the running prefix U V1 .. Vk,
// Y U^dag from the right with the running suffix Wk .. W3 U^dag), which keeps three
// 3x3 matrices live instead of a dozen.
// A block takes 32 sites of parity blockIdx.y and warp mu the links U_mu of those sites,
// so the four warps share the insertions and links they read through L1.
template <typename T>
constexpr int clover_force_min_blocks() {
  return sizeof(T) == 4 ? 3 : 1;  // FP32: 3 resident blocks (168 registers, a few spilled)
}
template <typename T>
__global__ void __launch_bounds__(128, clover_force_min_blocks<T>()) k_clover_force(double* F, const void* U64,
                                                                                  const T* Hc, Geom g) {
  const int cb = blockIdx.x * 32 + (threadIdx.x & 31);
  const int mu = threadIdx.x >> 5;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  int z[4];
  cb_coords(g, cb, p, z);
  const Mat3<T> U = glink<T>(U64, g, z, mu);
  Mat3<T> Zs = mat_zero<T>();
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int pl = plane_index(mu, nu);
    const T sg = mu < nu ? (T)1 : (T)-1;
    int zpm[4], zpmpn[4], zpn[4], zmn[4], zmnpm[4];
    shift(g, z, mu, 1, zpm);
    shift(g, zpm, nu, 1, zpmpn);
    shift(g, z, nu, 1, zpn);
    shift(g, z, nu, -1, zmn);
    shift(g, zmn, mu, 1, zmnpm);
    // upper: R = sum over the four leaves, L = running prefix U V1 .. Vk
    Mat3<T> L = U;
    Mat3<T> R = matmul(L, load_H<T>(Hc, g, zpm, pl, sg));
    {
      const Mat3<T> V1 = glink<T>(U64, g, zpm, nu);
      L = matmul(L, V1);
      R = mat_add(matmul(R, V1), matmul(L, load_H<T>(Hc, g, zpmpn, pl, sg)));
    }
    {
      const Mat3<T> V2 = dagger(glink<T>(U64, g, zpn, mu));
      L = matmul(L, V2);
      R = mat_add(matmul(R, V2), matmul(L, load_H<T>(Hc, g, zpn, pl, sg)));
    }
    {
      const Mat3<T> V3 = dagger(glink<T>(U64, g, z, nu));
      L = matmul(L, V3);
      R = mat_add(matmul(R, V3), matmul(L, load_H<T>(Hc, g, z, pl, sg)));
    }
    // lower: Q = sum over the four leaves, M = running suffix Wk .. W3 U^dag
    Mat3<T> M = dagger(U);
    Mat3<T> Q = matmul(load_H<T>(Hc, g, zpm, pl, sg), M);
    {
      const Mat3<T> W3 = glink<T>(U64, g, zmnpm, nu);
      M = matmul(W3, M);
      Q = mat_add(matmul(W3, Q), matmul(load_H<T>(Hc, g, zmnpm, pl, sg), M));
    }
    {
      const Mat3<T> W2 = glink<T>(U64, g, zmn, mu);
      M = matmul(W2, M);
      Q = mat_add(matmul(W2, Q), matmul(load_H<T>(Hc, g, zmn, pl, sg), M));
    }
    {
      const Mat3<T> W1 = dagger(glink<T>(U64, g, zmn, nu));
      M = matmul(W1, M);
      Q = mat_add(matmul(W1, Q), matmul(load_H<T>(Hc, g, z, pl, sg), M));
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Zs.m[i][j] = Zs.m[i][j] + R.m[i][j] - Q.m[i][j];
  }
  cplx<T> t[8];
  tr_lambda(Zs, t);
  // (1/8) Re tr(T_a Z) = (1/16) Re tr(lambda_a Z)
  for (int a = 0; a < 8; ++a) fptr(F, g, p, mu, a)[cb] += 0.0625 * (double)t[a].re;
}

// F += (beta/3) Im tr(T_a U S) = (beta/6) Im tr(lambda_a U S)
template <typename T>
__global__ void k_gauge_force(double* F, const void* U64, Geom g, int p, double beta) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  int z[4];
  cb_coords(g, cb, p, z);
  for (int mu = 0; mu < 4; ++mu) {
    Mat3<T> S = mat_zero<T>();
    int zpm[4];
    shift(g, z, mu, 1, zpm);
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      int zpn[4], zmn[4], zpmmn[4];
      shift(g, z, nu, 1, zpn);
      shift(g, z, nu, -1, zmn);
      shift(g, zpm, nu, -1, zpmmn);
      // upper staple U_nu(z+mu) U_mu(z+nu)^dag U_nu(z)^dag
      S = mat_add(S, matmul_nd(matmul_nd(glink<T>(U64, g, zpm, nu), glink<T>(U64, g, zpn, mu)), glink<T>(U64, g, z, nu)));
      // lower staple U_nu(z+mu-nu)^dag U_mu(z-nu)^dag U_nu(z-nu)
      S = mat_add(S, matmul(matmul_dn(glink<T>(U64, g, zpmmn, nu), dagger(glink<T>(U64, g, zmn, mu))), glink<T>(U64, g, zmn, nu)));
    }
    const Mat3<T> US = matmul(glink<T>(U64, g, z, mu), S);
    cplx<T> t[8];
    tr_lambda(US, t);
    for (int a = 0; a < 8; ++a) fptr(F, g, p, mu, a)[cb] += beta / 6.0 * (double)t[a].im;
  }
}

// ------------------------------------------------------------------ host side
void deriv_mhat_batch(pfmp_ctx* c, int prec, double* F, double* Hc, const DerivBatch& B) {
  if (B.n == 0) return;
  PFMP_REQUIRE(B.n <= kMaxDerivSets, PFMP_E_INVALID, "too many contractions in one force batch");
  bool clover = false;
  for (int k = 0; k < B.n; ++k) clover = clover || B.s[k].c_even != 0.0 || B.s[k].c_odd != 0.0;
  const dim3 grid(nblocks(c->g.Vh, 32), 2);
  if (prec == PFMP_F64) {
    k_force_hop<PFMP_F64><<<grid, 128, 0, c->stream>>>(F, c->U64, c->g, B);
    PFMP_CHECK_LAUNCH();
    if (clover) k_clover_insert<PFMP_F64><<<grid, 96, 0, c->stream>>>(Hc, c->g, B);
  } else {
    k_force_hop<PFMP_F32><<<grid, 128, 0, c->stream>>>(F, c->U32, c->g, B);
    PFMP_CHECK_LAUNCH();
    if (clover) k_clover_insert<PFMP_F32><<<grid, 96, 0, c->stream>>>(Hc, c->g, B);
  }
  PFMP_CHECK_LAUNCH();
}
void clover_insert_det(pfmp_op* op, double* Hc, double coef) {
  pfmp_ctx* c = op->ctx;
  k_clover_insert_det<<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(Hc, c->g, op->clov64[1], coef);
  PFMP_CHECK_LAUNCH();
}
// prec = PFMP_F64: FP64 arithmetic on the master links; PFMP_F32: FP32 arithmetic on the
// compressed FP32 links (the forces of an MD with FP32 forces), FP64 accumulation
// prec = PFMP_F32 reads an FP32 copy of Hc (converted once here, not per leaf)
void clover_force(pfmp_ctx* c, int prec, double* F, const double* Hc) {
  const dim3 grid(nblocks(c->g.Vh, 32), 2);
  if (prec == PFMP_F64) {
    k_clover_force<double><<<grid, 128, 0, c->stream>>>(F, c->U64, Hc, c->g);
  } else {
    const long n = 96L * c->g.Vh;
    if (!c->hc32) c->hc32 = (float*)dev_alloc(n * sizeof(float));
    k_to_f32<<<std::min(nblocks(n), 152 * 8), kBlock, 0, c->stream>>>(Hc, c->hc32, n);
    PFMP_CHECK_LAUNCH();
    k_clover_force<float><<<grid, 128, 0, c->stream>>>(F, c->U32, c->hc32, c->g);
  }
  PFMP_CHECK_LAUNCH();
}
void gauge_force(pfmp_ctx* c, int prec, double* F, double beta) {
  for (int p = 0; p < 2; ++p) {
    if (prec == PFMP_F64)
      k_gauge_force<double><<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(F, c->U64, c->g, p, beta);
    else
      k_gauge_force<float><<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(F, c->U32, c->g, p, beta);
    PFMP_CHECK_LAUNCH();
  }
}

}  // namespace pfmp
