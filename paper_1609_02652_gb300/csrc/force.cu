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

// H = sum_a h_a T_a (Hermitian traceless)
template <typename T>
__device__ __forceinline__ Mat3<T> from_algebra(const double h[8]) {
  Mat3<T> H;
  const double s = 0.5;
  H.m[0][0] = mk<T>((T)(s * (h[2] + kInvSqrt3 * h[7])), 0);
  H.m[1][1] = mk<T>((T)(s * (-h[2] + kInvSqrt3 * h[7])), 0);
  H.m[2][2] = mk<T>((T)(s * (-2.0 * kInvSqrt3 * h[7])), 0);
  H.m[0][1] = mk<T>((T)(s * h[0]), (T)(-s * h[1]));
  H.m[1][0] = mk<T>((T)(s * h[0]), (T)(s * h[1]));
  H.m[0][2] = mk<T>((T)(s * h[3]), (T)(-s * h[4]));
  H.m[2][0] = mk<T>((T)(s * h[3]), (T)(s * h[4]));
  H.m[1][2] = mk<T>((T)(s * h[5]), (T)(-s * h[6]));
  H.m[2][1] = mk<T>((T)(s * h[5]), (T)(s * h[6]));
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
__device__ __forceinline__ void shift(const Geom& g, const int x[4], int mu, int d, int y[4]) {
  for (int k = 0; k < 4; ++k) y[k] = x[k];
  y[mu] = (y[mu] + d + g.L[mu]) % g.L[mu];
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
// value only has to be a deterministic function of the gauge field), summed into the
// FP64 force
template <int PREC, int MU>
__device__ void hop_force_dir(double* F, const void* gauge, const Geom& g, int pz, int cb, const int z[4],
                              const typename Prec<PREC>::vec* Lf, const typename Prec<PREC>::vec* Rf,
                              const typename Prec<PREC>::vec* Lb, const typename Prec<PREC>::vec* Rb, double coef) {
  using T = typename Prec<PREC>::real;
  const Mat3<T> U = force_link<PREC>(gauge, g, pz, cb, z, MU);
  const int n = nbr_cb(g, z, MU, +1);
  Spinor<T> lf, rf, lb, rb;
  load_spinor(lf, Lf, cb, g.Vh);
  load_spinor(rf, Rf, n, g.Vh);
  load_spinor(lb, Lb, n, g.Vh);
  load_spinor(rb, Rb, cb, g.Vh);
  // Y_f = sum_s (U R_f)_s ((1 - g) L_f)_s^dag,  Y_b = sum_s R_b,s (U (1 + g) L_b)_s^dag
  Mat3<T> Yf = outer(umul(U, rf), proj_full<MU, -1>(lf));
  Mat3<T> Yb = outer(rb, umul(U, proj_full<MU, +1>(lb)));
  double c = coef;
  if (MU == 3 && z[3] == g.L[3] - 1) c *= g.bc_t;
  Mat3<T> Z;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Z.m[i][j] = Yf.m[i][j] - Yb.m[i][j];
  cplx<T> t[8];
  tr_lambda(Z, t);
  // Re(i tr(T_a Z)) = -Im tr(T_a Z) = -(1/2) Im tr(lambda_a Z)
  for (int a = 0; a < 8; ++a) fptr(F, g, pz, MU, a)[cb] += -0.5 * c * (double)t[a].im;
}

template <int PREC>
__global__ void k_force_hop(double* F, const void* gauge, Geom g, int pz, const typename Prec<PREC>::vec* Lf,
                            const typename Prec<PREC>::vec* Rf, const typename Prec<PREC>::vec* Lb,
                            const typename Prec<PREC>::vec* Rb, double coef) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  int z[4];
  cb_coords(g, cb, pz, z);
  hop_force_dir<PREC, 0>(F, gauge, g, pz, cb, z, Lf, Rf, Lb, Rb, coef);
  hop_force_dir<PREC, 1>(F, gauge, g, pz, cb, z, Lf, Rf, Lb, Rb, coef);
  hop_force_dir<PREC, 2>(F, gauge, g, pz, cb, z, Lf, Rf, Lb, Rb, coef);
  hop_force_dir<PREC, 3>(F, gauge, g, pz, cb, z, Lf, Rf, Lb, Rb, coef);
}

// G for the six planes from the chiral Pauli structure of sigma_{mu nu}:
// P1 = O01 + O10, P2 = -i O01 + i O10, P3 = O00 - O11 per chiral block B, O_ij = b_{2B+j} a_{2B+i}^dag;
// planes (01,02,03,12,13,23) = (P3+ + P3-, P2+ + P2-, -P1+ + P1-, P1+ + P1-, P2+ - P2-, -P3+ + P3-)
template <typename T>
__device__ void plane_G(const Spinor<T>& a, const Spinor<T>& b, Mat3<T> G[6]) {
  Mat3<T> P[2][3];
  for (int B = 0; B < 2; ++B) {
    Mat3<T> O[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) O[i][j].m[c][d] = mul_cj(b.s[2 * B + j][c], a.s[2 * B + i][d]);
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        P[B][0].m[c][d] = O[0][1].m[c][d] + O[1][0].m[c][d];
        P[B][1].m[c][d] = times_i(O[1][0].m[c][d] - O[0][1].m[c][d]);
        P[B][2].m[c][d] = O[0][0].m[c][d] - O[1][1].m[c][d];
      }
  }
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      G[0].m[c][d] = P[0][2].m[c][d] + P[1][2].m[c][d];
      G[1].m[c][d] = P[0][1].m[c][d] + P[1][1].m[c][d];
      G[2].m[c][d] = P[1][0].m[c][d] - P[0][0].m[c][d];
      G[3].m[c][d] = P[0][0].m[c][d] + P[1][0].m[c][d];
      G[4].m[c][d] = P[0][1].m[c][d] - P[1][1].m[c][d];
      G[5].m[c][d] = P[1][2].m[c][d] - P[0][2].m[c][d];
    }
}

__device__ __forceinline__ double* hptr(double* Hc, const Geom& g, int p, int plane, int a) {
  return Hc + (size_t)((p * 6 + plane) * 8 + a) * g.Vh;
}

// Hc[p] += coef (G~ + G~^dag) for G(a, b): h_a += 4 coef Re tr(T_a G) = 2 coef Re tr(lambda_a G)
template <int PREC>
__global__ void k_clover_insert(double* Hc, Geom g, int p, const typename Prec<PREC>::vec* A,
                                const typename Prec<PREC>::vec* B, double coef) {
  using T = typename Prec<PREC>::real;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  Spinor<T> a, b;
  load_spinor(a, A, cb, g.Vh);
  load_spinor(b, B, cb, g.Vh);
  Mat3<T> G[6];
  plane_G(a, b, G);
  for (int pl = 0; pl < 6; ++pl) {
    cplx<T> t[8];
    tr_lambda(G[pl], t);
    for (int k = 0; k < 8; ++k) hptr(Hc, g, p, pl, k)[cb] += 2.0 * coef * (double)t[k].re;
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

template <typename T>
__device__ __forceinline__ Mat3<T> load_H(const double* Hc, const Geom& g, const int x[4], int plane, double sgn) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(g, x);
  double h[8];
  for (int a = 0; a < 8; ++a) h[a] = sgn * Hc[(size_t)((p * 6 + plane) * 8 + a) * g.Vh + cb];
  return from_algebra<T>(h);
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
template <typename T>
__global__ void k_clover_force(double* F, const void* U64, const double* Hc, Geom g, int p) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (cb >= g.Vh) return;
  int z[4];
  cb_coords(g, cb, p, z);
  const Mat3<T> U = glink<T>(U64, g, z, mu);
  Mat3<T> Zs = mat_zero<T>();
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int pl = plane_index(mu, nu);
    const double sg = mu < nu ? 1.0 : -1.0;
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
void force_hop(pfmp_ctx* c, int prec, double* F, int pz, const void* Lf, const void* Rf, const void* Lb,
               const void* Rb, double coef) {
  if (prec == PFMP_F64)
    k_force_hop<PFMP_F64><<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(
        F, c->U64, c->g, pz, (const double2*)Lf, (const double2*)Rf, (const double2*)Lb, (const double2*)Rb, coef);
  else
    k_force_hop<PFMP_F32><<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(
        F, c->U32, c->g, pz, (const float4*)Lf, (const float4*)Rf, (const float4*)Lb, (const float4*)Rb, coef);
  PFMP_CHECK_LAUNCH();
}
void clover_insert(pfmp_ctx* c, int prec, double* Hc, int p, const void* a, const void* b, double coef) {
  if (prec == PFMP_F64)
    k_clover_insert<PFMP_F64><<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(Hc, c->g, p, (const double2*)a,
                                                                            (const double2*)b, coef);
  else
    k_clover_insert<PFMP_F32><<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(Hc, c->g, p, (const float4*)a,
                                                                            (const float4*)b, coef);
  PFMP_CHECK_LAUNCH();
}
void clover_insert_det(pfmp_op* op, double* Hc, double coef) {
  pfmp_ctx* c = op->ctx;
  k_clover_insert_det<<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(Hc, c->g, op->clov64[1], coef);
  PFMP_CHECK_LAUNCH();
}
// prec = PFMP_F64: FP64 arithmetic on the master links; PFMP_F32: FP32 arithmetic on the
// compressed FP32 links (the forces of an MD with FP32 forces), FP64 accumulation
void clover_force(pfmp_ctx* c, int prec, double* F, const double* Hc) {
  for (int p = 0; p < 2; ++p) {
    dim3 grid(nblocks(c->g.Vh, 64), 4);
    if (prec == PFMP_F64)
      k_clover_force<double><<<grid, 64, 0, c->stream>>>(F, c->U64, Hc, c->g, p);
    else
      k_clover_force<float><<<grid, 64, 0, c->stream>>>(F, c->U32, Hc, c->g, p);
    PFMP_CHECK_LAUNCH();
  }
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

// Re[a^dag dM-hat b] * coef  ->  F (hop terms) and Hc (clover terms); a, b even fields
// of precision prec (PFMP_F64 or PFMP_F32), y and w odd temporaries of that precision
void deriv_mhat(pfmp_op* op, int prec, double* F, double* Hc, const void* a, const void* b, double coef, void* y,
                void* w) {
  pfmp_ctx* c = op->ctx;
  const double k2 = op->kappa * op->kappa;
  const double kc = op->kappa * op->csw;
  // y = A_oo^{-1} H_oe b, w = A_oo^{-1} H^dag_oe a (odd)
  hop_clov_odd(op, prec, y, b, false);
  hop_clov_odd(op, prec, w, a, true);
  force_hop(c, prec, F, 0, a, y, w, b, -k2 * coef);
  force_hop(c, prec, F, 1, w, b, a, y, -k2 * coef);
  if (op->csw != 0.0) {
    clover_insert(c, prec, Hc, 0, a, b, -kc * coef);
    clover_insert(c, prec, Hc, 1, w, y, k2 * (-kc) * coef);
  }
}

}  // namespace pfmp
