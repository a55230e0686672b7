// SU(3) helpers in FP64 shared by field initialisation and the link update:
// anti-Hermitian algebra elements, the matrix exponential (scaling and squaring of the
// Taylor series) and reunitarisation.
#pragma once
#include "pfmp_internal.cuh"

namespace pfmp {

// Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): the result is in SU(3)
__device__ inline void reunitarise(Mat3<double>& U) {
  double n0 = 0;
  for (int j = 0; j < 3; ++j) n0 += norm2(U.m[0][j]);
  n0 = rsqrt(n0);
  for (int j = 0; j < 3; ++j) U.m[0][j] = n0 * U.m[0][j];
  cplx<double> d = mk(0.0, 0.0);
  for (int j = 0; j < 3; ++j) d = d + cj_mul(U.m[0][j], U.m[1][j]);
  for (int j = 0; j < 3; ++j) U.m[1][j] = U.m[1][j] - d * U.m[0][j];
  double n1 = 0;
  for (int j = 0; j < 3; ++j) n1 += norm2(U.m[1][j]);
  n1 = rsqrt(n1);
  for (int j = 0; j < 3; ++j) U.m[1][j] = n1 * U.m[1][j];
  reconstruct_row2(U);
}

// exp(X) for a small-ish 3x3 anti-Hermitian X: scaling by 2^-s until ||X||_F <= 1/4,
// Taylor series to order 14, then s squarings.
__device__ inline Mat3<double> expm3(Mat3<double> X) {
  double nf = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) nf += norm2(X.m[i][j]);
  nf = sqrt(nf);
  int s = 0;
  while (nf > 0.25 && s < 60) {
    nf *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X.m[i][j] = sc * X.m[i][j];
  // Horner: E = I + X (I + X/2 (I + X/3 ( ... )))
  Mat3<double> E = mat_zero<double>();
  for (int i = 0; i < 3; ++i) E.m[i][i] = mk(1.0, 0.0);
  for (int k = 14; k >= 1; --k) {
    Mat3<double> T = matmul(X, E);
    const double f = 1.0 / k;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) E.m[i][j] = (i == j ? mk(1.0, 0.0) : mk(0.0, 0.0)) + f * T.m[i][j];
  }
  for (int k = 0; k < s; ++k) E = matmul(E, E);
  return E;
}

// i * sum_a c_a T_a as an anti-Hermitian matrix (T_a = lambda_a / 2)
__device__ inline Mat3<double> i_algebra(const double c[8], double eps) {
  const double h = 0.5 * eps;
  const double s3 = 0.57735026918962576451;  // 1/sqrt(3)
  // H = sum c_a lambda_a / 2
  cplx<double> H[3][3];
  H[0][0] = mk(h * (c[2] + s3 * c[7]), 0.0);
  H[1][1] = mk(h * (-c[2] + s3 * c[7]), 0.0);
  H[2][2] = mk(h * (-2.0 * s3 * c[7]), 0.0);
  H[0][1] = mk(h * c[0], -h * c[1]);
  H[1][0] = mk(h * c[0], h * c[1]);
  H[0][2] = mk(h * c[3], -h * c[4]);
  H[2][0] = mk(h * c[3], h * c[4]);
  H[1][2] = mk(h * c[5], -h * c[6]);
  H[2][1] = mk(h * c[5], h * c[6]);
  Mat3<double> X;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X.m[i][j] = times_i(H[i][j]);
  return X;
}

}  // namespace pfmp
