// SU(3) helpers in FP64 shared by field initialisation and the link update:
// anti-Hermitian algebra elements, the matrix exponential (scaling and squaring of the
// Taylor series, reduced to three scalar series by Cayley-Hamilton) and reunitarisation.
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

// exp(X) for a 3x3 complex X.  By Cayley-Hamilton X^3 = e1 X^2 - e2 X + e3 I
// (e1 = tr X, e2 = (e1^2 - tr X^2) / 2, e3 = det X), so every term X^n / n! of the Taylor
// series is a_n I + b_n X + c_n X^2 with scalar coefficients, and
//   X^{n+1} / (n+1)! = (c_n e3, a_n - c_n e2, b_n + c_n e1) / (n + 1)   in that basis.
// The series runs in those three scalars until the last term's bound ||X||^n / n! is
// below 2^-56 (for ||X|| <= 1 it bounds the remainder too) and costs one
// matrix product (X^2) instead of one per order.  X is first scaled by 2^-s until
// ||X||_F <= 1 and the result squared s times; inside the MD ||eps P|| is well below 1.
__device__ inline Mat3<double> expm3(Mat3<double> X) {
  double nf = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) nf += norm2(X.m[i][j]);
  nf = sqrt(nf);
  int s = 0;
  while (nf > 1.0 && s < 60) {
    nf *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X.m[i][j] = sc * X.m[i][j];
  const Mat3<double> X2 = matmul(X, X);
  const cplx<double> e1 = X.m[0][0] + X.m[1][1] + X.m[2][2];
  const cplx<double> trX2 = X2.m[0][0] + X2.m[1][1] + X2.m[2][2];
  const cplx<double> e2 = 0.5 * (e1 * e1 - trX2);
  const cplx<double> e3 = X.m[0][0] * (X.m[1][1] * X.m[2][2] - X.m[1][2] * X.m[2][1]) -
                          X.m[0][1] * (X.m[1][0] * X.m[2][2] - X.m[1][2] * X.m[2][0]) +
                          X.m[0][2] * (X.m[1][0] * X.m[2][1] - X.m[1][1] * X.m[2][0]);
  // running term (a, b, c) = X^n / n! and the partial sums (f0, f1, f2)
  cplx<double> a = mk(0.0, 0.0), b = mk(1.0, 0.0), c = mk(0.0, 0.0);
  cplx<double> f0 = mk(1.0, 0.0), f1 = b, f2 = c;
  double term = nf;  // ||X||^n / n!
  for (int n = 1; n < 24 && term >= 1.3877787807814457e-17; ++n) {
    const double r = 1.0 / (n + 1);
    const cplx<double> a1 = r * (c * e3), b1 = r * (a - c * e2), c1 = r * (b + c * e1);
    a = a1;
    b = b1;
    c = c1;
    f0 = f0 + a;
    f1 = f1 + b;
    f2 = f2 + c;
    term *= nf * r;
  }
  Mat3<double> E;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      E.m[i][j] = f1 * X.m[i][j] + f2 * X2.m[i][j];
      if (i == j) E.m[i][j] = E.m[i][j] + f0;
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
