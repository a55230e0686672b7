// SU(3) helpers in FP64 shared by field initialisation and the link update: the
// exponential of an algebra element (scaling and squaring of the Taylor series, reduced
// to three scalar series by Cayley-Hamilton) and reunitarisation.
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

// exp(i H) for H = eps sum_a c_a lambda_a / 2 (Hermitian, traceless).  X = i H has
// tr X = 0, so Cayley-Hamilton gives X^3 = -e2 X + e3 with e2 = tr(H^2) / 2 (real) and
// e3 = det X = -i det H, and every Taylor term X^n / n! is a_n + b_n X + c_n X^2 with
//   (a, b, c)_{n+1} = (c_n e3, a_n - c_n e2, b_n) / (n + 1).
// The series runs in those three scalars until the last term's bound ||X||^n / n! is below
// 2^-56 (for ||X|| <= 1 it bounds the remainder too); exp(X) = f0 + i f1 H - f2 H^2 needs
// one Hermitian product H^2 (six entries) instead of one matrix product per order.  H is
// first scaled by 2^-s until ||H||_F <= 1 and the result squared s times; inside the MD
// ||eps P|| is well below 1.
__device__ inline Mat3<double> expm_algebra(const double c[8], double eps) {
  const double h = 0.5 * eps;
  const double s3 = 0.57735026918962576451;  // 1/sqrt(3)
  double hd[3] = {h * (c[2] + s3 * c[7]), h * (-c[2] + s3 * c[7]), h * (-2.0 * s3 * c[7])};
  cplx<double> h01 = mk(h * c[0], -h * c[1]), h02 = mk(h * c[3], -h * c[4]), h12 = mk(h * c[5], -h * c[6]);
  double q = hd[0] * hd[0] + hd[1] * hd[1] + hd[2] * hd[2] + 2.0 * (norm2(h01) + norm2(h02) + norm2(h12));
  double nf = sqrt(q);
  int s = 0;
  while (nf > 1.0 && s < 60) {
    nf *= 0.5;
    ++s;
  }
  if (s > 0) {
    const double sc = ldexp(1.0, -s);
    for (int k = 0; k < 3; ++k) hd[k] *= sc;
    h01 = sc * h01;
    h02 = sc * h02;
    h12 = sc * h12;
    q *= sc * sc;
  }
  // H^2 (Hermitian): diagonal and upper triangle
  const double n01 = norm2(h01), n02 = norm2(h02), n12 = norm2(h12);
  const double s00 = hd[0] * hd[0] + n01 + n02, s11 = hd[1] * hd[1] + n01 + n12, s22 = hd[2] * hd[2] + n02 + n12;
  const cplx<double> s01 = (hd[0] + hd[1]) * h01 + mul_cj(h02, h12);  // H01 (H00 + H11) + H02 H21
  const cplx<double> s02 = (hd[0] + hd[2]) * h02 + h01 * h12;          // H02 (H00 + H22) + H01 H12
  const cplx<double> s12 = (hd[1] + hd[2]) * h12 + cj_mul(h01, h02);   // H12 (H11 + H22) + H10 H02
  // det H = h00 h11 h22 + 2 Re(H01 H12 H20) - h00 |H12|^2 - h11 |H02|^2 - h22 |H01|^2
  const double d = hd[0] * hd[1] * hd[2] + 2.0 * mul_cj(h01 * h12, h02).re - hd[0] * n12 - hd[1] * n02 - hd[2] * n01;
  const double e2 = 0.5 * q;
  // running term (a, b, cc) = X^n / n! and the partial sums (f0, f1, f2); e3 = -i d
  cplx<double> a = mk(0.0, 0.0), b = mk(1.0, 0.0), cc = mk(0.0, 0.0);
  cplx<double> f0 = mk(1.0, 0.0), f1 = b, f2 = cc;
  double term = nf;  // ||X||^n / n!
  for (int n = 1; n < 24 && term >= 1.3877787807814457e-17; ++n) {
    const double r = 1.0 / (n + 1);
    const cplx<double> a1 = mk(r * d * cc.im, -r * d * cc.re);
    const cplx<double> b1 = mk(r * (a.re - e2 * cc.re), r * (a.im - e2 * cc.im));
    const cplx<double> c1 = r * b;
    a = a1;
    b = b1;
    cc = c1;
    f0 = f0 + a;
    f1 = f1 + b;
    f2 = f2 + cc;
    term *= nf * r;
  }
  // E = f0 + i f1 H - f2 H^2
  const cplx<double> g1 = times_i(f1);
  Mat3<double> E;
  E.m[0][0] = f0 + hd[0] * g1 - s00 * f2;
  E.m[1][1] = f0 + hd[1] * g1 - s11 * f2;
  E.m[2][2] = f0 + hd[2] * g1 - s22 * f2;
  E.m[0][1] = g1 * h01 - f2 * s01;
  E.m[1][0] = g1 * conj(h01) - f2 * conj(s01);
  E.m[0][2] = g1 * h02 - f2 * s02;
  E.m[2][0] = g1 * conj(h02) - f2 * conj(s02);
  E.m[1][2] = g1 * h12 - f2 * s12;
  E.m[2][1] = g1 * conj(h12) - f2 * conj(s12);
  for (int k = 0; k < s; ++k) E = matmul(E, E);
  return E;
}

}  // namespace pfmp
