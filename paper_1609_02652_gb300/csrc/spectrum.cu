// Extreme eigenvalues of K = M-hat^dag M-hat (or J) by the Lanczos recurrence.
//
// App. A: the Chebyshev filter approximates K^{-1} only inside its ellipse, which runs
// from 0 to 2 mu along the real axis, so (mu, nu) must be chosen with the spectrum
// [lambda_min, lambda_max] of K inside it.  The bounds come from Lanczos (Lanczos 1950):
//   beta_0 = 0, v_1 = s / |s|;  alpha_j = <v_j, K v_j>,
//   w = K v_j - alpha_j v_j - beta_{j-1} v_{j-1},  beta_j = |w|,  v_{j+1} = w / beta_j;
// the eigenvalues (Ritz values) of the tridiagonal T_k = tridiag(beta, alpha, beta) lie
// inside [lambda_min, lambda_max] and the extreme ones converge to the extreme
// eigenvalues first.  No reorthogonalisation: the loss of orthogonality only produces
// copies of converged Ritz values (Paige 1976), which leaves the extremes unchanged.
// FP64 throughout; the whole recurrence runs on the device (alpha_j from the reduction
// fused into K, beta_j from the update kernel), one host read at the end.  The extreme
// eigenvalues of T_k are found by Sturm-sequence bisection on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "context.h"

namespace pfmp {

// w -= alpha v + beta_prev vp; beta_out = |w|
__global__ void k_lanczos_w(double2* __restrict__ w, const double2* __restrict__ v, const double2* __restrict__ vp,
                            long n, const double* alpha, const double* beta_prev, ReduceBuf rb, double* beta_out) {
  const double a = *alpha, b = beta_prev ? *beta_prev : 0.0;
  double s[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 x = w[i];
    const double2 y = v[i];
    x.x -= a * y.x;
    x.y -= a * y.y;
    if (beta_prev) {
      const double2 z = vp[i];
      x.x -= b * z.x;
      x.y -= b * z.y;
    }
    w[i] = x;
    s[0] += x.x * x.x + x.y * x.y;
  }
  double t[1];
  if (grid_sum<1>(s, rb, t)) *beta_out = sqrt(t[0]);
}

// w /= beta (w = 0 when the Krylov space has closed, beta = 0)
__global__ void k_lanczos_scale(double2* __restrict__ w, long n, const double* beta) {
  const double b = *beta;
  const double f = b > 0.0 ? 1.0 / b : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 x = w[i];
    x.x *= f;
    x.y *= f;
    w[i] = x;
  }
}

static int lanczos_grid(long n) {
  long b = (n + kBlock - 1) / kBlock;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

// number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm sequence of
// the LDL^T pivots)
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double d = 1.0;
  const double tiny = 1e-300;
  for (size_t i = 0; i < a.size(); ++i) {
    const double off = i ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i ? off / d : 0.0);
    if (d == 0.0) d = -tiny;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// k-th smallest eigenvalue (0-based) of the tridiagonal by bisection
static double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
  double lo = a[0], hi = a[0];
  for (size_t i = 0; i < a.size(); ++i) {
    const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 4e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, mid) > k)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

void spectrum(pfmp_op* op, int nsteps, const void* v0, double* lmin, double* lmax, double* alpha_out,
              double* beta_out, int* steps) {
  pfmp_ctx* c = op->ctx;
  const Geom& g = c->g;
  const long n = 12L * g.Vh;
  const size_t bytes = spinor_bytes(g, PFMP_F64);
  double2* buf[3] = {nullptr, nullptr, nullptr};
  double* dab = nullptr;  // alpha[nsteps], beta[nsteps]
  try {
    for (auto& p : buf) p = (double2*)dev_alloc(bytes);
    dab = (double*)dev_alloc(2 * (size_t)nsteps * sizeof(double));
    // v_1 = s / |s|
    blas_norm2(c, PFMP_F64, v0, c->d_sums);
    double s2;
    PFMP_CUDA(cudaMemcpyAsync(&s2, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    PFMP_REQUIRE(s2 > 0 && std::isfinite(s2), PFMP_E_INVALID, "start vector must be non-zero and finite");
    blas_zero(c, PFMP_F64, buf[1]);
    caxpby(c, 1.0 / std::sqrt(s2), v0, 0.0, buf[1]);
    double2* vp = buf[0];
    double2* v = buf[1];
    double2* w = buf[2];
    double* alpha = dab;
    double* beta = dab + nsteps;
    for (int j = 0; j < nsteps; ++j) {
      kop(op, PFMP_F64, w, v, alpha + j, nullptr);
      k_lanczos_w<<<lanczos_grid(n), kBlock, 0, c->stream>>>(w, v, vp, n, alpha + j, j ? beta + j - 1 : nullptr,
                                                              c->rb, beta + j);
      PFMP_CHECK_LAUNCH();
      k_lanczos_scale<<<lanczos_grid(n), kBlock, 0, c->stream>>>(w, n, beta + j);
      PFMP_CHECK_LAUNCH();
      double2* t = vp;
      vp = v;
      v = w;
      w = t;
    }
    std::vector<double> ha(nsteps), hb(nsteps);
    PFMP_CUDA(cudaMemcpyAsync(ha.data(), alpha, nsteps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaMemcpyAsync(hb.data(), beta, nsteps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    // the Krylov space closes where beta_j vanishes (relative to the scale of T)
    double scale = 0;
    for (int j = 0; j < nsteps; ++j) scale = std::max(scale, std::fabs(ha[j]) + std::fabs(hb[j]));
    int k = nsteps;
    for (int j = 0; j < nsteps; ++j)
      if (!(hb[j] > 1e-13 * scale)) {
        k = j + 1;
        break;
      }
    for (int j = 0; j < k; ++j) PFMP_REQUIRE(std::isfinite(ha[j]) && std::isfinite(hb[j]), PFMP_E_NAN, "Lanczos NaN");
    std::vector<double> a(ha.begin(), ha.begin() + k), b(hb.begin(), hb.begin() + k);
    *lmin = tridiag_eig(a, b, 0);
    *lmax = tridiag_eig(a, b, k - 1);
    *steps = k;
    if (alpha_out) std::copy(ha.begin(), ha.begin() + k, alpha_out);
    if (beta_out) std::copy(hb.begin(), hb.begin() + k, beta_out);
  } catch (...) {
    for (auto p : buf) dev_free(p);
    dev_free(dab);
    throw;
  }
  for (auto p : buf) dev_free(p);
  dev_free(dab);
}

}  // namespace pfmp
