// Multi-shift CG with complex shifts and the Chebyshev polynomial filter.
//
// Multi-shift CG (the solver the paper pairs with the filter correction term, Sec. 3.1
// and App. C eq. force_polycorr): x_s = (K + sigma_s)^{-1} b for every shift from the
// Krylov space of the seed system K.  The shifted residuals stay collinear with the
// seed residual, r_s = zeta_s r, with the recurrences (Jegerlehner, hep-lat/9612014)
//   zeta_s' = zeta_s zeta_s^- a^- / [a^- zeta_s^- (1 + a sigma_s) + a b^- (zeta_s^- - zeta_s)]
//   alpha_s = a zeta_s' / zeta_s,  beta_s = b (zeta_s' / zeta_s)^2,
//   x_s += alpha_s p_s,  p_s = zeta_s' r + beta_s p_s,
// where a, b are the seed CG's alpha, beta and ^- marks the previous iteration.  All
// scalars live on the device: one CUDA graph-free loop of 6 kernels per iteration with
// no host round trip except a convergence check every `check` iterations.  FP64.
//
// Polynomial (App. A): P_n(K) v = a_n prod_{k=1}^{n} (K - z_k) v, roots
// z_k = mu (1 - cos t_k) - i sqrt(mu^2 - nu^2) sin t_k, t_k = 2 pi k/(n+1),
// a_n = 1/(mu prod_k (mu - z_k)); each factor is one K application and a complex axpby.
// R(K) = sqrt(a_n) prod_{Im z_k < 0} (K - z_k) (P = R^dag R for even n), R^dag with the
// conjugate roots.
#include <cmath>
#include <complex>
#include <vector>

#include "context.h"
#include "fields.cuh"

namespace pfmp {

struct MSShift {
  double2 sigma;
  double2 zeta_prev, zeta, zeta_next;
  double2 alpha, beta;
};
struct MSSeed {
  double alpha_prev, beta_prev;
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// zeta_next and alpha_s of every shift from the seed's alpha (just computed) and the
// previous alpha, beta
__global__ void k_ms_alpha(MSShift* sh, int ns, const CGScalars* s, const MSSeed* sd) {
  if (s->done) return;
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= ns) return;
  MSShift v = sh[i];
  const double a = s->alpha, ap = sd->alpha_prev, bp = sd->beta_prev;
  const double2 one_as = make_double2(1.0 + a * v.sigma.x, a * v.sigma.y);
  const double2 den = cadd(cs(ap, cm(v.zeta_prev, one_as)), cs(a * bp, csub(v.zeta_prev, v.zeta)));
  v.zeta_next = cdiv(cs(ap, cm(v.zeta, v.zeta_prev)), den);
  v.alpha = cs(a, cdiv(v.zeta_next, v.zeta));
  sh[i].zeta_next = v.zeta_next;
  sh[i].alpha = v.alpha;
}

// x_s += alpha_s p_s for all shifts
__global__ void k_ms_x(double2** x, double2* const* p, const MSShift* sh, int ns, long n, const CGScalars* s) {
  if (s->done) return;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    for (int k = 0; k < ns; ++k) {
      const double2 a = sh[k].alpha;
      double2 xx = x[k][i];
      const double2 pp = p[k][i];
      x[k][i] = cadd(xx, cm(a, pp));
    }
}

// seed residual r -= alpha Ap, |r|^2; finisher: beta, rr, iter, convergence (seed and all
// shifted residuals |zeta_s| |r| below stop), previous alpha/beta
__global__ void k_ms_r(double2* __restrict__ r, const double2* __restrict__ Ap, long n, ReduceBuf rb, CGScalars* s,
                       MSSeed* sd, const MSShift* sh, int ns) {
  if (s->done) return;
  const double al = s->alpha;
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 rr = r[i];
    const double2 aa = Ap[i];
    rr.x -= al * aa.x;
    rr.y -= al * aa.y;
    r[i] = rr;
    v[0] += rr.x * rr.x + rr.y * rr.y;
  }
  double t[1];
  if (grid_sum<1>(v, rb, t)) {
    const double beta = t[0] / s->rr;
    s->beta = beta;
    s->rr = t[0];
    s->iter += 1;
    sd->alpha_prev = al;
    sd->beta_prev = beta;
    bool conv = t[0] < s->stop_rr;
    for (int k = 0; k < ns && conv; ++k) {
      const double z2 = sh[k].zeta_next.x * sh[k].zeta_next.x + sh[k].zeta_next.y * sh[k].zeta_next.y;
      conv = z2 * t[0] < s->stop_rr;
    }
    if (conv || !(t[0] == t[0])) s->done_next = 1;
  }
}

// p_s = zeta_s' r + beta_s p_s, seed p = r + beta p; finisher rotates the zetas
__global__ void k_ms_p(double2* const* p, double2* pseed, const double2* __restrict__ r, MSShift* sh, int ns, long n,
                       ReduceBuf rb, CGScalars* s) {
  if (s->done) return;
  const double be = s->beta;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 rr = r[i];
    for (int k = 0; k < ns; ++k) {
      const double2 q = cdiv(sh[k].zeta_next, sh[k].zeta);
      const double2 bs = cs(be, cm(q, q));
      p[k][i] = cadd(cm(sh[k].zeta_next, rr), cm(bs, p[k][i]));
    }
    const double2 ps = pseed[i];
    pseed[i] = make_double2(rr.x + be * ps.x, rr.y + be * ps.y);
  }
  double v[1] = {0.0}, t[1];
  if (grid_sum<1>(v, rb, t)) {
    for (int k = 0; k < ns; ++k) {
      sh[k].zeta_prev = sh[k].zeta;
      sh[k].zeta = sh[k].zeta_next;
    }
    s->done = s->done_next;
  }
}

// y = a x + b y (complex a, b), FP64
__global__ void k_caxpby(double2 a, const double2* __restrict__ x, double2 b, double2* __restrict__ y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = cadd(cm(a, x[i]), cm(b, y[i]));
}

static int ms_grid(long n) {
  long b = (n + kBlock - 1) / kBlock;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

void caxpby(pfmp_ctx* c, std::complex<double> a, const void* x, std::complex<double> b, void* y) {
  const long n = 12L * c->g.Vh;
  k_caxpby<<<ms_grid(n), kBlock, 0, c->stream>>>(make_double2(a.real(), a.imag()), (const double2*)x,
                                                  make_double2(b.real(), b.imag()), (double2*)y, n);
  PFMP_CHECK_LAUNCH();
}

// per-operator workspace for the shifted search directions and device scalar arrays
struct MSWork {
  std::vector<double2*> p;
  double2** d_x = nullptr;
  double2** d_p = nullptr;
  MSShift* d_sh = nullptr;
  MSSeed* d_seed = nullptr;
  int cap = 0;
  ~MSWork() {
    for (auto q : p) dev_free(q);
    dev_free(d_x);
    dev_free(d_p);
    dev_free(d_sh);
    dev_free(d_seed);
  }
};

static MSWork& ms_work(pfmp_op* op, int ns) {
  if (!op->ms) op->ms = new MSWork();
  MSWork& w = *op->ms;
  if (w.cap < ns) {
    while ((int)w.p.size() < ns) w.p.push_back((double2*)dev_alloc(spinor_bytes(op->ctx->g, PFMP_F64)));
    dev_free(w.d_x);
    dev_free(w.d_p);
    dev_free(w.d_sh);
    w.d_x = (double2**)dev_alloc(ns * sizeof(double2*));
    w.d_p = (double2**)dev_alloc(ns * sizeof(double2*));
    w.d_sh = (MSShift*)dev_alloc(ns * sizeof(MSShift));
    if (!w.d_seed) w.d_seed = (MSSeed*)dev_alloc(sizeof(MSSeed));
    w.cap = ns;
  }
  return w;
}

void ms_work_free(pfmp_op* op) {
  delete op->ms;
  op->ms = nullptr;
}

// x[k] = (K + sigma_k)^{-1} b, FP64.  Returns iterations; true residuals optional.
int solve_multishift(pfmp_op* op, int ns, const std::complex<double>* sigma, void* const* x, const void* b, double tol,
                     int max_iter, int check, int* iters, double* max_true_res, long* kapply, bool want_true_res) {
  pfmp_ctx* c = op->ctx;
  PFMP_REQUIRE(ns >= 1 && ns <= 1024, PFMP_E_INVALID, "number of shifts must be in [1, 1024]");
  PFMP_REQUIRE(tol > 0 && max_iter > 0, PFMP_E_INVALID, "tol and max_iter must be positive");
  if (check <= 0) check = 8;
  MSWork& w = ms_work(op, ns);
  const size_t bytes = spinor_bytes(c->g, PFMP_F64);
  const long n = 12L * c->g.Vh;
  // |b|^2
  blas_norm2(c, PFMP_F64, b, c->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  const double bb = c->h_sums[0];
  *iters = 0;
  *kapply = 0;
  *max_true_res = 0;
  for (int k = 0; k < ns; ++k) blas_zero(c, PFMP_F64, x[k]);
  if (bb == 0.0) return PFMP_OK;
  PFMP_REQUIRE(std::isfinite(bb), PFMP_E_NAN, "right-hand side is not finite");
  void* r = op->cg64[0];
  void* pseed = op->cg64[1];
  void* Ap = op->cg64[2];
  PFMP_CUDA(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(pseed, b, bytes, cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double2*> hx(ns);
  std::vector<MSShift> hs(ns);
  for (int k = 0; k < ns; ++k) {
    hx[k] = (double2*)x[k];
    PFMP_CUDA(cudaMemcpyAsync(w.p[k], b, bytes, cudaMemcpyDeviceToDevice, c->stream));
    MSShift s{};
    s.sigma = make_double2(sigma[k].real(), sigma[k].imag());
    s.zeta_prev = s.zeta = s.zeta_next = make_double2(1.0, 0.0);
    hs[k] = s;
  }
  PFMP_CUDA(cudaMemcpyAsync(w.d_x, hx.data(), ns * sizeof(double2*), cudaMemcpyHostToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(w.d_p, w.p.data(), ns * sizeof(double2*), cudaMemcpyHostToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(w.d_sh, hs.data(), ns * sizeof(MSShift), cudaMemcpyHostToDevice, c->stream));
  MSSeed sd{1.0, 0.0};
  PFMP_CUDA(cudaMemcpyAsync(w.d_seed, &sd, sizeof(MSSeed), cudaMemcpyHostToDevice, c->stream));
  CGScalars* h = op->h_scal;
  *h = CGScalars{};
  h->rr = bb;
  h->stop_rr = tol * tol * bb;
  PFMP_CUDA(cudaMemcpyAsync(op->scal, h, sizeof(CGScalars), cudaMemcpyHostToDevice, c->stream));
  int done = 0;
  const long long kapply0 = op->kapply;  // queued iterations after convergence do no work
  while (done < max_iter) {
    const int chunk = check < max_iter - done ? check : max_iter - done;
    for (int k = 0; k < chunk; ++k) {
      kop(op, PFMP_F64, Ap, pseed, &op->scal->pAp, op->scal);
      k_ms_alpha<<<(ns + 127) / 128, 128, 0, c->stream>>>(w.d_sh, ns, op->scal, w.d_seed);
      PFMP_CHECK_LAUNCH();
      k_ms_x<<<ms_grid(n), kBlock, 0, c->stream>>>(w.d_x, w.d_p, w.d_sh, ns, n, op->scal);
      PFMP_CHECK_LAUNCH();
      k_ms_r<<<ms_grid(n), kBlock, 0, c->stream>>>((double2*)r, (const double2*)Ap, n, c->rb, op->scal, w.d_seed,
                                                    w.d_sh, ns);
      PFMP_CHECK_LAUNCH();
      k_ms_p<<<ms_grid(n), kBlock, 0, c->stream>>>(w.d_p, (double2*)pseed, (const double2*)r, w.d_sh, ns, n, c->rb,
                                                    op->scal);
      PFMP_CHECK_LAUNCH();
    }
    PFMP_CUDA(cudaMemcpyAsync(h, op->scal, sizeof(CGScalars), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    done = h->iter;
    PFMP_REQUIRE(std::isfinite(h->rr), PFMP_E_NAN, "multi-shift CG residual became NaN/Inf");
    if (h->done) break;
  }
  *iters = done;
  *kapply = done;
  op->kapply = kapply0 + done;
  if (want_true_res) {
    // || b - (K + sigma) x || / ||b|| for every shift, FP64
    for (int k = 0; k < ns; ++k) {
      kop(op, PFMP_F64, Ap, x[k], nullptr, nullptr);
      caxpby(c, sigma[k], x[k], 1.0, Ap);      // Ap = (K + sigma) x
      blas_xmy_norm(c, b, Ap, r, c->d_sums);
      PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      PFMP_CUDA(cudaStreamSynchronize(c->stream));
      const double res = std::sqrt(c->h_sums[0] / bb);
      if (res > *max_true_res) *max_true_res = res;
      *kapply += 1;
    }
  }
  return h->done ? PFMP_OK : PFMP_E_NOT_CONVERGED;
}

// ------------------------------------------------------------------ polynomial
std::vector<std::complex<double>> cheb_roots(int n, double mu, double nu) {
  std::vector<std::complex<double>> z(n);
  const double b = std::sqrt(mu * mu - nu * nu);
  for (int k = 1; k <= n; ++k) {
    const double t = 2.0 * M_PI * k / (n + 1);
    z[k - 1] = std::complex<double>(mu * (1.0 - std::cos(t)), -b * std::sin(t));
  }
  return z;
}
double cheb_norm(int n, double mu, double nu) {
  auto z = cheb_roots(n, mu, nu);
  std::complex<double> p = mu;
  for (auto zk : z) p *= (mu - zk);
  return (1.0 / p).real();
}

// out = scale * prod_k (K - z_k) in, factors applied in the given order; FP64
void poly_product(pfmp_op* op, const std::vector<std::complex<double>>& z, double scale, void* out, const void* in) {
  pfmp_ctx* c = op->ctx;
  const size_t bytes = spinor_bytes(c->g, PFMP_F64);
  void* w = op->cg64[2];
  PFMP_CUDA(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, c->stream));
  for (auto zk : z) {
    kop(op, PFMP_F64, w, out, nullptr, nullptr);   // w = K out
    caxpby(c, 1.0, w, -zk, out);                    // out = K out - z out
  }
  if (scale != 1.0) caxpby(c, 0.0, out, scale, out);
}

}  // namespace pfmp
