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
// scalars live on the device (FP64); one iteration is K (the reduction finisher writes
// a), the per-shift scalars, the seed residual (whose finisher writes b, the per-shift
// coefficients and which shifts have converged), and ONE pass that updates x_s and p_s
// of every shift still running and the seed direction.  A shift whose residual
// |zeta_s| |r| is below tol |b| takes this iteration's x update and then stops: the
// large shifts of a Chebyshev filter converge in a fraction of the seed's iterations,
// and their vectors leave the memory traffic.  The loop ends when every shift has
// converged (the seed system itself need not be one of them).
//
// Vectors (solutions, directions, seed residual) are FP64, or FP32 for the solves inside
// the MD forces (K on the FP32 stencil, FP64 global sums and scalars): a deterministic
// force needs no FP64 solve, and the trajectory's end actions stay FP64.
//
// Polynomial (App. A): P_n(K) v = a_n prod_{k=1}^{n} (K - z_k) v, roots
// z_k = mu (1 - cos t_k) - i sqrt(mu^2 - nu^2) sin t_k, t_k = 2 pi k/(n+1),
// a_n = 1/(mu prod_k (mu - z_k)); each factor is one K application and a complex axpby.
// R(K) = sqrt(a_n) prod_{Im z_k < 0} (K - z_k) (P = R^dag R for even n), R^dag with the
// conjugate roots.  The factors commute; they are applied in bit-reversed index order
// (stable_order), which keeps every partial product within a few orders of magnitude of
// the final one (in index order the partial products of P_64 reach 1e11 times it, and
// the rounding of each factor is amplified accordingly).
#include <cmath>
#include <complex>
#include <vector>

#include "context.h"
#include "fields.cuh"

namespace pfmp {

struct MSShift {
  double2 sigma;
  double2 zeta_prev, zeta, zeta_next;
  double2 alpha;   // x_s += alpha p_s
  double2 beta;    // p_s = zeta_next r + beta p_s
  int active;      // takes part in this iteration
  int keep;        // still running after it (its direction is updated)
};
struct MSSeed {
  double alpha_prev, beta_prev;
  int nact;        // shifts active this iteration, listed in act[]
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// complex words of a vector field: double2 = one complex number, float4 = two
__device__ __forceinline__ double2 axpy_c(double2 a, double2 x, double2 y) { return cadd(y, cm(a, x)); }
__device__ __forceinline__ float4 axpy_c(double2 a, float4 x, float4 y) {
  const float ar = (float)a.x, ai = (float)a.y;
  return make_float4(y.x + ar * x.x - ai * x.y, y.y + ar * x.y + ai * x.x, y.z + ar * x.z - ai * x.w,
                     y.w + ar * x.w + ai * x.z);
}
// a x + b y
__device__ __forceinline__ double2 axpby_c(double2 a, double2 x, double2 b, double2 y) { return cadd(cm(a, x), cm(b, y)); }
__device__ __forceinline__ float4 axpby_c(double2 a, float4 x, double2 b, float4 y) {
  const float ar = (float)a.x, ai = (float)a.y, br = (float)b.x, bi = (float)b.y;
  return make_float4(ar * x.x - ai * x.y + br * y.x - bi * y.y, ar * x.y + ai * x.x + br * y.y + bi * y.x,
                     ar * x.z - ai * x.w + br * y.z - bi * y.w, ar * x.w + ai * x.z + br * y.w + bi * y.z);
}
__device__ __forceinline__ double2 sub_real(double2 r, double a, double2 q) { return make_double2(r.x - a * q.x, r.y - a * q.y); }
__device__ __forceinline__ float4 sub_real(float4 r, double ad, float4 q) {
  const float a = (float)ad;
  return make_float4(r.x - a * q.x, r.y - a * q.y, r.z - a * q.z, r.w - a * q.w);
}
__device__ __forceinline__ double nrm(double2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double nrm(float4 v) { return (double)(v.x * v.x + v.y * v.y) + (double)(v.z * v.z + v.w * v.w); }
__device__ __forceinline__ double2 xpby_real(double2 r, double b, double2 p) { return make_double2(r.x + b * p.x, r.y + b * p.y); }
__device__ __forceinline__ float4 xpby_real(float4 r, double bd, float4 p) {
  const float b = (float)bd;
  return make_float4(r.x + b * p.x, r.y + b * p.y, r.z + b * p.z, r.w + b * p.w);
}

// zeta_next and alpha_s of every active shift from the seed's alpha (just computed) and
// the previous alpha, beta
__global__ void k_ms_alpha(MSShift* sh, int ns, const CGScalars* s, const MSSeed* sd) {
  if (s->done) return;
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= ns || !sh[i].active) return;
  MSShift v = sh[i];
  const double a = s->alpha, ap = sd->alpha_prev, bp = sd->beta_prev;
  const double2 one_as = make_double2(1.0 + a * v.sigma.x, a * v.sigma.y);
  const double2 den = cadd(cs(ap, cm(v.zeta_prev, one_as)), cs(a * bp, csub(v.zeta_prev, v.zeta)));
  v.zeta_next = cdiv(cs(ap, cm(v.zeta, v.zeta_prev)), den);
  v.alpha = cs(a, cdiv(v.zeta_next, v.zeta));
  sh[i].zeta_next = v.zeta_next;
  sh[i].alpha = v.alpha;
}

// seed residual r -= alpha Ap, |r|^2; finisher: beta, rr, iter, the shifts' direction
// coefficients, which shifts keep running (|zeta_s'|^2 |r|^2 >= stop), done when none
template <typename V>
__global__ void k_ms_r(V* __restrict__ r, const V* __restrict__ Ap, long n, ReduceBuf rb, CGScalars* s, MSSeed* sd,
                       MSShift* sh, int ns) {
  if (s->done) return;
  const double al = s->alpha;
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const V rr = sub_real(r[i], al, Ap[i]);
    r[i] = rr;
    v[0] += nrm(rr);
  }
  double t[1];
  if (grid_sum<1>(v, rb, t)) {
    const double beta = t[0] / s->rr;
    s->beta = beta;
    s->rr = t[0];
    s->iter += 1;
    sd->alpha_prev = al;
    sd->beta_prev = beta;
    bool any = false;
    for (int k = 0; k < ns; ++k) {
      if (!sh[k].active) continue;
      const double2 q = cdiv(sh[k].zeta_next, sh[k].zeta);
      sh[k].beta = cs(beta, cm(q, q));
      const int keep = nrm(sh[k].zeta_next) * t[0] >= s->stop_rr;
      sh[k].keep = keep;
      any = any || keep;
    }
    if (!any || !(t[0] == t[0])) s->done_next = 1;
  }
}

// x_s += alpha_s p_s and p_s = zeta_s' r + beta_s p_s for the active shifts (the
// direction only for those that keep running), the seed p = r + beta p; the finisher
// rotates the zetas and the active set
template <typename V>
__global__ void k_ms_xp(V* const* x, V* const* p, V* __restrict__ pseed, const V* __restrict__ r, MSShift* sh,
                        int ns, const int* act, MSSeed* sd, long n, ReduceBuf rb, CGScalars* s) {
  if (s->done) return;
  const double be = s->beta;
  const int na = sd->nact;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const V rr = r[i];
    for (int j = 0; j < na; ++j) {
      const int k = act[j];
      const V pk = p[k][i];
      x[k][i] = axpy_c(sh[k].alpha, pk, x[k][i]);
      if (sh[k].keep) p[k][i] = axpby_c(sh[k].zeta_next, rr, sh[k].beta, pk);
    }
    pseed[i] = xpby_real(rr, be, pseed[i]);
  }
  double v[1] = {0.0}, t[1];
  if (grid_sum<1>(v, rb, t)) {
    int m = 0;
    int* a = const_cast<int*>(act);
    for (int k = 0; k < ns; ++k) {
      if (!sh[k].active) continue;
      sh[k].zeta_prev = sh[k].zeta;
      sh[k].zeta = sh[k].zeta_next;
      sh[k].active = sh[k].keep;
      if (sh[k].keep) a[m++] = k;
    }
    sd->nact = m;
    s->done = s->done_next;
  }
}

// y = a x + b y (complex a, b) on FP64 or FP32 even fields; with b = 0, y = a x without
// reading y (its previous contents may be anything, NaN included)
template <typename V>
__global__ void k_caxpby(double2 a, const V* __restrict__ x, double2 b, V* __restrict__ y, long n) {
  const bool read_y = b.x != 0.0 || b.y != 0.0;
  const double2 zero = make_double2(0.0, 0.0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = read_y ? axpby_c(a, x[i], b, y[i]) : axpby_c(a, x[i], zero, x[i]);
}

static int ms_grid(long n) {
  long b = (n + kBlock - 1) / kBlock;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}
static long words(const Geom& g, int prec) { return (prec == PFMP_F64 ? 12L : 6L) * g.Vh; }

void caxpby(pfmp_ctx* c, int prec, std::complex<double> a, const void* x, std::complex<double> b, void* y) {
  const long n = words(c->g, prec);
  const double2 da = make_double2(a.real(), a.imag()), db = make_double2(b.real(), b.imag());
  if (prec == PFMP_F64)
    k_caxpby<double2><<<ms_grid(n), kBlock, 0, c->stream>>>(da, (const double2*)x, db, (double2*)y, n);
  else
    k_caxpby<float4><<<ms_grid(n), kBlock, 0, c->stream>>>(da, (const float4*)x, db, (float4*)y, n);
  PFMP_CHECK_LAUNCH();
}
void caxpby(pfmp_ctx* c, std::complex<double> a, const void* x, std::complex<double> b, void* y) {
  caxpby(c, PFMP_F64, a, x, b, y);
}

// per-operator workspace for the shifted search directions and device scalar arrays
struct MSWork {
  std::vector<double2*> p;
  void** d_x = nullptr;
  void** d_p = nullptr;
  MSShift* d_sh = nullptr;
  MSSeed* d_seed = nullptr;
  int* d_act = nullptr;
  int cap = 0;
  ~MSWork() {
    for (auto q : p) dev_free(q);
    dev_free(d_x);
    dev_free(d_p);
    dev_free(d_sh);
    dev_free(d_seed);
    dev_free(d_act);
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
    dev_free(w.d_act);
    w.d_x = (void**)dev_alloc(ns * sizeof(void*));
    w.d_p = (void**)dev_alloc(ns * sizeof(void*));
    w.d_sh = (MSShift*)dev_alloc(ns * sizeof(MSShift));
    w.d_act = (int*)dev_alloc(ns * sizeof(int));
    if (!w.d_seed) w.d_seed = (MSSeed*)dev_alloc(sizeof(MSSeed));
    w.cap = ns;
  }
  return w;
}

void ms_work_free(pfmp_op* op) {
  delete op->ms;
  op->ms = nullptr;
}

template <typename V>
static void ms_iteration(pfmp_op* op, int prec, MSWork& w, int ns, void* r, void* pseed, void* Ap, long n) {
  pfmp_ctx* c = op->ctx;
  kop(op, prec, Ap, pseed, &op->scal->pAp, op->scal);
  k_ms_alpha<<<(ns + 127) / 128, 128, 0, c->stream>>>(w.d_sh, ns, op->scal, w.d_seed);
  PFMP_CHECK_LAUNCH();
  k_ms_r<V><<<ms_grid(n), kBlock, 0, c->stream>>>((V*)r, (const V*)Ap, n, c->rb, op->scal, w.d_seed, w.d_sh, ns);
  PFMP_CHECK_LAUNCH();
  k_ms_xp<V><<<ms_grid(n), kBlock, 0, c->stream>>>((V* const*)w.d_x, (V* const*)w.d_p, (V*)pseed, (const V*)r,
                                                   w.d_sh, ns, w.d_act, w.d_seed, n, c->rb, op->scal);
  PFMP_CHECK_LAUNCH();
}

// x[k] = (K + sigma_k)^{-1} b in FP64 or FP32 (x, b of precision prec).  Returns the
// status; iterations, K applications and (FP64, on request) the largest true residual.
int solve_multishift(pfmp_op* op, int prec, int ns, const std::complex<double>* sigma, void* const* x, const void* b,
                     double tol, int max_iter, int check, int* iters, double* max_true_res, long* kapply,
                     bool want_true_res) {
  pfmp_ctx* c = op->ctx;
  PFMP_REQUIRE(prec == PFMP_F64 || prec == PFMP_F32, PFMP_E_INVALID, "multi-shift CG: precision must be F64 or F32");
  PFMP_REQUIRE(ns >= 1 && ns <= 1024, PFMP_E_INVALID, "number of shifts must be in [1, 1024]");
  PFMP_REQUIRE(tol > 0 && max_iter > 0, PFMP_E_INVALID, "tol and max_iter must be positive");
  // K is Hermitian positive definite, so K + sigma is singular only for real sigma < 0
  // (at sigma = -lambda for an eigenvalue lambda of K); such shifts are refused
  for (int k = 0; k < ns; ++k) {
    PFMP_REQUIRE(std::isfinite(sigma[k].real()) && std::isfinite(sigma[k].imag()), PFMP_E_INVALID,
                 "multi-shift CG: a shift is not finite");
    PFMP_REQUIRE(!(sigma[k].imag() == 0.0 && sigma[k].real() < 0.0), PFMP_E_INVALID,
                 "multi-shift CG: a real negative shift can make K + sigma singular");
  }
  if (check <= 0) check = 8;
  MSWork& w = ms_work(op, ns);
  const size_t bytes = spinor_bytes(c->g, prec);
  const long n = words(c->g, prec);
  blas_norm2(c, prec, b, c->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  const double bb = c->h_sums[0];
  *iters = 0;
  *kapply = 0;
  *max_true_res = 0;
  for (int k = 0; k < ns; ++k) blas_zero(c, prec, x[k]);
  if (bb == 0.0) return PFMP_OK;
  PFMP_REQUIRE(std::isfinite(bb), PFMP_E_NAN, "right-hand side is not finite");
  void* r = prec == PFMP_F64 ? (void*)op->cg64[0] : (void*)op->cg32[0];
  void* pseed = prec == PFMP_F64 ? (void*)op->cg64[1] : (void*)op->cg32[1];
  void* Ap = prec == PFMP_F64 ? (void*)op->cg64[2] : (void*)op->cg32[2];
  PFMP_CUDA(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(pseed, b, bytes, cudaMemcpyDeviceToDevice, c->stream));
  std::vector<void*> hx(ns), hp(ns);
  std::vector<MSShift> hs(ns);
  std::vector<int> act(ns);
  for (int k = 0; k < ns; ++k) {
    hx[k] = x[k];
    hp[k] = w.p[k];
    act[k] = k;
    PFMP_CUDA(cudaMemcpyAsync(w.p[k], b, bytes, cudaMemcpyDeviceToDevice, c->stream));
    MSShift s{};
    s.sigma = make_double2(sigma[k].real(), sigma[k].imag());
    s.zeta_prev = s.zeta = s.zeta_next = make_double2(1.0, 0.0);
    s.active = s.keep = 1;
    hs[k] = s;
  }
  PFMP_CUDA(cudaMemcpyAsync(w.d_x, hx.data(), ns * sizeof(void*), cudaMemcpyHostToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(w.d_p, hp.data(), ns * sizeof(void*), cudaMemcpyHostToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(w.d_sh, hs.data(), ns * sizeof(MSShift), cudaMemcpyHostToDevice, c->stream));
  PFMP_CUDA(cudaMemcpyAsync(w.d_act, act.data(), ns * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  MSSeed sd{1.0, 0.0, ns};
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
      if (prec == PFMP_F64)
        ms_iteration<double2>(op, prec, w, ns, r, pseed, Ap, n);
      else
        ms_iteration<float4>(op, prec, w, ns, r, pseed, Ap, n);
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
  if (want_true_res && prec == PFMP_F64) {
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

// bit-reversed order of 0..n-1 (indices >= n skipped): a permutation that interleaves
// roots from all around the ellipse, so that no partial product is dominated by one
// side of it
std::vector<int> stable_order(int n) {
  int b = 0;
  while ((1 << b) < n) ++b;
  std::vector<int> o;
  for (int i = 0; i < (1 << b); ++i) {
    int r = 0;
    for (int k = 0; k < b; ++k)
      if (i & (1 << k)) r |= 1 << (b - 1 - k);
    if (r < n) o.push_back(r);
  }
  return o;
}

std::vector<std::complex<double>> stable_ordered(const std::vector<std::complex<double>>& z) {
  std::vector<std::complex<double>> o;
  for (int k : stable_order((int)z.size())) o.push_back(z[k]);
  return o;
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

// out = scale * prod_k (K - z_k) in, factors applied in the given order (callers pass
// stable_ordered lists); FP64
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
