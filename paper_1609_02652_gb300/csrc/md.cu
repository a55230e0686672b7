// PF-MP action, heatbath, forces and the molecular-dynamics trajectory.
//
// Action (Sec. 2.5 eq. pfmp_action, with the Wilson gauge action and the even-odd clover
// determinant):
//   S = S_G + S_det + phi1^dag P(J) phi1 + phi2^dag [J P(J)]^{-1} phi2 + phi3^dag W K^{-1} W^dag phi3
//   S_G = beta sum_{x, mu<nu} (1 - Re tr U_{mu nu}/3),  S_det = -2 sum_{x odd} log det A(x),
//   K = M-hat^dag M-hat at kappa, J = W^dag W with W = M-hat at kappa' (same c_sw).
// Heatbath from Gaussian xi_i (density exp(-xi^dag xi)), so that S_i(phi_i) = xi_i^dag xi_i:
//   phi1 = R(J)^{-1} xi1,  phi2 = R(J)^dag W^dag xi2,  phi3 = W J^{-1} M-hat^dag xi3,
//   R(J) = sqrt(a_n) prod_{Im z_k<0} (J - z_k)  (P = R^dag R).
// Forces (App. C), as dS/d omega_a:
//   poly      F1 = sum_i Re eta_i^dag dJ chi_i, chi_i = a_n prod_{j>i}(J - z_j) phi1,
//             eta_i = prod_{j<i}(J - z_j^*) phi1  (eq. force_poly; 2n - 2 J products)
//   polycorr  F2 = -sum_{i<=n+1} Re eta-bar_i^dag dJ chi-bar_i, chi-bar_i = r_i (J - z_i)^{-1} phi2,
//             eta-bar_i = (J - z_i^*)^{-1} phi2, z_{n+1} = 0  (eq. force_polycorr, one multi-shift solve)
//   hasen     F3 = 2 Re chi^dag dW^dag phi3 - chi^dag dK chi, chi = K^{-1} W^dag phi3
//   det       dS_det = 2 kappa c_sw sum_x sum_{mu<nu} tr(dF_{mu nu} G), G = sum sigma A^{-1}
//   gauge     (beta/3) Im tr(T_a U S)
// Trajectory (Sec. 2.1, App. B): for each step of the merged schedule T-hat then the S-hat
// of every level with a non-zero step; Metropolis accept iff u < exp(-dH).
#include <cmath>
#include <complex>
#include <vector>

#include "context.h"
#include "fields.cuh"
#include "su3.cuh"

using cd = std::complex<double>;

namespace pfmp {

double plaquette(pfmp_ctx* c);
pfmp_op* op_new(pfmp_ctx* c, double kappa, double csw);
void op_delete(pfmp_op* op);
void spinor_unpack_any(pfmp_ctx* c, double* dst, int where, const void* src, int prec, int parity);
void spinor_pack_any(pfmp_ctx* c, void* dst, int prec, const double* src, int where, int parity);

// ------------------------------------------------------------------ kernels
__global__ void k_mom_update(double* __restrict__ p, const double* __restrict__ F, double eps, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] -= eps * F[i];
}

__global__ void k_sumsq(const double* __restrict__ p, long n, ReduceBuf rb, double* out) {
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) v[0] += p[i] * p[i];
  double t[1];
  if (grid_sum<1>(v, rb, t)) *out = t[0];
}

// U <- exp(i eps P) U, P = sum_a p_a T_a, then reunitarise (FP64 master field)
__global__ void k_link_update(double2* U, const double* __restrict__ mom, Geom g, double eps) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int pm = blockIdx.y;  // parity * 4 + mu
  if (cb >= g.Vh) return;
  double c[8];
  for (int a = 0; a < 8; ++a) c[a] = mom[(size_t)(pm * 8 + a) * g.Vh + cb];
  Mat3<double> E = expm3(i_algebra(c, eps));
  Mat3<double> L;
  double2* base = U + (size_t)(pm * 9) * g.Vh;
  load_link18(L, base, cb, g.Vh);
  Mat3<double> N = matmul(E, L);
  reunitarise(N);
  store_link18(base, N, cb, g.Vh);
}

// canonical [V][4][8] <-> device [2][4][8][Vh]
__global__ void k_alg_from_canonical(Geom g, const double* __restrict__ src, double* __restrict__ dst) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, p, x);
  const size_t s = lex_index(g, x);
  for (int mu = 0; mu < 4; ++mu)
    for (int a = 0; a < 8; ++a) dst[(size_t)((p * 4 + mu) * 8 + a) * g.Vh + cb] = src[(s * 4 + mu) * 8 + a];
}
__global__ void k_alg_to_canonical(Geom g, const double* __restrict__ src, double* __restrict__ dst) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, p, x);
  const size_t s = lex_index(g, x);
  for (int mu = 0; mu < 4; ++mu)
    for (int a = 0; a < 8; ++a) dst[(s * 4 + mu) * 8 + a] = src[(size_t)((p * 4 + mu) * 8 + a) * g.Vh + cb];
}

static int grid_for(long n) {
  long b = (n + kBlock - 1) / kBlock;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

}  // namespace pfmp

using namespace pfmp;

struct pfmp_action {
  pfmp_ctx* ctx = nullptr;
  pfmp_action_params prm{};
  pfmp_op* M = nullptr;  // kappa
  pfmp_op* W = nullptr;  // kappa'
  std::vector<cd> z;     // roots z_1..z_n
  double a_n = 0;
  std::vector<cd> sig;   // multi-shift shifts -z_i, i = 1..n+1 (z_{n+1} = 0)
  std::vector<cd> r;     // residues of 1/(z P(z))
  std::vector<int> conj_of;
  std::vector<cd> zh, sh;  // half roots (Im < 0) and residues of 1/prod(z - zh)
  double2* phi[3] = {nullptr, nullptr, nullptr};
  double* F = nullptr;    // [2][4][8][Vh]
  double* Hc = nullptr;   // [2][6][8][Vh]
  double* mom = nullptr;  // [2][4][8][Vh]
  double2* U0 = nullptr;  // saved master gauge field
  std::vector<double2*> ev;  // even FP64 temporaries
  std::vector<double2*> xs;  // multi-shift solutions
  double2* od[2] = {nullptr, nullptr};  // odd FP64 temporaries
  long long kapply0 = 0;
  int force_evals = 0;
};

namespace {

size_t spb(pfmp_action* A) { return spinor_bytes(A->ctx->g, PFMP_F64); }
void* E(pfmp_action* A, int i) { return A->ev[i]; }

void sync_read(pfmp_ctx* c, double* out, int n) {
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < n; ++i) out[i] = c->h_sums[i];
}

cd cdot(pfmp_ctx* c, const void* x, const void* y) {
  blas_cdot(c, PFMP_F64, x, y, c->d_sums);
  double v[2];
  sync_read(c, v, 2);
  return cd(v[0], v[1]);
}

void cg64(pfmp_action* A, pfmp_op* op, void* x, const void* b) {
  int it, rel;
  double res;
  long kap;
  int st = solve(op, PFMP_SOLVER_CG64, A->prm.tol, A->prm.max_iter, 0.1, 8, x, b, &it, &rel, &res, &kap);
  PFMP_REQUIRE(st == PFMP_OK, st, "CG inside the action did not converge");
}

void multishift(pfmp_action* A, pfmp_op* op, const std::vector<cd>& sig, const void* b) {
  while (A->xs.size() < sig.size()) A->xs.push_back((double2*)dev_alloc(spb(A)));
  std::vector<void*> x(sig.size());
  for (size_t k = 0; k < sig.size(); ++k) x[k] = A->xs[k];
  int it;
  double res;
  long kap;
  int st = solve_multishift(op, (int)sig.size(), sig.data(), x.data(), b, A->prm.tol, A->prm.max_iter, 8, &it, &res,
                            &kap, false);
  PFMP_REQUIRE(st == PFMP_OK, st, "multi-shift CG inside the action did not converge");
}

// Re eta^dag dK chi (coef) -> F, Hc for the operator op (K or J)
void deriv_K(pfmp_action* A, pfmp_op* op, const void* eta, const void* chi, double coef) {
  void* Mchi = E(A, 6);
  void* Meta = E(A, 7);
  mhat(op, PFMP_F64, Mchi, chi, false, nullptr, nullptr);
  mhat(op, PFMP_F64, Meta, eta, false, nullptr, nullptr);
  deriv_mhat(op, A->F, A->Hc, Mchi, eta, coef, A->od[0], A->od[1]);
  deriv_mhat(op, A->F, A->Hc, Meta, chi, coef, A->od[0], A->od[1]);
}

void refresh_ops(pfmp_action* A) {
  clover_build(A->M);
  clover_build(A->W);
}

}  // namespace

namespace pfmp {

void action_destroy(pfmp_action* A) {
  if (!A) return;
  cudaStreamSynchronize(A->ctx->stream);
  for (auto p : A->phi) dev_free(p);
  dev_free(A->F);
  dev_free(A->Hc);
  dev_free(A->mom);
  dev_free(A->U0);
  for (auto p : A->ev) dev_free(p);
  for (auto p : A->xs) dev_free(p);
  for (auto p : A->od) dev_free(p);
  op_delete(A->M);
  op_delete(A->W);
  delete A;
}

pfmp_action* action_create(pfmp_ctx* c, const pfmp_action_params* prm) {
  PFMP_REQUIRE(prm->n >= 2 && prm->n % 2 == 0, PFMP_E_UNSUPPORTED, "polynomial order must be even and >= 2");
  PFMP_REQUIRE(prm->mu >= prm->nu && prm->nu > 0, PFMP_E_INVALID, "need mu >= nu > 0");
  PFMP_REQUIRE(prm->tol > 0 && prm->max_iter > 0, PFMP_E_INVALID, "bad solver tolerance / iteration cap");
  pfmp_action* A = new pfmp_action();
  A->ctx = c;
  A->prm = *prm;
  try {
    A->M = op_new(c, prm->kappa, prm->csw);
    A->W = op_new(c, prm->kappa_h, prm->csw);
    const int n = prm->n;
    A->z = cheb_roots(n, prm->mu, prm->nu);
    A->a_n = cheb_norm(n, prm->mu, prm->nu);
    std::vector<cd> zz = A->z;
    zz.push_back(0.0);
    for (int i = 0; i <= n; ++i) {
      cd prod = A->a_n;
      for (int j = 0; j <= n; ++j)
        if (j != i) prod *= (zz[i] - zz[j]);
      A->r.push_back(1.0 / prod);
      A->sig.push_back(-zz[i]);
      int best = 0;
      for (int j = 0; j <= n; ++j)
        if (std::abs(zz[j] - std::conj(zz[i])) < std::abs(zz[best] - std::conj(zz[i]))) best = j;
      A->conj_of.push_back(best);
    }
    for (auto zk : A->z)
      if (zk.imag() < 0) A->zh.push_back(zk);
    for (size_t i = 0; i < A->zh.size(); ++i) {
      cd prod = 1.0;
      for (size_t j = 0; j < A->zh.size(); ++j)
        if (j != i) prod *= (A->zh[i] - A->zh[j]);
      A->sh.push_back(1.0 / prod);
    }
    const Geom& g = c->g;
    for (auto& p : A->phi) p = (double2*)dev_alloc(spb(A));
    A->F = (double*)dev_alloc((size_t)g.Vh * 64 * sizeof(double));
    A->Hc = (double*)dev_alloc((size_t)g.Vh * 96 * sizeof(double));
    A->mom = (double*)dev_alloc((size_t)g.Vh * 64 * sizeof(double));
    A->U0 = (double2*)dev_alloc((size_t)g.Vh * 72 * sizeof(double2));
    for (int i = 0; i < 8; ++i) A->ev.push_back((double2*)dev_alloc(spb(A)));
    for (auto& p : A->od) p = (double2*)dev_alloc(spb(A));
  } catch (...) {
    action_destroy(A);
    throw;
  }
  return A;
}

// phi_i from the noise xi_i (even FP64 device fields)
void action_heatbath(pfmp_action* A, const void* xi1, const void* xi2, const void* xi3) {
  pfmp_ctx* c = A->ctx;
  // phi1 = a_n^{-1/2} sum_k s_k (J - zh_k)^{-1} xi1
  std::vector<cd> sig;
  for (auto zk : A->zh) sig.push_back(-zk);
  multishift(A, A->W, sig, xi1);
  blas_zero(c, PFMP_F64, A->phi[0]);
  for (size_t k = 0; k < A->zh.size(); ++k) caxpby(c, A->sh[k] / std::sqrt(A->a_n), A->xs[k], 1.0, A->phi[0]);
  // phi2 = R(J)^dag W^dag xi2
  mhat(A->W, PFMP_F64, E(A, 0), xi2, true, nullptr, nullptr);
  std::vector<cd> zc;
  for (auto zk : A->zh) zc.push_back(std::conj(zk));
  poly_product(A->W, zc, std::sqrt(A->a_n), A->phi[1], E(A, 0));
  // phi3 = W J^{-1} M-hat^dag xi3
  mhat(A->M, PFMP_F64, E(A, 0), xi3, true, nullptr, nullptr);
  cg64(A, A->W, E(A, 1), E(A, 0));
  mhat(A->W, PFMP_F64, A->phi[2], E(A, 1), false, nullptr, nullptr);
}

void action_eval(pfmp_action* A, double S[5]) {
  pfmp_ctx* c = A->ctx;
  S[PFMP_TERM_GAUGE] = A->prm.beta * 6.0 * c->g.V * (1.0 - plaquette(c));
  S[PFMP_TERM_DET] = A->prm.csw != 0.0 ? -2.0 * A->M->logdet_oo : 0.0;
  // S1 = phi1^dag P(J) phi1
  poly_product(A->W, A->z, A->a_n, E(A, 0), A->phi[0]);
  S[PFMP_TERM_POLY] = cdot(c, A->phi[0], E(A, 0)).real();
  // S2 = sum_i r_i phi2^dag (J - z_i)^{-1} phi2
  multishift(A, A->W, A->sig, A->phi[1]);
  cd s2 = 0.0;
  for (size_t i = 0; i < A->sig.size(); ++i) s2 += A->r[i] * cdot(c, A->phi[1], A->xs[i]);
  S[PFMP_TERM_POLYCORR] = s2.real();
  // S3 = w^dag K^{-1} w, w = W^dag phi3
  mhat(A->W, PFMP_F64, E(A, 0), A->phi[2], true, nullptr, nullptr);
  cg64(A, A->M, E(A, 1), E(A, 0));
  S[PFMP_TERM_HASEN] = cdot(c, E(A, 0), E(A, 1)).real();
}

// F += dS_term/d omega (F must be zeroed by the caller for a fresh force)
void action_force(pfmp_action* A, int term) {
  pfmp_ctx* c = A->ctx;
  const Geom& g = c->g;
  A->force_evals++;
  if (term == PFMP_TERM_GAUGE) {
    gauge_force(c, A->F, A->prm.beta);
    return;
  }
  PFMP_CUDA(cudaMemsetAsync(A->Hc, 0, (size_t)g.Vh * 96 * sizeof(double), c->stream));
  bool clover = A->prm.csw != 0.0;
  if (term == PFMP_TERM_DET) {
    if (!clover) return;
    clover_insert_det(A->M, A->Hc, 2.0 * A->M->kappa * A->M->csw);
  } else if (term == PFMP_TERM_POLY) {
    const int n = A->prm.n;
    // chi_i, i = n-1 .. 0 (0-based): chi[n-1] = a_n phi1, chi[i] = (J - z_{i+1}) chi[i+1]
    while ((int)A->xs.size() < n) A->xs.push_back((double2*)dev_alloc(spb(A)));
    caxpby(c, A->a_n, A->phi[0], 0.0, A->xs[n - 1]);
    for (int i = n - 2; i >= 0; --i) {
      kop(A->W, PFMP_F64, A->xs[i], A->xs[i + 1], nullptr, nullptr);
      caxpby(c, -A->z[i + 1], A->xs[i + 1], 1.0, A->xs[i]);
    }
    // eta_0 = phi1, eta_i = (J - z_{i-1}^*) eta_{i-1}
    void* eta = E(A, 2);
    void* tmp = E(A, 3);
    PFMP_CUDA(cudaMemcpyAsync(eta, A->phi[0], spb(A), cudaMemcpyDeviceToDevice, c->stream));
    for (int i = 0; i < n; ++i) {
      if (i > 0) {
        kop(A->W, PFMP_F64, tmp, eta, nullptr, nullptr);
        caxpby(c, 1.0, tmp, -std::conj(A->z[i - 1]), eta);
      }
      deriv_K(A, A->W, eta, A->xs[i], 1.0);
    }
  } else if (term == PFMP_TERM_POLYCORR) {
    multishift(A, A->W, A->sig, A->phi[1]);
    void* chib = E(A, 2);
    for (size_t i = 0; i < A->sig.size(); ++i) {
      caxpby(c, A->r[i], A->xs[i], 0.0, chib);
      deriv_K(A, A->W, A->xs[A->conj_of[i]], chib, -1.0);
    }
  } else if (term == PFMP_TERM_HASEN) {
    mhat(A->W, PFMP_F64, E(A, 0), A->phi[2], true, nullptr, nullptr);
    void* chi = E(A, 1);
    cg64(A, A->M, chi, E(A, 0));
    // 2 Re chi^dag dW^dag phi3 = 2 Re phi3^dag dW chi
    deriv_mhat(A->W, A->F, A->Hc, A->phi[2], chi, 2.0, A->od[0], A->od[1]);
    deriv_K(A, A->M, chi, chi, -1.0);
  } else {
    PFMP_REQUIRE(false, PFMP_E_INVALID, "unknown action term");
  }
  if (clover) clover_force(c, A->F, A->Hc);
}

void action_zero_force(pfmp_action* A) {
  PFMP_CUDA(cudaMemsetAsync(A->F, 0, (size_t)A->ctx->g.Vh * 64 * sizeof(double), A->ctx->stream));
}

void alg_pack(pfmp_ctx* c, double* dst_dev, const double* src, int where) {
  const double* s = src;
  double* buf = nullptr;
  if (where == PFMP_HOST) {
    buf = (double*)dev_alloc((size_t)c->g.V * 32 * sizeof(double));
    PFMP_CUDA(cudaMemcpyAsync(buf, src, (size_t)c->g.V * 32 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    s = buf;
  }
  dim3 grid(nblocks(c->g.Vh), 2);
  k_alg_from_canonical<<<grid, kBlock, 0, c->stream>>>(c->g, s, dst_dev);
  PFMP_CHECK_LAUNCH();
  if (buf) {
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    dev_free(buf);
  }
}

void alg_unpack(pfmp_ctx* c, double* dst, int where, const double* src_dev) {
  double* d = dst;
  double* buf = nullptr;
  if (where == PFMP_HOST) {
    buf = (double*)dev_alloc((size_t)c->g.V * 32 * sizeof(double));
    d = buf;
  }
  dim3 grid(nblocks(c->g.Vh), 2);
  k_alg_to_canonical<<<grid, kBlock, 0, c->stream>>>(c->g, src_dev, d);
  PFMP_CHECK_LAUNCH();
  if (buf) {
    PFMP_CUDA(cudaMemcpyAsync(dst, buf, (size_t)c->g.V * 32 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    dev_free(buf);
  }
}

void action_force_out(pfmp_action* A, int term, double* out, int where) {
  action_zero_force(A);
  action_force(A, term);
  alg_unpack(A->ctx, out, where, A->F);
}

double kinetic(pfmp_action* A) {
  pfmp_ctx* c = A->ctx;
  const long n = 64L * c->g.Vh;
  k_sumsq<<<grid_for(n), kBlock, 0, c->stream>>>(A->mom, n, c->rb, c->d_sums);
  PFMP_CHECK_LAUNCH();
  double v;
  sync_read(c, &v, 1);
  return 0.5 * v;
}

void link_update(pfmp_action* A, double eps) {
  pfmp_ctx* c = A->ctx;
  dim3 grid(nblocks(c->g.Vh, 128), 8);
  k_link_update<<<grid, 128, 0, c->stream>>>(c->U64, A->mom, c->g, eps);
  PFMP_CHECK_LAUNCH();
  gauge_refresh_compressed(c);
  refresh_ops(A);
}

void mom_update(pfmp_action* A, double eps) {
  pfmp_ctx* c = A->ctx;
  const long n = 64L * c->g.Vh;
  k_mom_update<<<grid_for(n), kBlock, 0, c->stream>>>(A->mom, A->F, eps, n);
  PFMP_CHECK_LAUNCH();
}

void trajectory(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int term_level[5],
                const double* mom, int where, const void* const xi[3], double u, pfmp_traj_info* info) {
  pfmp_ctx* c = A->ctx;
  const Geom& g = c->g;
  PFMP_REQUIRE(len >= 1 && nlev >= 1, PFMP_E_INVALID, "empty schedule");
  for (int t = 0; t < 5; ++t)
    PFMP_REQUIRE(term_level[t] >= -1 && term_level[t] < nlev, PFMP_E_INVALID, "term level out of range");
  const long long k0 = A->M->kapply + A->W->kapply;
  A->force_evals = 0;
  PFMP_CUDA(cudaMemcpyAsync(A->U0, c->U64, (size_t)g.Vh * 72 * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  if (A->M->built_version != c->gauge_version || A->W->built_version != c->gauge_version) refresh_ops(A);
  alg_pack(c, A->mom, mom, where);
  action_heatbath(A, xi[0], xi[1], xi[2]);
  double S0[5], S1[5];
  action_eval(A, S0);
  double H0 = kinetic(A);
  for (int t = 0; t < 5; ++t)
    if (term_level[t] >= 0) H0 += S0[t];
  for (int i = 0; i < len; ++i) {
    if (T[i] != 0.0) link_update(A, T[i]);
    for (int l = 0; l < nlev; ++l) {
      const double eps = S[(size_t)l * len + i];
      if (eps == 0.0) continue;
      action_zero_force(A);
      for (int t = 0; t < 5; ++t)
        if (term_level[t] == l) action_force(A, t);
      mom_update(A, eps);
    }
  }
  action_eval(A, S1);
  double H1 = kinetic(A);
  for (int t = 0; t < 5; ++t)
    if (term_level[t] >= 0) H1 += S1[t];
  const double dH = H1 - H0;
  PFMP_REQUIRE(std::isfinite(dH), PFMP_E_NAN, "dH is not finite");
  const bool acc = u < std::exp(-dH);
  info->H0 = H0;
  info->H1 = H1;
  info->dH = dH;
  info->accepted = acc ? 1 : 0;
  for (int t = 0; t < 5; ++t) {
    info->S0[t] = term_level[t] >= 0 ? S0[t] : 0.0;
    info->S1[t] = term_level[t] >= 0 ? S1[t] : 0.0;
  }
  info->k_apply = A->M->kapply + A->W->kapply - k0;
  info->force_evals = A->force_evals;
  if (!acc) {
    PFMP_CUDA(cudaMemcpyAsync(c->U64, A->U0, (size_t)g.Vh * 72 * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    gauge_refresh_compressed(c);
    refresh_ops(A);
  }
  info->plaquette = plaquette(c);
}

// ------------------------------------------------------------------ schedules (host)
void schedule_2mn(int n, double tau, double lam, double* T, double* S) {
  const double h = tau / n;
  T[0] = 0.0;
  for (int k = 1; k <= 2 * n; ++k) T[k] = h / 2;
  S[0] = lam * h;
  for (int k = 0; k < n; ++k) {
    S[1 + 2 * k] = (1 - 2 * lam) * h;
    S[2 + 2 * k] = k < n - 1 ? 2 * lam * h : lam * h;
  }
}

// the generalised multi-scale merge (App. B): take the smallest pending time step, emit
// it with the space step of every scheme it completes (0 for the others), shorten the
// others' pending time steps; equality of time steps within eps * (sum of steps)
int schedule_merge(int ns, const int* len, const double* T, const double* S, int cap, double* Tout, double* Sout) {
  std::vector<std::vector<double>> t(ns), s(ns);
  size_t off = 0;
  double tot = 0;
  for (int i = 0; i < ns; ++i) {
    t[i].assign(T + off, T + off + len[i]);
    s[i].assign(S + off, S + off + len[i]);
    off += len[i];
    double sum = 0;
    for (double v : t[i]) sum += v;
    tot = std::max(tot, sum);
  }
  const double eps = 1e-12 * (tot > 0 ? tot : 1.0);
  std::vector<size_t> head(ns, 0);
  int m = 0;
  for (;;) {
    bool any = false;
    double d = 0;
    for (int i = 0; i < ns; ++i)
      if (head[i] < t[i].size()) {
        d = any ? std::min(d, t[i][head[i]]) : t[i][head[i]];
        any = true;
      }
    if (!any) break;
    PFMP_REQUIRE(m < cap, PFMP_E_INVALID, "merged schedule longer than the output capacity");
    Tout[m] = d;
    for (int i = 0; i < ns; ++i) {
      if (head[i] < t[i].size() && std::abs(t[i][head[i]] - d) <= eps) {
        Sout[(size_t)i * cap + m] = s[i][head[i]];
        head[i]++;
      } else {
        Sout[(size_t)i * cap + m] = 0.0;
        if (head[i] < t[i].size()) t[i][head[i]] -= d;
      }
    }
    ++m;
  }
  return m;
}

void action_get_phi(pfmp_action* A, int i, double* out, int where) {
  PFMP_REQUIRE(i >= 0 && i < 3, PFMP_E_INVALID, "pseudofermion index must be 0, 1 or 2");
  spinor_unpack_any(A->ctx, out, where, A->phi[i], PFMP_F64, 0);
}

void action_set_phi(pfmp_action* A, int i, const double* in, int where) {
  PFMP_REQUIRE(i >= 0 && i < 3, PFMP_E_INVALID, "pseudofermion index must be 0, 1 or 2");
  spinor_pack_any(A->ctx, A->phi[i], PFMP_F64, in, where, 0);
}

void action_refresh(pfmp_action* A) { refresh_ops(A); }
pfmp_ctx* action_ctx(pfmp_action* A) { return A->ctx; }

}  // namespace pfmp
