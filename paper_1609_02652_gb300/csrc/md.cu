// Actions, heatbath, forces and the molecular-dynamics trajectory.
//
// An action is a list of terms over hopping parameters kappa[0..] sharing c_sw (Sec. 2.2
// eq. hasenbusch, Sec. 2.3 eqs. 1poly/2poly, Sec. 2.5 eq. pfmp_action, Sec. 3.6):
//   GAUGE       S_G = beta sum_{x, mu<nu} (1 - Re tr U_{mu nu}/3)
//   DET         S_det = -2 sum_{x odd} log det A(x) at kappa[a]
//   FILTER      phi^dag Q(J_a) phi, Q = P_p2 / P_p1 = c prod_k (J_a - q_k)  (App. A factorisation)
//   FILTERCORR  phi^dag [J_a P_p2(J_a)]^{-1} phi = sum_i r_i phi^dag (J_a - z_i)^{-1} phi, z_{p2+1} = 0
//   RATIO       phi^dag W_a K_b^{-1} W_a^dag phi    (the Hermitian form of "J_a K_b^{-1}")
//   INV         phi^dag J_a^{-1} phi
// with K_b = M_b^dag M_b, J_a = W_a^dag W_a, M_b and W_a the even-odd M-hat at kappa[b], kappa[a].
// Heatbath from Gaussian xi (density exp(-xi^dag xi)), so that S_i(phi_i) = xi_i^dag xi_i:
//   FILTER phi = c^{-1/2} sum_k s_k (J_a - qh_k)^{-1} xi  (qh: roots with Im < 0, s_k the
//   residues of 1/prod(z - qh_k)),  FILTERCORR phi = R_p2(J_a)^dag W_a^dag xi,
//   RATIO phi = W_a J_a^{-1} M_b^dag xi,  INV phi = W_a^dag xi.
// Forces (App. C), as dS/d omega_a:
//   FILTER      sum_i Re eta_i^dag dJ chi_i, chi_i = c prod_{j>i}(J - q_j) phi,
//               eta_i = prod_{j<i}(J - q_j^*) phi  (eq. force_poly; 2q - 2 J products)
//   FILTERCORR  -sum_i Re eta-bar_i^dag dJ chi-bar_i, chi-bar_i = r_i (J - z_i)^{-1} phi,
//               eta-bar_i = (J - z_i^*)^{-1} phi  (eq. force_polycorr, one multi-shift solve)
//   RATIO       2 Re chi^dag dW_a^dag phi - chi^dag dK_b chi, chi = K_b^{-1} W_a^dag phi
//   INV         -chi^dag dJ_a chi, chi = J_a^{-1} phi
//   DET         2 kappa c_sw sum_x sum_{mu<nu} tr(dF_{mu nu} G), G = sum sigma A^{-1}
//   GAUGE       (beta/3) Im tr(T_a U S)
// Trajectory (Sec. 2.1, App. B): for each step of the merged schedule T-hat then the S-hat
// of every level with a non-zero step; Metropolis accept iff u < exp(-dH).
#include <algorithm>
#include <chrono>
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
  Mat3<double> E = expm_algebra(c, eps);
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

// per-link force norm |F_mu(x)| = sqrt(sum_a f_a^2) (F: [2][4][8][Vh]): out[0] = sum over
// links (deterministic grid sum), *maxbits = max over links (the bit patterns of
// non-negative doubles order like the values, so an integer atomicMax is exact and
// independent of scheduling); *maxbits must be zero on entry
__global__ void k_force_norm(const double* __restrict__ F, int Vh, ReduceBuf rb, double* out,
                             unsigned long long* maxbits) {
  double v[1] = {0.0};
  double mx = 0.0;
  const long nl = 8L * Vh;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nl; i += (long)gridDim.x * blockDim.x) {
    const long pm = i / Vh, cb = i - pm * Vh;
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double f = F[(size_t)(pm * 8 + a) * Vh + cb];
      s += f * f;
    }
    const double n = sqrt(s);
    v[0] += n;
    mx = fmax(mx, n);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(mx));
  double t[1];
  if (grid_sum<1>(v, rb, t)) out[0] = t[0];
}

}  // namespace pfmp

using namespace pfmp;

namespace {
struct Term {
  pfmp_term d{};
  int pf = -1;                   // pseudofermion index (fermion terms)
  std::vector<cd> q;             // FILTER: roots of Q, Q = c prod (z - q_k)
  double c = 0;
  std::vector<cd> qh, sh;        // FILTER: roots with Im < 0, residues of 1/prod(z - qh_k)
  std::vector<cd> sig, r;        // FILTERCORR: shifts -z_i (z_{p+1} = 0), residues of 1/(z P(z))
  std::vector<int> conj_of;      // FILTERCORR: index of the conjugate shift
  std::vector<cd> zh;            // FILTERCORR: roots of P_p with Im < 0 (heatbath R)
  double a_p = 0;
};
bool is_fermion(int kind) {
  return kind == PFMP_KIND_FILTER || kind == PFMP_KIND_FILTERCORR || kind == PFMP_KIND_RATIO || kind == PFMP_KIND_INV;
}
}  // namespace

struct pfmp_action {
  pfmp_ctx* ctx = nullptr;
  pfmp_action_def def{};
  std::vector<pfmp_op*> ops;  // one per kappa
  std::vector<Term> t;
  std::vector<double2*> phi;  // one per fermion term
  double* F = nullptr;    // [2][4][8][Vh]
  double* Hc = nullptr;   // [2][6][8][Vh]
  double* mom = nullptr;  // [2][4][8][Vh]
  double2* U0 = nullptr;  // saved master gauge field
  std::vector<double2*> ev;  // even FP64 temporaries
  std::vector<double2*> xs;  // multi-shift solutions
  // FP32 force path (force_prec = PFMP_F32): even temporaries, solutions and filter
  // chains
  std::vector<float4*> ev32;
  std::vector<float4*> xs32;
  // half-lattice scratch of the batched force contractions, FP64 [0] and FP32 [1]
  std::vector<void*> fbuf[2];
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

bool f32_forces(pfmp_action* A) { return A->def.force_prec == PFMP_F32; }
// relative residual of the solves inside the MD forces
double md_tol(pfmp_action* A) { return A->def.md_tol > 0 ? A->def.md_tol : A->def.tol; }
float4* E32(pfmp_action* A, int i) {
  while ((int)A->ev32.size() <= i) A->ev32.push_back((float4*)dev_alloc(spinor_bytes(A->ctx->g, PFMP_F32)));
  return A->ev32[i];
}

// the action's CG: FP64, or mixed (FP32 iterations with reliable updates, FP64-accurate
// true residual) when the action was created with PFMP_SOLVER_CG_MIXED
void cg_tol(pfmp_action* A, pfmp_op* op, void* x, const void* b, double tol) {
  int it, rel;
  double res;
  long kap;
  const bool mixed = A->def.solver == PFMP_SOLVER_CG_MIXED;
  int st = solve(op, mixed ? PFMP_SOLVER_CG_MIXED : PFMP_SOLVER_CG64, tol, A->def.max_iter, mixed ? 1e-4 : 0.1, 8, x,
                 b, &it, &rel, &res, &kap);
  PFMP_REQUIRE(st == PFMP_OK, st, "CG inside the action did not converge");
}
void cg64(pfmp_action* A, pfmp_op* op, void* x, const void* b) { cg_tol(A, op, x, b, A->def.tol); }

// multi-shift solutions into A->xs (FP64, at the action's tolerance) or A->xs32 (FP32,
// at the MD tolerance: the solves of the FP32 forces)
void multishift(pfmp_action* A, pfmp_op* op, const std::vector<cd>& sig, const void* b, int prec = PFMP_F64) {
  std::vector<void*> x(sig.size());
  if (prec == PFMP_F64) {
    while (A->xs.size() < sig.size()) A->xs.push_back((double2*)dev_alloc(spb(A)));
    for (size_t k = 0; k < sig.size(); ++k) x[k] = A->xs[k];
  } else {
    while (A->xs32.size() < sig.size()) A->xs32.push_back((float4*)dev_alloc(spinor_bytes(A->ctx->g, PFMP_F32)));
    for (size_t k = 0; k < sig.size(); ++k) x[k] = A->xs32[k];
  }
  int it;
  double res;
  long kap;
  const double tol = prec == PFMP_F64 ? A->def.tol : md_tol(A);
  int st = solve_multishift(op, prec, (int)sig.size(), sig.data(), x.data(), b, tol, A->def.max_iter, 8, &it, &res,
                            &kap, false);
  PFMP_REQUIRE(st == PFMP_OK, st, "multi-shift CG inside the action did not converge");
}

// half-lattice scratch field i of the force batches in precision prec
void* fscratch(pfmp_action* A, int prec, int i) {
  auto& v = A->fbuf[prec == PFMP_F64 ? 0 : 1];
  while ((int)v.size() <= i) v.push_back(dev_alloc(spinor_bytes(A->ctx->g, prec)));
  return v[i];
}

// The fermion-force contractions of one precision, collected and summed into F and Hc
// by one launch of each force kernel per kMaxDerivSets of them (App. C: every force is
// a sum of Re a^dag dM-hat b over the terms' fields).  The fields handed to add_mhat and
// add_K are read when the batch is flushed: they must stay unchanged until then, which a
// ring of kRing fields per caller guarantees (add_K flushes before it would overflow, so
// at most kMaxDerivSets / 2 K contractions are pending).
struct ForceBatch {
  static constexpr int kRing = kMaxDerivSets / 2 + 1;
  pfmp_action* A;
  int prec;
  DerivBatch b;
  ForceBatch(pfmp_action* a, int p) : A(a), prec(p) {}
  // callers flush before they read F or Hc; a batch dropped by an exception is lost
  // with the force it belonged to
  void flush() {
    deriv_mhat_batch(A->ctx, prec, A->F, A->Hc, b);
    b.n = 0;
  }
  // ring field j of this batch's precision (callers' chains of pending fields)
  void* ring(int j) { return fscratch(A, prec, 3 * kMaxDerivSets + j % kRing); }
  // Re a^dag dM-hat b (coef) for the operator op; a, b even fields
  void add_mhat(pfmp_op* op, const void* a, const void* bf, double coef) {
    if (b.n == kMaxDerivSets) flush();
    const int k = b.n;
    void* y = fscratch(A, prec, kMaxDerivSets + 2 * k);
    void* w = fscratch(A, prec, kMaxDerivSets + 2 * k + 1);
    hop_clov_odd(op, prec, y, bf, false);
    hop_clov_odd(op, prec, w, a, true);
    const double k2 = op->kappa * op->kappa, kc = op->kappa * op->csw;
    b.s[k] = DerivSet{a, bf, y, w, -k2 * coef, -kc * coef, k2 * (-kc) * coef};
    b.n++;
  }
  // Re eta^dag dK chi (coef) for K = M-hat^dag M-hat of op:
  //   Re (M-hat chi)^dag dM-hat eta + Re (M-hat eta)^dag dM-hat chi
  // (one contraction with twice the coefficient when eta and chi are the same field)
  void add_K(pfmp_op* op, const void* eta, const void* chi, double coef) {
    const int need = eta == chi ? 1 : 2;
    if (b.n + need > kMaxDerivSets) flush();
    void* Mchi = fscratch(A, prec, b.n);
    mhat(op, prec, Mchi, chi, false, nullptr, nullptr);
    if (eta == chi) {
      add_mhat(op, Mchi, eta, 2.0 * coef);
      return;
    }
    void* Meta = fscratch(A, prec, b.n + 1);
    mhat(op, prec, Meta, eta, false, nullptr, nullptr);
    add_mhat(op, Mchi, eta, coef);
    add_mhat(op, Meta, chi, coef);
  }
};

// clover terms of every operator after the gauge field changed; FP32 field strength
// (fprec = PFMP_F32) for the link updates inside an MD with FP32 forces
void refresh_ops(pfmp_action* A, int fprec = PFMP_F64) {
  for (auto op : A->ops) clover_build(op, fprec);
}

long long kapply_total(pfmp_action* A) {
  long long k = 0;
  for (auto op : A->ops) k += op->kapply;
  return k;
}

// residues of 1 / prod_k (z - w_k) over the list w
std::vector<cd> product_residues(const std::vector<cd>& w) {
  std::vector<cd> s;
  for (size_t i = 0; i < w.size(); ++i) {
    cd prod = 1.0;
    for (size_t j = 0; j < w.size(); ++j)
      if (j != i) prod *= (w[i] - w[j]);
    s.push_back(1.0 / prod);
  }
  return s;
}

// roots and normalisation of Q = P_p2 / P_p1 (App. A: with (p1 + 1) | (p2 + 1) the roots
// of P_p1 are those of P_p2 with index k = j (p2 + 1)/(p1 + 1); Q keeps the others and
// c = a_p2 / a_p1).  p1 = 0: Q = P_p2.
void filter_roots(int p1, int p2, double mu, double nu, std::vector<cd>& q, double& c) {
  PFMP_REQUIRE(p2 >= 2 && p2 % 2 == 0 && p1 >= 0 && p1 % 2 == 0, PFMP_E_UNSUPPORTED, "filter orders must be even");
  std::vector<cd> z = cheb_roots(p2, mu, nu);
  q.clear();
  if (p1 == 0) {
    q = z;
    c = cheb_norm(p2, mu, nu);
    return;
  }
  PFMP_REQUIRE(p2 > p1 && (p2 + 1) % (p1 + 1) == 0, PFMP_E_UNSUPPORTED,
               "P_p1 divides P_p2 only when (p1 + 1) divides (p2 + 1)");
  const int m = (p2 + 1) / (p1 + 1);
  for (int k = 1; k <= p2; ++k)
    if (k % m) q.push_back(z[k - 1]);
  c = cheb_norm(p2, mu, nu) / cheb_norm(p1, mu, nu);
}

void setup_term(Term& T, const pfmp_action_def& d) {
  const pfmp_term& x = T.d;
  if (x.kind == PFMP_KIND_FILTER) {
    filter_roots(x.p1, x.p2, d.mu, d.nu, T.q, T.c);
    for (auto qk : T.q)
      if (qk.imag() < 0) T.qh.push_back(qk);
    T.sh = product_residues(T.qh);
    T.q = stable_ordered(T.q);  // the order of the product's factors (action and force)
  } else if (x.kind == PFMP_KIND_FILTERCORR) {
    PFMP_REQUIRE(x.p2 >= 2 && x.p2 % 2 == 0, PFMP_E_UNSUPPORTED, "filter orders must be even");
    std::vector<cd> z = cheb_roots(x.p2, d.mu, d.nu);
    T.a_p = cheb_norm(x.p2, d.mu, d.nu);
    for (auto zk : z)
      if (zk.imag() < 0) T.zh.push_back(zk);
    z.push_back(0.0);
    const int n = x.p2;
    for (int i = 0; i <= n; ++i) {
      cd prod = T.a_p;
      for (int j = 0; j <= n; ++j)
        if (j != i) prod *= (z[i] - z[j]);
      T.r.push_back(1.0 / prod);
      T.sig.push_back(-z[i]);
      int best = 0;
      for (int j = 0; j <= n; ++j)
        if (std::abs(z[j] - std::conj(z[i])) < std::abs(z[best] - std::conj(z[i]))) best = j;
      T.conj_of.push_back(best);
    }
  }
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
  for (auto p : A->ev32) dev_free(p);
  for (auto p : A->xs32) dev_free(p);
  for (auto& v : A->fbuf)
    for (auto p : v) dev_free(p);
  for (auto op : A->ops) op_delete(op);
  delete A;
}

void action_scheme(int scheme, int p1, int p2, pfmp_action_def* d) {
  auto T = [](int kind, int a, int b, int q1, int q2) { return pfmp_term{kind, a, b, q1, q2}; };
  std::vector<pfmp_term> v = {T(PFMP_KIND_GAUGE, 0, 0, 0, 0), T(PFMP_KIND_DET, 0, 0, 0, 0)};
  switch (scheme) {
    case PFMP_SCHEME_1PF:
      v.push_back(T(PFMP_KIND_FILTER, 0, 0, 0, p2));
      v.push_back(T(PFMP_KIND_FILTERCORR, 0, 0, 0, p2));
      break;
    case PFMP_SCHEME_2PF:
      v.push_back(T(PFMP_KIND_FILTER, 0, 0, 0, p1));
      v.push_back(T(PFMP_KIND_FILTER, 0, 0, p1, p2));
      v.push_back(T(PFMP_KIND_FILTERCORR, 0, 0, 0, p2));
      break;
    case PFMP_SCHEME_1MP:
      v.push_back(T(PFMP_KIND_INV, 1, 0, 0, 0));
      v.push_back(T(PFMP_KIND_RATIO, 1, 0, 0, 0));
      break;
    case PFMP_SCHEME_2MP:
      v.push_back(T(PFMP_KIND_INV, 1, 0, 0, 0));
      v.push_back(T(PFMP_KIND_RATIO, 1, 2, 0, 0));
      v.push_back(T(PFMP_KIND_RATIO, 2, 0, 0, 0));
      break;
    case PFMP_SCHEME_PFMP:
      v.push_back(T(PFMP_KIND_FILTER, 1, 0, 0, p2));
      v.push_back(T(PFMP_KIND_FILTERCORR, 1, 0, 0, p2));
      v.push_back(T(PFMP_KIND_RATIO, 1, 0, 0, 0));
      break;
    case PFMP_SCHEME_2PF1MP:
      v.push_back(T(PFMP_KIND_FILTER, 1, 0, 0, p1));
      v.push_back(T(PFMP_KIND_FILTER, 1, 0, p1, p2));
      v.push_back(T(PFMP_KIND_FILTERCORR, 1, 0, 0, p2));
      v.push_back(T(PFMP_KIND_RATIO, 1, 0, 0, 0));
      break;
    case PFMP_SCHEME_1PF2MP:
      v.push_back(T(PFMP_KIND_FILTER, 1, 0, 0, p2));
      v.push_back(T(PFMP_KIND_FILTERCORR, 1, 0, 0, p2));
      v.push_back(T(PFMP_KIND_RATIO, 1, 2, 0, 0));
      v.push_back(T(PFMP_KIND_RATIO, 2, 0, 0, 0));
      break;
    default:
      PFMP_REQUIRE(false, PFMP_E_INVALID, "unknown scheme");
  }
  d->nterms = (int)v.size();
  for (size_t i = 0; i < v.size(); ++i) d->term[i] = v[i];
}

pfmp_action* action_create_def(pfmp_ctx* c, const pfmp_action_def* d) {
  PFMP_REQUIRE(d->nkappa >= 1 && d->nkappa <= PFMP_MAX_KAPPA, PFMP_E_INVALID, "nkappa out of range");
  PFMP_REQUIRE(d->nterms >= 1 && d->nterms <= PFMP_MAX_TERMS, PFMP_E_INVALID, "nterms out of range");
  PFMP_REQUIRE(d->mu >= d->nu && d->nu > 0, PFMP_E_INVALID, "need mu >= nu > 0");
  PFMP_REQUIRE(d->tol > 0 && d->max_iter > 0, PFMP_E_INVALID, "bad solver tolerance / iteration cap");
  PFMP_REQUIRE(d->solver == PFMP_SOLVER_CG64 || d->solver == PFMP_SOLVER_CG_MIXED, PFMP_E_INVALID,
               "action solver must be CG64 or CG_MIXED");
  PFMP_REQUIRE(d->force_prec == PFMP_F64 || d->force_prec == PFMP_F32, PFMP_E_INVALID,
               "force precision must be PFMP_F64 or PFMP_F32");
  PFMP_REQUIRE(d->md_tol >= 0 && d->md_tol < 1, PFMP_E_INVALID, "md_tol must be in [0, 1)");
  for (int i = 0; i < d->nkappa; ++i) PFMP_REQUIRE(d->kappa[i] > 0, PFMP_E_INVALID, "kappa must be positive");
  for (int i = 0; i < d->nterms; ++i) {
    const pfmp_term& x = d->term[i];
    PFMP_REQUIRE(x.kind >= PFMP_KIND_GAUGE && x.kind <= PFMP_KIND_INV, PFMP_E_INVALID, "unknown term kind");
    PFMP_REQUIRE(x.a >= 0 && x.a < d->nkappa, PFMP_E_INVALID, "term kappa index a out of range");
    PFMP_REQUIRE(x.kind != PFMP_KIND_RATIO || (x.b >= 0 && x.b < d->nkappa), PFMP_E_INVALID,
                 "term kappa index b out of range");
  }
  pfmp_action* A = new pfmp_action();
  A->ctx = c;
  A->def = *d;
  try {
    for (int i = 0; i < d->nterms; ++i) {
      Term T;
      T.d = d->term[i];
      setup_term(T, *d);
      if (is_fermion(T.d.kind)) T.pf = (int)A->phi.size(), A->phi.push_back(nullptr);
      A->t.push_back(T);
    }
    for (int i = 0; i < d->nkappa; ++i) A->ops.push_back(op_new(c, d->kappa[i], d->csw));
    const Geom& g = c->g;
    for (auto& p : A->phi) p = (double2*)dev_alloc(spb(A));
    A->F = (double*)dev_alloc((size_t)g.Vh * 64 * sizeof(double));
    A->Hc = (double*)dev_alloc((size_t)g.Vh * 96 * sizeof(double));
    A->mom = (double*)dev_alloc((size_t)g.Vh * 64 * sizeof(double));
    A->U0 = (double2*)dev_alloc((size_t)g.Vh * 72 * sizeof(double2));
    for (int i = 0; i < 8; ++i) A->ev.push_back((double2*)dev_alloc(spb(A)));
  } catch (...) {
    action_destroy(A);
    throw;
  }
  return A;
}

pfmp_action* action_create(pfmp_ctx* c, const pfmp_action_params* prm) {
  PFMP_REQUIRE(prm->n >= 2 && prm->n % 2 == 0, PFMP_E_UNSUPPORTED, "polynomial order must be even and >= 2");
  pfmp_action_def d{};
  d.beta = prm->beta;
  d.csw = prm->csw;
  d.nkappa = 2;
  d.kappa[0] = prm->kappa;
  d.kappa[1] = prm->kappa_h;
  d.mu = prm->mu;
  d.nu = prm->nu;
  d.tol = prm->tol;
  d.max_iter = prm->max_iter;
  action_scheme(PFMP_SCHEME_PFMP, 0, prm->n, &d);
  return action_create_def(c, &d);
}

int action_nterms(pfmp_action* A) { return (int)A->t.size(); }
int action_npf(pfmp_action* A) { return (int)A->phi.size(); }

// phi_i from the noise xi_i (even FP64 device fields, one per fermion term)
void action_heatbath(pfmp_action* A, const void* const* xi) {
  pfmp_ctx* c = A->ctx;
  for (auto& T : A->t) {
    if (T.pf < 0) continue;
    pfmp_op* W = A->ops[T.d.a];
    void* phi = A->phi[T.pf];
    const void* x = xi[T.pf];
    if (T.d.kind == PFMP_KIND_FILTER) {
      // phi = c^{-1/2} sum_k s_k (J - qh_k)^{-1} xi
      std::vector<cd> sig;
      for (auto qk : T.qh) sig.push_back(-qk);
      multishift(A, W, sig, x);
      blas_zero(c, PFMP_F64, phi);
      for (size_t k = 0; k < T.qh.size(); ++k) caxpby(c, T.sh[k] / std::sqrt(T.c), A->xs[k], 1.0, phi);
    } else if (T.d.kind == PFMP_KIND_FILTERCORR) {
      // phi = R(J)^dag W^dag xi
      mhat(W, PFMP_F64, E(A, 0), x, true, nullptr, nullptr);
      std::vector<cd> zc;
      for (auto zk : T.zh) zc.push_back(std::conj(zk));
      poly_product(W, stable_ordered(zc), std::sqrt(T.a_p), phi, E(A, 0));
    } else if (T.d.kind == PFMP_KIND_RATIO) {
      // phi = W_a J_a^{-1} M_b^dag xi
      mhat(A->ops[T.d.b], PFMP_F64, E(A, 0), x, true, nullptr, nullptr);
      cg64(A, W, E(A, 1), E(A, 0));
      mhat(W, PFMP_F64, phi, E(A, 1), false, nullptr, nullptr);
    } else {  // INV: phi = W^dag xi
      mhat(W, PFMP_F64, phi, x, true, nullptr, nullptr);
    }
  }
}

double action_term(pfmp_action* A, int i) {
  pfmp_ctx* c = A->ctx;
  Term& T = A->t[i];
  pfmp_op* W = A->ops[T.d.a];
  switch (T.d.kind) {
    case PFMP_KIND_GAUGE:
      return A->def.beta * 6.0 * c->g.V * (1.0 - plaquette(c));
    case PFMP_KIND_DET:
      return A->def.csw != 0.0 ? -2.0 * W->logdet_oo : 0.0;
    case PFMP_KIND_FILTER: {
      poly_product(W, T.q, T.c, E(A, 0), A->phi[T.pf]);
      return cdot(c, A->phi[T.pf], E(A, 0)).real();
    }
    case PFMP_KIND_FILTERCORR: {
      multishift(A, W, T.sig, A->phi[T.pf]);
      cd s = 0.0;
      for (size_t k = 0; k < T.sig.size(); ++k) s += T.r[k] * cdot(c, A->phi[T.pf], A->xs[k]);
      return s.real();
    }
    case PFMP_KIND_RATIO: {
      mhat(W, PFMP_F64, E(A, 0), A->phi[T.pf], true, nullptr, nullptr);
      cg64(A, A->ops[T.d.b], E(A, 1), E(A, 0));
      return cdot(c, E(A, 0), E(A, 1)).real();
    }
    default: {  // INV
      cg64(A, W, E(A, 1), A->phi[T.pf]);
      return cdot(c, A->phi[T.pf], E(A, 1)).real();
    }
  }
}

void action_eval(pfmp_action* A, double* S) {
  for (int i = 0; i < (int)A->t.size(); ++i) S[i] = action_term(A, i);
}

// The fermion forces with FP32 arithmetic (force_prec = PFMP_F32): the spinor products,
// the K chains of the filter force and the multi-shift solve of the correction force in
// FP32 (solves at the MD tolerance), the CG of the ratio and inverse terms mixed, every
// contraction summed into the FP64 force.  The MD only needs each force to be a fixed
// function of the gauge field (then every momentum update is a shear of phase space and
// the MD map stays reversible and area-preserving), so the trajectory is still exact;
// the actions at its ends are evaluated as before.
static void force_f32(pfmp_action* A, Term& T, pfmp_op* W, const void* phi) {
  pfmp_ctx* c = A->ctx;
  const size_t b32 = spinor_bytes(c->g, PFMP_F32);
  float4* phi32 = E32(A, 0);
  blas_copy(c, phi32, PFMP_F32, phi, PFMP_F64);
  if (T.d.kind == PFMP_KIND_FILTER) {
    const int m = (int)T.q.size();
    while ((int)A->xs32.size() < m) A->xs32.push_back((float4*)dev_alloc(b32));
    // chi_{m-1} = c phi, chi_k = (J - q_{k+1}) chi_{k+1}
    caxpby(c, PFMP_F32, T.c, phi32, 0.0, A->xs32[m - 1]);
    for (int k = m - 2; k >= 0; --k) {
      kop(W, PFMP_F32, A->xs32[k], A->xs32[k + 1], nullptr, nullptr);
      caxpby(c, PFMP_F32, -T.q[k + 1], A->xs32[k + 1], 1.0, A->xs32[k]);
    }
    // eta_0 = phi, eta_k = (J - q_{k-1}^*) eta_{k-1}, each in its own ring field
    ForceBatch fb(A, PFMP_F32);
    const void* eta = phi32;
    for (int k = 0; k < m; ++k) {
      if (k > 0) {
        void* next = fb.ring(k);
        kop(W, PFMP_F32, next, eta, nullptr, nullptr);
        caxpby(c, PFMP_F32, -std::conj(T.q[k - 1]), eta, 1.0, next);
        eta = next;
      }
      fb.add_K(W, eta, A->xs32[k], 1.0);
    }
    fb.flush();
  } else if (T.d.kind == PFMP_KIND_FILTERCORR) {
    multishift(A, W, T.sig, phi32, PFMP_F32);
    ForceBatch fb(A, PFMP_F32);
    for (size_t k = 0; k < T.sig.size(); ++k) {
      void* chib = fb.ring((int)k);
      caxpby(c, PFMP_F32, T.r[k], A->xs32[k], 0.0, chib);
      fb.add_K(W, A->xs32[T.conj_of[k]], chib, -1.0);
    }
    fb.flush();
  } else if (T.d.kind == PFMP_KIND_RATIO) {
    pfmp_op* Mb = A->ops[T.d.b];
    mhat(W, PFMP_F64, E(A, 0), phi, true, nullptr, nullptr);
    cg_tol(A, Mb, E(A, 1), E(A, 0), md_tol(A));
    float4* chi32 = E32(A, 1);
    blas_copy(c, chi32, PFMP_F32, E(A, 1), PFMP_F64);
    ForceBatch fb(A, PFMP_F32);
    fb.add_mhat(W, phi32, chi32, 2.0);
    fb.add_K(Mb, chi32, chi32, -1.0);
    fb.flush();
  } else {  // INV
    cg_tol(A, W, E(A, 1), phi, md_tol(A));
    float4* chi32 = E32(A, 1);
    blas_copy(c, chi32, PFMP_F32, E(A, 1), PFMP_F64);
    ForceBatch fb(A, PFMP_F32);
    fb.add_K(W, chi32, chi32, -1.0);
    fb.flush();
  }
}

// F += dS_i/d omega (F must be zeroed by the caller for a fresh force)
void action_force(pfmp_action* A, int i) {
  pfmp_ctx* c = A->ctx;
  const Geom& g = c->g;
  Term& T = A->t[i];
  pfmp_op* W = A->ops[T.d.a];
  A->force_evals++;
  const int fprec = f32_forces(A) ? PFMP_F32 : PFMP_F64;
  if (T.d.kind == PFMP_KIND_GAUGE) {
    gauge_force(c, fprec, A->F, A->def.beta);
    return;
  }
  const bool clover = A->def.csw != 0.0;
  if (T.d.kind == PFMP_KIND_DET && !clover) return;
  PFMP_CUDA(cudaMemsetAsync(A->Hc, 0, (size_t)g.Vh * 96 * sizeof(double), c->stream));
  void* phi = T.pf >= 0 ? A->phi[T.pf] : nullptr;
  if (T.d.kind != PFMP_KIND_DET && f32_forces(A)) {
    force_f32(A, T, W, phi);
  } else if (T.d.kind == PFMP_KIND_DET) {
    clover_insert_det(W, A->Hc, 2.0 * W->kappa * W->csw);
  } else if (T.d.kind == PFMP_KIND_FILTER) {
    const int m = (int)T.q.size();
    // chi_i, i = m-1 .. 0 (0-based): chi[m-1] = c phi, chi[i] = (J - q_{i+1}) chi[i+1]
    while ((int)A->xs.size() < m) A->xs.push_back((double2*)dev_alloc(spb(A)));
    caxpby(c, T.c, phi, 0.0, A->xs[m - 1]);
    for (int k = m - 2; k >= 0; --k) {
      kop(W, PFMP_F64, A->xs[k], A->xs[k + 1], nullptr, nullptr);
      caxpby(c, -T.q[k + 1], A->xs[k + 1], 1.0, A->xs[k]);
    }
    // eta_0 = phi, eta_i = (J - q_{i-1}^*) eta_{i-1}, each in its own ring field
    ForceBatch fb(A, PFMP_F64);
    const void* eta = phi;
    for (int k = 0; k < m; ++k) {
      if (k > 0) {
        void* next = fb.ring(k);
        kop(W, PFMP_F64, next, eta, nullptr, nullptr);
        caxpby(c, -std::conj(T.q[k - 1]), eta, 1.0, next);
        eta = next;
      }
      fb.add_K(W, eta, A->xs[k], 1.0);
    }
    fb.flush();
  } else if (T.d.kind == PFMP_KIND_FILTERCORR) {
    multishift(A, W, T.sig, phi);
    ForceBatch fb(A, PFMP_F64);
    for (size_t k = 0; k < T.sig.size(); ++k) {
      void* chib = fb.ring((int)k);
      caxpby(c, T.r[k], A->xs[k], 0.0, chib);
      fb.add_K(W, A->xs[T.conj_of[k]], chib, -1.0);
    }
    fb.flush();
  } else if (T.d.kind == PFMP_KIND_RATIO) {
    pfmp_op* Mb = A->ops[T.d.b];
    mhat(W, PFMP_F64, E(A, 0), phi, true, nullptr, nullptr);
    void* chi = E(A, 1);
    cg64(A, Mb, chi, E(A, 0));
    // 2 Re chi^dag dW^dag phi = 2 Re phi^dag dW chi
    ForceBatch fb(A, PFMP_F64);
    fb.add_mhat(W, phi, chi, 2.0);
    fb.add_K(Mb, chi, chi, -1.0);
    fb.flush();
  } else {  // INV
    void* chi = E(A, 1);
    cg64(A, W, chi, phi);
    ForceBatch fb(A, PFMP_F64);
    fb.add_K(W, chi, chi, -1.0);
    fb.flush();
  }
  if (clover) clover_force(c, fprec, A->F, A->Hc);
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
  PFMP_REQUIRE(term >= 0 && term < (int)A->t.size(), PFMP_E_INVALID, "term index out of range");
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
  refresh_ops(A, f32_forces(A) ? PFMP_F32 : PFMP_F64);
}

void mom_update(pfmp_action* A, double eps) {
  pfmp_ctx* c = A->ctx;
  const long n = 64L * c->g.Vh;
  k_mom_update<<<grid_for(n), kBlock, 0, c->stream>>>(A->mom, A->F, eps, n);
  PFMP_CHECK_LAUNCH();
}

// link sum and maximum of |F_mu(x)| over the current force buffer (synchronises)
void force_norms(pfmp_action* A, double* sum, double* mx) {
  pfmp_ctx* c = A->ctx;
  PFMP_CUDA(cudaMemsetAsync(c->d_sums, 0, 2 * sizeof(double), c->stream));
  const long nl = 8L * c->g.Vh;
  k_force_norm<<<grid_for(nl), kBlock, 0, c->stream>>>(A->F, c->g.Vh, c->rb, c->d_sums,
                                                       (unsigned long long*)(c->d_sums + 1));
  PFMP_CHECK_LAUNCH();
  double v[2];
  sync_read(c, v, 2);
  *sum = v[0];
  *mx = v[1];
}

// the MD part of a trajectory (Sec. 2.1, App. B): for each step of the merged schedule
// T-hat, then P -= eps F_t for every term t on each level with a non-zero step, one term
// at a time so that each term's force is measured (sums of the link averages into favg)
// clover terms built from an FP32 field strength inside the MD are rebuilt in FP64
static void fp64_clover(pfmp_action* A) {
  bool f32 = false;
  for (auto op : A->ops) f32 = f32 || op->built_prec != PFMP_F64;
  if (f32) refresh_ops(A, PFMP_F64);
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

static void md_steps(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level,
                     pfmp_traj_info* info) {
  const int nt = (int)A->t.size();
  const double nlinks = 4.0 * A->ctx->g.V;
  for (int i = 0; i < len; ++i) {
    if (T[i] != 0.0) {
      const auto t0 = std::chrono::steady_clock::now();
      link_update(A, T[i]);
      PFMP_CUDA(cudaStreamSynchronize(A->ctx->stream));
      info->ms_update += ms_since(t0);
    }
    for (int l = 0; l < nlev; ++l) {
      const double eps = S[(size_t)l * len + i];
      if (eps == 0.0) continue;
      for (int t = 0; t < nt; ++t) {
        if (term_level[t] != l) continue;
        const auto t0 = std::chrono::steady_clock::now();
        const long long kt = kapply_total(A);
        action_zero_force(A);
        action_force(A, t);
        mom_update(A, eps);
        info->k_apply_term[t] += kapply_total(A) - kt;
        double fs, fm;
        force_norms(A, &fs, &fm);  // synchronises
        info->nforce[t] += 1;
        info->fmax[t] = std::max(info->fmax[t], fm);
        info->favg[t] += fs / nlinks;
        info->ms_force[t] += ms_since(t0);
      }
    }
  }
}

// MD alone with the current pseudofermions: U and the momenta (canonical [V][4][8], in
// and out) evolve along the schedule; no heatbath, no Hamiltonian, no accept/reject
void action_md(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level,
               double* mom, int where) {
  pfmp_ctx* c = A->ctx;
  const int nt = (int)A->t.size();
  PFMP_REQUIRE(len >= 1 && nlev >= 1, PFMP_E_INVALID, "empty schedule");
  for (int t = 0; t < nt; ++t)
    PFMP_REQUIRE(term_level[t] >= -1 && term_level[t] < nlev, PFMP_E_INVALID, "term level out of range");
  bool stale = false;
  for (auto op : A->ops) stale = stale || op->built_version != c->gauge_version || op->built_prec != PFMP_F64;
  if (stale) refresh_ops(A);
  alg_pack(c, A->mom, mom, where);
  pfmp_traj_info scratch{};
  md_steps(A, len, T, nlev, S, term_level, &scratch);
  fp64_clover(A);
  alg_unpack(c, mom, where, A->mom);
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
}

void trajectory(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level,
                const double* mom, int where, const void* const* xi, double u, pfmp_traj_info* info) {
  pfmp_ctx* c = A->ctx;
  const Geom& g = c->g;
  const int nt = (int)A->t.size();
  PFMP_REQUIRE(len >= 1 && nlev >= 1, PFMP_E_INVALID, "empty schedule");
  for (int t = 0; t < nt; ++t)
    PFMP_REQUIRE(term_level[t] >= -1 && term_level[t] < nlev, PFMP_E_INVALID, "term level out of range");
  *info = pfmp_traj_info{};
  const auto t_start = std::chrono::steady_clock::now();
  const long long k0 = kapply_total(A);
  A->force_evals = 0;
  PFMP_CUDA(cudaMemcpyAsync(A->U0, c->U64, (size_t)g.Vh * 72 * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  bool stale = false;
  for (auto op : A->ops) stale = stale || op->built_version != c->gauge_version || op->built_prec != PFMP_F64;
  if (stale) refresh_ops(A);
  alg_pack(c, A->mom, mom, where);
  std::vector<double> S0(nt, 0.0), S1(nt, 0.0);
  double H0 = 0, H1 = 0;
  // a trajectory that fails (a NaN, a solve that does not converge) leaves the gauge
  // field as it found it
  auto restore = [&]() {
    cudaMemcpyAsync(c->U64, A->U0, (size_t)g.Vh * 72 * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream);
    gauge_refresh_compressed(c);
    refresh_ops(A);
  };
  try {
    action_heatbath(A, xi);
    H0 = kinetic(A);
    for (int t = 0; t < nt; ++t)
      if (term_level[t] >= 0) H0 += (S0[t] = action_term(A, t));
    md_steps(A, len, T, nlev, S, term_level, info);
    fp64_clover(A);  // the final Hamiltonian with FP64 clover terms
    H1 = kinetic(A);
    for (int t = 0; t < nt; ++t)
      if (term_level[t] >= 0) H1 += (S1[t] = action_term(A, t));
    PFMP_REQUIRE(std::isfinite(H1 - H0), PFMP_E_NAN, "dH is not finite");
  } catch (const Err&) {
    try {
      restore();
    } catch (const Err&) {
    }
    throw;
  }
  const double dH = H1 - H0;
  const bool acc = u < std::exp(-dH);
  info->H0 = H0;
  info->H1 = H1;
  info->dH = dH;
  info->accepted = acc ? 1 : 0;
  for (int t = 0; t < nt; ++t) {
    info->S0[t] = S0[t];
    info->S1[t] = S1[t];
    if (info->nforce[t] > 0) info->favg[t] /= info->nforce[t];
  }
  info->k_apply = kapply_total(A) - k0;
  info->force_evals = A->force_evals;
  if (!acc) restore();
  info->plaquette = plaquette(c);
  info->ms_total = ms_since(t_start);
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
  PFMP_REQUIRE(i >= 0 && i < (int)A->phi.size(), PFMP_E_INVALID, "pseudofermion index out of range");
  spinor_unpack_any(A->ctx, out, where, A->phi[i], PFMP_F64, 0);
}

void action_set_phi(pfmp_action* A, int i, const double* in, int where) {
  PFMP_REQUIRE(i >= 0 && i < (int)A->phi.size(), PFMP_E_INVALID, "pseudofermion index out of range");
  spinor_pack_any(A->ctx, A->phi[i], PFMP_F64, in, where, 0);
}

void action_refresh(pfmp_action* A) { refresh_ops(A); }
pfmp_ctx* action_ctx(pfmp_action* A) { return A->ctx; }

}  // namespace pfmp
