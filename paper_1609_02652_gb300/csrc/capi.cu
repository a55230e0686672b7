// extern "C" entry points: argument checks, exception-to-status translation, and the
// small amount of orchestration each call needs.  See include/pfmp.h for the contract.
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "context.h"

namespace pfmp {
const char* last_error();
pfmp_ctx* ctx_create(const int dims[4], int bc_t, void* stream);
void ctx_destroy(pfmp_ctx* c);
void gauge_set(pfmp_ctx* c, const double* U, int where);
void gauge_get(pfmp_ctx* c, double* U, int where);
void gauge_from_algebra(pfmp_ctx* c, const double* h, double eps, int where);
double plaquette(pfmp_ctx* c);
void spinor_pack_any(pfmp_ctx* c, void* dst, int prec, const double* src, int where, int parity);
void spinor_unpack_any(pfmp_ctx* c, double* dst, int where, const void* src, int prec, int parity);
void profile_begin(pfmp_ctx* c);
pfmp_action* action_create(pfmp_ctx* c, const pfmp_action_params* prm);
pfmp_action* action_create_def(pfmp_ctx* c, const pfmp_action_def* d);
void action_scheme(int scheme, int p1, int p2, pfmp_action_def* d);
int action_nterms(pfmp_action* A);
int action_npf(pfmp_action* A);
void action_destroy(pfmp_action* A);
void action_heatbath(pfmp_action* A, const void* const* xi);
void action_eval(pfmp_action* A, double* S);
void action_force_out(pfmp_action* A, int term, double* out, int where);
void action_get_phi(pfmp_action* A, int i, double* out, int where);
void action_set_phi(pfmp_action* A, int i, const double* in, int where);
void action_refresh(pfmp_action* A);
void schedule_2mn(int n, double tau, double lam, double* T, double* S);
int schedule_merge(int ns, const int* len, const double* T, const double* S, int cap, double* Tout, double* Sout);
void trajectory(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level,
                const double* mom, int where, const void* const* xi, double u, pfmp_traj_info* info);
pfmp_ctx* action_ctx(pfmp_action* A);
void action_md(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level,
               double* mom, int where);
pfmp_batch* batch_create(int nsys, pfmp_op* const* ops, const int* nrhs);
void batch_destroy(pfmp_batch* B);
int batch_solve(pfmp_batch* B, double tol, int max_iter, double delta, int check, void* const* x, const void* const* b,
                pfmp_solve_info* infos);
int batch_tune(pfmp_batch* B, int chunk, double* best_ms);
int batch_barrier_check(pfmp_batch* B, int rounds, int missing, double limit_s);
pfmp_nn* nn_create(pfmp_ctx* c, int nl, const int* ch, int prec);
void nn_destroy(pfmp_nn* N);
long nn_num_weights(const pfmp_nn* N);
void nn_set_weights(pfmp_nn* N, const double* w);
void nn_get_weights(pfmp_nn* N, double* w);
void nn_get_grads(pfmp_nn* N, double* w);
void nn_apply(pfmp_nn* N, void* out, const void* in, int prec_io);
void nn_set_tc(pfmp_nn* N, bool on);
void nn_check(pfmp_nn* N);
void nn_zero_grad(pfmp_nn* N);
double nn_loss_grad(pfmp_nn* N, pfmp_op* op, int kind, const void* b, const void* x, double scale);
double nn_train(pfmp_nn* N, pfmp_op* op, int kind, int npairs, const void* const* b, const void* const* x, int steps,
                int batch, double lr);
int solve_fgcr(pfmp_op* op, pfmp_nn* nn, double tol, int max_iter, int restart, double delta, void* x, const void* b,
               int* iters, int* outer, double* true_res, long* kapply, int* fallback_iters);
void profile_end(pfmp_ctx* c, int cls, long* launches, double* ms, double* bytes);
void spectrum(pfmp_op* op, int nsteps, const void* v0, double* lmin, double* lmax, double* alpha_out,
              double* beta_out, int* steps);
}  // namespace pfmp

using namespace pfmp;

#define API_BEGIN \
  try {           \
    set_last_error("");
#define API_END                                         \
  }                                                     \
  catch (const Err& e) {                                \
    return e.code;                                      \
  }                                                     \
  catch (const std::bad_alloc&) {                       \
    set_last_error("host allocation failed");           \
    return PFMP_E_NOMEM;                                \
  }                                                     \
  catch (...) {                                         \
    set_last_error("unexpected C++ exception");         \
    return PFMP_E_INVALID;                              \
  }                                                     \
  return PFMP_OK;

static void check_prec(int prec) { PFMP_REQUIRE(prec == PFMP_F64 || prec == PFMP_F32, PFMP_E_INVALID, "bad precision"); }
// the entry points that also take FP16 storage
static void check_prec_h(int prec) {
  PFMP_REQUIRE(prec == PFMP_F64 || prec == PFMP_F32 || prec == PFMP_H16, PFMP_E_INVALID, "bad precision");
}
static void check_where(int w) { PFMP_REQUIRE(w == PFMP_HOST || w == PFMP_DEVICE, PFMP_E_INVALID, "bad location"); }

namespace pfmp {
void op_delete(pfmp_op* op);
pfmp_op* op_new(pfmp_ctx* ctx, double kappa, double csw);
}

static void op_free(pfmp_op* op) { op_delete(op); }

void pfmp::op_delete(pfmp_op* op) {
  if (!op) return;
  for (int p = 0; p < 2; ++p) {
    dev_free(op->clov64[p]);
    dev_free(op->clov32[p]);
    dev_free(op->clovdf[p]);
    dev_free(op->clov16[p]);
  }
  dev_free(op->t16);
  dev_free(op->e16);
  for (auto q : op->cg16) dev_free(q);
  dev_free(op->tdf);
  dev_free(op->edf);
  dev_free(op->xdf);
  dev_free(op->kdf);
  dev_free(op->t64);
  dev_free(op->t32);
  dev_free(op->e64);
  dev_free(op->e32);
  for (int k = 0; k < 6; ++k) dev_free(op->cg64[k]);
  for (int k = 0; k < 4; ++k) dev_free(op->cg32[k]);
  dev_free(op->scal);
  if (op->h_scal) cudaFreeHost(op->h_scal);
  ms_work_free(op);
  if (op->fgcr && op->fgcr_free) op->fgcr_free(op->fgcr);
  for (auto& G : op->graph)
    if (G.exec) cudaGraphExecDestroy(G.exec);
  if (op->cap) cudaStreamDestroy(op->cap);
  delete op;
}

pfmp_op* pfmp::op_new(pfmp_ctx* ctx, double kappa, double csw) {
  PFMP_REQUIRE(kappa > 0 && csw >= 0, PFMP_E_INVALID, "kappa must be > 0 and c_sw >= 0");
  pfmp_op* op = new pfmp_op();
  op->ctx = ctx;
  op->kappa = kappa;
  op->csw = csw;
  try {
    const Geom& g = ctx->g;
    for (int p = 0; p < 2; ++p) {
      op->clov64[p] = (double2*)dev_alloc((size_t)g.Vh * 36 * sizeof(double2));
      op->clov32[p] = (float4*)dev_alloc((size_t)g.Vh * 18 * sizeof(float4));
      op->clovdf[p] = (float4*)dev_alloc((size_t)g.Vh * 36 * sizeof(float4));
      op->clov16[p] = (uint4*)dev_alloc((size_t)g.Vh * 9 * sizeof(uint4));
    }
    op->t16 = (uint4*)dev_alloc(spinor_bytes(g, PFMP_H16));
    op->e16 = (uint4*)dev_alloc(spinor_bytes(g, PFMP_H16));
    for (auto& q : op->cg16) q = (uint4*)dev_alloc(spinor_bytes(g, PFMP_H16));
    op->tdf = (float4*)dev_alloc((size_t)g.Vh * 12 * sizeof(float4));
    op->edf = (float4*)dev_alloc((size_t)g.Vh * 12 * sizeof(float4));
    op->xdf = (float4*)dev_alloc((size_t)g.Vh * 12 * sizeof(float4));
    op->kdf = (float4*)dev_alloc((size_t)g.Vh * 12 * sizeof(float4));
    op->t64 = (double2*)dev_alloc(spinor_bytes(g, PFMP_F64));
    op->e64 = (double2*)dev_alloc(spinor_bytes(g, PFMP_F64));
    op->t32 = (float4*)dev_alloc(spinor_bytes(g, PFMP_F32));
    op->e32 = (float4*)dev_alloc(spinor_bytes(g, PFMP_F32));
    for (int k = 0; k < 6; ++k) op->cg64[k] = (double2*)dev_alloc(spinor_bytes(g, PFMP_F64));
    for (int k = 0; k < 4; ++k) op->cg32[k] = (float4*)dev_alloc(spinor_bytes(g, PFMP_F32));
    op->scal = (CGScalars*)dev_alloc(sizeof(CGScalars));
    PFMP_CUDA(cudaMallocHost(&op->h_scal, sizeof(CGScalars)));
    clover_build(op);
  } catch (...) {
    op_delete(op);
    throw;
  }
  return op;
}

extern "C" {

const char* pfmp_strerror(int s) {
  switch (s) {
    case PFMP_OK: return "ok";
    case PFMP_E_INVALID: return "invalid argument";
    case PFMP_E_NOMEM: return "out of memory";
    case PFMP_E_CUDA: return "CUDA error";
    case PFMP_E_NOT_CONVERGED: return "solver did not converge";
    case PFMP_E_TIMEOUT: return "bounded device wait timed out";
    case PFMP_E_NAN: return "NaN or Inf encountered";
    case PFMP_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* pfmp_last_error(void) { return last_error(); }
int pfmp_version(void) { return 100; }
int64_t pfmp_launch_count(void) { return (int64_t)launch_count(); }

int pfmp_ctx_create(pfmp_ctx** ctx, const int dims[4], int bc_t, void* stream) {
  API_BEGIN
  PFMP_REQUIRE(ctx && dims, PFMP_E_INVALID, "null argument");
  *ctx = ctx_create(dims, bc_t, stream);
  API_END
}

int pfmp_ctx_destroy(pfmp_ctx* ctx) {
  API_BEGIN
  ctx_destroy(ctx);
  API_END
}

int pfmp_ctx_set_stream(pfmp_ctx* ctx, void* stream) {
  API_BEGIN
  PFMP_REQUIRE(ctx, PFMP_E_INVALID, "null context");
  ctx->stream = (cudaStream_t)stream;
  API_END
}

int64_t pfmp_half_volume(const pfmp_ctx* ctx) { return ctx ? ctx->g.Vh : -1; }
int64_t pfmp_spinor_bytes(const pfmp_ctx* ctx, int prec) {
  if (!ctx || (prec != PFMP_F64 && prec != PFMP_F32 && prec != PFMP_H16)) return -1;
  return (int64_t)spinor_bytes(ctx->g, prec);
}

int pfmp_gauge_set(pfmp_ctx* ctx, const double* U, int where) {
  API_BEGIN
  PFMP_REQUIRE(ctx && U, PFMP_E_INVALID, "null argument");
  check_where(where);
  gauge_set(ctx, U, where);
  API_END
}

int pfmp_gauge_get(pfmp_ctx* ctx, double* U, int where) {
  API_BEGIN
  PFMP_REQUIRE(ctx && U, PFMP_E_INVALID, "null argument");
  check_where(where);
  gauge_get(ctx, U, where);
  API_END
}

int pfmp_gauge_from_algebra(pfmp_ctx* ctx, const double* h, double eps, int where) {
  API_BEGIN
  PFMP_REQUIRE(ctx && h, PFMP_E_INVALID, "null argument");
  check_where(where);
  gauge_from_algebra(ctx, h, eps, where);
  API_END
}

int pfmp_plaquette(pfmp_ctx* ctx, double* plaq) {
  API_BEGIN
  PFMP_REQUIRE(ctx && plaq, PFMP_E_INVALID, "null argument");
  *plaq = plaquette(ctx);
  API_END
}

int pfmp_spinor_pack(pfmp_ctx* ctx, void* dst, int prec, const double* src, int where, int parity) {
  API_BEGIN
  PFMP_REQUIRE(ctx && dst && src && (parity == 0 || parity == 1), PFMP_E_INVALID, "bad argument");
  check_prec_h(prec);
  check_where(where);
  spinor_pack_any(ctx, dst, prec, src, where, parity);
  API_END
}

int pfmp_spinor_unpack(pfmp_ctx* ctx, double* dst, int where, const void* src, int prec, int parity) {
  API_BEGIN
  PFMP_REQUIRE(ctx && dst && src && (parity == 0 || parity == 1), PFMP_E_INVALID, "bad argument");
  check_prec_h(prec);
  check_where(where);
  spinor_unpack_any(ctx, dst, where, src, prec, parity);
  API_END
}

int pfmp_op_create(pfmp_ctx* ctx, double kappa, double csw, pfmp_op** out) {
  API_BEGIN
  PFMP_REQUIRE(ctx && out, PFMP_E_INVALID, "null argument");
  *out = op_new(ctx, kappa, csw);
  API_END
}

int pfmp_op_update(pfmp_op* op) {
  API_BEGIN
  PFMP_REQUIRE(op, PFMP_E_INVALID, "null operator");
  clover_build(op);
  API_END
}

int pfmp_op_destroy(pfmp_op* op) {
  API_BEGIN
  if (op) cudaStreamSynchronize(op->ctx->stream);
  op_free(op);
  API_END
}

int pfmp_op_logdet(pfmp_op* op, double* ld) {
  API_BEGIN
  PFMP_REQUIRE(op && ld, PFMP_E_INVALID, "null argument");
  *ld = op->logdet_oo;
  API_END
}

static int split_slot(int prec) { return prec == PFMP_F64 ? 0 : (prec == PFMP_F32 ? 1 : (prec == PFMP_DF ? 2 : -1)); }

int pfmp_op_set_split(pfmp_op* op, int prec, int ns) {
  API_BEGIN
  PFMP_REQUIRE(op && split_slot(prec) >= 0, PFMP_E_INVALID, "bad operator or precision");
  PFMP_REQUIRE(ns == 1 || ns == 2 || ns == 4 || ns == 8, PFMP_E_INVALID, "threads per site must be 1, 2, 4 or 8");
  op->nsplit[split_slot(prec)] = ns;
  for (auto& G : op->graph)
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
  API_END
}

int pfmp_op_set_block(pfmp_op* op, int threads) {
  API_BEGIN
  PFMP_REQUIRE(op && threads >= 32 && threads <= 128 && threads % 32 == 0, PFMP_E_INVALID,
               "threads per block must be 32, 64, 96 or 128");
  op->hop_block = threads;
  for (auto& G : op->graph)
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
  API_END
}

int pfmp_op_get_split(pfmp_op* op, int prec, int* ns) {
  API_BEGIN
  PFMP_REQUIRE(op && ns && split_slot(prec) >= 0, PFMP_E_INVALID, "bad argument");
  *ns = op->nsplit[split_slot(prec)];
  API_END
}

int pfmp_dslash(pfmp_op* op, int prec, void* out, const void* in, int out_parity, int dagger) {
  API_BEGIN
  PFMP_REQUIRE(op && out && in && out != in && (out_parity == 0 || out_parity == 1), PFMP_E_INVALID, "bad argument");
  check_prec_h(prec);
  hop(op, prec, out, in, out_parity, dagger != 0);
  API_END
}

int pfmp_clover_apply(pfmp_op* op, int prec, void* out, const void* in, int parity, int inverse) {
  API_BEGIN
  PFMP_REQUIRE(op && out && in, PFMP_E_INVALID, "null argument");
  PFMP_REQUIRE((parity == 0 && !inverse) || (parity == 1 && inverse), PFMP_E_UNSUPPORTED,
               "the library keeps A on even sites and A^{-1} on odd sites only");
  check_prec(prec);
  clover_mul(op, prec, out, in, parity);
  API_END
}

int pfmp_mhat(pfmp_op* op, int prec, void* out, const void* in, int dagger) {
  API_BEGIN
  PFMP_REQUIRE(op && out && in && out != in, PFMP_E_INVALID, "bad argument");
  check_prec_h(prec);
  mhat(op, prec, out, in, dagger != 0, nullptr, nullptr);
  API_END
}

int pfmp_kop(pfmp_op* op, int prec, void* out, const void* in, double* in_K_in) {
  API_BEGIN
  PFMP_REQUIRE(op && out && in && out != in, PFMP_E_INVALID, "bad argument");
  check_prec_h(prec);
  pfmp_ctx* c = op->ctx;
  kop(op, prec, out, in, in_K_in ? c->d_sums : nullptr, nullptr);
  if (in_K_in) {
    PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    *in_K_in = c->h_sums[0];
  }
  API_END
}

int pfmp_true_residual(pfmp_op* op, int arith, void* r, const void* x, const void* b, double* rel) {
  API_BEGIN
  PFMP_REQUIRE(op && r && x && b && r != x && r != b, PFMP_E_INVALID, "bad argument");
  PFMP_REQUIRE(arith == PFMP_F64 || arith == PFMP_DF, PFMP_E_INVALID, "arith must be PFMP_F64 or PFMP_DF");
  pfmp_ctx* c = op->ctx;
  double rr;
  if (arith == PFMP_DF) {
    rr = true_residual_df(op, x, b, r);
  } else {
    void* Ax = op->cg64[2];
    kop(op, PFMP_F64, Ax, x, nullptr, nullptr);
    blas_xmy_norm(c, b, Ax, r, c->d_sums);
    PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    rr = c->h_sums[0];
  }
  if (rel) {
    blas_norm2(c, PFMP_F64, b, c->d_sums);
    PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    *rel = c->h_sums[0] > 0 ? std::sqrt(rr / c->h_sums[0]) : 0.0;
  }
  API_END
}

int pfmp_norm2(pfmp_ctx* ctx, int prec, const void* x, double* result) {
  API_BEGIN
  PFMP_REQUIRE(ctx && x && result, PFMP_E_INVALID, "null argument");
  check_prec(prec);
  blas_norm2(ctx, prec, x, ctx->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(ctx->h_sums, ctx->d_sums, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PFMP_CUDA(cudaStreamSynchronize(ctx->stream));
  *result = ctx->h_sums[0];
  API_END
}

int pfmp_cdot(pfmp_ctx* ctx, int prec, const void* x, const void* y, double result[2]) {
  API_BEGIN
  PFMP_REQUIRE(ctx && x && y && result, PFMP_E_INVALID, "null argument");
  check_prec(prec);
  blas_cdot(ctx, prec, x, y, ctx->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(ctx->h_sums, ctx->d_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PFMP_CUDA(cudaStreamSynchronize(ctx->stream));
  result[0] = ctx->h_sums[0];
  result[1] = ctx->h_sums[1];
  API_END
}

int pfmp_axpy(pfmp_ctx* ctx, int prec, double a_re, double a_im, const void* x, void* y) {
  API_BEGIN
  PFMP_REQUIRE(ctx && x && y, PFMP_E_INVALID, "null argument");
  check_prec(prec);
  blas_axpy(ctx, prec, a_re, a_im, x, y);
  API_END
}

int pfmp_convert(pfmp_ctx* ctx, void* dst, int dst_prec, const void* src, int src_prec) {
  API_BEGIN
  PFMP_REQUIRE(ctx && dst && src, PFMP_E_INVALID, "null argument");
  check_prec_h(dst_prec);
  check_prec_h(src_prec);
  PFMP_REQUIRE(dst_prec == src_prec || (dst_prec != PFMP_H16 && src_prec != PFMP_H16) ||
                   dst_prec == PFMP_F32 || src_prec == PFMP_F32,
               PFMP_E_UNSUPPORTED, "FP16 fields convert to and from FP32 only");
  blas_copy(ctx, dst, dst_prec, src, src_prec);
  API_END
}

static int solve_impl(pfmp_op* op, const pfmp_solver_params* prm, void* x, const void* b, pfmp_solve_info* info) {
  int iters = 0, rel = 0;
  double res = 0;
  long kap = 0;
  int st = solve(op, prm->method, prm->tol, prm->max_iter, prm->delta, prm->check_every, x, b, &iters, &rel, &res, &kap);
  if (info) {
    info->iters = iters;
    info->reliable_updates = rel;
    info->true_rel_res = res;
    info->k_apply = kap;
    info->status = st;
  }
  if (st != PFMP_OK) set_last_error(pfmp_strerror(st));
  return st;
}

int pfmp_solve(pfmp_op* op, const pfmp_solver_params* prm, void* x, const void* b, pfmp_solve_info* info) {
  API_BEGIN
  PFMP_REQUIRE(op && prm && x && b, PFMP_E_INVALID, "null argument");
  int st = solve_impl(op, prm, x, b, info);
  if (st != PFMP_OK) return st;
  API_END
}

int pfmp_solve_host(pfmp_op* op, const pfmp_solver_params* prm, double* x_host, const double* b_host,
                    pfmp_solve_info* info) {
  API_BEGIN
  PFMP_REQUIRE(op && prm && x_host && b_host, PFMP_E_INVALID, "null argument");
  pfmp_ctx* c = op->ctx;
  // solver workspace slots 3 and 4 hold b and x of a host-memory solve
  void* b = op->cg64[3];
  void* x = op->cg64[4];
  spinor_pack_any(c, b, PFMP_F64, b_host, PFMP_HOST, 0);
  int st = solve_impl(op, prm, x, b, info);
  spinor_unpack_any(c, x_host, PFMP_HOST, x, PFMP_F64, 0);
  if (st != PFMP_OK) return st;
  API_END
}

int pfmp_solve_multishift(pfmp_op* op, int nshift, const double* sre, const double* sim, void* const* x, const void* b,
                          double tol, int max_iter, pfmp_solve_info* info) {
  API_BEGIN
  PFMP_REQUIRE(op && sre && sim && x && b && nshift >= 1, PFMP_E_INVALID, "bad argument");
  for (int k = 0; k < nshift; ++k) PFMP_REQUIRE(x[k] && x[k] != b, PFMP_E_INVALID, "bad solution pointer");
  std::vector<std::complex<double>> sig(nshift);
  for (int k = 0; k < nshift; ++k) sig[k] = std::complex<double>(sre[k], sim[k]);
  int it = 0;
  double res = 0;
  long kap = 0;
  int st = solve_multishift(op, PFMP_F64, nshift, sig.data(), x, b, tol, max_iter, 8, &it, &res, &kap,
                            info != nullptr);
  if (info) {
    info->iters = it;
    info->reliable_updates = 0;
    info->true_rel_res = res;
    info->k_apply = kap;
    info->status = st;
  }
  if (st != PFMP_OK) {
    set_last_error(pfmp_strerror(st));
    return st;
  }
  API_END
}

int pfmp_solve_multishift_prec(pfmp_op* op, int prec, int nshift, const double* sre, const double* sim, void* const* x,
                               const void* b, double tol, int max_iter, pfmp_solve_info* info) {
  API_BEGIN
  PFMP_REQUIRE(op && sre && sim && x && b && nshift >= 1, PFMP_E_INVALID, "bad argument");
  PFMP_REQUIRE(prec == PFMP_F64 || prec == PFMP_F32, PFMP_E_INVALID, "precision must be PFMP_F64 or PFMP_F32");
  for (int k = 0; k < nshift; ++k) PFMP_REQUIRE(x[k] && x[k] != b, PFMP_E_INVALID, "bad solution pointer");
  std::vector<std::complex<double>> sig(nshift);
  for (int k = 0; k < nshift; ++k) sig[k] = std::complex<double>(sre[k], sim[k]);
  int it = 0;
  double res = 0;
  long kap = 0;
  int st = solve_multishift(op, prec, nshift, sig.data(), x, b, tol, max_iter, 8, &it, &res, &kap,
                            info != nullptr && prec == PFMP_F64);
  if (info) {
    info->iters = it;
    info->reliable_updates = 0;
    info->true_rel_res = prec == PFMP_F64 ? res : -1.0;
    info->k_apply = kap;
    info->status = st;
  }
  if (st != PFMP_OK) {
    set_last_error(pfmp_strerror(st));
    return st;
  }
  API_END
}

int pfmp_poly_roots(int n, double mu, double nu, double* zre, double* zim, double* an) {
  API_BEGIN
  PFMP_REQUIRE(n >= 1 && mu >= nu && nu > 0, PFMP_E_INVALID, "need n >= 1 and mu >= nu > 0");
  auto z = cheb_roots(n, mu, nu);
  for (int k = 0; k < n; ++k) {
    if (zre) zre[k] = z[k].real();
    if (zim) zim[k] = z[k].imag();
  }
  if (an) *an = cheb_norm(n, mu, nu);
  API_END
}

int pfmp_poly_apply(pfmp_op* op, int n, double mu, double nu, int which, void* out, const void* in) {
  API_BEGIN
  PFMP_REQUIRE(op && out && in && out != in, PFMP_E_INVALID, "bad argument");
  PFMP_REQUIRE(mu >= nu && nu > 0 && n >= 1, PFMP_E_INVALID, "need n >= 1 and mu >= nu > 0");
  PFMP_REQUIRE(n % 2 == 0, PFMP_E_UNSUPPORTED, "odd polynomial orders are not supported");
  PFMP_REQUIRE(which >= 0 && which <= 2, PFMP_E_INVALID, "which must be 0 (P), 1 (R) or 2 (R^dag)");
  auto z = cheb_roots(n, mu, nu);
  const double an = cheb_norm(n, mu, nu);
  if (which == 0) {
    poly_product(op, stable_ordered(z), an, out, in);
  } else {
    std::vector<std::complex<double>> h;
    for (auto zk : z)
      if (zk.imag() < 0) h.push_back(which == 1 ? zk : std::conj(zk));
    poly_product(op, stable_ordered(h), std::sqrt(an), out, in);
  }
  API_END
}

int pfmp_spectrum(pfmp_op* op, int nsteps, const void* v0, double* lmin, double* lmax, double* alpha, double* beta,
                  int* steps) {
  API_BEGIN
  PFMP_REQUIRE(op && v0 && lmin && lmax && steps, PFMP_E_INVALID, "null argument");
  PFMP_REQUIRE(nsteps >= 1 && nsteps <= 100000, PFMP_E_INVALID, "nsteps must be in [1, 100000]");
  spectrum(op, nsteps, v0, lmin, lmax, alpha, beta, steps);
  API_END
}

int pfmp_balance_steps(int nlev, const double* fmax, int n_coarse, int* n) {
  API_BEGIN
  PFMP_REQUIRE(nlev >= 1 && fmax && n && n_coarse >= 1, PFMP_E_INVALID, "bad argument");
  int c = 0;
  for (int l = 0; l < nlev; ++l) {
    PFMP_REQUIRE(fmax[l] > 0 && std::isfinite(fmax[l]), PFMP_E_INVALID, "forces must be positive and finite");
    if (fmax[l] < fmax[c]) c = l;
  }
  for (int l = 0; l < nlev; ++l) {
    const double v = std::floor(n_coarse * fmax[l] / fmax[c] + 0.5);
    PFMP_REQUIRE(v < 1e9, PFMP_E_INVALID, "force ratio too large");
    n[l] = v < 1 ? 1 : (int)v;
  }
  API_END
}

int pfmp_cost(int ntraj, const int* accepted, const double* nmat, const double* dH, double tau_int,
              pfmp_cost_info* info) {
  API_BEGIN
  PFMP_REQUIRE(ntraj >= 2 && accepted && nmat && dH && info && tau_int > 0, PFMP_E_INVALID, "bad argument");
  auto mean_err = [&](auto f, double& m, double& e) {
    double s = 0;
    for (int i = 0; i < ntraj; ++i) s += f(i);
    m = s / ntraj;
    double v = 0;
    for (int i = 0; i < ntraj; ++i) v += (f(i) - m) * (f(i) - m);
    e = std::sqrt(2.0 * tau_int) * std::sqrt(v / (ntraj - 1)) / std::sqrt((double)ntraj);
  };
  pfmp_cost_info r{};
  mean_err([&](int i) { return accepted[i] ? 1.0 : 0.0; }, r.p_acc, r.p_acc_err);
  mean_err([&](int i) { return nmat[i]; }, r.nmat, r.nmat_err);
  mean_err([&](int i) { return std::exp(-dH[i]); }, r.exp_mdh, r.exp_mdh_err);
  if (r.p_acc > 0) {
    r.cost = r.nmat / r.p_acc;
    r.cost_err = r.cost * std::sqrt((r.nmat_err / r.nmat) * (r.nmat_err / r.nmat) +
                                    (r.p_acc_err / r.p_acc) * (r.p_acc_err / r.p_acc));
  } else {
    r.cost = r.cost_err = HUGE_VAL;
  }
  *info = r;
  API_END
}

int pfmp_action_scheme(int scheme, int p1, int p2, pfmp_action_def* def) {
  API_BEGIN
  PFMP_REQUIRE(def, PFMP_E_INVALID, "null argument");
  action_scheme(scheme, p1, p2, def);
  API_END
}

int pfmp_action_create_def(pfmp_ctx* ctx, const pfmp_action_def* def, pfmp_action** out) {
  API_BEGIN
  PFMP_REQUIRE(ctx && def && out, PFMP_E_INVALID, "null argument");
  *out = action_create_def(ctx, def);
  API_END
}

int pfmp_action_create(pfmp_ctx* ctx, const pfmp_action_params* prm, pfmp_action** out) {
  API_BEGIN
  PFMP_REQUIRE(ctx && prm && out, PFMP_E_INVALID, "null argument");
  *out = action_create(ctx, prm);
  API_END
}

int pfmp_action_destroy(pfmp_action* A) {
  API_BEGIN
  action_destroy(A);
  API_END
}

int pfmp_action_counts(pfmp_action* A, int* nterms, int* npf) {
  API_BEGIN
  PFMP_REQUIRE(A && nterms && npf, PFMP_E_INVALID, "null argument");
  *nterms = action_nterms(A);
  *npf = action_npf(A);
  API_END
}

int pfmp_action_refresh(pfmp_action* A) {
  API_BEGIN
  PFMP_REQUIRE(A, PFMP_E_INVALID, "null action");
  action_refresh(A);
  API_END
}

namespace {
// npf canonical host/device spinors -> temporary FP64 even device fields
struct NoiseFields {
  std::vector<double2*> d;
  NoiseFields(pfmp_action* A, const double* xi, int where) {
    pfmp_ctx* c = action_ctx(A);
    const size_t n = (size_t)c->g.V * 24;
    const int npf = action_npf(A);
    try {
      for (int i = 0; i < npf; ++i) {
        d.push_back((double2*)dev_alloc(spinor_bytes(c->g, PFMP_F64)));
        spinor_pack_any(c, d.back(), PFMP_F64, xi + i * n, where, 0);
      }
    } catch (...) {
      release();
      throw;
    }
  }
  void release() {
    for (auto p : d) dev_free(p);
    d.clear();
  }
  ~NoiseFields() { release(); }
  std::vector<const void*> ptrs() const { return std::vector<const void*>(d.begin(), d.end()); }
};
}  // namespace

int pfmp_action_heatbath(pfmp_action* A, const double* xi, int where) {
  API_BEGIN
  PFMP_REQUIRE(A && xi, PFMP_E_INVALID, "null argument");
  check_where(where);
  NoiseFields nf(A, xi, where);
  auto p = nf.ptrs();
  action_heatbath(A, p.data());
  PFMP_CUDA(cudaStreamSynchronize(action_ctx(A)->stream));
  API_END
}

int pfmp_action_get_phi(pfmp_action* A, int i, double* phi, int where) {
  API_BEGIN
  PFMP_REQUIRE(A && phi, PFMP_E_INVALID, "null argument");
  check_where(where);
  action_get_phi(A, i, phi, where);
  API_END
}

int pfmp_action_set_phi(pfmp_action* A, int i, const double* phi, int where) {
  API_BEGIN
  PFMP_REQUIRE(A && phi, PFMP_E_INVALID, "null argument");
  check_where(where);
  action_set_phi(A, i, phi, where);
  API_END
}

int pfmp_action_eval(pfmp_action* A, double* S) {
  API_BEGIN
  PFMP_REQUIRE(A && S, PFMP_E_INVALID, "null argument");
  action_eval(A, S);
  API_END
}

int pfmp_action_force(pfmp_action* A, int term, double* F, int where) {
  API_BEGIN
  PFMP_REQUIRE(A && F, PFMP_E_INVALID, "null argument");
  check_where(where);
  action_force_out(A, term, F, where);
  API_END
}

int pfmp_schedule_2mn(int n, double tau, double lambda, double* T, double* S) {
  API_BEGIN
  PFMP_REQUIRE(n >= 1 && T && S && tau > 0, PFMP_E_INVALID, "bad argument");
  schedule_2mn(n, tau, lambda, T, S);
  API_END
}

int pfmp_schedule_merge(int ns, const int* len, const double* T, const double* S, int cap, double* Tout, double* Sout,
                        int* len_out) {
  API_BEGIN
  PFMP_REQUIRE(ns >= 1 && len && T && S && Tout && Sout && len_out && cap >= 1, PFMP_E_INVALID, "bad argument");
  for (int i = 0; i < ns; ++i) PFMP_REQUIRE(len[i] >= 1, PFMP_E_INVALID, "empty scheme");
  *len_out = schedule_merge(ns, len, T, S, cap, Tout, Sout);
  API_END
}

int pfmp_trajectory(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level,
                    const double* mom, const double* xi, int where, double u, pfmp_traj_info* info) {
  API_BEGIN
  PFMP_REQUIRE(A && T && S && term_level && mom && xi && info, PFMP_E_INVALID, "null argument");
  check_where(where);
  NoiseFields nf(A, xi, where);
  auto p = nf.ptrs();
  trajectory(A, len, T, nlev, S, term_level, mom, where, p.data(), u, info);
  API_END
}

int pfmp_md(pfmp_action* A, int len, const double* T, int nlev, const double* S, const int* term_level, double* mom,
            int where) {
  API_BEGIN
  PFMP_REQUIRE(A && T && S && term_level && mom, PFMP_E_INVALID, "null argument");
  check_where(where);
  action_md(A, len, T, nlev, S, term_level, mom, where);
  API_END
}

int pfmp_batch_create(int nsys, pfmp_op* const* ops, const int* nrhs, pfmp_batch** out) {
  API_BEGIN
  PFMP_REQUIRE(out, PFMP_E_INVALID, "null argument");
  *out = batch_create(nsys, ops, nrhs);
  API_END
}

int pfmp_batch_destroy(pfmp_batch* B) {
  API_BEGIN
  batch_destroy(B);
  API_END
}

int pfmp_batch_tune(pfmp_batch* B, int chunk, int* block, double* ms) {
  API_BEGIN
  PFMP_REQUIRE(B && chunk >= 1, PFMP_E_INVALID, "bad argument");
  int bl = batch_tune(B, chunk, ms);
  if (block) *block = bl;
  API_END
}

int pfmp_batch_barrier_check(pfmp_batch* B, int rounds, int missing, double limit_s) {
  API_BEGIN
  PFMP_REQUIRE(B, PFMP_E_INVALID, "null argument");
  batch_barrier_check(B, rounds, missing, limit_s);
  API_END
}

int pfmp_batch_solve(pfmp_batch* B, const pfmp_solver_params* prm, void* const* x, const void* const* b,
                     pfmp_solve_info* infos) {
  API_BEGIN
  PFMP_REQUIRE(B && prm && x && b, PFMP_E_INVALID, "null argument");
  int st = batch_solve(B, prm->tol, prm->max_iter, prm->delta, prm->check_every, x, b, infos);
  if (st != PFMP_OK) {
    set_last_error(pfmp_strerror(st));
    return st;
  }
  API_END
}

int pfmp_nn_create(pfmp_ctx* ctx, int nl, const int* ch, int prec, pfmp_nn** out) {
  API_BEGIN
  PFMP_REQUIRE(ctx && ch && out, PFMP_E_INVALID, "null argument");
  *out = nn_create(ctx, nl, ch, prec);
  API_END
}

int pfmp_nn_destroy(pfmp_nn* nn) {
  API_BEGIN
  nn_destroy(nn);
  API_END
}

int64_t pfmp_nn_num_weights(const pfmp_nn* nn) { return nn ? (int64_t)nn_num_weights(nn) : -1; }

int pfmp_nn_set_weights(pfmp_nn* nn, const double* w) {
  API_BEGIN
  PFMP_REQUIRE(nn && w, PFMP_E_INVALID, "null argument");
  nn_set_weights(nn, w);
  API_END
}

int pfmp_nn_get_weights(pfmp_nn* nn, double* w) {
  API_BEGIN
  PFMP_REQUIRE(nn && w, PFMP_E_INVALID, "null argument");
  nn_get_weights(nn, w);
  API_END
}

int pfmp_nn_apply(pfmp_nn* nn, int prec, void* out, const void* in) {
  API_BEGIN
  PFMP_REQUIRE(nn && out && in && out != in, PFMP_E_INVALID, "bad argument");
  check_prec(prec);
  nn_apply(nn, out, in, prec);
  nn_check(nn);
  API_END
}

int pfmp_nn_set_tensor_cores(pfmp_nn* nn, int on) {
  API_BEGIN
  PFMP_REQUIRE(nn, PFMP_E_INVALID, "null network");
  nn_set_tc(nn, on != 0);
  API_END
}

int pfmp_nn_loss_grad(pfmp_nn* nn, pfmp_op* op, int kind, const void* b, const void* x, double* loss, double* grad) {
  API_BEGIN
  PFMP_REQUIRE(nn && b && x && loss, PFMP_E_INVALID, "null argument");
  nn_zero_grad(nn);
  *loss = nn_loss_grad(nn, op, kind, b, x, 1.0);
  if (grad) nn_get_grads(nn, grad);
  API_END
}

int pfmp_nn_train(pfmp_nn* nn, pfmp_op* op, int kind, int npairs, const void* const* b, const void* const* x, int steps,
                  int batch, double lr, double* final_loss) {
  API_BEGIN
  PFMP_REQUIRE(nn && b && x, PFMP_E_INVALID, "null argument");
  double l = nn_train(nn, op, kind, npairs, b, x, steps, batch, lr);
  if (final_loss) *final_loss = l;
  API_END
}

int pfmp_solve_fgcr(pfmp_op* op, pfmp_nn* nn, const pfmp_solver_params* prm, void* x, const void* b,
                    pfmp_solve_info* info) {
  API_BEGIN
  PFMP_REQUIRE(op && prm && x && b && x != b, PFMP_E_INVALID, "bad argument");
  int it = 0, outer = 0, fb = 0;
  double res = 0;
  long kap = 0;
  int st = solve_fgcr(op, nn, prm->tol, prm->max_iter, prm->restart, prm->delta, x, b, &it, &outer, &res, &kap, &fb);
  if (info) {
    info->iters = it;
    info->reliable_updates = fb;
    info->true_rel_res = res;
    info->k_apply = kap;
    info->status = st;
  }
  if (st != PFMP_OK) {
    set_last_error(pfmp_strerror(st));
    return st;
  }
  API_END
}

int pfmp_profile_begin(pfmp_ctx* ctx) {
  API_BEGIN
  PFMP_REQUIRE(ctx, PFMP_E_INVALID, "null context");
  profile_begin(ctx);
  API_END
}

int pfmp_profile_end(pfmp_ctx* ctx, int cls, int64_t* launches, double* total_ms, double* total_bytes) {
  API_BEGIN
  PFMP_REQUIRE(ctx && launches && total_ms && total_bytes, PFMP_E_INVALID, "null argument");
  PFMP_REQUIRE(cls == PFMP_KERNEL_HOP_F32 || cls == PFMP_KERNEL_HOP_F64 || cls == PFMP_KERNEL_HOP_DF ||
                   cls == PFMP_KERNEL_HOP_H16 || cls == PFMP_KERNEL_CG_F32,
               PFMP_E_INVALID,
               "bad kernel class");
  long n = 0;
  profile_end(ctx, cls, &n, total_ms, total_bytes);
  *launches = n;
  API_END
}

int pfmp_fma_rate(pfmp_ctx* ctx, int prec, double* tflops) {
  API_BEGIN
  PFMP_REQUIRE(ctx && tflops, PFMP_E_INVALID, "null argument");
  PFMP_REQUIRE(prec == PFMP_F64 || prec == PFMP_F32, PFMP_E_INVALID, "precision must be PFMP_F64 or PFMP_F32");
  *tflops = fma_rate(ctx, prec);
  API_END
}

}  // extern "C"
