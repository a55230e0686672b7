// Conjugate gradient on K = M-hat^dag M-hat (the paper's solver, Sec. 2.1, Sec. 3.1):
//  * CG64: FP64 throughout.
//  * half: as mixed, with the search direction p and K p in FP16 storage (per-site FP32
//    scales) and FP32 arithmetic; x and r stay FP32.
//  * mixed: FP32 CG ("sloppy") with FP64 reliable updates: every time the sloppy residual
//    has fallen by `delta` (or reached the target) the accumulated FP32 solution is
//    added to the FP64 solution and the true residual b - K x is recomputed (in
//    double-float on the FP32 pipe, and in FP64 once it is below the target: the FP64
//    value decides and is reported); the sloppy residual restarts from it while the
//    search direction is kept.
// The iteration runs on the device with no host round trip: alpha and beta come from
// device scalars written by the reduction finishers, and a `done` flag makes every
// queued kernel return at once after convergence.  The host looks at the scalars
// every `check_every` iterations.  Zero initial guess (history-free, reversible MD).
#include <cmath>

#include "context.h"

namespace pfmp {

// beta: the pending step of the fused FP32 iteration (p = r + beta p_old is formed by the
// next iteration); 0 starts from p = r
static void put_scalars(pfmp_op* op, double rr, double stop_rr, double beta = 0.0) {
  CGScalars* h = op->h_scal;
  h->rr = rr;
  h->rr_new = rr;
  h->pAp = 0;
  h->alpha = 0;
  h->beta = beta;
  h->stop_rr = stop_rr;
  h->done = 0;
  h->done_next = 0;
  h->iter = 0;
  PFMP_CUDA(cudaMemcpyAsync(op->scal, h, sizeof(CGScalars), cudaMemcpyHostToDevice, op->ctx->stream));
}
static void get_scalars(pfmp_op* op) {
  PFMP_CUDA(cudaMemcpyAsync(op->h_scal, op->scal, sizeof(CGScalars), cudaMemcpyDeviceToHost, op->ctx->stream));
  PFMP_CUDA(cudaStreamSynchronize(op->ctx->stream));
}
static double host_norm2(pfmp_op* op, int prec, const void* x) {
  pfmp_ctx* c = op->ctx;
  blas_norm2(c, prec, x, c->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_sums[0];
}

// r = b - K x in FP64; returns |r|^2
static double true_residual(pfmp_op* op, const void* x, const void* b, void* r, void* Ax) {
  pfmp_ctx* c = op->ctx;
  kop(op, PFMP_F64, Ax, x, nullptr, nullptr);
  blas_xmy_norm(c, b, Ax, r, c->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_sums[0];
}

// The fused FP32 iteration reads fewer CG-vector bytes but more per stencil site (two
// fields at every neighbour in its first phase) and runs at a lower occupancy; it wins
// where the solve's working set (links, clover, five FP32 fields: ~1440 B per
// half-lattice site) stays in L2 (16^3x32: 7.25 vs 8.43 ms per solve) and loses a few per
// cent where K streams from HBM (32^3x64: 102 vs 99 ms), so it is used up to the L2 size.
static bool fused_iteration(pfmp_op* op) {
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, op->ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return 1440.0 * op->ctx->g.Vh <= (double)l2;
}

static void launch_chunk(pfmp_op* op, int prec, void* x, void* r, void* p, void* Ap, int chunk) {
  pfmp_ctx* c = op->ctx;
  if (prec == PFMP_F32 && fused_iteration(op)) {  // four kernels per iteration, updates fused in
    for (int k = 0; k < chunk; ++k) cg_fused_iteration(op, (float4*)x, (float4*)r, (float4*)p);
    return;
  }
  for (int k = 0; k < chunk; ++k) {
    kop(op, prec, Ap, p, &op->scal->pAp, op->scal);
    cg_step_xr(c, prec, x, r, p, Ap, op->scal);
    cg_step_p(c, prec, p, r, op->scal);
  }
}

// One chunk of CG iterations.  Without kernel profiling the chunk is captured once into
// a CUDA graph (6 kernels per iteration, 4 for FP32; all parameters fixed: the scalars
// live on the device) and replayed on the context's stream, which removes the per-launch
// host cost.
// K applications are counted by run_cg from the iterations the device actually ran (the
// queued kernels of a converged chunk return at once), so the count kop keeps while the
// chunk is launched or captured is put back afterwards.
static void run_chunk(pfmp_op* op, int prec, void* x, void* r, void* p, void* Ap, int chunk) {
  pfmp_ctx* c = op->ctx;
  const long long kapply0 = op->kapply;
  if (c->prof.on) {
    launch_chunk(op, prec, x, r, p, Ap, chunk);
    op->kapply = kapply0;
    return;
  }
  pfmp_op::Graph& G = op->graph[prec];
  const void* key[4] = {x, r, p, Ap};
  bool hit = G.exec && G.chunk == chunk;
  for (int k = 0; k < 4 && hit; ++k) hit = G.key[k] == key[k];
  if (!hit) {
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
    if (!op->cap) PFMP_CUDA(cudaStreamCreateWithFlags(&op->cap, cudaStreamNonBlocking));
    cudaStream_t keep = c->stream;
    cudaGraph_t graph = nullptr;
    PFMP_CUDA(cudaStreamBeginCapture(op->cap, cudaStreamCaptureModeThreadLocal));
    c->stream = op->cap;
    const long long n0 = launch_count();
    try {
      launch_chunk(op, prec, x, r, p, Ap, chunk);
    } catch (...) {
      c->stream = keep;
      cudaStreamEndCapture(op->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    c->stream = keep;
    op->kapply = kapply0;
    G.kernels = launch_count() - n0;
    count_launches(-G.kernels);  // captured, not launched
    PFMP_CUDA(cudaStreamEndCapture(op->cap, &graph));
    cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    PFMP_CUDA(e);
    G.chunk = chunk;
    for (int k = 0; k < 4; ++k) G.key[k] = key[k];
  }
  PFMP_CUDA(cudaGraphLaunch(G.exec, c->stream));
  count_launches(G.kernels);
}

// run the device CG loop (prec) until `done` or the iteration cap; returns iterations
static int run_cg(pfmp_op* op, int prec, void* x, void* r, void* p, void* Ap, int max_iter, int check_every) {
  int done_iters = 0;
  for (;;) {
    const int chunk = check_every < max_iter - done_iters ? check_every : max_iter - done_iters;
    if (chunk <= 0) break;
    run_chunk(op, prec, x, r, p, Ap, chunk);
    get_scalars(op);
    op->kapply += op->h_scal->iter - done_iters;
    done_iters = op->h_scal->iter;
    if (op->h_scal->done) break;
  }
  return done_iters;
}

int solve(pfmp_op* op, int method, double tol, int max_iter, double delta, int check_every, void* x, const void* b,
          int* iters, int* rel_updates, double* true_res, long* kapply) {
  pfmp_ctx* c = op->ctx;
  PFMP_REQUIRE(x != b, PFMP_E_INVALID, "x and b must not alias");
  PFMP_REQUIRE(tol > 0 && max_iter > 0, PFMP_E_INVALID, "tol and max_iter must be positive");
  if (check_every <= 0) check_every = 8;
  if (!(delta > 0 && delta < 1)) delta = 0.1;
  *iters = 0;
  *rel_updates = 0;
  *kapply = 0;
  const double bb = host_norm2(op, PFMP_F64, b);
  blas_zero(c, PFMP_F64, x);
  if (bb == 0.0) {
    *true_res = 0.0;
    return PFMP_OK;
  }
  PFMP_REQUIRE(std::isfinite(bb), PFMP_E_NAN, "right-hand side is not finite");
  void* r = op->cg64[0];
  void* p = op->cg64[1];
  void* Ap = op->cg64[2];
  double rr_true = bb;
  int total = 0;
  if (method == PFMP_SOLVER_CG64) {
    // the solution accumulates in an operator-owned buffer (a stable CUDA-graph key) and
    // is copied to x at the end; restart from the true residual if the recursive one
    // drifted below it
    void* xa = op->cg64[5];
    blas_zero(c, PFMP_F64, xa);
    PFMP_CUDA(cudaMemcpyAsync(r, b, spinor_bytes(c->g, PFMP_F64), cudaMemcpyDeviceToDevice, c->stream));
    for (int restart = 0; restart < 8 && total < max_iter; ++restart) {
      PFMP_CUDA(cudaMemcpyAsync(p, r, spinor_bytes(c->g, PFMP_F64), cudaMemcpyDeviceToDevice, c->stream));
      put_scalars(op, rr_true, 0.25 * tol * tol * bb);
      const int it = run_cg(op, PFMP_F64, xa, r, p, Ap, max_iter - total, check_every);
      total += it;
      *kapply += it;
      PFMP_REQUIRE(std::isfinite(op->h_scal->rr), PFMP_E_NAN, "CG residual became NaN/Inf");
      rr_true = true_residual(op, xa, b, r, Ap);
      *kapply += 1;
      if (std::sqrt(rr_true / bb) < tol) break;
    }
    PFMP_CUDA(cudaMemcpyAsync(x, xa, spinor_bytes(c->g, PFMP_F64), cudaMemcpyDeviceToDevice, c->stream));
  } else if (method == PFMP_SOLVER_CG_MIXED || method == PFMP_SOLVER_CG_HALF) {
    // sloppy CG: x and r in FP32; p and Kp in FP32, or in FP16 storage for CG_HALF
    const int sp = method == PFMP_SOLVER_CG_HALF ? PFMP_H16 : PFMP_F32;
    float4* r32 = op->cg32[0];
    void* p32 = sp == PFMP_H16 ? (void*)op->cg16[0] : (void*)op->cg32[1];
    void* Ap32 = sp == PFMP_H16 ? (void*)op->cg16[1] : (void*)op->cg32[2];
    float4* xs32 = op->cg32[3];
    PFMP_CUDA(cudaMemcpyAsync(r, b, spinor_bytes(c->g, PFMP_F64), cudaMemcpyDeviceToDevice, c->stream));
    blas_copy(c, r32, PFMP_F32, r, PFMP_F64);
    blas_copy(c, p32, sp, r32, PFMP_F32);
    blas_zero(c, PFMP_F32, xs32);
    double rr_s = host_norm2(op, PFMP_F32, r32);
    double beta = 0.0;  // the fused FP32 iteration's pending step, kept across updates
    while (total < max_iter) {
      // sloppy target: a factor delta below the last true residual, not below tol
      double stop = delta * delta * rr_true;
      const double floor_rr = 0.25 * tol * tol * bb;
      if (stop < floor_rr) stop = floor_rr;
      put_scalars(op, rr_s, stop, sp == PFMP_F32 ? beta : 0.0);
      const int it = run_cg(op, sp, xs32, r32, p32, Ap32, max_iter - total, check_every);
      total += it;
      *kapply += it;
      PFMP_REQUIRE(std::isfinite(op->h_scal->rr), PFMP_E_NAN, "sloppy CG residual became NaN/Inf");
      beta = op->h_scal->beta;
      // reliable update: the true residual in double-float (FP32 pipe), confirmed in FP64
      // once it is below the target
      blas_add_lo(c, x, xs32);
      rr_true = true_residual_mixed(op, x, b, r, tol * tol * bb, kapply);
      *rel_updates += 1;
      if (std::sqrt(rr_true / bb) < tol) break;
      blas_copy(c, r32, PFMP_F32, r, PFMP_F64);
      blas_zero(c, PFMP_F32, xs32);
      rr_s = host_norm2(op, PFMP_F32, r32);
      if (it == 0) {  // stalled: restart the direction as well
        blas_copy(c, p32, sp, r32, PFMP_F32);
        beta = 0.0;
      }
    }
  } else {
    PFMP_REQUIRE(false, PFMP_E_INVALID, "unknown solver method");
  }
  *iters = total;
  *true_res = std::sqrt(rr_true / bb);
  PFMP_REQUIRE(std::isfinite(*true_res), PFMP_E_NAN, "true residual is not finite");
  return *true_res < tol ? PFMP_OK : PFMP_E_NOT_CONVERGED;
}

}  // namespace pfmp
