// Batched multi-system, multi-right-hand-side mixed-precision CG.
//
// Many independent systems K_s x_{s,r} = b_{s,r} (different lattices, gauge fields and
// kappa; R_s right-hand sides each) run as ONE set of grouped kernels: every launch
// covers all (system, site block, rhs) tiles, with the R_s tiles of one site block
// adjacent in the grid so that their link and clover reads share the L2.  Six grouped
// launches make one CG iteration for the whole batch (four stencil phases of K, the x/r
// update and the p update); a chunk of iterations is captured once as a CUDA graph and
// replayed, with per-(system, rhs) device scalars so that converged systems skip their
// work.  The FP32 iterations are corrected by FP64 reliable updates per (system, rhs),
// exactly as in the single-system mixed solver.  Block size per tile is chosen by a
// small autotuner (timed replays of one chunk).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hop.cuh"

namespace pfmp {

struct BatchSys {
  HopParams<PFMP_F32> hp;  // geometry, gauge, reduction buffer of the system's context
  const float4* clov_e;
  const float4* clov_o;
  double kappa2;
  int R, nsb, block0;
  long fw;  // float4 words per FP32 field (6 Vh)
  float4 *x, *r, *p, *Ap, *t, *e;  // R consecutive fields each
  CGScalars* scal;                 // [R]
  double* partials;                // [R][nsb]
  unsigned* tickets;               // [R]
};

struct TileRef {
  int s, sb, r;
};

__device__ __forceinline__ TileRef tile(const BatchSys* sys, const int* map) {
  TileRef t;
  t.s = map[blockIdx.x];
  const BatchSys& S = sys[t.s];
  const int local = blockIdx.x - S.block0;
  t.sb = local / S.R;
  t.r = local % S.R;
  return t;
}

// PHASE 1: t = A_oo^{-1} H_oe v; PHASE 2: w = A_ee v - kappa^2 H_eo t (v = p, w = e for
// M-hat; v = e, w = Ap for M-hat^dag); the non-dagger PHASE 2 reduces ||e||^2 = <p, K p>
template <bool DAG, int PHASE>
__global__ void __launch_bounds__(256) k_batch_hop(const BatchSys* __restrict__ sys, const int* __restrict__ map) {
  const TileRef T = tile(sys, map);
  const BatchSys& S = sys[T.s];
  CGScalars* sc = S.scal + T.r;
  if (sc->done) return;
  HopParams<PFMP_F32> a = S.hp;
  const long off = (long)T.r * S.fw;
  const float4* v = (DAG ? S.e : S.p) + off;
  if (PHASE == 1) {
    a.p = 1;
    a.in = v;
    a.out = S.t + off;
    a.clov = S.clov_o;
    a.coef = 1.0;
  } else {
    a.p = 0;
    a.in = S.t + off;
    a.x = v;
    a.out = (DAG ? S.Ap : S.e) + off;
    a.clov = S.clov_e;
    a.coef = -S.kappa2;
  }
  const int cb = T.sb * blockDim.x + threadIdx.x;
  constexpr bool RED = (PHASE == 2 && !DAG);
  double nrm[1] = {0.0};
  if (cb < a.g.Vh) {
    auto out = hop_site<PFMP_F32, DAG, PHASE == 1 ? EPI_CLOV : EPI_XPAY>(a, cb);
    store_spinor(a.out, out, cb, a.g.Vh);
    if (RED) nrm[0] = spinor_norm2(out);
  }
  if (RED) {
    double tot[1];
    if (group_sum<1>(nrm, S.partials + (size_t)T.r * S.nsb, S.tickets + T.r, S.nsb, T.sb, tot)) {
      sc->pAp = tot[0];
      sc->alpha = sc->rr / tot[0];
    }
  }
}

// x += alpha p, r -= alpha Ap, |r|^2 -> beta, rr, iter, done_next
__global__ void __launch_bounds__(256) k_batch_xr(const BatchSys* __restrict__ sys, const int* __restrict__ map) {
  const TileRef T = tile(sys, map);
  const BatchSys& S = sys[T.s];
  CGScalars* sc = S.scal + T.r;
  if (sc->done) return;
  const long off = (long)T.r * S.fw;
  const int Vh = S.hp.g.Vh;
  const int cb = T.sb * blockDim.x + threadIdx.x;
  const float al = (float)sc->alpha;
  double v[1] = {0.0};
  float acc = 0.f;  // the site's |r|^2 in FP32, across sites in FP64
  if (cb < Vh) {
    for (int k = 0; k < 6; ++k) {
      const long i = off + (long)k * Vh + cb;
      float4 xx = S.x[i], rr = S.r[i];
      const float4 pp = S.p[i], aa = S.Ap[i];
      xx.x += al * pp.x;
      xx.y += al * pp.y;
      xx.z += al * pp.z;
      xx.w += al * pp.w;
      rr.x -= al * aa.x;
      rr.y -= al * aa.y;
      rr.z -= al * aa.z;
      rr.w -= al * aa.w;
      S.x[i] = xx;
      S.r[i] = rr;
      acc += rr.x * rr.x + rr.y * rr.y + rr.z * rr.z + rr.w * rr.w;
    }
  }
  v[0] = acc;
  double t[1];
  if (group_sum<1>(v, S.partials + (size_t)T.r * S.nsb, S.tickets + T.r, S.nsb, T.sb, t)) {
    sc->rr_new = t[0];
    sc->beta = t[0] / sc->rr;
    sc->rr = t[0];
    sc->iter += 1;
    if (t[0] < sc->stop_rr || !(t[0] == t[0])) sc->done_next = 1;
  }
}

// p = r + beta p; the last tile of the (system, rhs) raises done if requested
__global__ void __launch_bounds__(256) k_batch_p(const BatchSys* __restrict__ sys, const int* __restrict__ map) {
  const TileRef T = tile(sys, map);
  const BatchSys& S = sys[T.s];
  CGScalars* sc = S.scal + T.r;
  if (sc->done) return;
  const long off = (long)T.r * S.fw;
  const int Vh = S.hp.g.Vh;
  const int cb = T.sb * blockDim.x + threadIdx.x;
  const float be = (float)sc->beta;
  if (cb < Vh) {
    for (int k = 0; k < 6; ++k) {
      const long i = off + (long)k * Vh + cb;
      const float4 rr = S.r[i], pp = S.p[i];
      S.p[i] = make_float4(rr.x + be * pp.x, rr.y + be * pp.y, rr.z + be * pp.z, rr.w + be * pp.w);
    }
  }
  double v[1] = {0.0}, t[1];
  if (group_sum<1>(v, S.partials + (size_t)T.r * S.nsb, S.tickets + T.r, S.nsb, T.sb, t)) sc->done = sc->done_next;
}

}  // namespace pfmp

using namespace pfmp;

struct pfmp_batch {
  std::vector<pfmp_op*> ops;
  std::vector<int> R;
  std::vector<BatchSys> sys;
  BatchSys* d_sys = nullptr;
  int* d_map = nullptr;
  int nblocks = 0, block = 128;
  std::vector<float4*> bufs;  // per system: one allocation of 6 R fields
  CGScalars* d_scal = nullptr;
  CGScalars* h_scal = nullptr;
  double* d_part = nullptr;
  unsigned* d_tick = nullptr;
  int total_rhs = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int exec_chunk = 0, exec_block = 0;
  long long graph_kernels = 0;
  bool tuned = false;
};

namespace pfmp {

static void batch_layout(pfmp_batch* B, int block) {
  B->block = block;
  int blk = 0;
  std::vector<int> map;
  for (size_t s = 0; s < B->sys.size(); ++s) {
    BatchSys& S = B->sys[s];
    S.nsb = (S.hp.g.Vh + block - 1) / block;
    S.block0 = blk;
    blk += S.nsb * S.R;
    for (int i = 0; i < S.nsb * S.R; ++i) map.push_back((int)s);
  }
  PFMP_REQUIRE(blk < (1 << 30), PFMP_E_INVALID, "batch too large");
  B->nblocks = blk;
  dev_free(B->d_map);
  dev_free(B->d_part);
  B->d_map = (int*)dev_alloc(map.size() * sizeof(int));
  // partials: per (system, rhs) nsb doubles
  size_t np = 0;
  for (auto& S : B->sys) np += (size_t)S.R * S.nsb;
  B->d_part = (double*)dev_alloc(np * sizeof(double));
  size_t off = 0;
  for (auto& S : B->sys) {
    S.partials = B->d_part + off;
    off += (size_t)S.R * S.nsb;
  }
  PFMP_CUDA(cudaMemcpy(B->d_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice));
  PFMP_CUDA(cudaMemcpy(B->d_sys, B->sys.data(), B->sys.size() * sizeof(BatchSys), cudaMemcpyHostToDevice));
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
}

void batch_destroy(pfmp_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (auto p : B->bufs) dev_free(p);
  dev_free(B->d_sys);
  dev_free(B->d_map);
  dev_free(B->d_scal);
  dev_free(B->d_part);
  dev_free(B->d_tick);
  if (B->h_scal) cudaFreeHost(B->h_scal);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
}

pfmp_batch* batch_create(int nsys, pfmp_op* const* ops, const int* nrhs) {
  PFMP_REQUIRE(nsys >= 1 && ops && nrhs, PFMP_E_INVALID, "bad batch description");
  pfmp_batch* B = new pfmp_batch();
  try {
    B->stream = ops[0]->ctx->stream;
    int tot = 0;
    for (int s = 0; s < nsys; ++s) {
      PFMP_REQUIRE(ops[s] && nrhs[s] >= 1 && nrhs[s] <= 64, PFMP_E_INVALID, "each system needs an operator and 1..64 rhs");
      B->ops.push_back(ops[s]);
      B->R.push_back(nrhs[s]);
      tot += nrhs[s];
    }
    B->total_rhs = tot;
    B->d_scal = (CGScalars*)dev_alloc(tot * sizeof(CGScalars));
    B->d_tick = (unsigned*)dev_alloc(tot * sizeof(unsigned));
    PFMP_CUDA(cudaMemset(B->d_tick, 0, tot * sizeof(unsigned)));
    PFMP_CUDA(cudaMallocHost(&B->h_scal, tot * sizeof(CGScalars)));
    int off = 0;
    for (int s = 0; s < nsys; ++s) {
      pfmp_op* op = ops[s];
      BatchSys S{};
      S.hp.g = op->ctx->g;
      S.hp.gauge = op->ctx->U32;
      S.hp.rb = op->ctx->rb;
      S.hp.scal = nullptr;
      S.hp.norm_out = nullptr;
      S.clov_e = op->clov32[0];
      S.clov_o = op->clov32[1];
      S.kappa2 = op->kappa * op->kappa;
      S.R = nrhs[s];
      S.fw = 6L * op->ctx->g.Vh;
      float4* buf = (float4*)dev_alloc((size_t)6 * S.R * S.fw * sizeof(float4));
      B->bufs.push_back(buf);
      S.x = buf;
      S.r = buf + 1 * S.R * S.fw;
      S.p = buf + 2 * S.R * S.fw;
      S.Ap = buf + 3 * S.R * S.fw;
      S.t = buf + 4 * S.R * S.fw;
      S.e = buf + 5 * S.R * S.fw;
      S.scal = B->d_scal + off;
      S.tickets = B->d_tick + off;
      off += S.R;
      B->sys.push_back(S);
    }
    B->d_sys = (BatchSys*)dev_alloc(nsys * sizeof(BatchSys));
    batch_layout(B, 128);
  } catch (...) {
    batch_destroy(B);
    throw;
  }
  return B;
}

static void batch_launch_chunk(pfmp_batch* B, cudaStream_t st, int chunk) {
  const int g = B->nblocks, b = B->block;
  for (int k = 0; k < chunk; ++k) {
    k_batch_hop<false, 1><<<g, b, 0, st>>>(B->d_sys, B->d_map);
    PFMP_CHECK_LAUNCH();
    k_batch_hop<false, 2><<<g, b, 0, st>>>(B->d_sys, B->d_map);
    PFMP_CHECK_LAUNCH();
    k_batch_hop<true, 1><<<g, b, 0, st>>>(B->d_sys, B->d_map);
    PFMP_CHECK_LAUNCH();
    k_batch_hop<true, 2><<<g, b, 0, st>>>(B->d_sys, B->d_map);
    PFMP_CHECK_LAUNCH();
    k_batch_xr<<<g, b, 0, st>>>(B->d_sys, B->d_map);
    PFMP_CHECK_LAUNCH();
    k_batch_p<<<g, b, 0, st>>>(B->d_sys, B->d_map);
    PFMP_CHECK_LAUNCH();
  }
}

static void batch_run_chunk(pfmp_batch* B, int chunk) {
  if (!B->exec || B->exec_chunk != chunk || B->exec_block != B->block) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    if (!B->cap) PFMP_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    PFMP_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    const long long n0 = launch_count();
    try {
      batch_launch_chunk(B, B->cap, chunk);
    } catch (...) {
      cudaStreamEndCapture(B->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    B->graph_kernels = launch_count() - n0;
    count_launches(-B->graph_kernels);
    PFMP_CUDA(cudaStreamEndCapture(B->cap, &graph));
    cudaError_t e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    PFMP_CUDA(e);
    B->exec_chunk = chunk;
    B->exec_block = B->block;
  }
  PFMP_CUDA(cudaGraphLaunch(B->exec, B->stream));
  count_launches(B->graph_kernels);
}

// per (system, rhs): x64 += xs, r64 = b - K x64 (FP64), returns |r64|^2 / |b|^2 and, if
// not converged, restarts the sloppy residual from r64
struct RhsState {
  double bb = 0, rr_true = 0;
  bool finished = false;
  int iters = 0, rel = 0;
  long kres = 0;  // K applications of the true residuals (double-float, FP64 confirmation)
  double res = 0;
};

static void put_scal(pfmp_batch* B, int idx, double rr, double stop) {
  CGScalars h{};
  h.rr = rr;
  h.rr_new = rr;
  h.stop_rr = stop;
  PFMP_CUDA(cudaMemcpyAsync(B->d_scal + idx, &h, sizeof(CGScalars), cudaMemcpyHostToDevice, B->stream));
  PFMP_CUDA(cudaStreamSynchronize(B->stream));
}

static double norm_sync(pfmp_ctx* c, int prec, const void* x) {
  blas_norm2(c, prec, x, c->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_sums[0];
}

int batch_solve(pfmp_batch* B, double tol, int max_iter, double delta, int check, void* const* x, const void* const* b,
                pfmp_solve_info* infos) {
  PFMP_REQUIRE(tol > 0 && max_iter > 0, PFMP_E_INVALID, "tol and max_iter must be positive");
  if (!(delta > 0 && delta < 1)) delta = 1e-4;
  if (check <= 0) check = 8;
  const int ns = (int)B->sys.size();
  // every context runs on the batch stream for the duration of the solve
  std::vector<cudaStream_t> keep(ns);
  for (int s = 0; s < ns; ++s) {
    keep[s] = B->ops[s]->ctx->stream;
    B->ops[s]->ctx->stream = B->stream;
  }
  std::vector<RhsState> st(B->total_rhs);
  int status = PFMP_OK;
  try {
    // initial residuals
    int idx = 0;
    for (int s = 0; s < ns; ++s) {
      pfmp_op* op = B->ops[s];
      pfmp_ctx* c = op->ctx;
      BatchSys& S = B->sys[s];
      for (int r = 0; r < S.R; ++r, ++idx) {
        const void* bb = b[idx];
        blas_zero(c, PFMP_F64, x[idx]);
        st[idx].bb = norm_sync(c, PFMP_F64, bb);
        float4* r32 = S.r + r * S.fw;
        blas_copy(c, r32, PFMP_F32, bb, PFMP_F64);
        PFMP_CUDA(cudaMemcpyAsync(S.p + r * S.fw, r32, spinor_bytes(c->g, PFMP_F32), cudaMemcpyDeviceToDevice, B->stream));
        PFMP_CUDA(cudaMemsetAsync(S.x + r * S.fw, 0, spinor_bytes(c->g, PFMP_F32), B->stream));
        st[idx].rr_true = st[idx].bb;
        if (st[idx].bb == 0.0) {
          st[idx].finished = true;
          CGScalars h{};
          h.done = 1;
          PFMP_CUDA(cudaMemcpyAsync(B->d_scal + idx, &h, sizeof(CGScalars), cudaMemcpyHostToDevice, B->stream));
          continue;
        }
        const double rr32 = norm_sync(c, PFMP_F32, r32);
        put_scal(B, idx, rr32, std::max(delta * delta * st[idx].bb, 0.25 * tol * tol * st[idx].bb));
      }
    }
    int done_iters = 0;
    int remaining = 0;
    for (auto& s : st) remaining += !s.finished;
    while (remaining > 0 && done_iters < max_iter) {
      batch_run_chunk(B, check);
      done_iters += check;
      PFMP_CUDA(cudaMemcpyAsync(B->h_scal, B->d_scal, B->total_rhs * sizeof(CGScalars), cudaMemcpyDeviceToHost,
                                B->stream));
      PFMP_CUDA(cudaStreamSynchronize(B->stream));
      idx = 0;
      for (int s = 0; s < ns; ++s) {
        pfmp_op* op = B->ops[s];
        pfmp_ctx* c = op->ctx;
        BatchSys& S = B->sys[s];
        for (int r = 0; r < S.R; ++r, ++idx) {
          RhsState& R = st[idx];
          if (R.finished || !B->h_scal[idx].done) continue;
          R.iters += B->h_scal[idx].iter;
          PFMP_REQUIRE(std::isfinite(B->h_scal[idx].rr), PFMP_E_NAN, "batched CG residual became NaN/Inf");
          // reliable update: double-float true residual, confirmed in FP64 below the target
          blas_add_lo(c, x[idx], S.x + r * S.fw);
          void* r64 = op->cg64[0];
          R.rr_true = true_residual_mixed(op, x[idx], b[idx], r64, tol * tol * R.bb, &R.kres);
          R.rel += 1;
          R.res = std::sqrt(R.rr_true / R.bb);
          if (R.res < tol) {
            R.finished = true;
            --remaining;
            continue;  // scalars keep done = 1
          }
          float4* r32 = S.r + r * S.fw;
          blas_copy(c, r32, PFMP_F32, r64, PFMP_F64);
          PFMP_CUDA(cudaMemsetAsync(S.x + r * S.fw, 0, spinor_bytes(c->g, PFMP_F32), B->stream));
          const double rr32 = norm_sync(c, PFMP_F32, r32);
          put_scal(B, idx, rr32, std::max(delta * delta * R.rr_true, 0.25 * tol * tol * R.bb));
        }
      }
    }
    for (auto& s : st)
      if (!s.finished) status = PFMP_E_NOT_CONVERGED;
    if (infos)
      for (int i = 0; i < B->total_rhs; ++i) {
        infos[i].iters = st[i].iters;
        infos[i].reliable_updates = st[i].rel;
        infos[i].true_rel_res = st[i].res;
        infos[i].k_apply = st[i].iters + st[i].kres;
        infos[i].status = st[i].finished ? PFMP_OK : PFMP_E_NOT_CONVERGED;
      }
  } catch (...) {
    for (int s = 0; s < ns; ++s) B->ops[s]->ctx->stream = keep[s];
    throw;
  }
  for (int s = 0; s < ns; ++s) B->ops[s]->ctx->stream = keep[s];
  return status;
}

// time one graph replay of `chunk` iterations for each candidate block size on the
// current (arbitrary) contents and keep the fastest; the solve afterwards starts afresh
int batch_tune(pfmp_batch* B, int chunk, double* best_ms) {
  const int cand[3] = {64, 128, 256};
  int best = B->block;
  double bms = 1e30;
  cudaEvent_t e0, e1;
  PFMP_CUDA(cudaEventCreate(&e0));
  PFMP_CUDA(cudaEventCreate(&e1));
  // scalars that never converge: stop_rr = 0, rr = 1
  std::vector<CGScalars> h(B->total_rhs);
  for (auto& v : h) {
    v = CGScalars{};
    v.rr = 1.0;
  }
  for (int c : cand) {
    batch_layout(B, c);
    PFMP_CUDA(cudaMemcpyAsync(B->d_scal, h.data(), h.size() * sizeof(CGScalars), cudaMemcpyHostToDevice, B->stream));
    // finite dummy contents (the byte 0x3f repeated is the float 0.747...)
    for (auto& S : B->sys) {
      PFMP_CUDA(cudaMemsetAsync(S.p, 0x3f, (size_t)S.R * S.fw * sizeof(float4), B->stream));
      PFMP_CUDA(cudaMemsetAsync(S.r, 0x3f, (size_t)S.R * S.fw * sizeof(float4), B->stream));
      PFMP_CUDA(cudaMemsetAsync(S.x, 0, (size_t)S.R * S.fw * sizeof(float4), B->stream));
    }
    batch_run_chunk(B, chunk);  // warm (and instantiate)
    PFMP_CUDA(cudaEventRecord(e0, B->stream));
    batch_run_chunk(B, chunk);
    PFMP_CUDA(cudaEventRecord(e1, B->stream));
    PFMP_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    PFMP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < bms) {
      bms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_layout(B, best);
  B->tuned = true;
  if (best_ms) *best_ms = bms;
  return best;
}

}  // namespace pfmp
