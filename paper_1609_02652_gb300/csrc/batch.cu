// Batched multi-system, multi-right-hand-side mixed-precision CG in one persistent launch.
//
// Many independent systems K_s x_{s,r} = b_{s,r} (different lattices, gauge fields and
// kappa; R_s right-hand sides each) are solved by ONE cooperative kernel whose blocks
// stay resident for the whole solve.  Each phase's work is cut into tiles (system, site
// block, rhs), the R_s tiles of one site block adjacent so that their link and clover
// reads share the L2; the blocks take the tiles in turn, and a grid barrier separates
// the phases.  A CG iteration of the whole batch is six phases: the four stencil phases
// of K = M-hat^dag M-hat, the x/r update and the p update, each rhs with its own scalars
// (the per-rhs sums are deterministic: fixed partial slots, summed in a fixed order by
// the rhs's last tile).  The FP32 iterations are corrected by reliable updates on the
// device: once a rhs's iterated residual has dropped by delta, x is accumulated in FP64
// and r = b - K x is recomputed with K in double-float (five more phases, only when some
// rhs asked for it); a rhs whose double-float residual is below the target stops.  The
// host then confirms each stopped rhs with K in FP64 and relaunches for any that FP64
// does not confirm (with a tighter double-float target for it).
//
// Fields and scalars that blocks rewrite during the launch are read through L2 only
// (ld.global.cg, volatile): L1 is not coherent across SMs.
//
// Every wait of the grid barrier is bounded by a wall-clock limit (the GPU's global
// timer): a block that waits longer raises an error flag and leaves, every other block
// leaves at its next barrier, and the host reports PFMP_E_TIMEOUT.  The launch is
// cooperative, with no more blocks than can be resident at once, so all blocks arrive.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "hop.cuh"

namespace pfmp {

// one system of the batch
struct PSys {
  Geom g;
  const float4* U32;
  const float4* Udf;
  const float4* clov32[2];  // A_ee, A_oo^{-1} (FP32)
  const float4* clovdf[2];  // the same in double-float
  double kappa2;
  int R, nsb, rhs0;
  long fw;                          // float4 words of one FP32 half-lattice field (6 Vh)
  float4 *x, *r, *p, *Ap, *t, *e;   // R FP32 fields each
  float4 *xdf, *edf, *tdf;          // R double-float fields each (2 fw words)
};

// per right-hand side
enum : int { RHS_ITER = 0, RHS_UPDATE = 1, RHS_DONE = 2, RHS_NAN = 3 };
struct PRhs {
  double2* x64;        // the caller's solution (FP64)
  const double2* b64;  // the caller's right-hand side (FP64)
  double bb, rr, pAp, alpha, beta, rr_true, stop_rr, tol2bb;
  int state, iters, updates, kres;
  long part0;          // first partial slot
};

struct PBatch {
  PSys* sys;
  PRhs* rhs;
  const int2* tiles;   // (system, site block * R + rhs)
  int ntiles;
  double* partials;    // per rhs: 2 nsb doubles
  unsigned* tickets;   // per rhs
  unsigned* bar;       // [0] arrivals, [1] generation
  int* err;            // raised by a barrier wait that timed out
  unsigned* nupd;      // reliable updates requested so far (monotonic)
  int* nactive;        // rhs still iterating or updating
  int* iters_done;     // batch iterations run by this launch
  unsigned nblocks;    // blocks that must reach each barrier
  unsigned long long limit_ns;
  int max_iter, fresh;
  double delta2, tol2;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a bounded wait.  Thread 0 of each block reads the generation,
// arrives, and the last arrival resets the count and opens the next generation; the
// others wait for the generation to change, for the error flag, or for limit_ns.
// Returns false on every thread of the block once the error flag is up.
__device__ bool grid_barrier(const PBatch& B) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = B.bar + 1;
    volatile int* err = B.err;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned a = atomicAdd(B.bar, 1u);
    if (a == B.nblocks - 1) {
      atomicExch(B.bar, 0u);
      __threadfence();
      atomicAdd(B.bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g0 && *err == 0) {
        if (global_ns() - t0 > B.limit_ns) {
          atomicExch(B.err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = *err == 0;
  }
  __syncthreads();
  return ok;
}

// per-rhs deterministic sum of N values over the rhs's nsb tiles: slot sb of the rhs's
// partials, the last tile to arrive sums the slots in order (true on its thread 0)
template <int N>
__device__ bool rhs_sum(const PBatch& B, const PRhs& R, int idx, int nsb, int sb, double v[N], double out[N]) {
  return group_sum<N>(v, B.partials + R.part0, B.tickets + idx, (unsigned)nsb, (unsigned)sb, out);
}

__device__ __forceinline__ int ld_state(const PRhs& R) { return *(volatile const int*)&R.state; }
__device__ __forceinline__ double ld_d(const double& v) { return __ldcg(&v); }

struct Tile {
  const PSys* S;
  PRhs* R;
  int idx, sb, r, cb;
};
__device__ __forceinline__ Tile tile_at(const PBatch& B, int t) {
  const int2 m = B.tiles[t];
  Tile T;
  T.S = B.sys + m.x;
  T.sb = m.y / T.S->R;
  T.r = m.y % T.S->R;
  T.idx = T.S->rhs0 + T.r;
  T.R = B.rhs + T.idx;
  T.cb = T.sb * blockDim.x + threadIdx.x;
  return T;
}

// ---------------------------------------------------------------- phases
// b -> r = p (FP32), x = 0 (FP32 and FP64); |b|^2 and |r|^2
__device__ void phase_init(const PBatch& B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const Tile T = tile_at(B, t);
    const PSys& S = *T.S;
    const int Vh = S.g.Vh;
    const long off = (long)T.r * S.fw;
    double v[2] = {0.0, 0.0};
    if (T.cb < Vh) {
      const double2* b = T.R->b64;
      double2* x = T.R->x64;
      float acc = 0.f;
      for (int k = 0; k < 6; ++k) {
        const double2 b0 = b[(size_t)(2 * k) * Vh + T.cb], b1 = b[(size_t)(2 * k + 1) * Vh + T.cb];
        v[0] += b0.x * b0.x + b0.y * b0.y + b1.x * b1.x + b1.y * b1.y;
        const float4 f = make_float4((float)b0.x, (float)b0.y, (float)b1.x, (float)b1.y);
        const long i = off + (long)k * Vh + T.cb;
        S.r[i] = f;
        S.p[i] = f;
        S.x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        acc += f.x * f.x + f.y * f.y + f.z * f.z + f.w * f.w;
        x[(size_t)(2 * k) * Vh + T.cb] = make_double2(0.0, 0.0);
        x[(size_t)(2 * k + 1) * Vh + T.cb] = make_double2(0.0, 0.0);
      }
      v[1] = acc;
    }
    double s[2];
    if (rhs_sum<2>(B, *T.R, T.idx, S.nsb * 1, T.sb, v, s)) {
      PRhs& R = *T.R;
      R.bb = s[0];
      R.rr = s[1];
      R.rr_true = s[0];
      R.tol2bb = B.tol2 * s[0];
      R.stop_rr = fmax(B.delta2 * s[0], 0.25 * R.tol2bb);
      R.iters = R.updates = R.kres = 0;
      if (!(s[0] == s[0]) || !(s[0] < 1e300)) {
        R.state = RHS_NAN;
        atomicSub(B.nactive, 1);
      } else if (s[0] == 0.0) {
        R.state = RHS_DONE;
        atomicSub(B.nactive, 1);
      } else {
        R.state = RHS_ITER;
      }
    }
  }
}

// the four stencil phases of K (FP32): PHASE 1 t = A_oo^{-1} H_oe v, PHASE 2
// w = A_ee v - kappa^2 H_eo t with v = p, w = e (DAG false) or v = e, w = Ap (DAG true);
// the non-adjoint PHASE 2 sums ||e||^2 = <p, K p> and sets alpha
template <bool DAG, int PHASE>
__device__ __noinline__ void phase_hop(const PBatch& B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const Tile T = tile_at(B, t);
    if (ld_state(*T.R) != RHS_ITER) continue;
    const PSys& S = *T.S;
    const long off = (long)T.r * S.fw;
    HopParams<PFMP_F32> a{};
    a.g = S.g;
    a.gauge = S.U32;
    const float4* v = (DAG ? S.e : S.p) + off;
    if (PHASE == 1) {
      a.p = 1;
      a.in = v;
      a.out = S.t + off;
      a.clov = S.clov32[1];
      a.coef = 1.0;
    } else {
      a.p = 0;
      a.in = S.t + off;
      a.x = v;
      a.out = (DAG ? S.Ap : S.e) + off;
      a.clov = S.clov32[0];
      a.coef = -S.kappa2;
    }
    constexpr bool RED = PHASE == 2 && !DAG;
    double nrm[1] = {0.0};
    if (T.cb < S.g.Vh) {
      const auto out = hop_site<PFMP_F32, DAG, PHASE == 1 ? EPI_CLOV : EPI_XPAY, true>(a, T.cb);
      store_spinor(a.out, out, T.cb, S.g.Vh);
      if (RED) nrm[0] = spinor_norm2(out);
    }
    if (RED) {
      double s[1];
      if (rhs_sum<1>(B, *T.R, T.idx, S.nsb, T.sb, nrm, s)) {
        T.R->pAp = s[0];
        T.R->alpha = ld_d(T.R->rr) / s[0];
      }
    }
  }
}

// x += alpha p, r -= alpha Ap; |r|^2 -> beta, rr; a rhs whose |r|^2 fell below stop_rr
// (or is not finite) asks for a reliable update
__device__ void phase_xr(const PBatch& B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const Tile T = tile_at(B, t);
    if (ld_state(*T.R) != RHS_ITER) continue;
    const PSys& S = *T.S;
    const int Vh = S.g.Vh;
    const long off = (long)T.r * S.fw;
    const float al = (float)ld_d(T.R->alpha);
    double v[1] = {0.0};
    if (T.cb < Vh) {
      float acc = 0.f;  // the site's |r|^2 in FP32, across sites in FP64
      for (int k = 0; k < 6; ++k) {
        const long i = off + (long)k * Vh + T.cb;
        float4 xx = __ldcg(S.x + i), rr = __ldcg(S.r + i);
        const float4 pp = __ldcg(S.p + i), aa = __ldcg(S.Ap + i);
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
      v[0] = acc;
    }
    double s[1];
    if (rhs_sum<1>(B, *T.R, T.idx, S.nsb, T.sb, v, s)) {
      PRhs& R = *T.R;
      R.beta = s[0] / ld_d(R.rr);
      R.rr = s[0];
      R.iters = *(volatile int*)&R.iters + 1;
      if (s[0] < ld_d(R.stop_rr) || !(s[0] == s[0]) || !(s[0] < 1e300)) {
        R.state = RHS_UPDATE;
        atomicAdd(B.nupd, 1u);
      }
    }
  }
}

// p = r + beta p for every rhs that ran this iteration
__device__ void phase_p(const PBatch& B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const Tile T = tile_at(B, t);
    const int st = ld_state(*T.R);
    if (st != RHS_ITER && st != RHS_UPDATE) continue;
    const PSys& S = *T.S;
    const int Vh = S.g.Vh;
    if (T.cb >= Vh) continue;
    const long off = (long)T.r * S.fw;
    const float be = (float)ld_d(T.R->beta);
    for (int k = 0; k < 6; ++k) {
      const long i = off + (long)k * Vh + T.cb;
      const float4 rr = __ldcg(S.r + i), pp = __ldcg(S.p + i);
      S.p[i] = make_float4(rr.x + be * pp.x, rr.y + be * pp.y, rr.z + be * pp.z, rr.w + be * pp.w);
    }
  }
}

// reliable update, step 1: x64 += x (FP32), x = 0, xdf = x64 split into FP32 pairs
__device__ void phase_accumulate(const PBatch& B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const Tile T = tile_at(B, t);
    if (ld_state(*T.R) != RHS_UPDATE) continue;
    const PSys& S = *T.S;
    const int Vh = S.g.Vh;
    if (T.cb >= Vh) continue;
    const long off = (long)T.r * S.fw;
    double2* x64 = T.R->x64;
    float4* xdf = S.xdf + 2 * off;
    for (int k = 0; k < 6; ++k) {
      const long i = off + (long)k * Vh + T.cb;
      const float4 xs = __ldcg(S.x + i);
      const size_t j0 = (size_t)(2 * k) * Vh + T.cb, j1 = (size_t)(2 * k + 1) * Vh + T.cb;
      double2 a = __ldcg(x64 + j0), b = __ldcg(x64 + j1);
      a.x += (double)xs.x;
      a.y += (double)xs.y;
      b.x += (double)xs.z;
      b.y += (double)xs.w;
      x64[j0] = a;
      x64[j1] = b;
      xdf[j0] = split2(a);
      xdf[j1] = split2(b);
      S.x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// reliable update, steps 2-5: K xdf in double-float (the same four stencil phases), then
// r = b - K x64 in FP64, its FP32 copy, |r|^2 in FP64 and of the FP32 copy
template <bool DAG, int PHASE>
__device__ __noinline__ void phase_hop_df(const PBatch& B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const Tile T = tile_at(B, t);
    if (ld_state(*T.R) != RHS_UPDATE) continue;
    const PSys& S = *T.S;
    const int Vh = S.g.Vh;
    const long off = 2 * (long)T.r * S.fw;
    HopParams<PREC_DF> a{};
    a.g = S.g;
    a.gauge = S.Udf;
    const float4* v = (DAG ? S.edf : S.xdf) + off;
    if (PHASE == 1) {
      a.p = 1;
      a.in = v;
      a.out = S.tdf + off;
      a.clov = S.clovdf[1];
      a.coef = 1.0;
    } else {
      a.p = 0;
      a.in = S.tdf + off;
      a.x = v;
      a.out = S.edf + off;
      a.clov = S.clovdf[0];
      a.coef = -S.kappa2;
    }
    constexpr bool LAST = DAG && PHASE == 2;
    double v2[2] = {0.0, 0.0};
    if (T.cb < Vh) {
      const auto out = hop_site_rolled<PREC_DF, DAG, PHASE == 1 ? EPI_CLOV : EPI_XPAY, true>(a, T.cb);
      if (!LAST) {
        store_spinor(a.out, out, T.cb, Vh);
      } else {
        const double2* b = T.R->b64;
        const long off32 = (long)T.r * S.fw;
        float acc = 0.f;
        for (int k = 0; k < 6; ++k) {
          const cplx<df> k0 = out.s[(2 * k) / 3][(2 * k) % 3], k1 = out.s[(2 * k + 1) / 3][(2 * k + 1) % 3];
          const double2 b0 = b[(size_t)(2 * k) * Vh + T.cb], b1 = b[(size_t)(2 * k + 1) * Vh + T.cb];
          const double r0 = b0.x - (double)k0.re, r1 = b0.y - (double)k0.im;
          const double r2 = b1.x - (double)k1.re, r3 = b1.y - (double)k1.im;
          v2[0] += r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3;
          const float4 f = make_float4((float)r0, (float)r1, (float)r2, (float)r3);
          S.r[off32 + (long)k * Vh + T.cb] = f;
          acc += f.x * f.x + f.y * f.y + f.z * f.z + f.w * f.w;
        }
        v2[1] = acc;
      }
    }
    if (LAST) {
      double s[2];
      if (rhs_sum<2>(B, *T.R, T.idx, S.nsb, T.sb, v2, s)) {
        PRhs& R = *T.R;
        R.rr_true = s[0];
        R.rr = s[1];
        R.updates = *(volatile int*)&R.updates + 1;
        R.kres = *(volatile int*)&R.kres + 1;
        const double tol2bb = ld_d(R.tol2bb);
        if (!(s[0] == s[0]) || !(s[0] < 1e300)) {
          R.state = RHS_NAN;
          atomicSub(B.nactive, 1);
        } else if (s[0] < tol2bb) {
          R.state = RHS_DONE;
          atomicSub(B.nactive, 1);
        } else {
          R.stop_rr = fmax(B.delta2 * s[0], 0.25 * tol2bb);
          R.state = RHS_ITER;
        }
      }
    }
  }
}

// 2 resident blocks of 256 threads per SM (128 registers): the FP32 stencil phases fit
// with a few spilled registers; the double-float phases (rare: reliable updates) are
// separate functions and spill more rather than cap the occupancy of the rest
__global__ void __launch_bounds__(256, 2) k_batch_persistent(PBatch B) {
  __shared__ unsigned s_nupd;
  __shared__ int s_active;
  if (B.fresh) {
    phase_init(B);
    if (!grid_barrier(B)) return;
  }
  unsigned seen = 0;
  int it = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_nupd = *(volatile unsigned*)B.nupd;
      s_active = *(volatile int*)B.nactive;
    }
    __syncthreads();
    const unsigned nupd = s_nupd;
    const int active = s_active;
    __syncthreads();
    if (nupd != seen) {
      seen = nupd;
      phase_accumulate(B);
      if (!grid_barrier(B)) return;
      phase_hop_df<false, 1>(B);
      if (!grid_barrier(B)) return;
      phase_hop_df<false, 2>(B);
      if (!grid_barrier(B)) return;
      phase_hop_df<true, 1>(B);
      if (!grid_barrier(B)) return;
      phase_hop_df<true, 2>(B);
      if (!grid_barrier(B)) return;
      continue;  // re-read the counters
    }
    if (active <= 0 || it >= B.max_iter) break;
    phase_hop<false, 1>(B);
    if (!grid_barrier(B)) return;
    phase_hop<false, 2>(B);
    if (!grid_barrier(B)) return;
    phase_hop<true, 1>(B);
    if (!grid_barrier(B)) return;
    phase_hop<true, 2>(B);
    if (!grid_barrier(B)) return;
    phase_xr(B);
    if (!grid_barrier(B)) return;
    phase_p(B);
    if (!grid_barrier(B)) return;
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *B.iters_done = it;
}

// the barrier alone: `rounds` barriers, for the barrier's own test (nblocks may exceed
// the grid, in which case every wait runs out and the error flag is raised)
__global__ void __launch_bounds__(256) k_barrier_check(PBatch B, int rounds) {
  for (int k = 0; k < rounds; ++k)
    if (!grid_barrier(B)) return;
}

}  // namespace pfmp

using namespace pfmp;

struct pfmp_batch {
  std::vector<pfmp_op*> ops;
  std::vector<int> R;
  std::vector<PSys> sys;
  PSys* d_sys = nullptr;
  PRhs* d_rhs = nullptr;
  std::vector<PRhs> h_rhs;
  int2* d_tiles = nullptr;
  int ntiles = 0, block = 128, grid = 0;
  std::vector<void*> bufs;
  double* d_part = nullptr;
  unsigned* d_tick = nullptr;
  unsigned* d_ctl = nullptr;  // bar[2], nupd, nactive, iters_done, err
  int total_rhs = 0;
  cudaStream_t stream = nullptr;
  double limit_s = 2.0;
  bool tuned = false;
};

namespace pfmp {

static void batch_layout(pfmp_batch* B, int block) {
  B->block = block;
  std::vector<int2> tiles;
  long np = 0;
  int idx = 0;
  for (size_t s = 0; s < B->sys.size(); ++s) {
    PSys& S = B->sys[s];
    S.nsb = (S.g.Vh + block - 1) / block;
    for (int i = 0; i < S.nsb * S.R; ++i) tiles.push_back(make_int2((int)s, i));
    for (int r = 0; r < S.R; ++r, ++idx) {
      B->h_rhs[idx].part0 = np;
      np += 2L * S.nsb;
    }
  }
  PFMP_REQUIRE(tiles.size() < (1u << 30), PFMP_E_INVALID, "batch too large");
  B->ntiles = (int)tiles.size();
  dev_free(B->d_tiles);
  dev_free(B->d_part);
  B->d_tiles = (int2*)dev_alloc(tiles.size() * sizeof(int2));
  B->d_part = (double*)dev_alloc(np * sizeof(double));
  PFMP_CUDA(cudaMemcpy(B->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice));
  PFMP_CUDA(cudaMemcpy(B->d_sys, B->sys.data(), B->sys.size() * sizeof(PSys), cudaMemcpyHostToDevice));
  int per_sm = 0, dev = 0, nsm = 0;
  PFMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent, block, 0));
  PFMP_CUDA(cudaGetDevice(&dev));
  PFMP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PFMP_REQUIRE(per_sm >= 1, PFMP_E_CUDA, "the persistent batch kernel cannot be resident");
  B->grid = std::min(per_sm * nsm, std::max(B->ntiles, 1));
}

void batch_destroy(pfmp_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (auto p : B->bufs) dev_free(p);
  dev_free(B->d_sys);
  dev_free(B->d_rhs);
  dev_free(B->d_tiles);
  dev_free(B->d_part);
  dev_free(B->d_tick);
  dev_free(B->d_ctl);
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
    B->h_rhs.assign(tot, PRhs{});
    B->d_rhs = (PRhs*)dev_alloc(tot * sizeof(PRhs));
    B->d_tick = (unsigned*)dev_alloc(tot * sizeof(unsigned));
    PFMP_CUDA(cudaMemset(B->d_tick, 0, tot * sizeof(unsigned)));
    B->d_ctl = (unsigned*)dev_alloc(8 * sizeof(unsigned));
    int off = 0;
    for (int s = 0; s < nsys; ++s) {
      pfmp_op* op = ops[s];
      PSys S{};
      S.g = op->ctx->g;
      S.U32 = op->ctx->U32;
      S.Udf = op->ctx->Udf;
      S.clov32[0] = op->clov32[0];
      S.clov32[1] = op->clov32[1];
      S.clovdf[0] = op->clovdf[0];
      S.clovdf[1] = op->clovdf[1];
      S.kappa2 = op->kappa * op->kappa;
      S.R = nrhs[s];
      S.rhs0 = off;
      S.fw = 6L * op->ctx->g.Vh;
      // 6 FP32 fields and 3 double-float fields (2 words each) per rhs
      float4* buf = (float4*)dev_alloc((size_t)12 * S.R * S.fw * sizeof(float4));
      B->bufs.push_back(buf);
      float4* q = buf;
      float4** f32[6] = {&S.x, &S.r, &S.p, &S.Ap, &S.t, &S.e};
      for (auto f : f32) {
        *f = q;
        q += (size_t)S.R * S.fw;
      }
      float4** fdf[3] = {&S.xdf, &S.edf, &S.tdf};
      for (auto f : fdf) {
        *f = q;
        q += (size_t)2 * S.R * S.fw;
      }
      off += S.R;
      B->sys.push_back(S);
    }
    B->d_sys = (PSys*)dev_alloc(nsys * sizeof(PSys));
    batch_layout(B, 128);
  } catch (...) {
    batch_destroy(B);
    throw;
  }
  return B;
}

static PBatch kernel_args(pfmp_batch* B, int max_iter, int fresh, double delta, double tol) {
  PBatch a{};
  a.sys = B->d_sys;
  a.rhs = B->d_rhs;
  a.tiles = B->d_tiles;
  a.ntiles = B->ntiles;
  a.partials = B->d_part;
  a.tickets = B->d_tick;
  a.bar = B->d_ctl;
  a.nupd = B->d_ctl + 2;
  a.nactive = (int*)(B->d_ctl + 3);
  a.iters_done = (int*)(B->d_ctl + 4);
  a.err = (int*)(B->d_ctl + 5);
  a.nblocks = (unsigned)B->grid;
  a.limit_ns = (unsigned long long)(B->limit_s * 1e9);
  a.max_iter = max_iter;
  a.fresh = fresh;
  a.delta2 = delta * delta;
  a.tol2 = tol * tol;
  return a;
}

// one cooperative launch; ctl = {nupd, nactive} before it; returns the batch iterations it
// ran and raises PFMP_E_TIMEOUT if a barrier wait ran out
static int launch_persistent(pfmp_batch* B, PBatch a, unsigned nupd, int nactive) {
  unsigned ctl[6] = {0u, 0u, nupd, (unsigned)nactive, 0u, 0u};
  PFMP_CUDA(cudaMemcpyAsync(B->d_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, B->stream));
  void* args[] = {&a};
  PFMP_CUDA(cudaLaunchCooperativeKernel((const void*)k_batch_persistent, dim3(B->grid), dim3(B->block), args, 0,
                                        B->stream));
  count_launches(1);
  PFMP_CUDA(cudaMemcpyAsync(ctl, B->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, B->stream));
  PFMP_CUDA(cudaStreamSynchronize(B->stream));
  PFMP_REQUIRE(ctl[5] == 0, PFMP_E_TIMEOUT, "batched solve: a grid barrier wait timed out");
  return (int)ctl[4];
}

int batch_solve(pfmp_batch* B, double tol, int max_iter, double delta, int check, void* const* x, const void* const* b,
                pfmp_solve_info* infos) {
  (void)check;
  PFMP_REQUIRE(tol > 0 && max_iter > 0, PFMP_E_INVALID, "tol and max_iter must be positive");
  if (!(delta > 0 && delta < 1)) delta = 1e-4;
  const int ns = (int)B->sys.size();
  for (int s = 0; s < ns; ++s)
    PFMP_REQUIRE(B->ops[s]->built_version == B->ops[s]->ctx->gauge_version && B->ops[s]->built_prec == PFMP_F64,
                 PFMP_E_INVALID, "gauge field changed since the clover term was built: call pfmp_op_update");
  for (int i = 0; i < B->total_rhs; ++i) {
    PFMP_REQUIRE(x[i] && b[i] && x[i] != b[i], PFMP_E_INVALID, "each rhs needs distinct x and b fields");
    B->h_rhs[i].x64 = (double2*)x[i];
    B->h_rhs[i].b64 = (const double2*)b[i];
  }
  PFMP_CUDA(cudaMemcpyAsync(B->d_rhs, B->h_rhs.data(), B->total_rhs * sizeof(PRhs), cudaMemcpyHostToDevice, B->stream));
  PFMP_CUDA(cudaMemsetAsync(B->d_tick, 0, B->total_rhs * sizeof(unsigned), B->stream));
  std::vector<long> kres64(B->total_rhs, 0);
  std::vector<int> finished(B->total_rhs, 0);
  std::vector<double> res(B->total_rhs, 0.0);
  int status = PFMP_OK, iters = 0, fresh = 1;
  unsigned nupd = 0;
  int nactive = B->total_rhs;
  for (int launch = 0; launch < 8 && nactive > 0 && iters < max_iter; ++launch) {
    iters += launch_persistent(B, kernel_args(B, max_iter - iters, fresh, delta, tol), nupd, nactive);
    fresh = 0;
    PFMP_CUDA(cudaMemcpyAsync(B->h_rhs.data(), B->d_rhs, B->total_rhs * sizeof(PRhs), cudaMemcpyDeviceToHost,
                              B->stream));
    PFMP_CUDA(cudaStreamSynchronize(B->stream));
    // the FP64 confirmation of every rhs that stopped on its double-float residual
    nupd = 0;
    nactive = 0;
    bool changed = false;
    for (int s = 0, i = 0; s < ns; ++s) {
      pfmp_op* op = B->ops[s];
      for (int r = 0; r < B->sys[s].R; ++r, ++i) {
        PRhs& R = B->h_rhs[i];
        PFMP_REQUIRE(R.state != RHS_NAN, PFMP_E_NAN, "batched CG residual became NaN/Inf");
        if (finished[i]) continue;
        if (R.state != RHS_DONE) {
          nactive += 1;
          continue;
        }
        if (R.bb == 0.0) {
          finished[i] = 1;
          continue;
        }
        cudaStream_t keep = op->ctx->stream;
        op->ctx->stream = B->stream;
        double rr = 0;
        try {
          rr = true_residual_f64(op, x[i], b[i], op->cg64[0]);
        } catch (...) {
          op->ctx->stream = keep;
          throw;
        }
        op->ctx->stream = keep;
        kres64[i] += 1;
        res[i] = std::sqrt(rr / R.bb);
        if (rr < tol * tol * R.bb) {
          finished[i] = 1;
        } else {  // continue from x64 with a tighter double-float target
          R.tol2bb = 0.25 * std::min(R.tol2bb, rr);
          R.state = RHS_UPDATE;
          nupd += 1;
          nactive += 1;
          changed = true;
        }
      }
    }
    if (changed)
      PFMP_CUDA(cudaMemcpyAsync(B->d_rhs, B->h_rhs.data(), B->total_rhs * sizeof(PRhs), cudaMemcpyHostToDevice,
                                B->stream));
  }
  for (int i = 0; i < B->total_rhs; ++i)
    if (!finished[i]) status = PFMP_E_NOT_CONVERGED;
  if (infos)
    for (int i = 0; i < B->total_rhs; ++i) {
      const PRhs& R = B->h_rhs[i];
      infos[i].iters = R.iters;
      infos[i].reliable_updates = R.updates;
      infos[i].true_rel_res = finished[i] ? res[i] : std::sqrt(R.rr_true / std::max(R.bb, 1e-300));
      infos[i].k_apply = R.iters + R.kres + kres64[i];
      infos[i].status = finished[i] ? PFMP_OK : PFMP_E_NOT_CONVERGED;
    }
  return status;
}

// time one persistent launch of `chunk` iterations for each candidate block size on
// finite dummy contents that never converge, keep the fastest; the solve afterwards
// starts afresh
int batch_tune(pfmp_batch* B, int chunk, double* best_ms) {
  const int cand[3] = {64, 128, 256};
  int best = B->block;
  double bms = 1e30;
  cudaEvent_t e0, e1;
  PFMP_CUDA(cudaEventCreate(&e0));
  PFMP_CUDA(cudaEventCreate(&e1));
  std::vector<PRhs> h(B->h_rhs);
  for (auto& v : h) {
    v.rr = 1.0;
    v.stop_rr = 0.0;
    v.state = RHS_ITER;
  }
  for (int c : cand) {
    for (size_t i = 0; i < h.size(); ++i) h[i].part0 = 0;
    batch_layout(B, c);
    for (size_t i = 0; i < h.size(); ++i) h[i].part0 = B->h_rhs[i].part0;
    PFMP_CUDA(cudaMemcpyAsync(B->d_rhs, h.data(), h.size() * sizeof(PRhs), cudaMemcpyHostToDevice, B->stream));
    PFMP_CUDA(cudaMemsetAsync(B->d_tick, 0, B->total_rhs * sizeof(unsigned), B->stream));
    // finite dummy contents (the byte 0x3f repeated is the float 0.747...)
    for (auto& S : B->sys) {
      PFMP_CUDA(cudaMemsetAsync(S.p, 0x3f, (size_t)S.R * S.fw * sizeof(float4), B->stream));
      PFMP_CUDA(cudaMemsetAsync(S.r, 0x3f, (size_t)S.R * S.fw * sizeof(float4), B->stream));
      PFMP_CUDA(cudaMemsetAsync(S.x, 0, (size_t)S.R * S.fw * sizeof(float4), B->stream));
    }
    launch_persistent(B, kernel_args(B, 1, 0, 0.5, 1e-30), 0, B->total_rhs);  // warm
    PFMP_CUDA(cudaMemcpyAsync(B->d_rhs, h.data(), h.size() * sizeof(PRhs), cudaMemcpyHostToDevice, B->stream));
    PFMP_CUDA(cudaEventRecord(e0, B->stream));
    launch_persistent(B, kernel_args(B, chunk, 0, 0.5, 1e-30), 0, B->total_rhs);
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

// `rounds` barriers on the batch's grid with `missing` blocks more expected than launched
// (0: every barrier passes; > 0: every wait runs out after limit_s and PFMP_E_TIMEOUT)
int batch_barrier_check(pfmp_batch* B, int rounds, int missing, double limit_s) {
  PFMP_REQUIRE(rounds >= 1 && missing >= 0 && limit_s > 0 && limit_s <= 10, PFMP_E_INVALID, "bad barrier check");
  PBatch a = kernel_args(B, 0, 0, 0.5, 1.0);
  a.nblocks = (unsigned)(B->grid + missing);
  a.limit_ns = (unsigned long long)(limit_s * 1e9);
  unsigned ctl[6] = {0u, 0u, 0u, 0u, 0u, 0u};
  PFMP_CUDA(cudaMemcpyAsync(B->d_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, B->stream));
  void* args[] = {&a, &rounds};
  PFMP_CUDA(cudaLaunchCooperativeKernel((const void*)k_barrier_check, dim3(B->grid), dim3(B->block), args, 0,
                                        B->stream));
  count_launches(1);
  PFMP_CUDA(cudaMemcpyAsync(ctl, B->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, B->stream));
  PFMP_CUDA(cudaStreamSynchronize(B->stream));
  PFMP_REQUIRE(ctl[5] == 0, PFMP_E_TIMEOUT, "grid barrier wait timed out");
  return PFMP_OK;
}

}  // namespace pfmp
