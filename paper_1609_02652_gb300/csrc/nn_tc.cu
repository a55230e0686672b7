// Tensor-core forward layers of the gauge-covariant network (C_in -> C_out channels with
// C_in, C_out in {1, 8}).
//
// The layer is a dense contraction per site and colour:
//   y[o][a](x, c) = sum_d sum_i sum_b W_d[o][i][a][b] t_d[i][b](x, c),
// t_d = the input channel parallel-transported from the neighbour in direction d (the
// site itself, four forward and four backward hops, fermion boundary factor included).
// As a real GEMM per colour: rows = 128 sites of a tile (M = 128, one TMEM lane each),
// K = 9 directions x C_in channels x 4 spins x (re, im), N = C_out x 4 spins x (re, im)
// (padded to 16), with B = [[Re W, -Im W], [Im W, Re W]] so that the complex product
// comes out in (re, im) column pairs.  Operands are FP16, the accumulator FP32 in
// tensor memory.  K is consumed in stages: one direction per stage (K = 8 C_in), or for
// C_in = 1 four directions per stage (K = 32, the last stage three quarters zero).
//
// Activations between the layers are FP16 complex [C][12][V], scaled by sigma = 1/rms of
// the network input so that FP16 keeps its precision (the network is linear; the last
// layer writes FP32 divided by sigma).  The directions are taken in the order site, +x,
// -x, +y, -y, +z, -z, +t, -t so that consecutive stages read overlapping neighbours.
//
// One CTA per SM loops over tiles of 128 sites.  Per stage, 512 threads (four per
// site) gather and transport the inputs (FP32 links) into a K-major shared-memory tile per
// colour (no-swizzle canonical layout: 8-row x 16-byte core matrices, K-adjacent cores
// 128 bytes apart, 8-row groups 16 K bytes apart), then one thread issues the
// tcgen05.mma instructions of the three colours and commits them to an mbarrier; the
// A tiles are double-buffered so that the gather of stage s + 1 overlaps the MMAs of
// stage s.  The packed weights of all stages (72 KB for 8 -> 8) stay in shared memory,
// brought in by bulk TMA copies.  The epilogue reads the accumulators with
// tcgen05.ld (lane = site) and writes the output activations.
// Every mbarrier wait is bounded; on a timeout the kernel raises a device error flag,
// waits (bounded) for the work it has in flight, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <cstdlib>

#include "context.h"
#include "fields.cuh"

namespace pfmp {
namespace tc {

constexpr int kM = 128;        // sites per tile = TMEM lanes
constexpr int kThreads = 512;  // four threads per site in the gather
// COUT = 9 marks the local mixing of the last layer: z_d = sum_i W_d[0][i] a_i at every
// site for the nine directions d (no gather; the transport follows in k_last_stencil)
template <int CIN, int COUT>
struct Shape {
  static constexpr bool LOCAL = COUT == 9;
  static constexpr int NST = LOCAL ? 1 : (CIN == 1 ? 3 : 9);  // K stages
  static constexpr int DPS = CIN == 1 ? 4 : 1;        // directions per stage
  static constexpr int K = CIN == 1 ? 32 : 8 * CIN;   // reals per stage
  static constexpr int N = (8 * COUT + 15) / 16 * 16;  // output reals per colour (padded to 16)
  static constexpr int A_TILE = kM * K * 2;
  static constexpr int A_BUF = 3 * A_TILE;
  static constexpr int B_ST = N * K * 2;
  static constexpr int B_ALL = NST * B_ST;
  static constexpr int SMEM = B_ALL + 2 * A_BUF;
  static constexpr int TMEM_COLS = 3 * N <= 32 ? 32 : (3 * N <= 64 ? 64 : (3 * N <= 128 ? 128 : 256));
  static constexpr uint32_t SBO = 16 * K;  // bytes between 8-row groups
  static_assert(3 * N <= 256 && N % 16 == 0 && K % 16 == 0, "tile shape");
  static_assert(CIN == 1 || CIN == 8, "the gather splits 8 channels over four threads per site");
};

// stage order of the nine directions (0 = site, 1 + mu = forward, 5 + mu = backward)
__host__ __device__ __forceinline__ int dir_of(int i) {
  return i == 0 ? 0 : (i & 1 ? 1 + (i >> 1) : 5 + ((i - 1) >> 1));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row r, column k) in a K-major no-swizzle tile with kdim columns
__host__ __device__ __forceinline__ uint32_t kmajor(int r, int k, int kdim) {
  return (uint32_t)((r >> 3) * (kdim / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4, leading (K) byte offset >> 4, stride
// (8-row group) byte offset >> 4, version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// non-blocking polls, backing off after the first thousand; gives up after ~2^20 polls
// (a fraction of a second) so that a lost completion cannot hang the GPU
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 1024) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// packed B operand of one layer: [NST][N x K] FP16, each stage a K-major canonical tile
template <int CIN, int COUT>
__global__ void k_pack_b(const float2* __restrict__ W, __half* __restrict__ B) {
  using S = Shape<CIN, COUT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S::NST * S::N * S::K) return;
  const int st = i / (S::N * S::K), rem = i % (S::N * S::K);
  const int n = rem / S::K, k = rem % S::K;
  const int di = st * S::DPS + (CIN == 1 ? (k >> 3) : 0);
  const int ic = CIN == 1 ? 0 : (k >> 3);
  const int o = n >> 3, a = (n >> 1) & 3, ro = n & 1;
  const int b = (k >> 1) & 3, ri = k & 1;
  float v = 0.f;
  if (S::LOCAL) {  // output block o is the direction d of the single output channel
    if (o < 9) {
      const float2 w = W[((size_t)o * CIN + ic) * 16 + a * 4 + b];
      v = ro == ri ? w.x : (ro == 0 ? -w.y : w.y);
    }
  } else {
    const int d = di < 9 ? dir_of(di) : 9;
    if (d < 9 && o < COUT) {
      const float2 w = W[(((size_t)d * COUT + o) * CIN + ic) * 16 + a * 4 + b];
      v = ro == ri ? w.x : (ro == 0 ? -w.y : w.y);
    }
  }
  B[(size_t)st * (S::B_ST / 2) + kmajor(n, k, S::K) / 2] = __float2half_rn(v);
}

// sigma = sqrt(n) / |in| (1 for a zero input) of an even FP32 field
__global__ void k_rms_scale(const float4* __restrict__ in, int Vh, ReduceBuf rb, float* sigma,
                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  float st = 0.f;  // per-thread sum in FP32, across threads in FP64
  const long n = 6L * Vh;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    st += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
  }
  double s[1] = {(double)st};
  double t[1];
  if (grid_sum<1>(s, rb, t)) *sigma = t[0] > 0 ? (float)sqrt(24.0 * Vh / t[0]) : 1.0f;
}

// neighbour, link and boundary factor of direction d at site x: the input of the item
// is f U a(y) (forward hop), f U^dag a(y) (backward hop) or a(x) (d = 0)
struct Hop {
  size_t sy;
  float f;
  int kind;
  Mat3<float> U;
};
__device__ __forceinline__ void make_hop(const Geom& g, const float4* __restrict__ U32, const int x[4], int d,
                                         Hop& h) {
  h.kind = d == 0 ? 0 : (d <= 4 ? 1 : 2);
  const int mu = d == 0 ? 0 : (d - 1) & 3;
  int y[4] = {x[0], x[1], x[2], x[3]};
  h.f = 1.0f;
  if (h.kind == 1) {
    y[mu] = y[mu] + 1 == g.L[mu] ? 0 : y[mu] + 1;
    if (mu == 3 && x[3] == g.L[3] - 1) h.f *= (float)g.bc_t;
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    load_link(h.U, U32 + (size_t)((p * 4 + mu) * 3) * g.Vh, cb_index(g, x), g.Vh);
  } else if (h.kind == 2) {
    y[mu] = y[mu] == 0 ? g.L[mu] - 1 : y[mu] - 1;
    if (mu == 3 && x[3] == 0) h.f *= (float)g.bc_t;
    const int p = (y[0] + y[1] + y[2] + y[3]) & 1;
    Mat3<float> L;
    load_link(L, U32 + (size_t)((p * 4 + mu) * 3) * g.Vh, cb_index(g, y), g.Vh);
    h.U = dagger(L);
  }
  h.sy = (size_t)lex_index(g, y);
}

// channel-major activations act[C][12][V] (half2 complex): component k of channel ic at
// site sy; the threads of a warp (consecutive sites) read consecutive words
template <int C>
__device__ __forceinline__ void load_channel(const __half2* __restrict__ in, size_t V, size_t sy, int ic,
                                             cplx<float> v[4][3]) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 w = __half22float2(__ldg(in + ((size_t)ic * 12 + sp * 3 + c) * V + sy));
      v[sp][c] = mk(w.x, w.y);
    }
}

// transport one channel and store it (FP16) at column col of the three colour tiles
template <int K>
__device__ __forceinline__ void store_channel(const Hop& h, const cplx<float> v[4][3], bool live, unsigned char* A,
                                              int row, int col, int a_tile) {
  cplx<float> t[4][3];
  if (live) {
    if (h.kind) {
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          t[sp][r] = h.f * (h.U.m[r][0] * v[sp][0] + h.U.m[r][1] * v[sp][1] + h.U.m[r][2] * v[sp][2]);
    } else {
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int r = 0; r < 3; ++r) t[sp][r] = h.f * v[sp][r];
    }
  } else {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int r = 0; r < 3; ++r) t[sp][r] = mk(0.f, 0.f);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    uint4 q;
    q.x = pack_h2(t[0][r].re, t[0][r].im);
    q.y = pack_h2(t[1][r].re, t[1][r].im);
    q.z = pack_h2(t[2][r].re, t[2][r].im);
    q.w = pack_h2(t[3][r].re, t[3][r].im);
    *reinterpret_cast<uint4*>(A + r * a_tile + kmajor(row, col, K)) = q;
  }
}

// the gather of one stage by one thread: part p of the site's (direction, channel) items.
// C_in = 8: one direction per stage, channels p and p + 4 (one link, 24 loads in flight);
// C_in = 1: the four parts take the stage's four directions (the last stage's parts
// 1 to 3 write the zero padding).
template <int CIN, int K>
__device__ __forceinline__ void gather_stage(const Geom& g, const float4* __restrict__ U32,
                                             const __half2* __restrict__ in, size_t V, bool live, const int x[4],
                                             int st, int part, unsigned char* A, int row, int a_tile) {
  if (CIN == 1) {
    const int di = 4 * st + part;
    const bool on = live && di < 9;
    Hop h;
    cplx<float> v[4][3];
    if (on) {
      make_hop(g, U32, x, dir_of(di), h);
      load_channel<1>(in, V, h.sy, 0, v);
    }
    store_channel<K>(h, v, on, A, row, part * 8, a_tile);
  } else {
    Hop h;
    cplx<float> v0[4][3], v1[4][3];
    const int ic0 = part, ic1 = part + 4;
    if (live) {
      make_hop(g, U32, x, dir_of(st), h);
      load_channel<8>(in, V, h.sy, ic0, v0);
      load_channel<8>(in, V, h.sy, ic1, v1);
    }
    store_channel<K>(h, v0, live, A, row, ic0 * 8, a_tile);
    store_channel<K>(h, v1, live, A, row, ic1 * 8, a_tile);
  }
}

// network input: sigma * (even FP32 field [6][Vh] float4) on even sites, 0 on odd sites,
// as FP16 complex [12][V] (lexicographic sites)
// rr (optional): |src|^2 already known to the caller (FGCR's residual norm); sigma is then
// computed here, stored for the later kernels, and no separate reduction is needed
__global__ void k_embed16(Geom g, const float4* __restrict__ src, float* __restrict__ sigma_p,
                          __half2* __restrict__ dst, const int* __restrict__ skip, const double* __restrict__ rr) {
  if (skip && *skip) return;
  if (rr) {
    const double t = *rr;
    const float sg0 = t > 0 ? (float)sqrt(24.0 * g.Vh / t) : 1.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) *sigma_p = sg0;
  }
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int r = s, x[4];
  x[0] = r % g.L[0];
  r /= g.L[0];
  x[1] = r % g.L[1];
  r /= g.L[1];
  x[2] = r % g.L[2];
  x[3] = r / g.L[2];
  const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
  const float sg = rr ? (*rr > 0 ? (float)sqrt(24.0 * g.Vh / *rr) : 1.0f) : *sigma_p;
  const int cb = s >> 1;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float4 v = even ? src[(size_t)k * g.Vh + cb] : make_float4(0.f, 0.f, 0.f, 0.f);
    dst[(size_t)(2 * k) * g.V + s] = __floats2half2_rn(sg * v.x, sg * v.y);
    dst[(size_t)(2 * k + 1) * g.V + s] = __floats2half2_rn(sg * v.z, sg * v.w);
  }
}

// last layer, second half: out(x) = sum_d U_d(x) z_d(x + d) on even sites (the only ones
// the network output is read on): z_0(x) + sum_mu [U_mu(x) z_{1+mu}(x + mu)
// + U_mu(x - mu)^dag z_{5+mu}(x - mu)] with the fermion boundary factor on time hops; z
// is FP16 [9][12][V] scaled by sigma, out the even FP32 field [6][Vh] divided by sigma
__global__ void k_last_stencil(Geom g, const float4* __restrict__ U32, const __half2* __restrict__ z,
                               float4* __restrict__ out, const float* __restrict__ sigma_p,
                               const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, 0, x);
  const size_t V = (size_t)g.V;
  cplx<float> acc[12];
  {
    const size_t s0 = (size_t)lex_index(g, x);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 v = __half22float2(__ldg(z + (size_t)k * V + s0));
      acc[k] = mk(v.x, v.y);
    }
  }
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      int y[4] = {x[0], x[1], x[2], x[3]};
      float f = 1.0f;
      Mat3<float> Um;
      if (dir == 0) {
        y[mu] = y[mu] + 1 == g.L[mu] ? 0 : y[mu] + 1;
        if (mu == 3 && x[3] == g.L[3] - 1) f = (float)g.bc_t;
        load_link(Um, U32 + (size_t)(mu * 3) * g.Vh, cb, g.Vh);  // x is even: parity 0
      } else {
        y[mu] = y[mu] == 0 ? g.L[mu] - 1 : y[mu] - 1;
        if (mu == 3 && x[3] == 0) f = (float)g.bc_t;
        Mat3<float> L;
        load_link(L, U32 + (size_t)((4 + mu) * 3) * g.Vh, cb_index(g, y), g.Vh);  // y is odd
        Um = dagger(L);
      }
      const int d = dir == 0 ? 1 + mu : 5 + mu;
      const size_t sy = (size_t)lex_index(g, y);
      cplx<float> v[4][3];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 w = __half22float2(__ldg(z + ((size_t)d * 12 + sp * 3 + c) * V + sy));
          v[sp][c] = mk(w.x, w.y);
        }
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          acc[sp * 3 + r] = acc[sp * 3 + r] + f * (Um.m[r][0] * v[sp][0] + Um.m[r][1] * v[sp][1] + Um.m[r][2] * v[sp][2]);
    }
  }
  const float inv = 1.0f / *sigma_p;
#pragma unroll
  for (int j = 0; j < 6; ++j)
    out[(size_t)j * g.Vh + cb] =
        make_float4(inv * acc[2 * j].re, inv * acc[2 * j].im, inv * acc[2 * j + 1].re, inv * acc[2 * j + 1].im);
}

// OUT16: FP16 scaled output for the next layer; otherwise FP32 output divided by sigma
template <int CIN, int COUT, bool OUT16>
__global__ void __launch_bounds__(kThreads, 1)
    k_nn_layer_tc(Geom g, const float4* __restrict__ U32, const __half* __restrict__ Bg, const __half2* __restrict__ in,
                  void* __restrict__ out, const float* __restrict__ sigma_p, int* __restrict__ err,
                  const int* __restrict__ skip) {
  using S = Shape<CIN, COUT>;
  if (skip && *skip) return;  // block-uniform: nothing allocated yet
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t bar_w, bar_a[2];
  unsigned char* sB = sm;
  unsigned char* sA = sm + S::B_ALL;
  const int tid = threadIdx.x;
  const int row = tid & (kM - 1);  // site in the tile
  const int part = tid >> 7;       // which of the site's (direction, channel) items
  const size_t V = (size_t)g.V;
  const float inv_sigma = OUT16 ? 1.0f : 1.0f / *sigma_p;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_w)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_a[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_a[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(S::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // weights of all stages: bulk TMA copies completing on bar_w
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar_w)), "r"(S::B_ALL)
                 : "memory");
    for (int st = 0; st < S::NST; ++st)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(sB + st * S::B_ST)),
          "l"(Bg + (size_t)st * (S::B_ST / 2)), "r"(S::B_ST), "r"(smem_addr(&bar_w))
          : "memory");
  }
  bool fail = !mbar_wait(smem_addr(&bar_w), 0);
  if (fail) atomicExch(err, 1);
  // every abort decision below is block-uniform (__syncthreads_or of the threads' own
  // wait results), so all threads leave the loops together
  bool aborted = __syncthreads_or(fail);

  const int ntiles = (g.V + kM - 1) / kM;
  uint32_t use = 0;           // A-buffer uses issued so far (buffer = use & 1)
  int pending[2] = {-1, -1};  // use index of the last commit on each buffer (thread 0 view)
  const uint32_t id = idesc(kM, S::N);
  for (int tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
    const int s = tile * kM + row;
    const bool live = s < g.V;
    int x[4] = {0, 0, 0, 0};
    if (live) {
      int r = s;
      x[0] = r % g.L[0];
      r /= g.L[0];
      x[1] = r % g.L[1];
      r /= g.L[1];
      x[2] = r % g.L[2];
      x[3] = r / g.L[2];
    }
    for (int st = 0; st < S::NST; ++st, ++use) {
      const int buf = use & 1;
      // the MMAs that last read this buffer (use - 2) must be complete
      fail = use >= 2 && !mbar_wait(smem_addr(&bar_a[buf]), ((use >> 1) - 1) & 1);
      if (fail) atomicExch(err, 2);
      unsigned char* A = sA + buf * S::A_BUF;
      // ---- gather of the stage's inputs into the three colour tiles
      gather_stage<CIN, S::K>(g, U32, in, V, live, x, st, part, A, row, S::A_TILE);
      // ---- make the tiles visible to the tensor core, then one thread issues the MMAs
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (__syncthreads_or(fail)) {
        aborted = true;
        break;
      }
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int r = 0; r < 3; ++r) {
          const uint32_t a0 = smem_addr(A + r * S::A_TILE);
          const uint32_t b0 = smem_addr(sB + st * S::B_ST);
#pragma unroll 1
          for (int kk = 0; kk < S::K / 16; ++kk)
            mma_f16(tmem + r * S::N, sdesc(a0 + kk * 256, 128, S::SBO), sdesc(b0 + kk * 256, 128, S::SBO), id,
                    (st > 0 || kk > 0) ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&bar_a[buf]))
                     : "memory");
        pending[buf] = (int)use;
      }
    }
    if (aborted) break;
    // ---- epilogue: all MMAs of the tile are complete when the last commit has arrived
    const uint32_t last = use - 1;
    fail = !mbar_wait(smem_addr(&bar_a[last & 1]), (last >> 1) & 1);
    if (fail) atomicExch(err, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(fail)) {
      aborted = true;
      break;
    }
    if (tid == 0) pending[0] = pending[1] = -1;
    {
      // warp w reads TMEM lanes 32 (w % 4) .. + 31; the 16-column chunks are dealt out
      // to the four column groups w / 4
      const int w = tid >> 5, q = w & 3, grp = w >> 2;
      const int srow = tile * kM + q * 32 + (tid & 31);
      constexpr int NCHUNK = 3 * S::N / 16;
#pragma unroll 1
      for (int chunk = grp; chunk < NCHUNK; chunk += kThreads / 128) {
        const int c0 = chunk * 16;
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + c0, v);
        if (srow < g.V) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int col = c0 + j;
            const int r = col / S::N, n = col % S::N;
            const int o = n >> 3, a = (n >> 1) & 3;
            if (o < COUT) {
              const size_t idx = ((size_t)o * 12 + a * 3 + r) * V + srow;
              if (OUT16)
                reinterpret_cast<__half2*>(out)[idx] = __floats2half2_rn(v[j], v[j + 1]);
              else
                reinterpret_cast<float2*>(out)[idx] = make_float2(v[j] * inv_sigma, v[j + 1] * inv_sigma);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // ---- teardown: nothing of this CTA may still be running on the tensor core
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if (pending[b] >= 0) mbar_wait(smem_addr(&bar_a[b]), ((uint32_t)pending[b] >> 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS));
}

// ---------------------------------------------------------------- pipelined layer (C_out = 8)
// The same contraction with the gather split in two: the raw neighbour activations go
// global -> shared by 4-byte cp.async copies (no registers held; the threads of a warp,
// consecutive sites, copy consecutive words), one stage ahead of the stage being
// transported; the links of the next stage are prefetched into registers.  Per stage:
// issue the copies of stage u + 1, wait for those of stage u, transport them from the
// staging buffer into the FP16 A tiles, one thread issues the MMAs.  Staging layout
// [slot][component][row] (slot: the input channel, or for C_in = 1 the direction of the
// stage), so the warp's reads in the transport are conflict-free.  The A tiles are
// single-buffered: the transport of stage u waits for the MMAs of stage u - 1.
template <int CIN>
struct Pipe {
  using S = Shape<CIN, 8>;
  static constexpr int SLOTS = CIN == 1 ? 4 : 8;
  static constexpr int STAGE_BYTES = SLOTS * 12 * kM * 4;
  static constexpr int SMEM = S::B_ALL + S::A_BUF + 2 * STAGE_BYTES;
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}


// the next stage's item of one thread: neighbour site, boundary factor, kind and the raw
// 12-real link (rebuilt and daggered at transport time)
struct HopRaw {
  float4 l[3];
  float f;
  int kind;  // 0 site, 1 forward, 2 backward, -1 nothing (padding or a dead row)
};

__device__ __forceinline__ void hop_prefetch(const Geom& g, const float4* __restrict__ U32, const int x[4], int d,
                                             HopRaw& h, size_t& sy) {
  h.kind = d == 0 ? 0 : (d <= 4 ? 1 : 2);
  const int mu = d == 0 ? 0 : (d - 1) & 3;
  int y[4] = {x[0], x[1], x[2], x[3]};
  h.f = 1.0f;
  if (h.kind == 1) {
    y[mu] = y[mu] + 1 == g.L[mu] ? 0 : y[mu] + 1;
    if (mu == 3 && x[3] == g.L[3] - 1) h.f = (float)g.bc_t;
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const float4* l = U32 + (size_t)((p * 4 + mu) * 3) * g.Vh + cb_index(g, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) h.l[k] = __ldg(l + (size_t)k * g.Vh);
  } else if (h.kind == 2) {
    y[mu] = y[mu] == 0 ? g.L[mu] - 1 : y[mu] - 1;
    if (mu == 3 && x[3] == 0) h.f = (float)g.bc_t;
    const int p = (y[0] + y[1] + y[2] + y[3]) & 1;
    const float4* l = U32 + (size_t)((p * 4 + mu) * 3) * g.Vh + cb_index(g, y);
#pragma unroll
    for (int k = 0; k < 3; ++k) h.l[k] = __ldg(l + (size_t)k * g.Vh);
  }
  sy = (size_t)lex_index(g, y);
}

__device__ __forceinline__ void site_coords(const Geom& g, int s, int x[4]) {
  int r = s;
  x[0] = r % g.L[0];
  r /= g.L[0];
  x[1] = r % g.L[1];
  r /= g.L[1];
  x[2] = r % g.L[2];
  x[3] = r / g.L[2];
}

template <int CIN>
__global__ void __launch_bounds__(kThreads, 1)
    k_nn_layer_tc2(Geom g, const float4* __restrict__ U32, const __half* __restrict__ Bg, const __half2* __restrict__ in,
                   __half2* __restrict__ out, int* __restrict__ err, const int* __restrict__ skip) {
  using S = Shape<CIN, 8>;
  using PP = Pipe<CIN>;
  if (skip && *skip) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t bar_w, bar_a;
  unsigned char* sB = sm;
  unsigned char* sA = sm + S::B_ALL;
  unsigned char* sR = sm + S::B_ALL + S::A_BUF;  // two staging buffers
  const int tid = threadIdx.x;
  const int row = tid & (kM - 1);
  const int part = tid >> 7;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_w)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_a)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(S::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar_w)), "r"(S::B_ALL)
                 : "memory");
    for (int st = 0; st < S::NST; ++st)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(sB + st * S::B_ST)),
          "l"(Bg + (size_t)st * (S::B_ST / 2)), "r"(S::B_ST), "r"(smem_addr(&bar_w))
          : "memory");
  }
  bool fail = !mbar_wait(smem_addr(&bar_w), 0);
  if (fail) atomicExch(err, 1);
  bool aborted = __syncthreads_or(fail);

  const int ntiles = (g.V + kM - 1) / kM;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nwork = my_tiles * S::NST;
  const uint32_t id = idesc(kM, S::N);

  // issue the copies (and link loads) of work item u into staging buffer u & 1
  auto issue = [&](int u, HopRaw& h) {
    h.kind = -1;
    if (u >= nwork) return;
    const int tile = blockIdx.x + (u / S::NST) * gridDim.x, st = u % S::NST;
    const int s = tile * kM + row;
    if (s >= g.V) return;
    int x[4];
    site_coords(g, s, x);
    const int di = CIN == 1 ? 4 * st + part : st;
    if (di >= 9) return;
    size_t sy;
    hop_prefetch(g, U32, x, dir_of(di), h, sy);
    const uint32_t base = smem_addr(sR + (u & 1) * PP::STAGE_BYTES) + row * 4;
    const size_t V = (size_t)g.V;
    // C_in = 8: channels 2 part, 2 part + 1; C_in = 1: the part's direction slot
#pragma unroll
    for (int q = 0; q < (CIN == 1 ? 1 : 2); ++q) {
      const int ic = CIN == 1 ? 0 : 2 * part + q;
      const int slot = CIN == 1 ? part : ic;
#pragma unroll
      for (int k = 0; k < 12; ++k)
        cp_async4(base + (uint32_t)((slot * 12 + k) * kM) * 4, in + ((size_t)ic * 12 + k) * V + sy);
    }
  };

  HopRaw cur, nxt;
  if (!aborted) issue(0, cur);
  asm volatile("cp.async.commit_group;" ::: "memory");
  uint32_t commits = 0;  // MMA commits issued on bar_a
  for (int u = 0; u < nwork && !aborted; ++u) {
    const int tl = u / S::NST, st = u % S::NST;
    const int tile = blockIdx.x + tl * gridDim.x;
    issue(u + 1, nxt);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    // the MMAs of the previous stage read the A tiles: wait for them
    fail = commits > 0 && !mbar_wait(smem_addr(&bar_a), (commits - 1) & 1);
    if (fail) atomicExch(err, 2);
    if (__syncthreads_or(fail)) {
      aborted = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- transport the staged inputs into the three colour tiles
    {
      const uint32_t* R = reinterpret_cast<const uint32_t*>(sR + (u & 1) * PP::STAGE_BYTES) + row;
      Hop h;
      h.kind = cur.kind < 0 ? 0 : cur.kind;
      h.f = cur.f;
      if (cur.kind > 0) {
        Mat3<float> L;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          L.m[(2 * k) / 3][(2 * k) % 3] = mk(cur.l[k].x, cur.l[k].y);
          L.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(cur.l[k].z, cur.l[k].w);
        }
        reconstruct_row2(L);
        h.U = cur.kind == 1 ? L : dagger(L);
      }
      const bool live = cur.kind >= 0;
      constexpr int NCH = CIN == 1 ? 1 : 2;
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        const int slot = CIN == 1 ? part : 2 * part + q;
        cplx<float> v[4][3];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float2 f = live ? h2_to_f2(R[(slot * 12 + k) * kM]) : make_float2(0.f, 0.f);
          v[k / 3][k % 3] = mk(f.x, f.y);
        }
        const int col = CIN == 1 ? part * 8 : (2 * part + q) * 8;
        store_channel<S::K>(h, v, live, sA, row, col, S::A_TILE);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int r = 0; r < 3; ++r) {
        const uint32_t a0 = smem_addr(sA + r * S::A_TILE);
        const uint32_t b0 = smem_addr(sB + st * S::B_ST);
#pragma unroll 1
        for (int kk = 0; kk < S::K / 16; ++kk)
          mma_f16(tmem + r * S::N, sdesc(a0 + kk * 256, 128, S::SBO), sdesc(b0 + kk * 256, 128, S::SBO), id,
                  (st > 0 || kk > 0) ? 1u : 0u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar_a))
                   : "memory");
    }
    ++commits;
    cur = nxt;
    if (st == S::NST - 1) {
      // ---- epilogue of the tile: accumulators complete when the last commit arrived
      fail = !mbar_wait(smem_addr(&bar_a), (commits - 1) & 1);
      if (fail) atomicExch(err, 3);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (__syncthreads_or(fail)) {
        aborted = true;
        break;
      }
      // warp w: TMEM lanes 32 (w % 4) .. + 31 (sites), output channels 2 (w / 4), + 1;
      // channel-major output [8][12][V]: consecutive lanes write consecutive sites
      const int w = tid >> 5, qd = w & 3, grp = w >> 2;
      const int srow = tile * kM + qd * 32 + (tid & 31);
      const size_t V = (size_t)g.V;
      float v[3][16];
#pragma unroll
      for (int r = 0; r < 3; ++r) tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + r * S::N + grp * 16, v[r]);
      if (srow < g.V) {
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int k = 0; k < 12; ++k) {  // complex k = spin a * 3 + colour r
            const int a = k / 3, r = k % 3;
            out[((size_t)(2 * grp + o) * 12 + k) * V + srow] =
                __floats2half2_rn(v[r][o * 8 + a * 2], v[r][o * 8 + a * 2 + 1]);
          }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  // ---- teardown: no copy in flight, nothing of this CTA running on the tensor core
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (tid == 0 && commits > 0) mbar_wait(smem_addr(&bar_a), (commits - 1) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS));
}

}  // namespace tc

// ---------------------------------------------------------------- host side
// layers with (C_in, C_out) in {(1, 8), (8, 8), (8, 1)} run on the tensor cores
bool nn_tc_supported(int cin, int cout) {
  return (cin == 1 && cout == 8) || (cin == 8 && cout == 8) || (cin == 8 && cout == 1);
}

// the last layer (8 -> 1) is packed for the local mixing (Shape<8, 9>)
size_t nn_tc_packed_bytes(int cin, int cout) {
  if (cin == 1) return tc::Shape<1, 8>::B_ALL;
  if (cout == 1) return tc::Shape<8, 9>::B_ALL;
  return tc::Shape<8, 8>::B_ALL;
}

template <int CIN, int COUT>
static void pack_t(pfmp_ctx* c, const void* W, void* Bp) {
  using S = tc::Shape<CIN, COUT>;
  const int n = S::NST * S::N * S::K;
  tc::k_pack_b<CIN, COUT><<<nblocks(n, 256), 256, 0, c->stream>>>((const float2*)W, (__half*)Bp);
  PFMP_CHECK_LAUNCH();
}

void nn_tc_pack(pfmp_ctx* c, int cin, int cout, const void* W, void* Bp) {
  if (cin == 1)
    pack_t<1, 8>(c, W, Bp);
  else if (cout == 1)
    pack_t<8, 9>(c, W, Bp);
  else
    pack_t<8, 8>(c, W, Bp);
}

void nn_tc_scale(pfmp_ctx* c, const void* in_even_f32, float* sigma_dev, const int* skip) {
  const long n = 6L * c->g.Vh;
  long b = (n + kBlock - 1) / kBlock;
  const int grid = (int)(b < 152 * 4 ? b : 152 * 4);
  tc::k_rms_scale<<<grid, kBlock, 0, c->stream>>>((const float4*)in_even_f32, c->g.Vh, c->rb, sigma_dev, skip);
  PFMP_CHECK_LAUNCH();
}

template <int CIN, int COUT, bool OUT16>
static int layer_init() {
  using S = tc::Shape<CIN, COUT>;
  static int sms = 0;
  if (!sms) {
    PFMP_CUDA(cudaFuncSetAttribute(tc::k_nn_layer_tc<CIN, COUT, OUT16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   S::SMEM));
    int dev = 0;
    PFMP_CUDA(cudaGetDevice(&dev));
    PFMP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

template <int CIN>
static int layer2_init() {
  static int sms = 0;
  if (!sms) {
    PFMP_CUDA(cudaFuncSetAttribute(tc::k_nn_layer_tc2<CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   tc::Pipe<CIN>::SMEM));
    int dev = 0;
    PFMP_CUDA(cudaGetDevice(&dev));
    PFMP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

// kernel attributes set outside any stream capture
void nn_tc_init() {
  layer_init<1, 8, true>();
  layer_init<8, 8, true>();
  layer_init<8, 9, true>();
  layer2_init<1>();
  layer2_init<8>();
}

// The staged variant (k_nn_layer_tc2) measured slower than the single-stage kernel at
// 16^3 x 32 (one network application 0.77 vs 0.57 ms): with one stage of lookahead it holds
// about the same bytes in flight per SM (one stage, ~48 KB) and adds a barrier and a
// shared-memory round trip per stage.  It is kept selectable (PFMP_NN_TC_PIPE=1 in the
// environment) for profiling; the single-stage kernel is the default.
static bool use_pipe() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("PFMP_NN_TC_PIPE");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

template <int CIN>
static void layer2_t(pfmp_ctx* c, const void* Bp, const void* in, void* out, int* err, const int* skip) {
  const int sms = layer2_init<CIN>();
  const int ntiles = (c->g.V + tc::kM - 1) / tc::kM;
  const int grid = ntiles < sms ? ntiles : sms;
  tc::k_nn_layer_tc2<CIN><<<grid, tc::kThreads, tc::Pipe<CIN>::SMEM, c->stream>>>(
      c->g, c->U32, (const __half*)Bp, (const __half2*)in, (__half2*)out, err, skip);
  PFMP_CHECK_LAUNCH();
}

template <int CIN, int COUT, bool OUT16>
static void layer_t(pfmp_ctx* c, const void* Bp, const void* in, void* out, const float* sigma, int* err,
                    const int* skip) {
  using S = tc::Shape<CIN, COUT>;
  const int sms = layer_init<CIN, COUT, OUT16>();
  const int ntiles = (c->g.V + tc::kM - 1) / tc::kM;
  const int grid = ntiles < sms ? ntiles : sms;
  tc::k_nn_layer_tc<CIN, COUT, OUT16><<<grid, tc::kThreads, S::SMEM, c->stream>>>(
      c->g, c->U32, (const __half*)Bp, (const __half2*)in, out, sigma, err, skip);
  PFMP_CHECK_LAUNCH();
}

// in: FP16 scaled activations; out: FP16 scaled (last = false) or FP32 / sigma (last)
void nn_tc_layer(pfmp_ctx* c, int cin, int cout, bool last, const void* Bp, const void* in, void* out,
                 const float* sigma, int* err, const int* skip) {
  PFMP_REQUIRE(!last && cout == 8, PFMP_E_INVALID, "tensor-core layer sequence (the last layer: nn_tc_last)");
  if (use_pipe()) {
    if (cin == 1)
      layer2_t<1>(c, Bp, in, out, err, skip);
    else
      layer2_t<8>(c, Bp, in, out, err, skip);
  } else if (cin == 1) {
    layer_t<1, 8, true>(c, Bp, in, out, sigma, err, skip);
  } else {
    layer_t<8, 8, true>(c, Bp, in, out, sigma, err, skip);
  }
}

// the last layer (8 -> 1) as local mixing on the tensor cores (z, FP16 [9][12][V]) and
// the even-site transport stencil, straight into the even FP32 output field
void nn_tc_last(pfmp_ctx* c, const void* Bp, const void* in, void* z16, void* out_even_f32, const float* sigma,
                int* err, const int* skip) {
  layer_t<8, 9, true>(c, Bp, in, z16, sigma, err, skip);
  tc::k_last_stencil<<<nblocks(c->g.Vh, 128), 128, 0, c->stream>>>(c->g, c->U32, (const __half2*)z16,
                                                                   (float4*)out_even_f32, sigma, skip);
  PFMP_CHECK_LAUNCH();
}

void nn_tc_embed(pfmp_ctx* c, const void* in_even_f32, float* sigma, void* act16, const int* skip, const double* rr) {
  tc::k_embed16<<<nblocks(c->g.V, 256), 256, 0, c->stream>>>(c->g, (const float4*)in_even_f32, sigma,
                                                             (__half2*)act16, skip, rr);
  PFMP_CHECK_LAUNCH();
}

}  // namespace pfmp
