// Context, gauge field, layout conversion and field initialisation.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "context.h"
#include "fields.cuh"
#include "su3.cuh"
#include "dfloat.cuh"

namespace pfmp {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }
void set_last_error(const std::string& s) { g_last_error = s; }
const char* last_error() { return g_last_error.c_str(); }

void* dev_alloc(size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    throw Err{PFMP_E_NOMEM};
  }
  return p;
}
void dev_free(void* p) {
  if (p) cudaFree(p);
}

// ------------------------------------------------------------------ master link access
__device__ __forceinline__ const double2* master_ptr(const double2* U, const Geom& g, int parity, int mu) {
  return U + (size_t)((parity * 4 + mu) * 9) * g.Vh;
}
__device__ __forceinline__ Mat3<double> link_at(const double2* U, const Geom& g, const int x[4], int mu) {
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  Mat3<double> M;
  load_link18(M, master_ptr(U, g, p, mu), cb_index(g, x), g.Vh);
  return M;
}

// ------------------------------------------------------------------ kernels
__global__ void k_gauge_from_canonical(Geom g, const double* __restrict__ src, double2* __restrict__ U) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, p, x);
  const size_t s = lex_index(g, x);
  for (int mu = 0; mu < 4; ++mu) {
    double2* dst = U + (size_t)((p * 4 + mu) * 9) * g.Vh;
    const double* q = src + (s * 4 + mu) * 18;
    for (int k = 0; k < 9; ++k) dst[(size_t)k * g.Vh + cb] = make_double2(q[2 * k], q[2 * k + 1]);
  }
}

__global__ void k_gauge_to_canonical(Geom g, const double2* __restrict__ U, double* __restrict__ dst) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, p, x);
  const size_t s = lex_index(g, x);
  for (int mu = 0; mu < 4; ++mu) {
    const double2* src = U + (size_t)((p * 4 + mu) * 9) * g.Vh;
    double* q = dst + (s * 4 + mu) * 18;
    for (int k = 0; k < 9; ++k) {
      double2 v = src[(size_t)k * g.Vh + cb];
      q[2 * k] = v.x;
      q[2 * k + 1] = v.y;
    }
  }
}

__global__ void k_gauge_compress(Geom g, const double2* __restrict__ U, float4* __restrict__ U32,
                                 float4* __restrict__ Udf, uint4* __restrict__ U16) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int pm = blockIdx.y;  // parity*4 + mu
  if (cb >= g.Vh) return;
  const double2* src = U + (size_t)(pm * 9) * g.Vh;
  double2 v[6];
  for (int k = 0; k < 6; ++k) v[k] = src[(size_t)k * g.Vh + cb];
  float4* ddf = Udf + (size_t)(pm * 9) * g.Vh;
  for (int k = 0; k < 9; ++k) ddf[(size_t)k * g.Vh + cb] = split2(src[(size_t)k * g.Vh + cb]);
  float4* d32 = U32 + (size_t)(pm * 3) * g.Vh;
  for (int k = 0; k < 3; ++k)
    d32[(size_t)k * g.Vh + cb] =
        make_float4((float)v[2 * k].x, (float)v[2 * k].y, (float)v[2 * k + 1].x, (float)v[2 * k + 1].y);
  uint4* d16 = U16 + (size_t)pm * 3 * (g.Vh / 2);  // link planes of 24 bytes per link
  uint32_t h[6];
  for (int k = 0; k < 6; ++k) h[k] = f2_to_h2((float)v[k].x, (float)v[k].y);
  d16[cb] = make_uint4(h[0], h[1], h[2], h[3]);
  reinterpret_cast<uint2*>(d16 + g.Vh)[cb] = make_uint2(h[4], h[5]);
}

__global__ void k_gauge_from_algebra(Geom g, const double* __restrict__ h, double eps, double2* __restrict__ U) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, p, x);
  const size_t s = lex_index(g, x);
  for (int mu = 0; mu < 4; ++mu) {
    double c[8];
    for (int a = 0; a < 8; ++a) c[a] = h[(s * 4 + mu) * 8 + a];
    Mat3<double> E = expm_algebra(c, eps);
    reunitarise(E);
    store_link18(U + (size_t)((p * 4 + mu) * 9) * g.Vh, E, cb, g.Vh);
  }
}

__global__ void k_plaquette(Geom g, const double2* __restrict__ U, ReduceBuf rb, double* out) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  double v[1] = {0.0};
  if (cb < g.Vh) {
    int x[4];
    cb_coords(g, cb, p, x);
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
        xm[mu] = (xm[mu] + 1) % g.L[mu];
        xn[nu] = (xn[nu] + 1) % g.L[nu];
        Mat3<double> A = matmul(link_at(U, g, x, mu), link_at(U, g, xm, nu));
        Mat3<double> B = matmul(link_at(U, g, x, nu), link_at(U, g, xn, mu));
        Mat3<double> P = matmul_nd(A, B);
        v[0] += P.m[0][0].re + P.m[1][1].re + P.m[2][2].re;
      }
  }
  // 2-D grid: flatten block id for the reduction
  double tot[1];
  if (grid_sum<1>(v, rb, tot)) *out = tot[0];
}

template <int PREC>
__global__ void k_spinor_pack(Geom g, const double* __restrict__ src, typename Prec<PREC>::vec* dst, int parity) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, parity, x);
  const double* q = src + (size_t)lex_index(g, x) * 24;
  Spinor<typename Prec<PREC>::real> s;
  for (int k = 0; k < 12; ++k) s.s[k / 3][k % 3] = mk((typename Prec<PREC>::real)q[2 * k], (typename Prec<PREC>::real)q[2 * k + 1]);
  store_spinor(dst, s, cb, g.Vh);
}

template <int PREC>
__global__ void k_spinor_unpack(Geom g, double* __restrict__ dst, const typename Prec<PREC>::vec* src, int parity) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, parity, x);
  double* q = dst + (size_t)lex_index(g, x) * 24;
  Spinor<typename Prec<PREC>::real> s;
  load_spinor(s, src, cb, g.Vh);
  for (int k = 0; k < 12; ++k) {
    q[2 * k] = (double)s.s[k / 3][k % 3].re;
    q[2 * k + 1] = (double)s.s[k / 3][k % 3].im;
  }
}

// ------------------------------------------------------------------ host side
static double* canon_scratch(pfmp_ctx* c, size_t doubles) {
  // grows on demand; sized for a gauge field (72 doubles per site) at most
  static_assert(sizeof(double) == 8, "");
  if (!c->canon) c->canon = (double*)dev_alloc((size_t)c->g.V * 72 * sizeof(double));
  (void)doubles;
  return c->canon;
}

void gauge_refresh_compressed(pfmp_ctx* c) {
  dim3 grid(nblocks(c->g.Vh), 8);
  k_gauge_compress<<<grid, kBlock, 0, c->stream>>>(c->g, c->U64, c->U32, c->Udf, c->U16);
  PFMP_CHECK_LAUNCH();
  c->gauge_version++;
}

void spinor_pack(pfmp_ctx* c, void* dst, int prec, const double* src_dev, int parity) {
  if (prec == PFMP_F64)
    k_spinor_pack<PFMP_F64><<<nblocks(c->g.Vh), kBlock, 0, c->stream>>>(c->g, src_dev, (double2*)dst, parity);
  else if (prec == PFMP_H16)
    k_spinor_pack<PFMP_H16><<<nblocks(c->g.Vh), kBlock, 0, c->stream>>>(c->g, src_dev, (uint4*)dst, parity);
  else
    k_spinor_pack<PFMP_F32><<<nblocks(c->g.Vh), kBlock, 0, c->stream>>>(c->g, src_dev, (float4*)dst, parity);
  PFMP_CHECK_LAUNCH();
}
void spinor_unpack(pfmp_ctx* c, double* dst_dev, const void* src, int prec, int parity) {
  if (prec == PFMP_F64)
    k_spinor_unpack<PFMP_F64><<<nblocks(c->g.Vh), kBlock, 0, c->stream>>>(c->g, dst_dev, (const double2*)src, parity);
  else if (prec == PFMP_H16)
    k_spinor_unpack<PFMP_H16><<<nblocks(c->g.Vh), kBlock, 0, c->stream>>>(c->g, dst_dev, (const uint4*)src, parity);
  else
    k_spinor_unpack<PFMP_F32><<<nblocks(c->g.Vh), kBlock, 0, c->stream>>>(c->g, dst_dev, (const float4*)src, parity);
  PFMP_CHECK_LAUNCH();
}

pfmp_ctx* ctx_create(const int dims[4], int bc_t, void* stream) {
  for (int m = 0; m < 4; ++m) PFMP_REQUIRE(dims[m] >= 2 && dims[m] % 2 == 0, PFMP_E_INVALID, "lattice extents must be even and >= 2");
  PFMP_REQUIRE(bc_t == 1 || bc_t == -1, PFMP_E_INVALID, "bc_t must be +1 or -1");
  const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  PFMP_REQUIRE(V / 2 < (1L << 30), PFMP_E_INVALID, "lattice too large for 32-bit site indices");
  pfmp_ctx* c = new pfmp_ctx();
  try {
    for (int m = 0; m < 4; ++m) c->g.L[m] = dims[m];
    c->g.V = (int)V;
    c->g.Vh = (int)(V / 2);
    c->g.bc_t = bc_t;
    c->stream = (cudaStream_t)stream;
    PFMP_CUDA(cudaGetDevice(&c->device));
    c->U64 = (double2*)dev_alloc((size_t)c->g.Vh * 2 * 4 * 9 * sizeof(double2));
    c->U32 = (float4*)dev_alloc((size_t)c->g.Vh * 2 * 4 * 3 * sizeof(float4));
    c->Udf = (float4*)dev_alloc((size_t)c->g.Vh * 2 * 4 * 9 * sizeof(float4));
    c->U16 = (uint4*)dev_alloc((size_t)c->g.Vh * 2 * 4 * 24);
    c->rb.partials = (double*)dev_alloc((size_t)kMaxReduceBlocks * kMaxSums * sizeof(double));
    c->rb.counter = (unsigned*)dev_alloc(sizeof(unsigned));
    PFMP_CUDA(cudaMemset(c->rb.counter, 0, sizeof(unsigned)));
    c->d_sums = (double*)dev_alloc(64 * sizeof(double));
    PFMP_CUDA(cudaMallocHost(&c->h_sums, 64 * sizeof(double)));
  } catch (...) {
    dev_free(c->U64);
    dev_free(c->U32);
    dev_free(c->Udf);
    dev_free(c->U16);
    dev_free(c->rb.partials);
    dev_free(c->rb.counter);
    dev_free(c->d_sums);
    if (c->h_sums) cudaFreeHost(c->h_sums);
    delete c;
    throw;
  }
  return c;
}

static cudaEvent_t prof_event(pfmp_ctx* c) {
  KernelProfile& P = c->prof;
  if (P.used == P.pool.size()) {
    cudaEvent_t e;
    PFMP_CUDA(cudaEventCreate(&e));
    P.pool.push_back(e);
  }
  return P.pool[P.used++];
}

void prof_start(pfmp_ctx* c, cudaEvent_t* a) {
  *a = nullptr;
  if (!c->prof.on) return;
  *a = prof_event(c);
  PFMP_CUDA(cudaEventRecord(*a, c->stream));
}

void prof_stop(pfmp_ctx* c, int cls, double bytes, cudaEvent_t a) {
  if (!c->prof.on || !a) return;
  cudaEvent_t b = prof_event(c);
  PFMP_CUDA(cudaEventRecord(b, c->stream));
  c->prof.recs.push_back({cls, bytes, a, b});
}

void profile_begin(pfmp_ctx* c) {
  c->prof.on = true;
  c->prof.used = 0;
  c->prof.recs.clear();
}

// totals of one kernel class since profile_begin; stops recording
void profile_end(pfmp_ctx* c, int cls, long* launches, double* ms, double* bytes) {
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  *launches = 0;
  *ms = 0;
  *bytes = 0;
  for (auto& r : c->prof.recs) {
    if (r.cls != cls) continue;
    float t = 0;
    PFMP_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    *launches += 1;
    *ms += t;
    *bytes += r.bytes;
  }
  c->prof.on = false;
}

void ctx_destroy(pfmp_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  dev_free(c->U64);
  dev_free(c->U32);
  dev_free(c->Udf);
  dev_free(c->U16);
  dev_free(c->rb.partials);
  dev_free(c->rb.counter);
  dev_free(c->d_sums);
  dev_free(c->canon);
  dev_free(c->fmunu);
  dev_free(c->hc32);
  if (c->h_sums) cudaFreeHost(c->h_sums);
  delete c;
}

void gauge_set(pfmp_ctx* c, const double* U, int where) {
  const double* src = U;
  if (where == PFMP_HOST) {
    double* buf = canon_scratch(c, (size_t)c->g.V * 72);
    PFMP_CUDA(cudaMemcpyAsync(buf, U, (size_t)c->g.V * 72 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = buf;
  }
  dim3 grid(nblocks(c->g.Vh), 2);
  k_gauge_from_canonical<<<grid, kBlock, 0, c->stream>>>(c->g, src, c->U64);
  PFMP_CHECK_LAUNCH();
  gauge_refresh_compressed(c);
  if (where == PFMP_HOST) PFMP_CUDA(cudaStreamSynchronize(c->stream));
}

void gauge_get(pfmp_ctx* c, double* U, int where) {
  double* dst = where == PFMP_HOST ? canon_scratch(c, (size_t)c->g.V * 72) : U;
  dim3 grid(nblocks(c->g.Vh), 2);
  k_gauge_to_canonical<<<grid, kBlock, 0, c->stream>>>(c->g, c->U64, dst);
  PFMP_CHECK_LAUNCH();
  if (where == PFMP_HOST) {
    PFMP_CUDA(cudaMemcpyAsync(U, dst, (size_t)c->g.V * 72 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
  }
}

void gauge_from_algebra(pfmp_ctx* c, const double* h, double eps, int where) {
  const double* src = h;
  if (where == PFMP_HOST) {
    double* buf = canon_scratch(c, (size_t)c->g.V * 32);
    PFMP_CUDA(cudaMemcpyAsync(buf, h, (size_t)c->g.V * 32 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = buf;
  }
  dim3 grid(nblocks(c->g.Vh), 2);
  k_gauge_from_algebra<<<grid, kBlock, 0, c->stream>>>(c->g, src, eps, c->U64);
  PFMP_CHECK_LAUNCH();
  gauge_refresh_compressed(c);
  if (where == PFMP_HOST) PFMP_CUDA(cudaStreamSynchronize(c->stream));
}

double plaquette(pfmp_ctx* c) {
  dim3 grid(nblocks(c->g.Vh), 2);
  k_plaquette<<<grid, kBlock, 0, c->stream>>>(c->g, c->U64, c->rb, c->d_sums);
  PFMP_CHECK_LAUNCH();
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_sums[0] / (18.0 * c->g.V);
}

void spinor_pack_any(pfmp_ctx* c, void* dst, int prec, const double* src, int where, int parity) {
  const double* s = src;
  if (where == PFMP_HOST) {
    double* buf = canon_scratch(c, (size_t)c->g.V * 24);
    PFMP_CUDA(cudaMemcpyAsync(buf, src, (size_t)c->g.V * 24 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    s = buf;
  }
  spinor_pack(c, dst, prec, s, parity);
  if (where == PFMP_HOST) PFMP_CUDA(cudaStreamSynchronize(c->stream));
}

void spinor_unpack_any(pfmp_ctx* c, double* dst, int where, const void* src, int prec, int parity) {
  if (where == PFMP_HOST) {
    // host destination: the other parity's sites are written as zero
    double* buf = canon_scratch(c, (size_t)c->g.V * 24);
    PFMP_CUDA(cudaMemsetAsync(buf, 0, (size_t)c->g.V * 24 * sizeof(double), c->stream));
    spinor_unpack(c, buf, src, prec, parity);
    PFMP_CUDA(cudaMemcpyAsync(dst, buf, (size_t)c->g.V * 24 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
  } else {
    spinor_unpack(c, dst, src, prec, parity);
  }
}

}  // namespace pfmp
