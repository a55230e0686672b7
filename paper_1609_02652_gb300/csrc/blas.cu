// BLAS-1 on single-parity spinor fields and the fused CG vector updates.  All sums are
// accumulated in FP64 and reduced deterministically (reduce.cuh).  Grid-stride loops
// over 16-byte words with a grid of a few blocks per SM.
#include "context.h"
#include "fields.cuh"

namespace pfmp {

static int blas_grid(long n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  long b = (n + kBlock - 1) / kBlock;
  long cap = (long)sms * 8;
  return (int)(b < cap ? b : cap);
}

__device__ __forceinline__ double dot2(double2 a) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------------------------- elementwise
// F64 [12][Vh] double2 -> F32 [6][Vh] float4 and back
__global__ void k_f64_to_f32(const double2* __restrict__ s, float4* __restrict__ d, int Vh) {
  const long n = 6L * Vh;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long k = i / Vh, cb = i % Vh;
    double2 a = s[(2 * k) * Vh + cb], b = s[(2 * k + 1) * Vh + cb];
    d[i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}
__global__ void k_f32_to_f64(const float4* __restrict__ s, double2* __restrict__ d, int Vh, int accumulate) {
  const long n = 6L * Vh;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long k = i / Vh, cb = i % Vh;
    float4 v = s[i];
    double2 a = make_double2(v.x, v.y), b = make_double2(v.z, v.w);
    if (accumulate) {
      double2 a0 = d[(2 * k) * Vh + cb], b0 = d[(2 * k + 1) * Vh + cb];
      a.x += a0.x;
      a.y += a0.y;
      b.x += b0.x;
      b.y += b0.y;
    }
    d[(2 * k) * Vh + cb] = a;
    d[(2 * k + 1) * Vh + cb] = b;
  }
}

__global__ void k_axpy64(double are, double aim, const double2* __restrict__ x, double2* __restrict__ y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 a = x[i], b = y[i];
    b.x += are * a.x - aim * a.y;
    b.y += are * a.y + aim * a.x;
    y[i] = b;
  }
}
__global__ void k_axpy32(float are, float aim, const float4* __restrict__ x, float4* __restrict__ y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float4 a = x[i], b = y[i];
    b.x += are * a.x - aim * a.y;
    b.y += are * a.y + aim * a.x;
    b.z += are * a.z - aim * a.w;
    b.w += are * a.w + aim * a.z;
    y[i] = b;
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double sq(double2 a) { return dot2(a); }
__device__ __forceinline__ float sq(float4 a) { return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w; }

// FP32 fields: each thread's few terms summed in FP32 (GB300's FP64 pipe is a small
// fraction of the FP32 one), the sums across threads and blocks in FP64
template <typename V>
__global__ void k_norm2(const V* __restrict__ x, long n, ReduceBuf rb, double* out) {
  decltype(sq(x[0])) acc = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) acc += sq(x[i]);
  double v[1] = {(double)acc};
  double t[1];
  if (grid_sum<1>(v, rb, t)) *out = t[0];
}

// <x, y> = sum conj(x) y  (re, im)
__global__ void k_cdot64(const double2* __restrict__ x, const double2* __restrict__ y, long n, ReduceBuf rb,
                         double* out) {
  double v[2] = {0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 a = x[i], b = y[i];
    v[0] += a.x * b.x + a.y * b.y;
    v[1] += a.x * b.y - a.y * b.x;
  }
  double t[2];
  if (grid_sum<2>(v, rb, t)) {
    out[0] = t[0];
    out[1] = t[1];
  }
}
__global__ void k_cdot32(const float4* __restrict__ x, const float4* __restrict__ y, long n, ReduceBuf rb,
                         double* out) {
  double v[2] = {0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float4 a = x[i], b = y[i];
    v[0] += (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z + (double)a.w * b.w;
    v[1] += (double)a.x * b.y - (double)a.y * b.x + (double)a.z * b.w - (double)a.w * b.z;
  }
  double t[2];
  if (grid_sum<2>(v, rb, t)) {
    out[0] = t[0];
    out[1] = t[1];
  }
}

// r = b - Ax, out = |r|^2 (FP64)
__global__ void k_xmy_norm(const double2* __restrict__ b, const double2* __restrict__ Ax, double2* __restrict__ r,
                           long n, ReduceBuf rb, double* out) {
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 a = b[i], c = Ax[i];
    double2 d = make_double2(a.x - c.x, a.y - c.y);
    r[i] = d;
    v[0] += dot2(d);
  }
  double t[1];
  if (grid_sum<1>(v, rb, t)) *out = t[0];
}

// ---------------------------------------------------------------- CG updates
// x += alpha p, r -= alpha Ap, rr_new = |r|^2; finisher: beta = rr_new/rr, rr = rr_new,
// iter++, done = (rr < stop_rr)
__global__ void k_cg_xr64(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                          const double2* __restrict__ Ap, long n, ReduceBuf rb, CGScalars* s) {
  if (s->done) return;
  const double al = s->alpha;
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 xx = x[i], rr = r[i], pp = p[i], aa = Ap[i];
    xx.x += al * pp.x;
    xx.y += al * pp.y;
    rr.x -= al * aa.x;
    rr.y -= al * aa.y;
    x[i] = xx;
    r[i] = rr;
    v[0] += dot2(rr);
  }
  double t[1];
  if (grid_sum<1>(v, rb, t)) {
    s->rr_new = t[0];
    s->beta = t[0] / s->rr;
    s->rr = t[0];
    s->iter += 1;
    if (t[0] < s->stop_rr || !(t[0] == t[0])) s->done_next = 1;
  }
}
__global__ void k_cg_xr32(float4* __restrict__ x, float4* __restrict__ r, const float4* __restrict__ p,
                          const float4* __restrict__ Ap, long n, ReduceBuf rb, CGScalars* s) {
  if (s->done) return;
  const float al = (float)s->alpha;
  float acc = 0.f;  // per-thread |r|^2 in FP32, across threads in FP64
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float4 xx = x[i], rr = r[i], pp = p[i], aa = Ap[i];
    xx.x += al * pp.x;
    xx.y += al * pp.y;
    xx.z += al * pp.z;
    xx.w += al * pp.w;
    rr.x -= al * aa.x;
    rr.y -= al * aa.y;
    rr.z -= al * aa.z;
    rr.w -= al * aa.w;
    x[i] = xx;
    r[i] = rr;
    acc += sq(rr);
  }
  double v[1] = {(double)acc};
  double t[1];
  if (grid_sum<1>(v, rb, t)) {
    s->rr_new = t[0];
    s->beta = t[0] / s->rr;
    s->rr = t[0];
    s->iter += 1;
    if (t[0] < s->stop_rr || !(t[0] == t[0])) s->done_next = 1;
  }
}
// p = r + beta p; the last block then raises `done` if the x/r update asked for it, so
// that an iteration always completes its three updates before the loop stops
__global__ void k_cg_p64(double2* __restrict__ p, const double2* __restrict__ r, long n, ReduceBuf rb,
                         CGScalars* s) {
  if (s->done) return;
  const double be = s->beta;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double2 pp = p[i], rr = r[i];
    p[i] = make_double2(rr.x + be * pp.x, rr.y + be * pp.y);
  }
  double v[1] = {0.0}, t[1];
  if (grid_sum<1>(v, rb, t)) s->done = s->done_next;
}
__global__ void k_cg_p32(float4* __restrict__ p, const float4* __restrict__ r, long n, ReduceBuf rb,
                         CGScalars* s) {
  if (s->done) return;
  const float be = (float)s->beta;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float4 pp = p[i], rr = r[i];
    p[i] = make_float4(rr.x + be * pp.x, rr.y + be * pp.y, rr.z + be * pp.z, rr.w + be * pp.w);
  }
  double v[1] = {0.0}, t[1];
  if (grid_sum<1>(v, rb, t)) s->done = s->done_next;
}

// ---------------------------------------------------------------- FP16 storage
// (site-parallel: a site's scale covers its 24 reals)
__global__ void k_f32_to_h16(const float4* __restrict__ s, uint4* __restrict__ d, int Vh) {
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
    Spinor<float> v;
    load_spinor(v, s, cb, Vh);
    store_spinor(d, v, cb, Vh);
  }
}
__global__ void k_h16_to_f32(const uint4* __restrict__ s, float4* __restrict__ d, int Vh) {
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
    Spinor<float> v;
    load_spinor(v, s, cb, Vh);
    store_spinor(d, v, cb, Vh);
  }
}

__device__ __forceinline__ float h16_scale(const uint4* f, int cb, int Vh) {
  return reinterpret_cast<const float*>(f + (size_t)3 * Vh)[cb];
}

// FP32 x, r with FP16 p, Ap: x += alpha p, r -= alpha Ap, |r|^2 -> beta, rr, iter, done_next
__global__ void k_cg_xr_h(float4* __restrict__ x, float4* __restrict__ r, const uint4* __restrict__ p,
                          const uint4* __restrict__ Ap, int Vh, ReduceBuf rb, CGScalars* s) {
  if (s->done) return;
  const float al = (float)s->alpha;
  float acc = 0.f;
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
    const float ap = al * h16_scale(p, cb, Vh), aa = al * h16_scale(Ap, cb, Vh);
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // FP16 word k = FP32 words 2k and 2k + 1
      const uint4 pv = p[(size_t)k * Vh + cb], av = Ap[(size_t)k * Vh + cb];
      const uint32_t pw[4] = {pv.x, pv.y, pv.z, pv.w}, aw[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const size_t i = (size_t)(2 * k + h) * Vh + cb;
        const float2 p0 = h2_to_f2(pw[2 * h]), p1 = h2_to_f2(pw[2 * h + 1]);
        const float2 a0 = h2_to_f2(aw[2 * h]), a1 = h2_to_f2(aw[2 * h + 1]);
        float4 xx = x[i], rr = r[i];
        xx.x += ap * p0.x;
        xx.y += ap * p0.y;
        xx.z += ap * p1.x;
        xx.w += ap * p1.y;
        rr.x -= aa * a0.x;
        rr.y -= aa * a0.y;
        rr.z -= aa * a1.x;
        rr.w -= aa * a1.y;
        x[i] = xx;
        r[i] = rr;
        acc += sq(rr);
      }
    }
  }
  double v[1] = {(double)acc};
  double t[1];
  if (grid_sum<1>(v, rb, t)) {
    s->rr_new = t[0];
    s->beta = t[0] / s->rr;
    s->rr = t[0];
    s->iter += 1;
    if (t[0] < s->stop_rr || !(t[0] == t[0])) s->done_next = 1;
  }
}

// FP16 p = r + beta p (new per-site scale); the last block then raises `done` if asked
__global__ void k_cg_p_h(uint4* __restrict__ p, const float4* __restrict__ r, int Vh, ReduceBuf rb, CGScalars* s) {
  if (s->done) return;
  const float be = (float)s->beta;
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
    Spinor<float> pp, rr;
    load_spinor(pp, p, cb, Vh);
    load_spinor(rr, r, cb, Vh);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) pp.s[a][c] = rr.s[a][c] + be * pp.s[a][c];
    store_spinor(p, pp, cb, Vh);
  }
  double v[1] = {0.0}, t[1];
  if (grid_sum<1>(v, rb, t)) s->done = s->done_next;
}

// ---------------------------------------------------------------- host
static long words(const pfmp_ctx* c, int prec) { return prec == PFMP_F64 ? 12L * c->g.Vh : 6L * c->g.Vh; }

void blas_zero(pfmp_ctx* c, int prec, void* x) {
  PFMP_CUDA(cudaMemsetAsync(x, 0, spinor_bytes(c->g, prec), c->stream));
}

void blas_copy(pfmp_ctx* c, void* dst, int dprec, const void* src, int sprec) {
  const int Vh = c->g.Vh;
  if (dprec == sprec) {
    PFMP_CUDA(cudaMemcpyAsync(dst, src, spinor_bytes(c->g, dprec), cudaMemcpyDeviceToDevice, c->stream));
    return;
  }
  if (dprec == PFMP_H16) {
    PFMP_REQUIRE(sprec == PFMP_F32, PFMP_E_UNSUPPORTED, "FP16 fields are converted from FP32");
    k_f32_to_h16<<<blas_grid(Vh), kBlock, 0, c->stream>>>((const float4*)src, (uint4*)dst, Vh);
  } else if (sprec == PFMP_H16) {
    PFMP_REQUIRE(dprec == PFMP_F32, PFMP_E_UNSUPPORTED, "FP16 fields are converted to FP32");
    k_h16_to_f32<<<blas_grid(Vh), kBlock, 0, c->stream>>>((const uint4*)src, (float4*)dst, Vh);
  } else if (dprec == PFMP_F32) {
    k_f64_to_f32<<<blas_grid(6L * Vh), kBlock, 0, c->stream>>>((const double2*)src, (float4*)dst, Vh);
  } else {
    k_f32_to_f64<<<blas_grid(6L * Vh), kBlock, 0, c->stream>>>((const float4*)src, (double2*)dst, Vh, 0);
  }
  PFMP_CHECK_LAUNCH();
}

void blas_add_lo(pfmp_ctx* c, void* x64, const void* x32) {
  const int Vh = c->g.Vh;
  k_f32_to_f64<<<blas_grid(6L * Vh), kBlock, 0, c->stream>>>((const float4*)x32, (double2*)x64, Vh, 1);
  PFMP_CHECK_LAUNCH();
}

void blas_axpy(pfmp_ctx* c, int prec, double are, double aim, const void* x, void* y) {
  const long n = words(c, prec);
  if (prec == PFMP_F64)
    k_axpy64<<<blas_grid(n), kBlock, 0, c->stream>>>(are, aim, (const double2*)x, (double2*)y, n);
  else
    k_axpy32<<<blas_grid(n), kBlock, 0, c->stream>>>((float)are, (float)aim, (const float4*)x, (float4*)y, n);
  PFMP_CHECK_LAUNCH();
}

void blas_norm2(pfmp_ctx* c, int prec, const void* x, double* out_dev) {
  const long n = words(c, prec);
  if (prec == PFMP_F64)
    k_norm2<double2><<<blas_grid(n), kBlock, 0, c->stream>>>((const double2*)x, n, c->rb, out_dev);
  else
    k_norm2<float4><<<blas_grid(n), kBlock, 0, c->stream>>>((const float4*)x, n, c->rb, out_dev);
  PFMP_CHECK_LAUNCH();
}

void blas_cdot(pfmp_ctx* c, int prec, const void* x, const void* y, double* out_dev) {
  const long n = words(c, prec);
  if (prec == PFMP_F64)
    k_cdot64<<<blas_grid(n), kBlock, 0, c->stream>>>((const double2*)x, (const double2*)y, n, c->rb, out_dev);
  else
    k_cdot32<<<blas_grid(n), kBlock, 0, c->stream>>>((const float4*)x, (const float4*)y, n, c->rb, out_dev);
  PFMP_CHECK_LAUNCH();
}

void blas_xmy_norm(pfmp_ctx* c, const void* b, const void* Ax, void* r, double* out_dev) {
  const long n = words(c, PFMP_F64);
  k_xmy_norm<<<blas_grid(n), kBlock, 0, c->stream>>>((const double2*)b, (const double2*)Ax, (double2*)r, n, c->rb,
                                                     out_dev);
  PFMP_CHECK_LAUNCH();
}

// prec = PFMP_H16: x and r FP32, p and Ap FP16
void cg_step_xr(pfmp_ctx* c, int prec, void* x, void* r, const void* p, const void* Ap, CGScalars* s) {
  if (prec == PFMP_H16) {
    k_cg_xr_h<<<blas_grid(c->g.Vh), kBlock, 0, c->stream>>>((float4*)x, (float4*)r, (const uint4*)p,
                                                           (const uint4*)Ap, c->g.Vh, c->rb, s);
    PFMP_CHECK_LAUNCH();
    return;
  }
  const long n = words(c, prec);
  if (prec == PFMP_F64)
    k_cg_xr64<<<blas_grid(n), kBlock, 0, c->stream>>>((double2*)x, (double2*)r, (const double2*)p,
                                                      (const double2*)Ap, n, c->rb, s);
  else
    k_cg_xr32<<<blas_grid(n), kBlock, 0, c->stream>>>((float4*)x, (float4*)r, (const float4*)p, (const float4*)Ap,
                                                      n, c->rb, s);
  PFMP_CHECK_LAUNCH();
}

// prec = PFMP_H16: p FP16, r FP32
void cg_step_p(pfmp_ctx* c, int prec, void* p, const void* r, CGScalars* s) {
  if (prec == PFMP_H16) {
    k_cg_p_h<<<blas_grid(c->g.Vh), kBlock, 0, c->stream>>>((uint4*)p, (const float4*)r, c->g.Vh, c->rb, s);
    PFMP_CHECK_LAUNCH();
    return;
  }
  const long n = words(c, prec);
  if (prec == PFMP_F64)
    k_cg_p64<<<blas_grid(n), kBlock, 0, c->stream>>>((double2*)p, (const double2*)r, n, c->rb, s);
  else
    k_cg_p32<<<blas_grid(n), kBlock, 0, c->stream>>>((float4*)p, (const float4*)r, n, c->rb, s);
  PFMP_CHECK_LAUNCH();
}

}  // namespace pfmp
