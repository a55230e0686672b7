// The true residual r = b - K x of the mixed solvers with K applied in double-float on
// the FP32 pipe (dfloat.cuh): x is split once into FP32 pairs, K runs through the same
// stencil templates as the FP32 and FP64 paths, and only the final b - (hi + lo) and
// |r|^2 use FP64.  About 48 significant bits: the residual is accurate to ~1e-13
// relative to |K| |x|, far below the 1e-10 stopping tolerance.
#include "context.h"
#include "dfloat.cuh"

namespace pfmp {

__global__ void k_split_df(const double2* __restrict__ x, float4* __restrict__ y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] = split2(x[i]);
}

__global__ void k_residual_df(const double2* __restrict__ b, const float4* __restrict__ kx, double2* __restrict__ r,
                              long n, ReduceBuf rb, double* out) {
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 bb = b[i];
    const float4 k = kx[i];
    const double2 d = make_double2(bb.x - ((double)k.x + (double)k.y), bb.y - ((double)k.z + (double)k.w));
    r[i] = d;
    v[0] += d.x * d.x + d.y * d.y;
  }
  double t[1];
  if (grid_sum<1>(v, rb, t)) *out = t[0];
}

static int rgrid(long n) {
  long b = (n + kBlock - 1) / kBlock;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

double true_residual_df(pfmp_op* op, const void* x64, const void* b64, void* r64) {
  pfmp_ctx* c = op->ctx;
  const long n = 12L * c->g.Vh;
  k_split_df<<<rgrid(n), kBlock, 0, c->stream>>>((const double2*)x64, op->xdf, n);
  PFMP_CHECK_LAUNCH();
  kop_df(op, op->kdf, op->xdf);
  k_residual_df<<<rgrid(n), kBlock, 0, c->stream>>>((const double2*)b64, op->kdf, (double2*)r64, n, c->rb, c->d_sums);
  PFMP_CHECK_LAUNCH();
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_sums[0];
}

}  // namespace pfmp
