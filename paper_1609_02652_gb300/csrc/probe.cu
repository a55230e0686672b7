// Measured FMA throughput of this GPU in FP64 and FP32: the ALU roofline of the FP64
// stencil (and so of the FP64 CG baseline) and of the double-float stencil, which run
// on those pipes.  Every thread runs 8 independent FMA chains for `iters` rounds on
// register operands (no memory traffic in the loop); the grid is 8 blocks of 256
// threads per SM; the time is taken with CUDA events around the launch on the context's
// stream after one warm-up launch.
#include "context.h"

namespace pfmp {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T* out, int iters, T seed) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + (T)(threadIdx.x + k);
  const T b = (T)0.999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // never true; keeps the chains live
}

double fma_rate(pfmp_ctx* c, int prec) {
  int dev = 0, sms = 0;
  PFMP_CUDA(cudaGetDevice(&dev));
  PFMP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  double* out = (double*)dev_alloc((size_t)blocks * sizeof(double));
  cudaEvent_t e0, e1;
  PFMP_CUDA(cudaEventCreate(&e0));
  PFMP_CUDA(cudaEventCreate(&e1));
  float ms = 0;
  for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
    PFMP_CUDA(cudaEventRecord(e0, c->stream));
    if (prec == PFMP_F64)
      k_fma_rate<double><<<blocks, threads, 0, c->stream>>>(out, iters, 1.0);
    else
      k_fma_rate<float><<<blocks, threads, 0, c->stream>>>((float*)out, iters, 1.0f);
    PFMP_CHECK_LAUNCH();
    PFMP_CUDA(cudaEventRecord(e1, c->stream));
    PFMP_CUDA(cudaEventSynchronize(e1));
    PFMP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(out);
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace pfmp
