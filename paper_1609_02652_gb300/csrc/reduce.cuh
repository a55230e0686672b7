// Deterministic one-launch global sums in FP64: warp shuffles, then shared memory, one
// partial per block, and the last block to finish (atomic ticket) adds the partials in
// a fixed order.  The result therefore does not depend on block scheduling.
#pragma once
#include "pfmp_internal.cuh"

namespace pfmp {

struct ReduceBuf {
  double* partials;   // [max_blocks * kMaxSums]
  unsigned* counter;  // one ticket counter, left at 0 after each use
};
constexpr int kMaxSums = 4;
constexpr int kMaxReduceBlocks = 65536;

template <int N>
__device__ __forceinline__ void block_sum(double v[N], double* sh /* [N][32] */) {
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sh[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double w = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
      v[k] = w;
    }
  }
  __syncthreads();
}

// Adds v[0..N) over the whole grid.  Returns true in exactly one thread (thread 0 of the
// last block), whose out[0..N) then holds the grid totals.  Every thread of every block
// must call this (no early return before it).
template <int N>
__device__ __forceinline__ bool grid_sum(double v[N], ReduceBuf rb, double out[N]) {
  __shared__ double sh[N * 32];
  __shared__ bool last;
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_sum<N>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) rb.partials[(size_t)bid * N + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(rb.counter, 1u);
    last = (t == nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double w[N];
#pragma unroll
  for (int k = 0; k < N; ++k) w[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] += ((volatile double*)rb.partials)[(size_t)b * N + k];
  block_sum<N>(w, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = w[k];
    *rb.counter = 0u;
    return true;
  }
  return false;
}

}  // namespace pfmp

namespace pfmp {

// The same deterministic sum over a group of blocks that belong together (e.g. one
// system of a batch): block `idx` of `nblk` writes its partials to partials[idx*N..],
// takes a ticket from *ticket, and the last one adds the partials in index order.
template <int N>
__device__ __forceinline__ bool group_sum(double v[N], double* partials, unsigned* ticket, unsigned nblk, unsigned idx,
                                          double out[N]) {
  __shared__ double sh[N * 32];
  __shared__ bool last;
  block_sum<N>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) partials[(size_t)idx * N + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double w[N];
#pragma unroll
  for (int k = 0; k < N; ++k) w[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] += ((volatile double*)partials)[(size_t)b * N + k];
  block_sum<N>(w, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = w[k];
    *ticket = 0u;
    return true;
  }
  return false;
}

}  // namespace pfmp
