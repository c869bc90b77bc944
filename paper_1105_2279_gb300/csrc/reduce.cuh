// Deterministic FP64 block reduction: warp shuffles, then one warp over the
// per-warp sums, then a single-block pass over the per-block partials in a
// fixed order.  The grid of every reducing kernel depends only on the problem
// size, so results are bit-identical run to run.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

namespace lq {

constexpr int kReduceThreads = 256;

template <int NV> __device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
}

// Sums v over the block; thread 0 writes the NV totals to out[0..NV).
template <int NV> __device__ __forceinline__ void block_sum_store(double (&v)[NV], double* out) {
  __shared__ double sm[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum<NV>(v);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[warp][i] = v[i];
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = lane < nw ? sm[lane][i] : 0.0;
    warp_sum<NV>(v);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < NV; ++i) out[i] = v[i];
  }
}

// Second pass: one block sums nparts partial NV-vectors in a fixed order.
template <int NV> __global__ void k_reduce_partials(const double* __restrict__ parts, int nparts, double* out) {
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += parts[(long long)p * NV + i];
  block_sum_store<NV>(v, out);
}

#ifndef __CUDACC_RTC__
// Grid size of a reducing kernel over n items: a function of n only (the cap
// is 8 blocks of 256 threads on each of the 152 SMs of a GB300).
constexpr int kReduceMaxBlocks = 1216;
inline int reduce_grid(long long n) {
  long long b = (n + kReduceThreads - 1) / kReduceThreads;
  if (b > kReduceMaxBlocks) b = kReduceMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}
#endif

}  // namespace lq
