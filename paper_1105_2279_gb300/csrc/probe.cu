// Measured CUDA-core FMA throughput (the denominators of the FP64- and
// FP32-pipe rooflines): every thread of a full-occupancy grid runs eight
// independent FMA chains, so the pipe, not the chain latency, sets the time.
#include "lq_internal.h"

namespace lq {

constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T b, T c, int iters, T* sink) {
  T a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == (T)-1.2345) *sink = s;   // never true for these inputs; keeps the chains live
}

template <typename T>
static lq_status probe(int iters, double* tflops, cudaStream_t s) {
  void* sink = nullptr;
  lq_status st = scratch_alloc(&sink, sizeof(T), s, "lq_peak_probe");
  if (st != LQ_OK) return st;
  const int blocks = device_sm_count() * 8;   // 8 x 256 threads: 64 warps per SM
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // b slightly below 1 and c = 0 keep every chain finite and normal
  k_fma_probe<T><<<blocks, 256, 0, s>>>((T)0.999999, (T)0, iters, (T*)sink);   // warm-up (clocks)
  cudaEventRecord(e0, s);
  k_fma_probe<T><<<blocks, 256, 0, s>>>((T)0.999999, (T)0, iters, (T*)sink);
  cudaEventRecord(e1, s);
  st = launch_check("k_fma_probe");
  if (st == LQ_OK) st = cuda_check(cudaEventSynchronize(e1), "lq_peak_probe timing");
  float ms = 0.0f;
  if (st == LQ_OK) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  scratch_free(sink, s);
  if (st == LQ_OK) *tflops = 2.0 * kProbeChains * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
  return st;
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_peak_probe(int prec, double* tflops, void* stream) {
  clear_error();
  if (!tflops || (prec != LQ_F32 && prec != LQ_F64)) {
    set_error("lq_peak_probe: need prec LQ_F32 or LQ_F64 and an output pointer");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  // about 50 ms per timed launch at the expected rates (1.2 / 75 TFLOP/s)
  if (prec == LQ_F64) return probe<double>(4096, tflops, s);
  return probe<float>(262144, tflops, s);
}
