// ig_peak.cu -- measured arithmetic peaks of the device, for the rooflines of the kernels that are
// bound by FP64 (or FP32) instructions rather than by HBM: a grid of one wave of resident CTAs on
// every SM, each thread running 8 independent fused multiply-add chains for a fixed number of
// steps, timed with CUDA events on the caller's stream. Each step of a chain is one FMA (2 flops).
#include <cuda_runtime.h>

#include "../../include/iskra_gb300.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakBlock) fma_chain_kernel(T* __restrict__ sink, int steps, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x & 15) * T(0.001) + T(i);
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T tot = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) tot += x[i];
  // the chains stay live: the sum is stored only if it takes an impossible value
  if (tot == T(-1.2345e30)) sink[blockIdx.x * blockDim.x + threadIdx.x] = tot;
}

template <typename T>
cudaError_t run(cudaStream_t st, int steps, double* flops_per_s, double* seconds) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kPeakBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMalloc(&sink, sizeof(T) * (size_t)grid * kPeakBlock)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    const T a = T(0.9999999), b = T(1e-7);
    fma_chain_kernel<T><<<grid, kPeakBlock, 0, st>>>(sink, steps / 8 > 0 ? steps / 8 : 1, a, b);  // warm-up
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<grid, kPeakBlock, 0, st>>>(sink, steps, a, b);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
      const double flops = 2.0 * kChains * (double)steps * (double)grid * kPeakBlock;
      if (seconds) *seconds = ms * 1e-3;
      if (flops_per_s) *flops_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return e;
}

}  // namespace

extern "C" ig_status ig_measure_fma_peak(int precision, int steps, void* cuda_stream, double* flops_per_s,
                                         double* seconds) {
  if (!flops_per_s || steps < 1) return IG_ERR_INVALID_ARG;
  if (precision != IG_PRECISION_FP64 && precision != IG_PRECISION_MIXED) return IG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const cudaError_t e = precision == IG_PRECISION_FP64 ? run<double>(st, steps, flops_per_s, seconds)
                                                       : run<float>(st, steps, flops_per_s, seconds);
  if (e == cudaErrorMemoryAllocation) return IG_ERR_OOM;
  return e == cudaSuccess ? IG_OK : IG_ERR_CUDA;
}
