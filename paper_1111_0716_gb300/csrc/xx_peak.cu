// xx_peak.cu -- measured CUDA-core FMA rates of the device, the denominators of
// the ALU rooflines the benchmark reports for the FP32 passes and the all-FP64
// path.  Not part of the exchange method: a measurement helper.
#include <cuda_runtime.h>

#include "../../include/xx.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;        // independent FMA chains per thread (hides the FMA latency)
constexpr int kIters = 4096;      // FMAs per chain

// keeps the chains live: written only if a result equals the (unreachable) sentinel
__device__ double xx_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T b, T c, T sentinel) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == sentinel) xx_peak_sink = (double)s;
}

template <typename T>
int measure(cudaStream_t s, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return XX_ERR_NO_DEVICE;
  }
  const int blocks = sms * 8;
  // b slightly below 1 keeps the values finite over the chain
  const T b = (T)0.999999, c = (T)1e-3, sentinel = (T)-12345.678;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return XX_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return XX_ERR_CUDA;
  }
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(b, c, sentinel);   // warm-up
  const int reps = 5;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, kThreads, 0, s>>>(b, c, sentinel);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) {
    cudaGetLastError();
    return XX_ERR_CUDA;
  }
  const double flops = 2.0 * (double)reps * blocks * kThreads * kChains * (double)kIters;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return XX_OK;
}

}  // namespace

extern "C" int xx_measure_fma_rate(int precision, double* tflops_out, void* stream) {
  if (!tflops_out || (precision != XX_FP32_MIXED && precision != XX_FP64)) return XX_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == XX_FP64 ? measure<double>(s, tflops_out) : measure<float>(s, tflops_out);
}
