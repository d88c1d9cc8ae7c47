// Measured arithmetic peaks of the GPU the library runs on: dense FP32 and FP64
// fused multiply-add throughput of the CUDA cores.  These are the denominators
// of the ALU rooflines (the FP64 patch factorisation, the FP64 smoother, the
// FP32 operator apply), measured rather than taken from a data sheet.
//
// Each thread runs NCH independent FMA chains (enough to cover the pipeline
// latency) for `iters` steps on values that depend on runtime arguments, and
// stores one value only if it matches an impossible sentinel, so nothing can be
// folded away.  The grid fills every SM at full occupancy.
#include <cuda_runtime.h>

#include "../../include/alstokes.h"

namespace {

constexpr int NCH = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T a, T b, T* sink) {
  T v[NCH];
#pragma unroll
  for (int k = 0; k < NCH; ++k) v[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) v[k] = v[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < NCH; ++k) s += v[k];
  if (s == (T)-12345.678) sink[threadIdx.x] = s;   // never true for the arguments used
}

template <typename T>
double measure(int iters, cudaStream_t s, T* sink) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned blocks = (unsigned)sms * 8;
  // a slightly below 1 keeps the chains bounded: v -> b / (1 - a)
  const T a = (T)0.999, b = (T)0.001;
  k_fma_peak<T><<<blocks, 256, 0, s>>>(iters / 8, a, b, sink);   // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  k_fma_peak<T><<<blocks, 256, 0, s>>>(iters, a, b, sink);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * NCH * (double)iters * blocks * 256.0;
  return ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
}

}  // namespace

extern "C" als_status als_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, void* stream) {
  if (!fp32_tflops || !fp64_tflops) return ALS_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  double* sink = nullptr;
  if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return ALS_ENOMEM;
  *fp32_tflops = measure<float>(1 << 16, s, reinterpret_cast<float*>(sink));
  *fp64_tflops = measure<double>(1 << 12, s, sink);
  const cudaError_t e = cudaGetLastError();
  cudaFree(sink);
  return e == cudaSuccess ? ALS_OK : ALS_ECUDA;
}
