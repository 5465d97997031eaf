// FP32-pipe throughput probe: the roofline denominator for the FP32 filter.
//
// Every thread runs 8 independent FMA chains (scalar FFMA) or 8 independent
// packed two-lane chains (fma.rn.f32x2, 2 FMAs per instruction); the grid
// fills every SM.  Throughput = 2 flops x FMAs / event-timed duration.
#include <cuda_runtime.h>

#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) ffma_probe(float *out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live, never taken
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long x, unsigned long long a,
                                                   unsigned long long b) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x), "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

__global__ void __launch_bounds__(256) ffma2_probe(float *out, int iters, float a, float b) {
  unsigned long long x[kChains];
  const unsigned long long a2 = pack2(a, a), b2 = pack2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = pack2(1e-3f * (float)(threadIdx.x + c), 2e-3f * (float)c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma2(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    s += __uint_as_float((unsigned)x[c]) + __uint_as_float((unsigned)(x[c] >> 32));
  if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace fbf

// Measures the FP32 FMA throughput of `device` in TFLOP/s (2 flops per FMA):
// packed == 0 uses scalar FFMA, packed != 0 the two-lane fma.rn.f32x2.
// Allocates and frees a small result buffer and synchronises the device.
extern "C" fbf_status fbf_measure_fp32_peak(int device, int packed, double *tflops) {
  using namespace fbf;
  if (!tflops) return FBF_ERR_INVALID_ARGUMENT;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return FBF_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return FBF_ERR_INVALID_ARGUMENT;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  float *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fbf_status st = FBF_OK;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) st = FBF_ERR_CUDA;
  if (st == FBF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = FBF_ERR_CUDA;
  if (st == FBF_OK) {
    for (int rep = 0; rep < 2; ++rep) {  // first launch warms up clocks and caches
      cudaEventRecord(e0, 0);
      if (packed)
        ffma2_probe<<<blocks, threads>>>(out, iters, 0.9999999f, 1e-7f);
      else
        ffma_probe<<<blocks, threads>>>(out, iters, 0.9999999f, 1e-7f);
      cudaEventRecord(e1, 0);
    }
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      st = FBF_ERR_CUDA;
  }
  if (st == FBF_OK) {
    const double fmas = (double)blocks * threads * iters * kUnroll * kChains * (packed ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaSetDevice(prev);
  return st;
}
