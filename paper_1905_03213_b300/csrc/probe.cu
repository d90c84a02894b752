// FP32 FMA throughput probe: the denominator of the gridding roofline, measured.
//
// Gridding spends 8 flop (one complex multiply-add, four FMAs) per kernel tap, so its
// roofline's compute bound is the device's FP32 FMA rate. This kernel measures that rate
// directly: every thread runs kChains independent FMA chains (enough to cover the FMA
// pipeline's latency), either as scalar fma.rn.f32 or as packed fma.rn.f32x2 (two FMAs per
// instruction, the form the gridding kernels use), for a fixed number of iterations, on
// every SM at full occupancy. The result is written out so that nothing is optimised away.
#include <cuda_runtime.h>

#include "internal.h"

namespace wp {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 512;

__device__ __forceinline__ unsigned long long fma2p(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ float fma1p(float a, float b, float c) {
  float d;
  asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// packed: kChains chains of f32x2 FMAs; scalar: 2 kChains chains of f32 FMAs (same flops per
// iteration). a and b are close to 1 so the values stay finite for any iteration count.
template <bool kPacked>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int64_t iters, float seed, float* out) {
  const float a = 1.0f + 1e-7f * (float)(threadIdx.x & 7), b = 0.999999f;
  float r = 0.f;
  if constexpr (kPacked) {
    unsigned long long acc[kChains];
    const unsigned long long A = (unsigned long long)__float_as_uint(a) | ((unsigned long long)__float_as_uint(a) << 32);
    const unsigned long long B = (unsigned long long)__float_as_uint(b) | ((unsigned long long)__float_as_uint(b) << 32);
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      const float v = seed + (float)k;
      acc[k] = (unsigned long long)__float_as_uint(v) | ((unsigned long long)__float_as_uint(v + 0.5f) << 32);
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) acc[k] = fma2p(acc[k], A, B);
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) r += __uint_as_float((uint32_t)acc[k]) + __uint_as_float((uint32_t)(acc[k] >> 32));
  } else {
    float acc[2 * kChains];
#pragma unroll
    for (int k = 0; k < 2 * kChains; ++k) acc[k] = seed + 0.5f * (float)k;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < 2 * kChains; ++k) acc[k] = fma1p(acc[k], a, b);
    }
#pragma unroll
    for (int k = 0; k < 2 * kChains; ++k) r += acc[k];
  }
  if (r == 12345.678f) out[0] = r;        // practically never: keeps the chains alive
  if (threadIdx.x == 0 && blockIdx.x == 0 && iters < 0) out[1] = r;
}

}  // namespace
}  // namespace wp

extern "C" int wp_probe_fp32_fma(int32_t device, int32_t packed, int64_t iters, int32_t reps, double* tflops_out,
                                 double* ms_out) {
  if (iters < 1 || reps < 1 || !tflops_out) return WP_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return WP_EINVAL;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return WP_ECUDA;
  const int blocks = prop.multiProcessorCount * (prop.maxThreadsPerMultiProcessor / wp::kProbeThreads);
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = WP_OK;
  if (cudaMalloc(&out, 2 * sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = WP_ECUDA;
  }
  float ms = 0.f;
  if (rc == WP_OK) {
    auto launch = [&]() {
      if (packed) wp::k_fma_probe<true><<<blocks, wp::kProbeThreads>>>(iters, 1.0f, out);
      else wp::k_fma_probe<false><<<blocks, wp::kProbeThreads>>>(iters, 1.0f, out);
    };
    launch();                                   // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      rc = WP_ECUDA;
  }
  if (rc == WP_OK) {
    // flop per launch: threads x iterations x 2 kChains FMAs x 2 flop
    const double flop = (double)blocks * wp::kProbeThreads * (double)iters * 2.0 * wp::kChains * 2.0 * reps;
    *tflops_out = flop / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms / reps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return rc;
}
