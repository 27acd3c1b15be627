// Arithmetic throughput of the device's SMs for the roofline of the recursive step: a
// loop of independent multiply-add chains held in registers, on every SM, in the three
// forms the kernels of this library issue (FP64 fma, FP32 fma, paired FP32 fma.rn.f32x2).
// The paper has no counterpart; this is a measurement helper (bfly_measure_peak).
#include <algorithm>
#include <string>
#include <vector>

#include "plan_state.hpp"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;  // 32 warps per SM: 8 per sub-partition
constexpr int kChains = 8;           // independent accumulators per thread

// Written only when a result equals a value the loop cannot produce, so that the
// compiler keeps the loop and nothing is stored in practice.
static __device__ double g_peak_sink[1];

// kind 0: FP64 fma; 1: FP32 fma; 2: paired FP32 fma (fma.rn.f32x2).  Every iteration does
// kChains multiply-adds (paired: 2 kChains) per thread, a = a * m + c with m = 1/2, so the
// accumulators stay at normal magnitudes.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(int iters, float seed) {
  const float c = seed * (1.0f + threadIdx.x * 1e-7f);
  if constexpr (KIND == 0) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = c + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], 0.5, (double)c);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0) g_peak_sink[0] = s;
  } else if constexpr (KIND == 1) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = c + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], 0.5f, c);
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0f) g_peak_sink[0] = s;
  } else {
    float2 a[kChains];
    const float2 m = make_float2(0.5f, 0.5f), cc = make_float2(c, c);
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = make_float2(c + j, c - j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], m, cc);
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
    if (s == -1.0f) g_peak_sink[0] = s;
  }
}

#define PEAK_CUDA(call)                                                                          \
  do {                                                                                           \
    const cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                       \
      return bfly_state::set_error(BFLY_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaError_t launch_peak(int kind, int grid, int iters, cudaStream_t s) {
  if (kind == 0) peak_kernel<0><<<grid, kPeakThreads, 0, s>>>(iters, 0.75f);
  else if (kind == 1) peak_kernel<1><<<grid, kPeakThreads, 0, s>>>(iters, 0.75f);
  else peak_kernel<2><<<grid, kPeakThreads, 0, s>>>(iters, 0.75f);
  return cudaGetLastError();
}

}  // namespace

extern "C" bfly_status bfly_measure_peak(int kind, double *flops_per_s, double *ms) {
  bfly_state::set_error(BFLY_OK, "");
  if (kind < 0 || kind > 2 || !flops_per_s) return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "kind must be 0, 1 or 2 and flops_per_s non-NULL");
  int dev = 0, sms = 0;
  PEAK_CUDA(cudaGetDevice(&dev));
  PEAK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * kPeakBlocksPerSm;
  // about 20-40 ms per launch at the expected rates (FP64 is far slower than FP32 on this part)
  const int iters = kind == 0 ? 8192 : kind == 1 ? 262144 : 131072;
  const double fma_per_iter = kind == 2 ? 2.0 * kChains : (double)kChains;
  cudaStream_t s = nullptr;
  PEAK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // one warm-up launch, then the best of 3
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_peak(kind, grid, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.0f || t < best)) best = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return bfly_state::set_error(BFLY_ERR_CUDA, std::string("peak measurement: ") + cudaGetErrorString(e));
  if (!(best > 0.0f)) return bfly_state::set_error(BFLY_ERR_CUDA, "peak measurement: no time recorded");
  const double flops = 2.0 * fma_per_iter * iters * (double)grid * kPeakThreads;
  *flops_per_s = flops / (best * 1e-3);
  if (ms) *ms = best;
  return BFLY_OK;
}
