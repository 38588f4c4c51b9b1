// Measured float32 FMA rate of the current device: the denominator of the arithmetic side
// of the sweeps' roofline (8 W^2 flops per visibility for gridding plus degridding). Not
// part of the method; a measurement helper for benchmarks.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "lmg.h"
#include "lmg_internal.h"

namespace lmg {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hide the FMA latency)
constexpr int kIters = 2048;    // loop trips; kChains FMAs each
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fma_rate(float seed, float* sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 0.001f * float(threadIdx.x + c);
  const float m = 0.99993f, q = 1.0e-4f;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, q);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true for these values; keeps the chains live
}

}  // namespace
}  // namespace lmg

extern "C" int lmg_fp32_fma_rate(double* flops_per_s, void* stream) {
  using namespace lmg;
  if (!flops_per_s) return set_error(LMG_EINVAL, "flops_per_s is NULL");
  *flops_per_s = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate, kPeakThreads, 0);
  if (e != cudaSuccess) return cuda_error(e, "lmg_fp32_fma_rate setup");
  // every SM fully occupied, several waves so that the tail is a small part of the time
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 8;
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_error(e, "lmg_fp32_fma_rate events");
  }
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a, st);
    k_fma_rate<<<blocks, kPeakThreads, 0, st>>>(1.0f, nullptr);
    cudaEventRecord(b, st);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) break;
    const double flops = 2.0 * double(blocks) * kPeakThreads * kChains * double(kIters);
    if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (double(ms) * 1e-3));  // rep 0 warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_error(e, "lmg_fp32_fma_rate");
  *flops_per_s = best;
  return LMG_OK;
}
