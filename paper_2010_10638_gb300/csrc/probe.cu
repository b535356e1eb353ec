// Instrumentation: the FP32 FMA rate of this GPU, measured (no counterpart in the paper).
// The roofline of the FP32 TTMc is reported against it instead of a figure derived from
// unit counts and the nominal clock.  Every thread runs eight independent FMA chains, so
// the pipe, not the FMA latency, bounds the loop; the chains' sums are stored only when
// a runtime flag says so, which keeps the work live without memory traffic.
#include <algorithm>

#include "internal.cuh"

namespace tk {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, float seed, int store, float *out) {
  float v[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) v[c] = seed + (float)(threadIdx.x + c);
  const float a = 0.999999f, b = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += v[c];
  if (store) out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace tk

extern "C" double tucker_fp32_fma_tflops(int iters, void *stream) {
  if (iters < 1) return -1.0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tk::fma_probe_kernel, tk::kProbeThreads, 0) !=
      cudaSuccess)
    return -1.0;
  const int blocks = sms * std::max(per_sm, 1);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.0;
  }
  double best = -1.0;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms the clocks; the best of the rest counts
    cudaEventRecord(e0, s);
    tk::fma_probe_kernel<<<blocks, tk::kProbeThreads, 0, s>>>(iters, 1.0f, 0, nullptr);
    ::tk::count_launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) break;
    const double flops = 2.0 * blocks * tk::kProbeThreads * (double)iters * 16.0 * tk::kProbeChains;
    if (rep > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? best : -1.0;
}
