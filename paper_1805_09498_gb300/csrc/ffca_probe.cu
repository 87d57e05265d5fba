// Measured FP64 FMA rate of the current device: the denominator of the FP64
// ALU roofline of the plain FP64 path (whose per-point work is bound by this
// part's FP64 throughput, not by HBM).  Not part of the method.
#include <cuda_runtime.h>

#include "ffca.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (hide the FP64 latency)
constexpr int kProbeIters = 4096;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

// Written only under a condition that never holds (the sums are positive),
// so that the compiler keeps the chains.
__device__ double g_probe_sink;

// Every thread runs kChains independent chains x <- x a + b for `iters`
// steps (x starts at 1 or above, a slightly below 1 and b > 0: the values
// stay positive and finite).
__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) g_probe_sink = s;
}

}  // namespace

extern "C" ffca_status ffca_peak_fp64(void* stream_, double* gflops) {
  if (!gflops) return FFCA_ERR_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FFCA_ERR_CUDA;
  const int grid = nsm * kProbeBlocksPerSm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FFCA_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FFCA_ERR_CUDA;
  }
  ffca_status st = FFCA_OK;
  float best = 0.f;
  for (int rep = 0; rep < 4 && st == FFCA_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, stream);
    k_fp64_fma<<<grid, kProbeThreads, 0, stream>>>(kProbeIters, 0.999999999, 1e-9);
    cudaEventRecord(e1, stream);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      st = FFCA_ERR_CUDA;
    else if (rep > 0 && (best == 0.f || ms < best))
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FFCA_OK) return st;
  const double fmas = (double)grid * kProbeThreads * kProbeIters * kChains;
  *gflops = 2.0 * fmas / (best * 1e-3) / 1e9;
  return FFCA_OK;
}
