// sv_peak.cu -- measured FP64 throughput of the device, the denominator of the
// FP64 step kernels' roofline (those kernels are bound by the FP64 pipe, not
// by HBM, on a GPU whose double-precision rate is a small fraction of its
// float rate).  Not part of the paper's method.
//
// Every thread advances eight independent FMA chains x <- x a + b (a just
// below 1, so the values stay finite and normal); with four 256-thread blocks
// per SM that is 64 independent DFMAs in flight per SM scheduler, far more
// than the FP64 pipe's latency needs.  The count of FMAs is exact, the time
// comes from CUDA events on the caller's stream, and the best of three
// launches is reported.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sv.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 4096;

__device__ double g_sink;

__global__ void __launch_bounds__(kThreads) dfma_chains_kernel(double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * c + 1e-9 * threadIdx.x;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot drop: it depends on every chain (the chains
  // converge to b / (1 - a) = 1, so it never happens)
  if (s == -1.0) g_sink = s;
}

}  // namespace

extern "C" int sv_measure_fp64_peak(void* cuda_stream, double* tflops) {
  if (!tflops) return SV_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return SV_ECUDA;
  const int grid = 4 * sms;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SV_ECUDA;
  }
  int rc = SV_OK;
  float best = 0.0f;
  for (int rep = 0; rep < 4 && rc == SV_OK; ++rep) {   // one warm-up, three timed
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = SV_ECUDA; break; }
    dfma_chains_kernel<<<grid, kThreads, 0, st>>>(0.9999999, 1e-7);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess) {
      rc = SV_ECUDA;
      break;
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = SV_ECUDA; break; }
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SV_OK) return rc;
  if (!(best > 0.0f)) return SV_ECUDA;
  const double flops = 2.0 * kChains * (double)kIters * kThreads * (double)grid;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SV_OK;
}
