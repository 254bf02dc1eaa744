// Measured FP64 fused multiply-add rate of the current GPU: the denominator
// against which the FP64 stage kernels (bound by the FP64 pipe, not by HBM)
// are rated.  Plain DFMA chains, eight independent accumulators per thread,
// every SM filled; timed with CUDA events; the GPU's clocks and settings are
// only read, never changed.
#include <cuda_runtime.h>

#include "../../include/rad.h"

namespace {

constexpr int kChains = 8, kUnroll = 16, kThreads = 256, kCtasPerSm = 8;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(double *out, long long iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * c + 1e-9 * threadIdx.x;
  const double m = 0.9999999999, add = 1e-12;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, add);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" int rad_fp64_fma_rate(double seconds, double *tflops_out) {
  if (!tflops_out || !(seconds > 0.0 && seconds <= 30.0)) return RAD_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RAD_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RAD_ECUDA;
  const int grid = nsm * kCtasPerSm;
  double *out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * kThreads * sizeof(double)) != cudaSuccess) return RAD_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int st = RAD_OK;
  double best = 0.0;
  long long iters = 64;
  const double flops_per_iter = 2.0 * kChains * kUnroll * (double)grid * kThreads;
  // calibrate: grow the loop until one launch takes a tenth of the budget,
  // then time three launches of about a third of it each
  for (int pass = 0; pass < 24 && st == RAD_OK; ++pass) {
    cudaEventRecord(e0);
    k_dfma_rate<<<grid, kThreads>>>(out, iters, 1.0 + pass);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = RAD_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 100.0f * seconds) {
      const long long target = (long long)((double)iters * (1000.0 * seconds / 3.0) / ms) + 1;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_dfma_rate<<<grid, kThreads>>>(out, target, 2.0 + rep);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = RAD_ECUDA;
          break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        const double r = flops_per_iter * (double)target / (ms * 1e-3) * 1e-12;
        if (r > best) best = r;
      }
      break;
    }
    iters *= 2;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (st == RAD_OK && best <= 0.0) st = RAD_ECUDA;
  if (st == RAD_OK) *tflops_out = best;
  return st;
}
