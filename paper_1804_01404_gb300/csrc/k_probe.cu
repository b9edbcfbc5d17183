// FP64 throughput probe: the FP64 path of the method is bound by the FP64 pipes, which run at a
// small fraction of the FP32 rate on this GPU, so its roofline needs a measured FP64 peak.  Every
// thread runs eight independent FMA chains (enough to cover the pipe latency) for a fixed count.
#include <cuda_runtime.h>

#include "../../include/tdks.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;                  // keeps the chains live; practically never taken
}

}  // namespace

extern "C" tdks_status tdks_probe_fp64(double* tflops) {
  if (!tflops) return TDKS_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TDKS_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TDKS_ECUDA;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return TDKS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = nsm * 8, threads = 256, iters = 4096;
  k_dfma<<<blocks, threads>>>(out, 64, 0.999999, 1e-7);           // warm-up
  cudaEventRecord(e0);
  k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e1);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return TDKS_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return TDKS_OK;
}
