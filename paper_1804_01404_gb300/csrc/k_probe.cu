// FMA throughput probes.  The FP64 path of the method is bound by the FP64 pipes, which run at a
// small fraction of the FP32 rate on this GPU, so its roofline needs a measured FP64 peak; the FP32
// cell kernels are bound on chip by FP32 arithmetic, issue and shared memory, and their roofline is
// reported against the measured FP32 FMA rate.  Every thread runs eight independent FMA chains
// (enough to cover the pipe latency) for a fixed count.
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

__global__ void __launch_bounds__(256) k_sfma(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;
}

// packed form: one instruction does the FMAs of both halves of a float2 (the cell kernels' complex
// arithmetic uses it)
__global__ void __launch_bounds__(256) k_sfma2(float* out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
  const float2 av = make_float2(a, a), bv = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], av, bv);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 12345.678f) out[0] = s;
}

// Time one launch of `kern` (blocks x 256 threads, iters iterations) after a short warm-up; ms <= 0 on
// failure.
template <typename K, typename V>
float time_probe(K kern, V* out, int blocks, int iters, V a, V b) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.f; }
  kern<<<blocks, 256>>>(out, 64, a, b);
  cudaEventRecord(e0);
  kern<<<blocks, 256>>>(out, iters, a, b);
  cudaEventRecord(e1);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (err == cudaSuccess && cudaGetLastError() == cudaSuccess) ? ms : -1.f;
}

}  // namespace

extern "C" tdks_status tdks_probe_fp32(double* tflops) {
  if (!tflops) return TDKS_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TDKS_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TDKS_ECUDA;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return TDKS_ENOMEM;
  const int blocks = nsm * 8, iters = 16384;
  const float ms1 = time_probe(k_sfma, out, blocks, iters, 0.999999f, 1e-7f);
  const float ms2 = time_probe(k_sfma2, out, blocks, iters, 0.999999f, 1e-7f);
  cudaFree(out);
  if (ms1 <= 0.f || ms2 <= 0.f) return TDKS_ECUDA;
  const double fl = 2.0 * kChains * (double)iters * blocks * 256;   // scalar kernel; the packed one does 2x
  const double r1 = fl / (ms1 * 1e-3) / 1e12, r2 = 2.0 * fl / (ms2 * 1e-3) / 1e12;
  *tflops = r1 > r2 ? r1 : r2;
  return TDKS_OK;
}

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
