// Sums over a whole grid of CTAs in one launch.
//
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, and a chain of dependent FP64
// additions waits on the narrow FP64 pipe at every link, so a reduction keeps its chains short:
// every CTA reduces its threads' values (warp shuffles, then one thread per value over the warps),
// writes them to partials[blockIdx.x], and the CTA that finishes last (an atomic ticket, after a
// memory fence) loads all CTAs' partials at once -- thread t takes CTAs t, t + blockDim.x, ... -- and
// reduces them the same way.  The grouping of the additions depends only on CTA and thread indices,
// so the total does not depend on the order in which CTAs ran.  The last CTA resets the ticket for
// the next launch.
#pragma once

#include <cuda_runtime.h>

namespace tdks {

// v: this thread's NV values.  partials: [gridDim.x][NV] doubles; ticket: one unsigned, zero before
// the first launch.  Returns true in every thread of the last CTA, where tot[NV] (shared) holds the
// totals after the call.
template <int NV>
__device__ __forceinline__ bool grid_sum(const double (&v)[NV], double* partials, unsigned* ticket,
                                         double* tot) {
  __shared__ double red[NV][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[j][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double x = 0;
    for (int w = 0; w < nw; ++w) x += red[threadIdx.x][w];
    partials[(size_t)blockIdx.x * NV + threadIdx.x] = x;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double x = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) x += __ldcg(&partials[(size_t)b * NV + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[j][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double x = 0;
    for (int w = 0; w < nw; ++w) x += red[threadIdx.x][w];
    tot[threadIdx.x] = x;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();
  return true;
}

// CTAs for a grid_sum over n items with `threads` per CTA: one item per thread, at most 2 per SM.
inline int grid_sum_blocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 304) b = 304;
  return b < 1 ? 1 : (int)b;
}

}  // namespace tdks
