// Warp-level sums of several values per lane.
#pragma once

#include <cuda_runtime.h>

namespace tdks {

// Warp sums of N = 2^K values per lane with N - 1 + 5 - K shuffles instead of 5 N: at each of the
// first K steps a lane keeps one half of its values and trades the other half with the partner lane
// (lane ^ 16, then ^ 8, ...), the last 5 - K steps add a single value.  On return lane L holds the
// warp total of value (L >> (5 - K)).
template <int N, typename T>
__device__ __forceinline__ T warp_split_sum(T* v) {
  constexpr int K = (N >= 32) ? 5 : (N >= 16) ? 4 : (N >= 8) ? 3 : (N >= 4) ? 2 : (N >= 2) ? 1 : 0;
  static_assert((1 << K) == N, "N must be a power of two up to 32");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int st = 0; st < K; ++st) {
    const int n = N >> st, o = 16 >> st;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < n / 2; ++j) {
      const T send = up ? v[j] : v[j + n / 2];
      const T keep = up ? v[j + n / 2] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T r = v[0];
#pragma unroll
  for (int st = K; st < 5; ++st) r += __shfl_xor_sync(0xffffffffu, r, 16 >> st);
  return r;
}

}  // namespace tdks
