// Compensated float-float arithmetic: a value is the unevaluated sum hi + lo of two floats, added
// with Knuth's two-sum, which keeps about 44 significant bits.  Used where a sum must be nearly as
// accurate as FP64 but FP64 arithmetic, at a small fraction of the FP32 rate on this GPU, would
// bound the kernel.
#pragma once

#include <cuda_runtime.h>

namespace tdks {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
  const float h = s + e;
  return FF{h, e - (h - s)};
}

// the product of w = wh + wl (a split FP64 weight) and a float r, as a float-float
__device__ __forceinline__ FF ff_mul(float wh, float wl, float r) {
  const float p = wh * r;
  return FF{p, fmaf(wh, r, -p) + wl * r};
}

__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

}  // namespace tdks
