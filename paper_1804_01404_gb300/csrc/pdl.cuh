// Programmatic dependent launch between the short kernels of a step's serial chain (the Hartree
// solve, the misfit): a kernel launched with launch_pdl may be scheduled while the kernel before it
// in the stream is still running, once every CTA of that kernel has called pdl_trigger (or exited);
// it calls pdl_wait before its first access to memory the earlier kernel writes or reads, which
// returns when that kernel has completed and its writes are visible.  So only the launch latency
// overlaps.  Both instructions are no-ops for a kernel launched without the attribute.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace tdks {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// kern<<<grid, block, smem, s>>>(args...) with programmatic stream serialisation allowed, and an
// optional cluster size (x) for kernels that need one.  While s is being captured into a graph the
// kernel is launched without the attribute: inside the step graphs the programmatic edges measured
// slower than plain ones (learned step 2403 against 2414 steps/s), while stream launches gain (the
// predictor-corrector step 1523 -> 1552 steps/s).
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int cluster_x,
                       A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (cs == cudaStreamCaptureStatusNone) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cluster_x > 0) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cluster_x;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = na > 0 ? at : nullptr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

}  // namespace tdks
