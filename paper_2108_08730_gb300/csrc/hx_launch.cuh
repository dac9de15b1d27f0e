// Kernel launches with programmatic dependent launch (PDL, sm_90 and later).
//
// A kernel launched through launch_k may be scheduled while its predecessor
// in the stream is still draining: its CTAs become resident early and block in
// pdl_enter() until the predecessor grid has completed and its memory is
// visible, so the launch latency between two dependent kernels overlaps the
// predecessor's tail.  Every kernel launched through launch_k therefore calls
// pdl_enter() before its first global-memory access.  griddepcontrol.wait is
// a hardware wait on the predecessor grid (no spinning in this code) and
// returns at once for a kernel launched without the attribute.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace hx {

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Process-wide switch, read once from HX_PDL ("0" disables; default on).
bool pdl_enabled();

template <typename... K, typename... A>
cudaError_t launch_k(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

}  // namespace hx
