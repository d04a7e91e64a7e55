// Programmatic dependent launch between kernels that follow one another on a
// stream (the steps of the LB loop, the layers of the network): a kernel
// launched by launch_pdl may be scheduled, and run its prologue (barrier
// set-up, tensor-memory allocation), while the kernel before it on the stream
// finishes.  Such a kernel calls pdl_trigger() at its start and pdl_wait()
// before its first access to global memory; pdl_wait returns once the kernel
// before it has completed and its writes are visible.  Without the launch
// attribute both are no-ops.
#pragma once

#include <cuda_runtime.h>

namespace lbk {

__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace lbk
