// Kernel launch with programmatic dependent launch (PDL).
//
// Every kernel of the step is launched with programmatic stream
// serialisation, so the next kernel on the stream is scheduled while the
// current one finishes. Each kernel therefore starts with pdl_wait(), which
// returns once the preceding grid has completed and its writes are visible,
// and then calls pdl_launch() to let its own successor be scheduled. A
// kernel launched without the attribute treats both as no-ops.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace edpc {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches from the calling thread use the PDL attribute while this is true.
inline thread_local bool g_pdl_enabled = true;

// Turns the PDL attribute off for the launches made in its scope (kernels whose
// stream also waits on an event, i.e. with more than one incoming dependency).
struct NoPdl {
  bool saved;
  NoPdl() : saved(g_pdl_enabled) { g_pdl_enabled = false; }
  ~NoPdl() { g_pdl_enabled = saved; }
};

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_pdl_enabled ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

}  // namespace edpc
