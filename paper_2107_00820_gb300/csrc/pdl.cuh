// Programmatic dependent launch for the chains of small kernels of the cycle.
//
// A kernel launched with launch_pdl may be scheduled while its predecessor on
// the stream is still finishing: its CTAs start, run their prologue (index
// arithmetic, shared-memory set-up, loads of data no kernel of the chain writes),
// and then wait in pdl_wait() until the predecessor has completed and its writes
// are visible.  Each kernel calls pdl_trigger() once a CTA has done its main
// work, so the successor is launched while the last CTAs run.  Every kernel that
// is launched this way calls pdl_wait() before it touches memory another kernel
// of the chain writes; launched normally, both calls are no-ops.  Captured into
// a CUDA graph the launches become programmatic dependency edges.
// ALS_PDL=0 in the environment launches every kernel normally.
#pragma once
#include <cuda_runtime.h>
#include <stdlib.h>

namespace als {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

inline bool pdl_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("ALS_PDL");
    v = (e && e[0] == '0') ? 0 : 1;
  }
  return v == 1;
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace als
