// pdl.cuh -- programmatic dependent launch for the short kernels of a solver
// iteration (vector updates, dot products).  At the solvers' small sizes a
// kernel runs for a few microseconds, about as long as the gap between two
// dependent launches; a kernel launched with programmatic stream
// serialization may be scheduled while its predecessor in the stream is
// still running and waits on the device instead (griddepcontrol), so the
// launch latency overlaps the predecessor's work.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace mpk {

// The first statement of every kernel that launch_pdl may launch: allows the
// next kernel in the stream to begin launching, then waits until the
// previous kernel has completed and its memory writes are visible.  Both
// instructions have no effect on a kernel launched without the attribute.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;\n\tgriddepcontrol.wait;" ::: "memory");
}

// kernel<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialization allowed (also inside stream capture, where it becomes a
// programmatic graph edge).  Errors are reported as for <<<>>> (the return
// value and cudaGetLastError).
template <class... P, class... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace mpk
