// Programmatic dependent launch (PDL) between the kernels of one Arnoldi step.
//
// A kernel launched with launch_pdl() may start while the kernel before it on
// the stream is still running: its CTAs become resident as soon as every CTA
// of the previous kernel has executed pdl_trigger() (or exited), run their
// prologue, and block in pdl_wait() until the previous kernel has completed
// and its memory is visible.  The solver's kernels trigger at the end of each
// CTA's main work (triggering at the start let the next kernel's CTAs take SM
// resources from the running one), after their own wait, so when a kernel
// starts, the kernel two launches back has completed: its outputs may be read
// before the kernel's own wait.  Both instructions are no-ops in a kernel
// launched without the attribute.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace pn {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches kern<<<grid, block, smem, s>>>(args...), with programmatic stream
// serialisation when pdl is true.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace pn
