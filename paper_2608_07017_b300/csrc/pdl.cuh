// pdl.cuh -- programmatic dependent launch for chains of short dependent kernels (the panels of
// the LU).  A kernel launched with launch_pdl may be scheduled once every CTA of its predecessor
// in the stream has started (each CTA signals that with pdl_trigger on entry); it must call
// pdl_wait, which returns when the predecessor has completed and its writes are visible, before
// it reads or writes memory the predecessor touches.  Both are no-ops for a normal launch.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace ewos {

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace ewos
