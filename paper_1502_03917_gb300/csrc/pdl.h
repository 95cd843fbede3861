// pdl.h -- launches with programmatic dependent launch (internal).
//
// Consecutive kernels of a cycle depend on each other through global memory.
// Launched with programmatic stream serialisation, a kernel may be scheduled
// while its predecessor is still draining; it calls pdl_wait() first, which
// returns once the predecessor has completed and its writes are visible, so
// only the launch latency overlaps.  Stream capture records the launch as a
// programmatic edge of the CUDA graph.
#pragma once
#include <cuda_runtime.h>

namespace aaomg {

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
#endif

// Set while recording a graph that must not contain programmatic edges (the
// launches then serialise fully; griddepcontrol.wait returns at once).
inline thread_local bool g_pdl_off = false;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl_off ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace aaomg
