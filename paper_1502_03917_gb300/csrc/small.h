// small.h -- one-launch smoothing calls for small levels (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "edge.h"

namespace aaomg {

// threads per block of the one-launch smoothing kernels (FP64 needs more
// registers per thread)
template <typename T>
constexpr int small_threads() {
    return sizeof(T) == 4 ? 1024 : 512;
}
constexpr int kBlockSmemMax = 227 * 1024;
// dynamic shared memory of the cluster kernel (it also has a small static table)
constexpr int kClusterSmemMax = kBlockSmemMax - 8 * 1024;

// shared memory of the single-block kernel for a level with n cells
template <typename T>
size_t block_smooth_smem(int n);
template <typename T>
cudaError_t small_prepare();
// `steps` smoothing steps (smoother 0 NE, 1 LSGS, 2 sLSGS) on one level in one
// launch of one thread block (rh in shared memory)
template <typename T>
void launch_smooth_block(const LevelP<T>& P, const EdgeTable<T>& E, int smoother, int steps, T* x, const T* f,
                         cudaStream_t s);

}  // namespace aaomg
