// cluster.h -- one-launch smoothing calls on mid-size levels, one thread-block
// cluster per call (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace aaomg {

// level sizes (cells per side) with a cluster kernel
constexpr bool cluster_level(int n) { return n == 64 || n == 128 || n == 256; }
constexpr int kClusterMax = 16;  // 16 needs the non-portable cluster size

// rows [row_lo(k), row_lo(k+1)) of a level with `rows` grid rows belong to
// block k of a cluster of cs blocks
AAOMG_HD int cluster_row_lo(int k, int rows, int cs) { return (int)(((long long)k * rows) / cs); }

// shared memory per block: x and rh pairs of the largest strip
template <typename T>
size_t cluster_smem(int n, int cs);
template <typename T>
cudaError_t cluster_prepare();
// clusters of cs blocks that can be resident at once on this device (0: the
// configuration cannot run)
template <typename T>
int cluster_max_active(int n, int cs);
// `steps` smoothing steps (smoother 0 NE, 1 LSGS, 2 sLSGS) on one level in one
// launch of one cluster of cs blocks
template <typename T>
cudaError_t launch_smooth_cluster(const LevelP<T>& P, int smoother, int steps, T* x, const T* f, int cs,
                                  cudaStream_t s);

}  // namespace aaomg
