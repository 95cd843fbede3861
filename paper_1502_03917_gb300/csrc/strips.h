// strips.h -- one-launch smoothing calls on small and mid-size levels
// (internal): one thread block, or one thread-block cluster whose blocks each
// own a strip of grid rows.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace aaomg {

// threads per block (FP64 needs more registers per thread)
template <typename T>
constexpr int strip_threads() {
    return sizeof(T) == 4 ? 1024 : 512;
}
// dynamic shared memory per block: 227 KB less room for a small static table
constexpr int kStripSmemMax = 227 * 1024 - 12 * 1024;
constexpr int kClusterMax = 16;  // blocks per cluster; above 8 needs the non-portable size

// level sizes (cells per side) with a single-block kernel and with a cluster kernel
constexpr bool block_level(int n) { return n == 4 || n == 8 || n == 16 || n == 32 || n == 64; }
constexpr bool cluster_level(int n) { return n == 64 || n == 128 || n == 256; }

// rows [row_lo(k), row_lo(k+1)) of a level with `rows` grid rows belong to
// block k of cs blocks
AAOMG_HD int strip_row_lo(int k, int rows, int cs) { return (int)(((long long)k * rows) / cs); }

// Coefficients of the nodes of one boundary class cls5(i) + 5 cls5(j) (25
// classes per level; class 12 is the deep interior): mass and bare stiffness
// weights of the 7 offsets, L_y^-1 of each neighbour (0 outside the grid),
// N_ii^-1 of both fields, and the LSGS scatter weights of both fields (the
// column of A scaled by the neighbours' L^-1).  Built on the host in FP64.
template <typename T>
struct EdgeClass {
    T m[7], kd[7], il[7];
    T iny, inl;
    T sc[2][7][2];
};

// shared memory per block: x and rh pairs of the largest strip
template <typename T>
size_t strips_smem(int n, int cs);
template <typename T>
cudaError_t strips_prepare();
// whether cs blocks (1: a single block) have a kernel for n and fit in shared memory
template <typename T>
bool strips_fit(int n, int cs);
// clusters of cs blocks that can be resident at once on this device (0: the
// configuration cannot run; 1 for a fitting single block)
template <typename T>
int strips_max_active(int n, int cs);
// `steps` smoothing steps (smoother 0 NE, 1 LSGS, 2 sLSGS) on one level in one
// launch of cs blocks (cs = 1: a single block; else one cluster)
template <typename T>
cudaError_t launch_smooth_strips(const LevelP<T>& P, const EdgeClass<T>* ctab, int smoother, int steps, T* x,
                                 const T* f, int cs, cudaStream_t s);

// The level with 512 cells per side (FP32, LSGS or sLSGS): a whole smoothing
// call in one launch of a 16-block cluster that keeps the residual in shared
// memory and updates the iterate in global memory.  Clusters that can be
// resident at once (0: cannot run: FP64, another size, no room).
template <typename T>
int rg_max_active(int n);
template <typename T>
cudaError_t launch_smooth_rg(const LevelP<T>& P, const EdgeClass<T>* ctab, int smoother, int steps, T* x,
                             const T* f, cudaStream_t s);

}  // namespace aaomg
