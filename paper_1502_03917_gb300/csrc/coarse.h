// coarse.h -- the single-block coarse-grid cycle kernel (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace aaomg {

constexpr int kMaxCtaLevel = 6;

// deepest level whose whole hierarchy (x, f, L^{-1} r for levels 1..l) fits in
// shared memory: 65x65 nodes in FP32, 33x33 in FP64
template <typename T>
constexpr int max_cta_level() {
    return sizeof(T) == 4 ? 6 : 5;
}

template <typename T>
struct CtaParams {
    LevelP<T> P[kMaxCtaLevel + 1];  // levels 1..lc, shared-memory layout (ld = n+1, fs = (n+1)^2)
    int lc;                         // finest level handled by the block
    int smoother, nu_pre, nu_post, gamma;
    int64_t g_ld, g_fs;             // layout of the level-lc vectors in global memory
};

template <typename T>
size_t coarse_smem_bytes(int lc);
template <typename T>
cudaError_t coarse_prepare();
template <typename T>
void launch_coarse_cycle(const CtaParams<T>& C, const T* f, T* x, const double* ainv, int ncycles, cudaStream_t s);

}  // namespace aaomg
