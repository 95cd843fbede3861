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
// FP64 columns of the dense map "ncycles cycles from zero on level C.lc"
// (row-major, m x m with m = 2 (2^lc+1)^2)
template <typename T>
cudaError_t launch_coarse_basis(const CtaParams<T>& C, const double* ainv, int ncycles, double* Bd, cudaStream_t s);

// x = B f for a dense row-major m x m operator (one warp per row)
template <typename T>
void launch_dense_apply(const T* B, int m, const T* f, T* x, cudaStream_t s);
void launch_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);

template <typename T>
void launch_coarse_cycle(const CtaParams<T>& C, const T* f, T* x, const double* ainv, int ncycles, cudaStream_t s);

}  // namespace aaomg
