// launch.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace aaomg {

template <typename T>
void launch_resid_hat(const LevelP<T>& P, const T* f, const T* x, T* rh, cudaStream_t s);
template <typename T>
void launch_ne_update(const LevelP<T>& P, T* x, const T* rh, cudaStream_t s);
template <typename T>
void launch_lsgs_phase(const LevelP<T>& P, int field, int colour, T* x, T* rh, cudaStream_t s);
// one colour phase (colour of (i + j) mod 3) of the CGS smoother, in place on x
template <typename T>
void launch_cgs_phase(const LevelP<T>& P, int colour, const T* f, T* x, cudaStream_t s);
template <typename T>
void launch_restrict(const LevelP<T>& Pf, const LevelP<T>& Pc, const T* f, const T* x, T* fc, T* xc, cudaStream_t s);
template <typename T>
void launch_prolong(const LevelP<T>& Pf, const LevelP<T>& Pc, const T* xc, T* x, cudaStream_t s);
template <typename T>
void launch_coarsest(const double* ainv, const T* f, T* x, int64_t fs, cudaStream_t s);

// FP64 residual of the paper's system with norms; r and fin optional.
// out[0] = ||f - A x||^2_{L^-1}, out[1] = ||f||^2_{L^-1} (device).
void launch_resid64(const LevelP<double>& P, const double* f, const double* x, double* r, float* fin, int64_t fin_ld,
                    int64_t fin_fs, double* part, int nblk, double* out, cudaStream_t s);
// out[0] = ||x||^2_L, out[1] = ||x||^2_{L^-1} on the paper's system (device)
void launch_norms64(const LevelP<double>& P, const double* x, double* part, int nblk, double* out, cudaStream_t s);
void launch_refine_update(const LevelP<double>& P, double* x, const float* d, int64_t d_ld, int64_t d_fs,
                          cudaStream_t s);
void launch_to_f32(int n, const double* v, int64_t v_ld, int64_t v_fs, float* out, int64_t o_ld, int64_t o_fs,
                   double s_l, cudaStream_t s);
void launch_to_f64(int n, const float* v, int64_t v_ld, int64_t v_fs, double* out, int64_t o_ld, int64_t o_fs,
                   double s_l, cudaStream_t s);
void launch_rhs(const LevelP<double>& P, const double* yD, double* f, cudaStream_t s);

void launch_control(int64_t nn, const double* x, double alpha, double* u, cudaStream_t s);
void launch_adjoint_rhs(int64_t nn, const double* ubar, double alpha, double* g, cudaStream_t s);
// gyD = M z_y; out[0] = ubar . lambda, out[1] = (M z_lambda) . lambda (device)
void launch_adjoint_terms(const LevelP<double>& P, const double* x, const double* ubar, const double* z, double* gyD,
                          double* part, int nblk, double* out, cudaStream_t s);

constexpr int kResidBlocks = 304;  // 2 x 152 SMs

}  // namespace aaomg
