// coarse.cu -- the coarse end of the multigrid cycle in one thread block.
//
// Below a few thousand nodes per level the cycle of section 2 is latency
// bound: a W-cycle from level L visits level l 2^(L-l) times, and every visit
// of a grid-wide kernel costs a launch.  This kernel keeps every level from
// `lc` down to the coarsest (h = 1/2) in shared memory and runs whole cycles
// there -- smoothing (Algorithm 1 or the colour phases of Algorithm 2), defect
// restriction, the recursive coarse-grid steps, the exact coarsest solve,
// prolongation and post-smoothing -- with a block barrier between dependent
// phases.  It performs `ncycles` consecutive cycles on level lc for one
// right-hand side, i.e. the gamma coarse-grid steps a finer level asks for.
#include <cuda_runtime.h>

#include "coarse.h"
#include "pdl.h"
#include "stencil.cuh"

namespace aaomg {

namespace {

// threads per block: FP64 needs more registers per thread than 64
template <typename T>
constexpr int cta_threads() {
    return sizeof(T) == 4 ? 1024 : 512;
}

template <typename T>
struct CtaState {
    T* x[kMaxCtaLevel + 1];
    T* f[kMaxCtaLevel + 1];
    T* rh[kMaxCtaLevel + 1];
    double* ainv;
};

template <typename T>
__device__ void cta_lsgs_phase(const LevelP<T>& P, int field, int colour, T* x, T* rh) {
    const int n1 = P.n + 1;
    const int cpr = (n1 + 6) / 7;  // nodes of one colour per row (at most)
    for (int t = threadIdx.x; t < n1 * cpr; t += blockDim.x) {
        int j = t / cpr, k = t - j * cpr;
        int i = ((colour - 2 * j) % 7 + 7) % 7 + 7 * k;
        if (i <= P.n) lsgs_update_at(P, field, x, rh, i, j);
    }
    __syncthreads();
}

template <typename T>
__device__ void cta_cgs_phase(const LevelP<T>& P, int colour, const T* f, T* x) {
    const int n1 = P.n + 1;
    const int spr = (n1 + 2) / 3;  // nodes of one colour per row (at most)
    for (int t = threadIdx.x; t < n1 * spr; t += blockDim.x) {
        int j = t / spr, k = t - j * spr;
        int i = ((colour - j) % 3 + 3) % 3 + 3 * k;
        if (i <= P.n) cgs_update_at(P, f, x, i, j);
    }
    __syncthreads();
}

template <typename T>
__device__ void cta_smooth(const CtaParams<T>& C, const CtaState<T>& S, int l, int steps) {
    if (steps <= 0) return;
    const LevelP<T>& P = C.P[l];
    const int n1 = P.n + 1, nn = n1 * n1;
    T *x = S.x[l], *f = S.f[l], *rh = S.rh[l];
    if (C.smoother == 3) {
        for (int m = 0; m < steps; ++m)
            for (int c = 0; c < 3; ++c) cta_cgs_phase(P, c, f, x);
        return;
    }
    if (C.smoother == 0) {
        for (int m = 0; m < steps; ++m) {
            for (int t = threadIdx.x; t < nn; t += blockDim.x) resid_hat_at(P, f, x, rh, t % n1, t / n1);
            __syncthreads();
            for (int t = threadIdx.x; t < nn; t += blockDim.x) ne_update_at(P, x, rh, t % n1, t / n1);
            __syncthreads();
        }
        return;
    }
    for (int t = threadIdx.x; t < nn; t += blockDim.x) resid_hat_at(P, f, x, rh, t % n1, t / n1);
    __syncthreads();
    for (int m = 0; m < steps; ++m) {
        for (int field = 0; field < 2; ++field)
            for (int c = 0; c < 7; ++c) cta_lsgs_phase(P, field, colour_seq(c), x, rh);
        if (C.smoother == 2)
            for (int field = 1; field >= 0; --field)
                for (int c = 6; c >= 0; --c) cta_lsgs_phase(P, field, colour_seq(c), x, rh);
    }
}

template <typename T>
__device__ void cta_coarsest(const CtaState<T>& S) {
    T* f = S.f[1];
    T* x = S.x[1];
    double v = 0.0;
    int t = threadIdx.x;
    if (t < 18) {
        for (int c = 0; c < 18; ++c) v += S.ainv[t * 18 + c] * (double)f[c];
    }
    __syncthreads();  // every read of f before x is written (x and f are distinct, kept for clarity)
    if (t < 18) x[t] = (T)v;
    __syncthreads();
}

template <typename T>
__device__ void cta_restrict(const CtaParams<T>& C, const CtaState<T>& S, int l) {
    const LevelP<T>& P = C.P[l];
    const LevelP<T>& Pc = C.P[l - 1];
    const int nc1 = Pc.n + 1;
    for (int t = threadIdx.x; t < nc1 * nc1; t += blockDim.x) {
        int I = t % nc1, J = t / nc1;
        T sy, sl;
        restrict_at(P, S.f[l], S.x[l], I, J, sy, sl);
        int64_t c = nidx(Pc, I, J);
        S.f[l - 1][c] = sy;
        S.f[l - 1][c + Pc.fs] = sl;
        S.x[l - 1][c] = T(0);
        S.x[l - 1][c + Pc.fs] = T(0);
    }
    __syncthreads();
}

template <typename T>
__device__ void cta_prolong(const CtaParams<T>& C, const CtaState<T>& S, int l) {
    const LevelP<T>& P = C.P[l];
    const LevelP<T>& Pc = C.P[l - 1];
    const int n1 = P.n + 1;
    for (int t = threadIdx.x; t < n1 * n1; t += blockDim.x) {
        int i = t % n1, j = t / n1;
        T vy, vl;
        prolong_at(P, Pc, S.x[l - 1], i, j, vy, vl);
        int64_t p = nidx(P, i, j);
        S.x[l][p] += vy;
        S.x[l][p + P.fs] += vl;
    }
    __syncthreads();
}

// `ncycles` cycles on level `top`, each recursing gamma times per level (the
// recursion of section 2 unrolled into a loop with one counter per level, so
// that the stack size is static).
template <typename T>
__device__ void cta_cycles(const CtaParams<T>& C, const CtaState<T>& S, int top, int ncycles) {
    int todo[kMaxCtaLevel + 2];
    todo[top + 1] = ncycles;
    int l = top;
    for (;;) {
        // start a cycle on level l: pre-smooth and restrict down to level 1
        while (l > 1) {
            cta_smooth(C, S, l, C.nu_pre);
            cta_restrict(C, S, l);
            todo[l] = C.gamma;
            --l;
        }
        cta_coarsest(S);
        // the cycle on level l is complete; climb while parents are complete
        for (;;) {
            int parent = l + 1;
            if (--todo[parent] > 0) break;  // another cycle on level l
            if (parent > top) return;
            cta_prolong(C, S, parent);
            cta_smooth(C, S, parent, C.nu_post);
            l = parent;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(cta_threads<T>()) k_coarse_cycle(CtaParams<T> C, const T* __restrict__ fg,
                                                              T* __restrict__ xg, const double* __restrict__ ainv,
                                                              int ncycles) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem[];
    CtaState<T> S;
    double* a = reinterpret_cast<double*>(smem);
    T* p = reinterpret_cast<T*>(smem + 18 * 18 * sizeof(double));
    for (int l = 1; l <= C.lc; ++l) {
        int64_t sz = 2 * C.P[l].fs;
        S.x[l] = p;
        S.f[l] = p + sz;
        S.rh[l] = p + 2 * sz;
        p += 3 * sz;
    }
    S.ainv = a;
    for (int t = threadIdx.x; t < 18 * 18; t += blockDim.x) a[t] = ainv[t];
    const LevelP<T>& P = C.P[C.lc];
    const int n1 = P.n + 1;
    for (int t = threadIdx.x; t < n1 * n1; t += blockDim.x) {
        int i = t % n1, j = t / n1;
        int64_t g = (int64_t)j * C.g_ld + i, q = nidx(P, i, j);
        S.f[C.lc][q] = fg[g];
        S.f[C.lc][q + P.fs] = fg[g + C.g_fs];
        S.x[C.lc][q] = xg[g];
        S.x[C.lc][q + P.fs] = xg[g + C.g_fs];
    }
    __syncthreads();
    cta_cycles(C, S, C.lc, ncycles);
    for (int t = threadIdx.x; t < n1 * n1; t += blockDim.x) {
        int i = t % n1, j = t / n1;
        int64_t g = (int64_t)j * C.g_ld + i, q = nidx(P, i, j);
        xg[g] = S.x[C.lc][q];
        xg[g + C.g_fs] = S.x[C.lc][q + P.fs];
    }
}

// Columns of the dense operator of `ncycles` cycles from a zero initial guess
// on level lc: block k runs the cycles with f = e_k and stores the result as
// column k of Bd (row-major m x m, m = 2 (n+1)^2), in FP64.
template <typename T>
__global__ void __launch_bounds__(cta_threads<T>()) k_coarse_basis(CtaParams<T> C, const double* __restrict__ ainv,
                                                                   int ncycles, double* __restrict__ Bd) {
    extern __shared__ __align__(16) unsigned char smem[];
    CtaState<T> S;
    double* a = reinterpret_cast<double*>(smem);
    T* p = reinterpret_cast<T*>(smem + 18 * 18 * sizeof(double));
    for (int l = 1; l <= C.lc; ++l) {
        int64_t sz = 2 * C.P[l].fs;
        S.x[l] = p;
        S.f[l] = p + sz;
        S.rh[l] = p + 2 * sz;
        p += 3 * sz;
    }
    S.ainv = a;
    for (int t = threadIdx.x; t < 18 * 18; t += blockDim.x) a[t] = ainv[t];
    const int64_t m = 2 * C.P[C.lc].fs;
    const int k = blockIdx.x;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
        S.f[C.lc][t] = T(t == k ? 1 : 0);
        S.x[C.lc][t] = T(0);
    }
    __syncthreads();
    cta_cycles(C, S, C.lc, ncycles);
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) Bd[t * m + k] = (double)S.x[C.lc][t];
}

}  // namespace

template <typename T>
size_t coarse_smem_bytes(int lc) {
    size_t s = 18 * 18 * sizeof(double);
    for (int l = 1; l <= lc; ++l) {
        size_t n1 = (size_t(1) << l) + 1;
        s += 3 * 2 * n1 * n1 * sizeof(T);
    }
    return s;
}

template <typename T>
cudaError_t coarse_prepare() {
    return cudaFuncSetAttribute(k_coarse_cycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarse_smem_bytes<T>(max_cta_level<T>()));
}

template <typename T>
void launch_coarse_cycle(const CtaParams<T>& C, const T* f, T* x, const double* ainv, int ncycles, cudaStream_t s) {
    launch_pdl(k_coarse_cycle<T>, 1, cta_threads<T>(), coarse_smem_bytes<T>(C.lc), s, C, f, x, ainv, ncycles);
}

template <typename T>
cudaError_t launch_coarse_basis(const CtaParams<T>& C, const double* ainv, int ncycles, double* Bd, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_basis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)coarse_smem_bytes<T>(max_cta_level<T>()));
    if (e != cudaSuccess) return e;
    int m = (int)(2 * C.P[C.lc].fs);
    k_coarse_basis<T><<<m, cta_threads<T>(), coarse_smem_bytes<T>(C.lc), s>>>(C, ainv, ncycles, Bd);
    return cudaGetLastError();
}

template cudaError_t launch_coarse_basis<float>(const CtaParams<float>&, const double*, int, double*, cudaStream_t);
template cudaError_t launch_coarse_basis<double>(const CtaParams<double>&, const double*, int, double*, cudaStream_t);
template size_t coarse_smem_bytes<float>(int);
template size_t coarse_smem_bytes<double>(int);
template cudaError_t coarse_prepare<float>();
template cudaError_t coarse_prepare<double>();
template void launch_coarse_cycle<float>(const CtaParams<float>&, const float*, float*, const double*, int,
                                         cudaStream_t);
template void launch_coarse_cycle<double>(const CtaParams<double>&, const double*, double*, const double*, int,
                                          cudaStream_t);

}  // namespace aaomg
