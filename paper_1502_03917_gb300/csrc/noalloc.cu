// noalloc.cu -- the FP64 residual r = f - A x and its relative norm without any
// handle and without allocating device memory.
//
// Some callers cannot allocate: a program whose device memory budget is fixed
// when it starts, a framework whose caching allocator owns every device byte,
// or a real-time loop in which the device-wide synchronisation that cudaMalloc
// and cudaFree may cause is not allowed.  For them this variant of the
// handle's residual kernel keeps its scratch (one partial sum pair per grid row
// and the final pair) in file-scope __device__ arrays that every device which
// loads the library holds until the process exits.
//
// The host never passes the arrays' names to a kernel: in host code they are
// stand-ins, not device addresses.  The first call on a device, with that device
// current, looks up their device addresses with cudaGetSymbolAddress and caches
// them; make that first call before any stream capture.  All calls share the
// arrays and every call overwrites them completely, so calls that overlap on
// the GPU (on different streams) race and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "aaomg.h"
#include "stencil.cuh"

namespace aaomg {
namespace {

constexpr int kNoAllocMaxRows = 4097;  // grid rows of the finest level: levels <= 12
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) double g_row_sums[2 * kNoAllocMaxRows];
__device__ __align__(256) double g_total[2];

std::mutex g_mu;
double* g_rows_addr[kNoAllocMaxDevices];
double* g_total_addr[kNoAllocMaxDevices];

// one block per grid row j: r = f - A x on that row (paper's scaling, FP64) and
// the row's partial sums of ||r||^2_{L^-1} and ||f||^2_{L^-1}
__global__ void k_resid_rows(LevelP<double> P, const double* __restrict__ f, const double* __restrict__ x,
                             double* __restrict__ r, double* __restrict__ rows) {
    const int j = blockIdx.x;
    double srr = 0.0, sff = 0.0;
    for (int i = threadIdx.x; i <= P.n; i += blockDim.x) {
        double ay, al;
        apply_A(P, x, i, j, ay, al);
        int64_t p = nidx(P, i, j);
        double fy = f[p], fl = f[p + P.fs];
        double ry = fy - ay, rl = fl - al;
        double il = inv_ly(P, i, j), ill = il * P.invd;
        srr += ry * ry * il + rl * rl * ill;
        sff += fy * fy * il + fl * fl * ill;
        if (r) {
            r[p] = ry;
            r[p + P.fs] = rl;
        }
    }
    __shared__ double sa[32], sb[32];
    for (int o = 16; o > 0; o >>= 1) {
        srr += __shfl_down_sync(0xffffffffu, srr, o);
        sff += __shfl_down_sync(0xffffffffu, sff, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = srr;
        sb[w] = sff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += sa[k];
            b += sb[k];
        }
        rows[2 * j] = a;
        rows[2 * j + 1] = b;
    }
}

// sum the row partials in row order (deterministic)
__global__ void k_rows_total(const double* __restrict__ rows, int nrows, double* __restrict__ total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nrows; ++k) {
            a += rows[2 * k];
            b += rows[2 * k + 1];
        }
        total[0] = a;
        total[1] = b;
    }
}

// coefficients of the paper's system (c = 1, d = 1/alpha) on the finest level,
// as far as the residual and the norms need them
LevelP<double> residual_params(int levels, double alpha, int k_variant) {
    LevelP<double> P{};
    const int n = 1 << levels;
    const double h = 1.0 / n, h2 = h * h, beta = std::sqrt(alpha), km = k_variant == 0 ? 1.0 : 0.0;
    P.n = n;
    P.ld = n + 1;
    P.fs = (int64_t)(n + 1) * (n + 1);
    P.h2 = h2;
    P.c = 1.0;
    P.d = 1.0 / alpha;
    P.invd = alpha;
    P.beta = beta;
    P.km = km;
    P.tau = 0.4;
    auto ly = [&](int i, int j) {
        double m[7], kd[7];
        row_coeffs_general<double>(i, j, n, h2, m, kd);
        return m[0] + beta * (kd[0] + km * m[0]);
    };
    double m[7], kd[7];
    row_coeffs_general<double>(1, 1, n, h2, m, kd);
    P.mC = m[0];
    P.mO = m[1];
    P.invLy_int = 1.0 / ly(1, 1);
    const int rep[3] = {0, 1, n};
    for (int cy = 0; cy < 3; ++cy)
        for (int cx = 0; cx < 3; ++cx) P.invLy[cx + 3 * cy] = 1.0 / ly(rep[cx], rep[cy]);
    return P;
}

}  // namespace
}  // namespace aaomg

using namespace aaomg;

extern "C" {

int mg_residual_noalloc(int levels, double alpha, int k_variant, const double* f, const double* x, double* r,
                        double* relres, void* stream) {
    // levels > 12: the 8193 grid rows of h = 2^-13 exceed the static scratch
    if (levels < 1 || levels > 12) return AAOMG_ERR_BAD_ARG;
    if (!(alpha > 0.0) || !std::isfinite(alpha) || (k_variant != 0 && k_variant != 1) || !f || !x)
        return AAOMG_ERR_BAD_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return AAOMG_ERR_NO_DEVICE;
    double* rows = nullptr;
    double* total = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_rows_addr[dev]) {
            void* a = nullptr;
            void* b = nullptr;
            e = cudaGetSymbolAddress(&a, g_row_sums);
            if (e == cudaSuccess) e = cudaGetSymbolAddress(&b, g_total);
            if (e != cudaSuccess) return AAOMG_ERR_CUDA;
            g_rows_addr[dev] = (double*)a;
            g_total_addr[dev] = (double*)b;
        }
        rows = g_rows_addr[dev];
        total = g_total_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    LevelP<double> P = residual_params(levels, alpha, k_variant);
    k_resid_rows<<<P.n + 1, 256, 0, s>>>(P, f, x, r, rows);
    k_rows_total<<<1, 32, 0, s>>>(rows, P.n + 1, total);
    e = cudaGetLastError();
    if (e == cudaSuccess && relres) {
        double h[2];
        e = cudaMemcpyAsync(h, total, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) *relres = std::sqrt(h[0] / (h[1] > 0.0 ? h[1] : 1.0));
    }
    return e == cudaSuccess ? AAOMG_OK : AAOMG_ERR_CUDA;
}

}  // extern "C"
