// kernels.cu -- per-level stencil kernels: residual, NE update, one LSGS colour
// phase, defect restriction, prolongation, coarsest solve, FP64 refinement and
// norm reductions.  One thread per node (or per coarse node); the operator is
// applied matrix-free from the coefficients of common.cuh.
#include <cuda_runtime.h>

#include "coarse.h"
#include "common.cuh"
#include "launch.h"
#include "pdl.h"
#include "lean.cuh"
#include "stencil.cuh"

namespace aaomg {

namespace {

// ---------------------------------------------------------------- kernels --

// Thread t of the launch -> node: the deep-interior nodes first (their count
// rounded up to a warp), then the edge nodes, so that no warp mixes the
// constant-stencil path with the general one.

// rh = L^{-1} (f - A x) on every node
// N > 0: kernel instantiated for n = N cells (strides are compile-time
// constants); N = 0: any n
template <typename T, int N>
__global__ void k_resid_hat(LevelP<T> P, const T* __restrict__ f, const T* __restrict__ x, T* __restrict__ rhv) {
    pdl_wait();
    using V2 = typename P2<T>::t;
    V2* rh = reinterpret_cast<V2*>(rhv);  // (y, lambda) pairs
    const int n = N > 0 ? N : P.n, ld = n + 1, fs = ld * ld;
    InteriorAll ia(n);
    EdgeNodes ed(n, -1);
    const int ni = ia.count(), nip = (ni + 31) & ~31;
    int t = blockIdx.x * blockDim.x + threadIdx.x, i, j;
    if (t < nip) {
        if (t < ni) {
            ia.node(t, i, j);
            resid_fast(P, f, x, rh, i, j, ld, fs);
        }
    } else if (t - nip < ed.count() && ed.node(t - nip, i, j)) {
        resid_hat_acc(P, f, x, RhPair<T>{rh}, i, j);
    }
}

// Algorithm 1 update: x += tau L^{-1} A rh (A symmetric), with rh = L^{-1} r
template <typename T, int N>
__global__ void k_ne_update(LevelP<T> P, T* __restrict__ x, const T* __restrict__ rhv) {
    pdl_wait();
    using V2 = typename P2<T>::t;
    V2* rh = reinterpret_cast<V2*>(const_cast<T*>(rhv));
    const int n = N > 0 ? N : P.n, ld = n + 1, fs = ld * ld;
    InteriorAll ia(n);
    EdgeNodes ed(n, -1);
    const int ni = ia.count(), nip = (ni + 31) & ~31;
    int t = blockIdx.x * blockDim.x + threadIdx.x, i, j;
    if (t < nip) {
        if (t < ni) {
            ia.node(t, i, j);
            ne_fast(P, x, rh, i, j, ld, fs);
        }
    } else if (t - nip < ed.count() && ed.node(t - nip, i, j)) {
        ne_update_acc(P, x, RhPair<T>{rh}, i, j);
    }
}

// One colour phase of Algorithm 2: every unknown of field `field` on a node of
// colour `colour` does q = sum_j A_ij rh_j, p = q / N_ii, x_i += p and
// rh_j -= A_ji p / L_jj on its neighbourhood.  Nodes of one colour share no
// neighbour, so the updates of a phase are independent and race-free.
template <typename T, int N>
__global__ void k_lsgs_phase(LevelP<T> P, int field, int colour, T* __restrict__ x, T* __restrict__ rhv) {
    pdl_wait();
    using V2 = typename P2<T>::t;
    V2* rh = reinterpret_cast<V2*>(rhv);
    const int n = N > 0 ? N : P.n, ld = n + 1, fs = ld * ld;
    InteriorColour ic(n, colour);
    EdgeNodes ed(n, colour);
    const int ni = ic.count(), nip = (ni + 31) & ~31;
    int t = blockIdx.x * blockDim.x + threadIdx.x, i, j;
    if (t < nip) {
        if (t < ni && ic.node(t, i, j)) lsgs_fast(P, field, x, rh, i, j, ld, fs);
    } else if (t - nip < ed.count() && ed.node(t - nip, i, j)) {
        lsgs_update_acc(P, field, x, RhPair<T>{rh}, i, j);
    }
}

// One colour phase of the CGS smoother: every node of colour c of (i + j) mod 3
// (no two coupled) solves its 2x2 block against the residual of the current
// iterate.  One thread per slot; slot t is row t / spr, the k-th node of the
// colour in that row.
template <typename T>
__global__ void k_cgs_phase(LevelP<T> P, int colour, const T* __restrict__ f, T* __restrict__ x) {
    pdl_wait();
    const int spr = (P.n + 1 + 2) / 3;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (P.n + 1) * spr) return;
    const int j = t / spr, k = t - j * spr;
    const int i = ((colour - j) % 3 + 3) % 3 + 3 * k;
    if (i <= P.n) cgs_update_at(P, f, x, i, j);
}

// Defect restriction: fc = P^T (f - A x) on a coarse node (I,J) -- weight 1 at
// the fine node (2I,2J) and 1/2 at its six neighbours, the midpoints of the
// coarse edges; also zeroes the coarse iterate xc.
template <typename T>
__global__ void k_restrict(LevelP<T> Pf, LevelP<T> Pc, const T* __restrict__ f, const T* __restrict__ x,
                           T* __restrict__ fc, T* __restrict__ xc) {
    pdl_wait();
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I > Pc.n || J > Pc.n) return;
    T sy, sl;
    restrict_at(Pf, f, x, I, J, sy, sl);
    int64_t c = nidx(Pc, I, J);
    fc[c] = sy;
    fc[c + Pc.fs] = sl;
    xc[c] = T(0);
    xc[c + Pc.fs] = T(0);
}

// x += P xc: nodal interpolation of the coarse P1 function at the fine node
template <typename T>
__global__ void k_prolong(LevelP<T> Pf, LevelP<T> Pc, const T* __restrict__ xc, T* __restrict__ x) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > Pf.n || j > Pf.n) return;
    T vy, vl;
    prolong_at(Pf, Pc, xc, i, j, vy, vl);
    int64_t p = nidx(Pf, i, j);
    x[p] += vy;
    x[p + Pf.fs] += vl;
}

// exact solve on the coarsest grid (18 unknowns): x = A_1^{-1} f in FP64
template <typename T>
__global__ void k_coarsest(const double* __restrict__ ainv, const T* __restrict__ f, T* __restrict__ x, int64_t fs) {
    pdl_wait();
    __shared__ double fb[18];
    int t = threadIdx.x;
    if (t < 18) fb[t] = (double)f[(t < 9 ? t : fs + t - 9)];
    __syncthreads();
    if (t < 18) {
        double s = 0.0;
        for (int c = 0; c < 18; ++c) s += ainv[t * 18 + c] * fb[c];
        x[(t < 9 ? t : fs + t - 9)] = (T)s;
    }
}

// ---------------------------------------------------------- reductions --

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block sum of two values; result valid in thread 0
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[32], sb[32];
    a = warp_sum(a);
    b = warp_sum(b);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        a = l < nw ? sa[l] : 0.0;
        b = l < nw ? sb[l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

// FP64 residual r = f - A x on the paper's system (c = 1, d = 1/alpha) with
// ||r||^2_{L^-1} and ||f||^2_{L^-1} partial sums per block.  Optional outputs:
// r (FP64) and the scaled single-precision defect fin = (r_y, beta r_lambda)
// for the FP32 cycles.
__global__ void k_resid64(LevelP<double> P, const double* __restrict__ f, const double* __restrict__ x,
                          double* __restrict__ r, float* __restrict__ fin, int64_t fin_ld, int64_t fin_fs,
                          double* __restrict__ part) {
    int64_t nn = (int64_t)(P.n + 1) * (P.n + 1);
    double srr = 0.0, sff = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(t / (P.n + 1)), i = (int)(t - (int64_t)j * (P.n + 1));
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
        if (fin) {
            int64_t q = (int64_t)j * fin_ld + i;
            fin[q] = (float)ry;
            fin[q + fin_fs] = (float)(P.beta * rl);
        }
    }
    block_sum2(srr, sff);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = srr;
        part[2 * blockIdx.x + 1] = sff;
    }
}

// ||x||^2_L and ||x||^2_{L^-1} partial sums per block, L = diag(Q) of the
// paper's system: L_y = M_ii + alpha^{1/2} K_ii, L_lambda = alpha^{-1} L_y
__global__ void k_norms64(LevelP<double> P, const double* __restrict__ x, double* __restrict__ part) {
    int64_t nn = (int64_t)(P.n + 1) * (P.n + 1);
    double sl = 0.0, sinv = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(t / (P.n + 1)), i = (int)(t - (int64_t)j * (P.n + 1));
        int64_t p = nidx(P, i, j);
        double il = inv_ly(P, i, j), xy = x[p], xl = x[p + P.fs];
        sl += xy * xy / il + xl * xl * (P.d / il);
        sinv += xy * xy * il + xl * xl * (il * P.invd);
    }
    block_sum2(sl, sinv);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sl;
        part[2 * blockIdx.x + 1] = sinv;
    }
}

// sum the per-block partials in a fixed order (deterministic)
__global__ void k_reduce_parts(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
        a += part[2 * t];
        b += part[2 * t + 1];
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// x += S^{-1} d: y += d_y, lambda += beta d_lambda (undo the FP32 scaling)
__global__ void k_refine_update(LevelP<double> P, double* __restrict__ x, const float* __restrict__ d, int64_t d_ld,
                                int64_t d_fs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > P.n || j > P.n) return;
    int64_t p = nidx(P, i, j), q = (int64_t)j * d_ld + i;
    x[p] += (double)d[q];
    x[p + P.fs] += P.beta * (double)d[q + d_fs];
}

// v (paper's scaling, FP64) -> out (FP32 symmetric scaling): lambda * s_l
__global__ void k_to_f32(int n, const double* __restrict__ v, int64_t v_ld, int64_t v_fs, float* __restrict__ out,
                         int64_t o_ld, int64_t o_fs, double s_l) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > n || j > n) return;
    int64_t p = (int64_t)j * v_ld + i, q = (int64_t)j * o_ld + i;
    out[q] = (float)v[p];
    out[q + o_fs] = (float)(v[p + v_fs] * s_l);
}

__global__ void k_to_f64(int n, const float* __restrict__ v, int64_t v_ld, int64_t v_fs, double* __restrict__ out,
                         int64_t o_ld, int64_t o_fs, double s_l) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > n || j > n) return;
    int64_t p = (int64_t)j * v_ld + i, q = (int64_t)j * o_ld + i;
    out[q] = (double)v[p];
    out[q + o_fs] = (double)v[p + v_fs] * s_l;
}

// f = (M yD, 0)
__global__ void k_rhs(LevelP<double> P, const double* __restrict__ yD, double* __restrict__ f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > P.n || j > P.n) return;
    double m[7], kd[7], y[7];
    row_coeffs(P, i, j, m, kd);
    // yD is packed with stride n+1
    LevelP<double> Q = P;
    Q.ld = P.n + 1;
    load7(Q, yD, i, j, y);
    double s = 0.0;
    for (int o = 0; o < 7; ++o) s += m[o] * y[o];
    int64_t p = nidx(P, i, j);
    f[p] = s;
    f[p + P.fs] = 0.0;
}

inline dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

}  // namespace

// ------------------------------------------------------------- launchers --
const dim3 kBlk2(32, 8);

// threads for the interior/edge split: interior slots rounded to a warp + edge slots
inline int split_threads(int n, bool colour) {
    int ni = n >= 4 ? (n - 3) * (colour ? (n - 3 + 6) / 7 : (n - 3)) : 0;
    int rows = n >= 4 ? 4 : n + 1;
    int full = colour ? (n + 7) / 7 : n + 1;
    int ne = rows * full + (n >= 4 ? 4 * (n - 3) : 0);
    return ((ni + 31) & ~31) + ne;
}
// instantiate the level kernels for the grid sizes of the middle levels
#define AAOMG_BY_N(N_, CALL)                  \
    switch (N_) {                             \
    case 128: CALL(128); break;               \
    case 256: CALL(256); break;               \
    case 512: CALL(512); break;               \
    case 1024: CALL(1024); break;             \
    default: CALL(0); break;                  \
    }
template <typename T>
void launch_resid_hat(const LevelP<T>& P, const T* f, const T* x, T* rh, cudaStream_t s) {
    int nb = (split_threads(P.n, false) + 255) / 256;
#define L_(N) launch_pdl(k_resid_hat<T, N>, nb, 256, 0, s, P, f, x, rh)
    AAOMG_BY_N(P.n, L_)
#undef L_
}
template <typename T>
void launch_ne_update(const LevelP<T>& P, T* x, const T* rh, cudaStream_t s) {
    int nb = (split_threads(P.n, false) + 255) / 256;
#define L_(N) launch_pdl(k_ne_update<T, N>, nb, 256, 0, s, P, x, rh)
    AAOMG_BY_N(P.n, L_)
#undef L_
}
template <typename T>
void launch_lsgs_phase(const LevelP<T>& P, int field, int colour, T* x, T* rh, cudaStream_t s) {
    int nb = (split_threads(P.n, true) + 255) / 256;
#define L_(N) launch_pdl(k_lsgs_phase<T, N>, nb, 256, 0, s, P, field, colour, x, rh)
    AAOMG_BY_N(P.n, L_)
#undef L_
}
template <typename T>
void launch_cgs_phase(const LevelP<T>& P, int colour, const T* f, T* x, cudaStream_t s) {
    const int slots = (P.n + 1) * ((P.n + 1 + 2) / 3);
    launch_pdl(k_cgs_phase<T>, (slots + 255) / 256, 256, 0, s, P, colour, f, x);
}
template <typename T>
void launch_restrict(const LevelP<T>& Pf, const LevelP<T>& Pc, const T* f, const T* x, T* fc, T* xc, cudaStream_t s) {
    launch_pdl(k_restrict<T>, grid2(Pc.n + 1, Pc.n + 1, kBlk2), kBlk2, 0, s, Pf, Pc, f, x, fc, xc);
}
template <typename T>
void launch_prolong(const LevelP<T>& Pf, const LevelP<T>& Pc, const T* xc, T* x, cudaStream_t s) {
    launch_pdl(k_prolong<T>, grid2(Pf.n + 1, Pf.n + 1, kBlk2), kBlk2, 0, s, Pf, Pc, xc, x);
}
template <typename T>
void launch_coarsest(const double* ainv, const T* f, T* x, int64_t fs, cudaStream_t s) {
    launch_pdl(k_coarsest<T>, 1, 32, 0, s, ainv, f, x, fs);
}

void launch_resid64(const LevelP<double>& P, const double* f, const double* x, double* r, float* fin, int64_t fin_ld,
                    int64_t fin_fs, double* part, int nblk, double* out, cudaStream_t s) {
    k_resid64<<<nblk, 256, 0, s>>>(P, f, x, r, fin, fin_ld, fin_fs, part);
    k_reduce_parts<<<1, 256, 0, s>>>(part, nblk, out);
}
void launch_norms64(const LevelP<double>& P, const double* x, double* part, int nblk, double* out, cudaStream_t s) {
    k_norms64<<<nblk, 256, 0, s>>>(P, x, part);
    k_reduce_parts<<<1, 256, 0, s>>>(part, nblk, out);
}
void launch_refine_update(const LevelP<double>& P, double* x, const float* d, int64_t d_ld, int64_t d_fs,
                          cudaStream_t s) {
    k_refine_update<<<grid2(P.n + 1, P.n + 1, kBlk2), kBlk2, 0, s>>>(P, x, d, d_ld, d_fs);
}
void launch_to_f32(int n, const double* v, int64_t v_ld, int64_t v_fs, float* out, int64_t o_ld, int64_t o_fs,
                   double s_l, cudaStream_t s) {
    k_to_f32<<<grid2(n + 1, n + 1, kBlk2), kBlk2, 0, s>>>(n, v, v_ld, v_fs, out, o_ld, o_fs, s_l);
}
void launch_to_f64(int n, const float* v, int64_t v_ld, int64_t v_fs, double* out, int64_t o_ld, int64_t o_fs,
                   double s_l, cudaStream_t s) {
    k_to_f64<<<grid2(n + 1, n + 1, kBlk2), kBlk2, 0, s>>>(n, v, v_ld, v_fs, out, o_ld, o_fs, s_l);
}
void launch_rhs(const LevelP<double>& P, const double* yD, double* f, cudaStream_t s) {
    k_rhs<<<grid2(P.n + 1, P.n + 1, kBlk2), kBlk2, 0, s>>>(P, yD, f);
}

#define AAOMG_INST(T)                                                                                          \
    template void launch_resid_hat<T>(const LevelP<T>&, const T*, const T*, T*, cudaStream_t);                \
    template void launch_ne_update<T>(const LevelP<T>&, T*, const T*, cudaStream_t);                          \
    template void launch_lsgs_phase<T>(const LevelP<T>&, int, int, T*, T*, cudaStream_t);                     \
    template void launch_cgs_phase<T>(const LevelP<T>&, int, const T*, T*, cudaStream_t);                      \
    template void launch_restrict<T>(const LevelP<T>&, const LevelP<T>&, const T*, const T*, T*, T*,          \
                                     cudaStream_t);                                                           \
    template void launch_prolong<T>(const LevelP<T>&, const LevelP<T>&, const T*, T*, cudaStream_t);          \
    template void launch_coarsest<T>(const double*, const T*, T*, int64_t, cudaStream_t);
AAOMG_INST(float)
AAOMG_INST(double)

}  // namespace aaomg

// ------------------------------------------------------ dense coarse map --
namespace aaomg {
namespace {

// x = B f, B dense row-major m x m: one warp per output row, f staged in
// shared memory; the row sum is reduced in a fixed lane order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply(const T* __restrict__ B, int m, const T* __restrict__ f,
                                                     T* __restrict__ x) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* fs = reinterpret_cast<T*>(smem_raw);
    for (int t = threadIdx.x; t < m; t += blockDim.x) fs[t] = f[t];
    __syncthreads();
    int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= m) return;
    const T* row = B + (int64_t)r * m;
    T s = T(0);
    for (int k = lane; k < m; k += 32) s += row[k] * fs[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] = s;
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}

}  // namespace

template <typename T>
void launch_dense_apply(const T* B, int m, const T* f, T* x, cudaStream_t s) {
    launch_pdl(k_dense_apply<T>, (m + 7) / 8, 256, m * sizeof(T), s, B, m, f, x);
}
void launch_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
    k_f64_to_f32<<<1024, 256, 0, s>>>(a, b, n);
}
template void launch_dense_apply<float>(const float*, int, const float*, float*, cudaStream_t);
template void launch_dense_apply<double>(const double*, int, const double*, double*, cudaStream_t);

}  // namespace aaomg

// ------------------------------------------------------------- adjoint --
namespace aaomg {
namespace {

// u = lambda / alpha
__global__ void k_control(int64_t nn, const double* __restrict__ x, double invalpha, double* __restrict__ u) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x)
        u[t] = x[nn + t] * invalpha;
}

// g = (0, ubar / alpha)
__global__ void k_adjoint_rhs(int64_t nn, const double* __restrict__ ubar, double invalpha, double* __restrict__ g) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        g[t] = 0.0;
        g[nn + t] = ubar[t] * invalpha;
    }
}

// gyD = M z_y, and per-block partials of ubar . lambda and (M z_lambda) . lambda
__global__ void k_adjoint_terms(LevelP<double> P, const double* __restrict__ x, const double* __restrict__ ubar,
                                const double* __restrict__ z, double* __restrict__ gyD, double* __restrict__ part) {
    const int64_t nn = (int64_t)(P.n + 1) * (P.n + 1);
    double a = 0.0, b = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(t / (P.n + 1)), i = (int)(t - (int64_t)j * (P.n + 1));
        double m[7], kd[7], zy[7], zl[7];
        row_coeffs(P, i, j, m, kd);
        load7(P, z, i, j, zy);
        load7(P, z + P.fs, i, j, zl);
        double mzy = 0.0, mzl = 0.0;
        for (int o = 0; o < 7; ++o) {
            mzy += m[o] * zy[o];
            mzl += m[o] * zl[o];
        }
        gyD[t] = mzy;
        double lam = x[nn + t];
        a += ubar[t] * lam;
        b += mzl * lam;
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

}  // namespace

void launch_control(int64_t nn, const double* x, double alpha, double* u, cudaStream_t s) {
    k_control<<<608, 256, 0, s>>>(nn, x, 1.0 / alpha, u);
}
void launch_adjoint_rhs(int64_t nn, const double* ubar, double alpha, double* g, cudaStream_t s) {
    k_adjoint_rhs<<<608, 256, 0, s>>>(nn, ubar, 1.0 / alpha, g);
}
void launch_adjoint_terms(const LevelP<double>& P, const double* x, const double* ubar, const double* z, double* gyD,
                          double* part, int nblk, double* out, cudaStream_t s) {
    k_adjoint_terms<<<nblk, 256, 0, s>>>(P, x, ubar, z, gyD, part);
    k_reduce_parts<<<1, 256, 0, s>>>(part, nblk, out);
}

}  // namespace aaomg
