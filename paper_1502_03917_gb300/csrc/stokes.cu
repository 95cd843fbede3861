// stokes.cu -- the Stokes control solver (include/aaomg_stokes.h): Taylor-Hood
// discretisation of the optimality system of eq. (mp3), assembled on the host,
// and its all-at-once multigrid iteration (section 2) on the GPU in FP64.
//
// Storage.  Every level keeps A with its rows in the LSGS visiting order:
// block by block (v_1, v_2, p, lambda_1, lambda_2, mu), colour by colour, each
// colour padded to whole warps and sorted by row length inside (vertex nodes
// of the P2 grid have 45 entries, edge nodes 22, pressure rows 38).  A row's
// entries (column, A_ij and A_ij / L_jj, the weight of the gather of
// Algorithm 2) are contiguous, their count padded to a multiple of 8, and 8
// lanes of a warp share a row, so that the lanes read consecutive words.
// Vectors stay in the natural block order of the ABI.
//
// Kernels.  A colour of LSGS is one launch over its rows (gather q = sum_j
// A_ij r_j / L_jj, p = q / N_ii, x_i += p, scatter r_j -= A_ji p; the rows of a
// colour touch disjoint entries of r, so the updates of a launch commute and
// each row's scatter reuses the values its gather loaded); on levels up to 4
// (at most 4422 unknowns) a whole smoothing call runs in one single-block
// launch with x and r in shared memory and a barrier between colours.
// Residual, restriction (the transposes of the embeddings) and prolongation are
// row-parallel kernels over CSR matrices; the coarsest level applies a
// precomputed dense solution operator.  The coarse-grid correction of level 5
// or 4 (the gamma iterations of all coarser levels from zero, a fixed linear
// map of the restricted defect) is applied as one dense matrix built at
// set-up by running those iterations on every unit vector (multi-vector forms
// of the same kernels), so the cycle does not pay the colour phases' launch
// latency on the coarse levels.  Launches use programmatic dependent launch;
// one cycle is recorded once into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "aaomg_stokes.h"
#include "errors.h"
#include "pdl.h"
#include "trace.h"

namespace {

using aaomg::set_error;
using aaomg::TraceRange;
using aaomg::launch_pdl;
using aaomg::pdl_wait;

#define SCK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return set_error(AAOMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

constexpr int kGroup = 8;  // lanes per row of A
constexpr int kVCol = 19;  // colours (a + 7 b) mod 19 of the P2 half-step grid
constexpr int kPCol = 7;   // colours (i + 2 j) mod 7 of the vertices
constexpr int kSmallThreads = 1024;
constexpr int kNormBlocks = 296;
constexpr int kMaxPerLane = 6;  // entries of the longest row (45) per lane, rounded up

// ============================================================ kernels ==

// A in the LSGS visiting order: row `row` holds the entries [start, start +
// len) of col / a / al, its length padded to a multiple of kGroup (padding:
// column 0, weight 0).  Rows are padded per colour to whole warps (rowid -1).
struct RowsDev {
    int m;                   // unknowns
    int nrows;               // rows in the visiting order, padding included
    const int* rowid;        // natural index of each row, -1 for padding
    const int* len;          // padded length of each row
    const long long* start;  // first entry of each row
    const int* col;          // natural column of each entry
    const double* a;         // A_ij
    const double* al;        // A_ij / L_jj
    const double* invN;      // 1 / N_ii per row
    const double* invL;      // 1 / L_ii, natural order
};

// A row's data, loaded together (none of these loads waits for another):
// natural index (-1: padding or no row), padded length, first entry, 1 / N_ii.
struct RowHead {
    int i, n;
    long long b;
    double invN;
};

__device__ __forceinline__ RowHead row_head(const RowsDev& S, int row) {
    RowHead h{-1, 0, 0, 0.0};
    if (row >= 0 && row < S.nrows) {
        h.i = S.rowid[row];
        h.n = S.len[row];
        h.b = S.start[row];
        h.invN = S.invN[row];
    }
    if (h.i < 0) h.n = 0;
    return h;
}

// The kGroup lanes of a group (aligned within a warp) share one row: lane l
// takes the entries l, l + kGroup, ...; all its loads are issued before their
// first use, the partial sums meet by shuffles.  Every lane of the group gets
// the row's sum; an empty row (n = 0) gives zero (every lane of the warp still
// takes part in the shuffles).
__device__ __forceinline__ double group_dot(const RowsDev& S, const RowHead& h, int lane, const double* v,
                                           const double* w) {
    double acc = 0.0;
    int c[kMaxPerLane];
    double wk[kMaxPerLane];
#pragma unroll
    for (int u = 0; u < kMaxPerLane; ++u) {
        const bool on = lane + u * kGroup < h.n;
        c[u] = on ? S.col[h.b + lane + u * kGroup] : 0;
        wk[u] = on ? w[h.b + lane + u * kGroup] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kMaxPerLane; ++u) acc += wk[u] * v[c[u]];
#pragma unroll
    for (int o = kGroup / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, kGroup);
    return acc;
}

// one row of Algorithm 2 on (x, r) (global or shared memory) by a group:
// gather q = sum_j A_ij r_j / L_jj, p = q / N_ii, x_i += p, scatter
// r_j -= A_ji p (A symmetric: the row's own entries).  No other row of the
// colour touches these r_j, so the scatter reuses the gathered values and
// indices: a row costs three dependent memory round trips (its head, its
// entries, the residual entries they address).  row < 0 or a padding row:
// shuffles only.
__device__ __forceinline__ void group_lsgs(const RowsDev& S, int row, int lane, double* x, double* r) {
    const RowHead h = row_head(S, row);
    int c[kMaxPerLane];
    double wl[kMaxPerLane], ak[kMaxPerLane], rk[kMaxPerLane];
#pragma unroll
    for (int u = 0; u < kMaxPerLane; ++u) {
        const bool on = lane + u * kGroup < h.n;
        c[u] = on ? S.col[h.b + lane + u * kGroup] : -1;
        wl[u] = on ? S.al[h.b + lane + u * kGroup] : 0.0;
        ak[u] = on ? S.a[h.b + lane + u * kGroup] : 0.0;
    }
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < kMaxPerLane; ++u) rk[u] = c[u] >= 0 ? r[c[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < kMaxPerLane; ++u) acc += wl[u] * rk[u];
#pragma unroll
    for (int o = kGroup / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, kGroup);
    if (h.i < 0) return;
    const double p = acc * h.invN;
    if (lane == 0) x[h.i] += p;
#pragma unroll
    for (int u = 0; u < kMaxPerLane; ++u)
        if (c[u] >= 0 && ak[u] != 0.0) r[c[u]] = rk[u] - ak[u] * p;
}

// the rows [r0, r0 + cnt) of one colour, a group per row; vector blockIdx.y
// of multi-vectors at stride m
__global__ void k_st_phase(RowsDev S, int r0, int cnt, double* x, double* r) {
    pdl_wait();
    x += (size_t)blockIdx.y * S.m;
    r += (size_t)blockIdx.y * S.m;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t / kGroup, lane = t % kGroup;
    group_lsgs(S, g < cnt ? r0 + g : -1, lane, x, r);
}

// r = f - A x over all rows
__global__ void k_st_resid(RowsDev S, const double* f, const double* x, double* r) {
    pdl_wait();
    const size_t vo = (size_t)blockIdx.y * S.m;
    f += vo;
    x += vo;
    r += vo;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = t / kGroup, lane = t % kGroup;
    const RowHead h = row_head(S, row);
    const int i = h.i;
    const double s = group_dot(S, h, lane, x, S.a);
    if (i >= 0 && lane == 0) r[i] = f[i] - s;
}

// Algorithm 1, first loop: p_i = tau (sum_j A_ij r_j / L_jj) / L_ii
__global__ void k_st_ne_p(RowsDev S, double tau, const double* r, double* p) {
    pdl_wait();
    const size_t vo = (size_t)blockIdx.y * S.m;
    r += vo;
    p += vo;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = t / kGroup, lane = t % kGroup;
    const RowHead h = row_head(S, row);
    const int i = h.i;
    const double q = group_dot(S, h, lane, r, S.al);
    if (i >= 0 && lane == 0) p[i] = tau * q * S.invL[i];
}

// Algorithm 1, second loop (gather form, A symmetric): x_i += p_i,
// r_i -= sum_j A_ij p_j
__global__ void k_st_ne_update(RowsDev S, const double* p, double* x, double* r) {
    pdl_wait();
    const size_t vo = (size_t)blockIdx.y * S.m;
    p += vo;
    x += vo;
    r += vo;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = t / kGroup, lane = t % kGroup;
    const RowHead h = row_head(S, row);
    const int i = h.i;
    const double s = group_dot(S, h, lane, p, S.a);
    if (i >= 0 && lane == 0) {
        x[i] += p[i];
        r[i] -= s;
    }
}

// A whole smoothing call on a small level in one block: x and r (and the NE
// update p) in shared memory, a barrier between dependent passes, a group of
// kGroup lanes per row; block b works on vector b of a multi-vector.
// smoother: 0 NE, 1 LSGS, 2 sLSGS.
__global__ void __launch_bounds__(kSmallThreads)
    k_st_small(RowsDev S, const int* __restrict__ poff, int nph, int smoother, int steps, double tau,
               const double* __restrict__ f, double* __restrict__ x) {
    pdl_wait();
    extern __shared__ double sm[];
    double* xs = sm;
    double* rs = sm + S.m;
    double* ps = sm + 2 * S.m;
    f += (size_t)blockIdx.x * S.m;
    x += (size_t)blockIdx.x * S.m;
    const int g = threadIdx.x, G = blockDim.x;
    const int grp = g / kGroup, lane = g % kGroup, NG = G / kGroup;
    const int nrow_pad = (S.nrows + NG - 1) / NG * NG;  // whole rounds: every group meets the shuffles
    for (int i = g; i < S.m; i += G) xs[i] = x[i];
    __syncthreads();
    for (int row = grp; row < nrow_pad; row += NG) {
        const RowHead h = row_head(S, row);
        const int i = h.i;
        const double s = group_dot(S, h, lane, xs, S.a);
        if (i >= 0 && lane == 0) rs[i] = f[i] - s;
    }
    __syncthreads();
    for (int m = 0; m < steps; ++m) {
        if (smoother == 0) {
            for (int row = grp; row < nrow_pad; row += NG) {
                const RowHead h = row_head(S, row);
                const int i = h.i;
                const double q = group_dot(S, h, lane, rs, S.al);
                if (i >= 0 && lane == 0) ps[i] = tau * q * S.invL[i];
            }
            __syncthreads();
            for (int row = grp; row < nrow_pad; row += NG) {
                const RowHead h = row_head(S, row);
                const int i = h.i;
                const double s = group_dot(S, h, lane, ps, S.a);
                if (i >= 0 && lane == 0) {
                    xs[i] += ps[i];
                    rs[i] -= s;
                }
            }
            __syncthreads();
            continue;
        }
        for (int pass = 0; pass < (smoother == 2 ? 2 : 1); ++pass)
            for (int q = 0; q < nph; ++q) {
                const int ph = pass == 0 ? q : nph - 1 - q;
                const int r0 = poff[ph], cnt = poff[ph + 1] - r0;
                const int cnt_pad = (cnt + NG - 1) / NG * NG;
                for (int k = grp; k < cnt_pad; k += NG) group_lsgs(S, k < cnt ? r0 + k : -1, lane, xs, rs);
                __syncthreads();
            }
    }
    for (int i = g; i < S.m; i += G) x[i] = xs[i];
}

struct CsrDev {
    const int* ptr;
    const int* col;
    const double* val;
};

// block layout of a level's vectors: v_1, v_2, p, lambda_1, lambda_2, mu
struct Blocks {
    int nv, np;
    __host__ __device__ int off(int b) const {
        return b < 2 ? b * nv : b == 2 ? 2 * nv : b < 5 ? 2 * nv + np + (b - 3) * nv : 4 * nv + np;
    }
    __host__ __device__ bool vel(int b) const { return b != 2 && b != 5; }
    __host__ __device__ int m() const { return 4 * nv + 2 * np; }
};

__device__ __forceinline__ void locate(const Blocks& B, int u, int& blk, int& j) {
    if (u < 2 * B.nv) {
        blk = u / B.nv;
        j = u - blk * B.nv;
    } else if (u < 2 * B.nv + B.np) {
        blk = 2;
        j = u - 2 * B.nv;
    } else if (u < 4 * B.nv + B.np) {
        const int v = u - 2 * B.nv - B.np;
        blk = 3 + v / B.nv;
        j = v - (blk - 3) * B.nv;
    } else {
        blk = 5;
        j = u - 4 * B.nv - B.np;
    }
}

// fc = I^T rf, block by block: R2 = P2^T on velocities, R1 = P1^T on pressures
__global__ void k_st_restrict(Blocks Bf, Blocks Bc, CsrDev R2, CsrDev R1, const double* __restrict__ rf,
                              double* __restrict__ fc, double* __restrict__ xc) {
    pdl_wait();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= Bc.m()) return;
    rf += (size_t)blockIdx.y * Bf.m();  // vector blockIdx.y of multi-vectors
    fc += (size_t)blockIdx.y * Bc.m();
    xc += (size_t)blockIdx.y * Bc.m();
    int blk, j;
    locate(Bc, u, blk, j);
    const CsrDev& R = Bc.vel(blk) ? R2 : R1;
    const double* src = rf + Bf.off(blk);
    double s = 0.0;
    for (int k = R.ptr[j]; k < R.ptr[j + 1]; ++k) s += R.val[k] * src[R.col[k]];
    fc[u] = s;
    xc[u] = 0.0;
}

// xf += I xc, block by block
__global__ void k_st_prolong(Blocks Bf, Blocks Bc, CsrDev P2, CsrDev P1, const double* __restrict__ xc,
                             double* __restrict__ xf) {
    pdl_wait();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= Bf.m()) return;
    xc += (size_t)blockIdx.y * Bc.m();
    xf += (size_t)blockIdx.y * Bf.m();
    int blk, j;
    locate(Bf, u, blk, j);
    const CsrDev& P = Bf.vel(blk) ? P2 : P1;
    const double* src = xc + Bc.off(blk);
    double s = 0.0;
    for (int k = P.ptr[j]; k < P.ptr[j + 1]; ++k) s += P.val[k] * src[P.col[k]];
    xf[u] += s;
}

// coarsest level: x = G f (G the solution operator with int p = int mu = 0);
// block b solves for vector b of a multi-vector
__global__ void k_st_coarse(int m, const double* __restrict__ G, const double* __restrict__ f, double* __restrict__ x) {
    pdl_wait();
    f += (size_t)blockIdx.x * m;
    x += (size_t)blockIdx.x * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += G[(size_t)i * m + j] * f[j];
        x[i] = s;
    }
}

// x = B f with the dense map B of the coarse levels (column-major, m x m):
// block (bx, by) sums the columns [by ck, (by + 1) ck) for the rows of tile bx
// into part[by]; k_st_dense_sum adds the partial sums in a fixed order
constexpr int kDenseChunks = 32;
__global__ void k_st_dense(int m, int ck, const double* __restrict__ B, const double* __restrict__ f,
                           double* __restrict__ part) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j0 = blockIdx.y * ck, j1 = min(m, j0 + ck);
    double s0 = 0.0, s1 = 0.0;
    int j = j0;
    for (; j + 1 < j1; j += 2) {
        s0 += B[(size_t)j * m + i] * f[j];
        s1 += B[(size_t)(j + 1) * m + i] * f[j + 1];
    }
    if (j < j1) s0 += B[(size_t)j * m + i] * f[j];
    part[(size_t)blockIdx.y * m + i] = s0 + s1;
}

__global__ void k_st_dense_sum(int m, const double* __restrict__ part, double* __restrict__ x) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int c = 0; c < kDenseChunks; ++c) s += part[(size_t)c * m + i];
    x[i] = s;
}

// the unit vectors e_{j0} .. e_{j0 + nc - 1} of R^m as a multi-vector
__global__ void k_st_identity(int m, int j0, int nc, double* __restrict__ e) {
    pdl_wait();
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (size_t)m * nc) e[t] = ((size_t)j0 + t / m == t % m) ? 1.0 : 0.0;
}

// f = (M v_D, 0, 0, 0): Mf holds the interior rows of the full P2 mass matrix
__global__ void k_st_rhs(Blocks B, int ng2, CsrDev Mf, const double* __restrict__ vD, double* __restrict__ f) {
    pdl_wait();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.m()) return;
    double s = 0.0;
    if (u < 2 * B.nv) {
        const int c = u / B.nv, i = u - c * B.nv;
        for (int k = Mf.ptr[i]; k < Mf.ptr[i + 1]; ++k) s += Mf.val[k] * vD[(size_t)c * ng2 + Mf.col[k]];
    }
    f[u] = s;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// the means of p and mu: out[0] = sum_q w_q p_q, out[1] = sum_q w_q mu_q
// (sum_q w_q = |Omega| = 1); one block
__global__ void k_st_means(Blocks B, const double* __restrict__ w, const double* __restrict__ x, double* out) {
    pdl_wait();
    double sp = 0.0, sm = 0.0;
    for (int q = threadIdx.x; q < B.np; q += blockDim.x) {
        sp += w[q] * x[B.off(2) + q];
        sm += w[q] * x[B.off(5) + q];
    }
    sp = block_sum(sp);
    sm = block_sum(sm);
    if (threadIdx.x == 0) {
        out[0] = sp;
        out[1] = sm;
    }
}

// u = lambda / alpha: the control (both components) from the adjoint velocity
__global__ void k_st_control(Blocks B, double inv_alpha, const double* __restrict__ x, double* __restrict__ u) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 * B.nv) u[t] = x[B.off(3) + t] * inv_alpha;
}

__global__ void k_st_shift(Blocks B, const double* __restrict__ means, double* __restrict__ x) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B.np) return;
    x[B.off(2) + q] -= means[0];
    x[B.off(5) + q] -= means[1];
}

// partial sums of the norms: mode 0: part = (sum v_i^2 / L_i, sum g_i^2 / L_i)
// (residual and right-hand side in ||.||_{L^-1}); mode 1: part = (sum L_i
// (v_i - s_i)^2, sum (v_i - s_i)^2 / L_i) with s the mean shift of p and mu
// (means may be null: no shift)
__global__ void k_st_norm_part(Blocks B, int mode, const double* __restrict__ invL, const double* __restrict__ v,
                               const double* __restrict__ g, const double* __restrict__ means, double* part) {
    pdl_wait();
    double s0 = 0.0, s1 = 0.0;
    const int m = B.m();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double vi = v[i];
        if (mode == 0) {
            s0 += vi * vi * invL[i];
            if (g) s1 += g[i] * g[i] * invL[i];
        } else {
            if (means) {
                if (i >= B.off(2) && i < B.off(2) + B.np) vi -= means[0];
                if (i >= B.off(5)) vi -= means[1];
            }
            s0 += vi * vi / invL[i];
            s1 += vi * vi * invL[i];
        }
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

__global__ void k_st_norm_final(const double* __restrict__ part, int nblk, double* out) {
    pdl_wait();
    double s0 = 0.0, s1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        s0 += part[2 * b];
        s1 += part[2 * b + 1];
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) {
        out[0] = s0;
        out[1] = s1;
    }
}

// ====================================================== host assembly ==

// Rows with a small fixed capacity; an entry added twice is summed.
struct Rows {
    int cap = 0;
    std::vector<int> cnt, col;
    std::vector<double> val;
    void init(int nrows, int c) {
        cap = c;
        cnt.assign(nrows, 0);
        col.assign((size_t)nrows * c, 0);
        val.assign((size_t)nrows * c, 0.0);
    }
    bool add(int r, int c, double v) {
        int* cs = &col[(size_t)r * cap];
        double* vs = &val[(size_t)r * cap];
        for (int k = 0; k < cnt[r]; ++k)
            if (cs[k] == c) {
                vs[k] += v;
                return true;
            }
        if (cnt[r] == cap) return false;
        cs[cnt[r]] = c;
        vs[cnt[r]] = v;
        ++cnt[r];
        return true;
    }
    int nrows() const { return (int)cnt.size(); }
    double get(int r, int c) const {
        for (int k = 0; k < cnt[r]; ++k)
            if (col[(size_t)r * cap + k] == c) return val[(size_t)r * cap + k];
        return 0.0;
    }
};

// Local P2 / P1 matrices of a triangle with counterclockwise vertices, local
// P2 nodes 0..2 the vertices and 3, 4, 5 the midpoints of edges (0,1), (1,2),
// (2,0).  Integrals by the 7-point rule of degree 5 on the triangle (the
// integrands have degree 4 at most, so the rule is exact): the centroid, and
// the two orbits (a, a, 1-2a) with a = (6 -+ sqrt 15) / 21.
struct Local {
    double M[6][6], K[6][6], D[2][3][6];  // D[c][q][t] = -int l_q d_c phi_t
};

void local_matrices(const double px[3], const double py[3], Local& E) {
    const double det = (px[1] - px[0]) * (py[2] - py[0]) - (px[2] - px[0]) * (py[1] - py[0]);
    const double area = std::fabs(det) / 2.0;
    double gx[3], gy[3];  // gradients of the barycentric coordinates
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        gx[a] = (py[b] - py[c]) / det;
        gy[a] = (px[c] - px[b]) / det;
    }
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    double qp[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                       {a1, a1, 1 - 2 * a1}, {a1, 1 - 2 * a1, a1}, {1 - 2 * a1, a1, a1},
                       {a2, a2, 1 - 2 * a2}, {a2, 1 - 2 * a2, a2}, {1 - 2 * a2, a2, a2}};
    const double qw[7] = {9.0 / 40, w1, w1, w1, w2, w2, w2};
    static const int EG[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    std::memset(&E, 0, sizeof(E));
    for (int k = 0; k < 7; ++k) {
        const double* l = qp[k];
        double phi[6], dx[6], dy[6];
        for (int a = 0; a < 3; ++a) {
            phi[a] = l[a] * (2.0 * l[a] - 1.0);
            dx[a] = (4.0 * l[a] - 1.0) * gx[a];
            dy[a] = (4.0 * l[a] - 1.0) * gy[a];
        }
        for (int e = 0; e < 3; ++e) {
            const int a = EG[e][0], b = EG[e][1];
            phi[3 + e] = 4.0 * l[a] * l[b];
            dx[3 + e] = 4.0 * (l[b] * gx[a] + l[a] * gx[b]);
            dy[3 + e] = 4.0 * (l[b] * gy[a] + l[a] * gy[b]);
        }
        const double w = qw[k] * area;
        for (int s = 0; s < 6; ++s)
            for (int t = 0; t < 6; ++t) {
                E.M[s][t] += w * phi[s] * phi[t];
                E.K[s][t] += w * (dx[s] * dx[t] + dy[s] * dy[t]);
            }
        for (int q = 0; q < 3; ++q)
            for (int t = 0; t < 6; ++t) {
                E.D[0][q][t] -= w * l[q] * dx[t];
                E.D[1][q][t] -= w * l[q] * dy[t];
            }
    }
}

// one level of the hierarchy on the host
struct HostLevel {
    int n = 0, ng = 0, nv = 0, np = 0, m = 0;
    Rows M, K, Mf, D[2], DT[2];  // Mf: interior rows, columns over all ng^2 half-step nodes
    std::vector<double> Ld, Nd, w;
    int vidx(int a, int b) const { return (a < 1 || b < 1 || a > ng - 2 || b > ng - 2) ? -1 : (b - 1) * (ng - 2) + a - 1; }
    Blocks blocks() const { return Blocks{nv, np}; }
};

bool assemble(int n, double alpha, HostLevel& H) {
    H.n = n;
    H.ng = 2 * n + 1;
    H.nv = (H.ng - 2) * (H.ng - 2);
    H.np = (n + 1) * (n + 1);
    H.m = 4 * H.nv + 2 * H.np;
    const double h = 1.0 / n;
    static const int TV[2][3][2] = {{{0, 0}, {1, 0}, {1, 1}}, {{0, 0}, {1, 1}, {0, 1}}};
    static const int EG[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    Local E[2];
    for (int t = 0; t < 2; ++t) {
        double px[3], py[3];
        for (int a = 0; a < 3; ++a) {
            px[a] = TV[t][a][0] * h;
            py[a] = TV[t][a][1] * h;
        }
        local_matrices(px, py, E[t]);
    }
    H.M.init(H.nv, 19);
    H.K.init(H.nv, 19);
    H.Mf.init(H.nv, 19);
    H.D[0].init(H.np, 19);
    H.D[1].init(H.np, 19);
    H.w.assign(H.np, 0.0);
    bool ok = true;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            for (int t = 0; t < 2; ++t) {
                int ga[6], gb[6], q[3];
                for (int a = 0; a < 3; ++a) {
                    ga[a] = 2 * (i + TV[t][a][0]);
                    gb[a] = 2 * (j + TV[t][a][1]);
                    q[a] = (j + TV[t][a][1]) * (n + 1) + i + TV[t][a][0];
                    H.w[q[a]] += h * h / 6.0;  // int of a hat function over the triangle: |T| / 3
                }
                for (int e = 0; e < 3; ++e) {
                    ga[3 + e] = (ga[EG[e][0]] + ga[EG[e][1]]) / 2;
                    gb[3 + e] = (gb[EG[e][0]] + gb[EG[e][1]]) / 2;
                }
                int vi[6];
                for (int s = 0; s < 6; ++s) vi[s] = H.vidx(ga[s], gb[s]);
                for (int s = 0; s < 6; ++s) {
                    if (vi[s] < 0) continue;
                    for (int u = 0; u < 6; ++u) {
                        ok = ok && H.Mf.add(vi[s], gb[u] * H.ng + ga[u], E[t].M[s][u]);
                        if (vi[u] < 0) continue;
                        ok = ok && H.M.add(vi[s], vi[u], E[t].M[s][u]) && H.K.add(vi[s], vi[u], E[t].K[s][u]);
                    }
                }
                for (int a = 0; a < 3; ++a)
                    for (int u = 0; u < 6; ++u)
                        if (vi[u] >= 0)
                            ok = ok && H.D[0].add(q[a], vi[u], E[t].D[0][a][u]) && H.D[1].add(q[a], vi[u], E[t].D[1][a][u]);
            }
    if (!ok) return false;
    for (int c = 0; c < 2; ++c) {
        H.DT[c].init(H.nv, 7);
        for (int q = 0; q < H.np; ++q)
            for (int k = 0; k < H.D[c].cnt[q]; ++k)
                ok = ok && H.DT[c].add(H.D[c].col[(size_t)q * 19 + k], q, H.D[c].val[(size_t)q * 19 + k]);
    }
    if (!ok) return false;
    // L of section 2 and N_ii of Algorithm 2
    const Blocks B = H.blocks();
    H.Ld.assign(H.m, 0.0);
    std::vector<double> W(H.nv);
    for (int i = 0; i < H.nv; ++i) W[i] = H.M.get(i, i) + std::sqrt(alpha) * H.K.get(i, i);
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < H.nv; ++i) {
            H.Ld[B.off(c) + i] = W[i];
            H.Ld[B.off(3 + c) + i] = W[i] / alpha;
        }
    for (int q = 0; q < H.np; ++q) {
        double s = 0.0;
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < H.D[c].cnt[q]; ++k) {
                const double d = H.D[c].val[(size_t)q * 19 + k];
                s += d * d / W[H.D[c].col[(size_t)q * 19 + k]];
            }
        H.Ld[B.off(2) + q] = alpha * s;
        H.Ld[B.off(5) + q] = s;
    }
    return true;
}

// the entries of row u of A (natural order), eq. (mp3)
void a_row(const HostLevel& H, double alpha, int u, std::vector<int>& cols, std::vector<double>& vals) {
    cols.clear();
    vals.clear();
    const Blocks B = H.blocks();
    auto put = [&](const Rows& R, int r, int off, double scale) {
        for (int k = 0; k < R.cnt[r]; ++k) {
            cols.push_back(off + R.col[(size_t)r * R.cap + k]);
            vals.push_back(scale * R.val[(size_t)r * R.cap + k]);
        }
    };
    int blk = 0, j = u;
    for (int b = 5; b >= 0; --b)
        if (u >= B.off(b)) {
            blk = b;
            j = u - B.off(b);
            break;
        }
    switch (blk) {
    case 0:
    case 1:  // v_c rows: M v_c + K lambda_c + D_c^T mu
        put(H.M, j, B.off(blk), 1.0);
        put(H.K, j, B.off(3 + blk), 1.0);
        put(H.DT[blk], j, B.off(5), 1.0);
        break;
    case 2:  // p rows: D lambda
        put(H.D[0], j, B.off(3), 1.0);
        put(H.D[1], j, B.off(4), 1.0);
        break;
    case 3:
    case 4:  // lambda_c rows: K v_c + D_c^T p - alpha^-1 M lambda_c
        put(H.K, j, B.off(blk - 3), 1.0);
        put(H.DT[blk - 3], j, B.off(2), 1.0);
        put(H.M, j, B.off(blk), -1.0 / alpha);
        break;
    default:  // mu rows: D v
        put(H.D[0], j, B.off(0), 1.0);
        put(H.D[1], j, B.off(1), 1.0);
        break;
    }
}

// canonical embeddings into level f from level c = f - 1: P2 on the interior
// nodes of the half-step grids (the coarse P2 function evaluated at the fine
// node through the coarse triangle holding it), P1 on the vertices (linear
// interpolation along the fine vertex's coarse edge)
struct Csr {
    std::vector<int> ptr, col;
    std::vector<double> val;
    int nrows = 0, ncols = 0;
};

Csr embed_p2(const HostLevel& F, const HostLevel& C) {
    Csr P;
    P.nrows = F.nv;
    P.ncols = C.nv;
    P.ptr.push_back(0);
    static const int LOWER[6][2] = {{0, 0}, {2, 0}, {2, 2}, {1, 0}, {2, 1}, {1, 1}};  // coarse half-step offsets
    static const int UPPER[6][2] = {{0, 0}, {2, 2}, {0, 2}, {1, 1}, {1, 2}, {0, 1}};
    static const int EG[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int b = 1; b <= F.ng - 2; ++b)
        for (int a = 1; a <= F.ng - 2; ++a) {
            const int I = a / 4, J = b / 4;  // coarse cell; a, b <= 4 nc - 1
            const double s = (a - 4 * I) / 4.0, t = (b - 4 * J) / 4.0;
            const bool lower = s >= t;
            const double lam[3] = {lower ? 1.0 - s : 1.0 - t, lower ? s - t : s, lower ? t : t - s};
            const int(*nodes)[2] = lower ? LOWER : UPPER;
            for (int k = 0; k < 6; ++k) {
                const double wgt = k < 3 ? lam[k] * (2.0 * lam[k] - 1.0) : 4.0 * lam[EG[k - 3][0]] * lam[EG[k - 3][1]];
                const int cv = C.vidx(2 * I + nodes[k][0], 2 * J + nodes[k][1]);
                if (wgt != 0.0 && cv >= 0) {
                    P.col.push_back(cv);
                    P.val.push_back(wgt);
                }
            }
            P.ptr.push_back((int)P.col.size());
        }
    return P;
}

Csr embed_p1(const HostLevel& F, const HostLevel& C) {
    Csr P;
    P.nrows = F.np;
    P.ncols = C.np;
    P.ptr.push_back(0);
    const int nc = C.n;
    for (int j = 0; j <= F.n; ++j)
        for (int i = 0; i <= F.n; ++i) {
            // the fine vertex is a coarse vertex or the midpoint of a coarse
            // edge: horizontal, vertical or the SW-NE diagonal
            const int i0 = i / 2, j0 = j / 2, i1 = (i + 1) / 2, j1 = (j + 1) / 2;
            if (i0 == i1 && j0 == j1) {
                P.col.push_back(j0 * (nc + 1) + i0);
                P.val.push_back(1.0);
            } else {
                P.col.push_back(j0 * (nc + 1) + i0);
                P.val.push_back(0.5);
                P.col.push_back(j1 * (nc + 1) + i1);
                P.val.push_back(0.5);
            }
            P.ptr.push_back((int)P.col.size());
        }
    return P;
}

Csr transpose(const Csr& P) {
    Csr R;
    R.nrows = P.ncols;
    R.ncols = P.nrows;
    R.ptr.assign(R.nrows + 1, 0);
    for (int c : P.col) ++R.ptr[c + 1];
    for (int r = 0; r < R.nrows; ++r) R.ptr[r + 1] += R.ptr[r];
    R.col.resize(P.col.size());
    R.val.resize(P.val.size());
    std::vector<int> fill(R.ptr.begin(), R.ptr.end() - 1);
    for (int r = 0; r < P.nrows; ++r)
        for (int k = P.ptr[r]; k < P.ptr[r + 1]; ++k) {
            R.col[fill[P.col[k]]] = r;
            R.val[fill[P.col[k]]++] = P.val[k];
        }
    return R;
}

// the LSGS visiting order: (block, colour) classes, rows of a class by
// decreasing length then increasing index
std::vector<std::vector<int>> colour_classes(const HostLevel& H, const std::vector<int>& rowlen) {
    const Blocks B = H.blocks();
    std::vector<std::vector<int>> cls;
    for (int blk = 0; blk < 6; ++blk) {
        const int ncol = B.vel(blk) ? kVCol : kPCol;
        std::vector<std::vector<int>> c(ncol);
        if (B.vel(blk)) {
            for (int b = 1; b <= H.ng - 2; ++b)
                for (int a = 1; a <= H.ng - 2; ++a) c[(a + 7 * b) % kVCol].push_back(B.off(blk) + H.vidx(a, b));
        } else {
            for (int j = 0; j <= H.n; ++j)
                for (int i = 0; i <= H.n; ++i) c[(i + 2 * j) % kPCol].push_back(B.off(blk) + j * (H.n + 1) + i);
        }
        for (auto& v : c) {
            std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return rowlen[x] > rowlen[y]; });
            cls.push_back(std::move(v));
        }
    }
    return cls;
}

// FP64 Gauss-Jordan inverse with partial pivoting (row-major, in place)
bool invert(int m, std::vector<double>& a) {
    std::vector<double> inv((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) inv[(size_t)i * m + i] = 1.0;
    for (int c = 0; c < m; ++c) {
        int p = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(a[(size_t)r * m + c]) > std::fabs(a[(size_t)p * m + c])) p = r;
        if (a[(size_t)p * m + c] == 0.0) return false;
        if (p != c)
            for (int k = 0; k < m; ++k) {
                std::swap(a[(size_t)p * m + k], a[(size_t)c * m + k]);
                std::swap(inv[(size_t)p * m + k], inv[(size_t)c * m + k]);
            }
        const double d = 1.0 / a[(size_t)c * m + c];
        for (int k = 0; k < m; ++k) {
            a[(size_t)c * m + k] *= d;
            inv[(size_t)c * m + k] *= d;
        }
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = a[(size_t)r * m + c];
            if (f == 0.0) continue;
            for (int k = 0; k < m; ++k) {
                a[(size_t)r * m + k] -= f * a[(size_t)c * m + k];
                inv[(size_t)r * m + k] -= f * inv[(size_t)c * m + k];
            }
        }
    }
    a.swap(inv);
    return true;
}

}  // namespace

// ============================================================ handle ==

struct ms_ctx {
    struct Lev {
        int n = 0, nv = 0, np = 0, m = 0, nrows = 0, nph = 0;
        std::vector<int> poff;  // phase offsets into the padded rows (host)
        int *rowid = nullptr, *len = nullptr, *col = nullptr, *poff_d = nullptr;
        long long* start = nullptr;
        double *a = nullptr, *al = nullptr, *invN = nullptr, *invL = nullptr, *w = nullptr;
        // embeddings from the next coarser level (P2, P1) and their transposes
        int *p2p = nullptr, *p2c = nullptr, *p1p = nullptr, *p1c = nullptr;
        int *r2p = nullptr, *r2c = nullptr, *r1p = nullptr, *r1c = nullptr;
        double *p2v = nullptr, *p1v = nullptr, *r2v = nullptr, *r1v = nullptr;
        double *x = nullptr, *f = nullptr, *r = nullptr, *p = nullptr;
        bool small = false;
        long long nnz = 0, stored = 0;  // entries of A; entries held (rows padded to multiples of kGroup)
        RowsDev rows() const {
            return RowsDev{m, nrows, rowid, len, start, col, a, al, invN, invL};
        }
        Blocks blocks() const { return Blocks{nv, np}; }
    };
    int L = 0;
    double alpha = 0.0;
    ms_options o{};
    int kd = 0;               // levels <= kd are replaced by their dense map (0: none)
    double* B = nullptr;      // the dense map on level kd, column-major
    double* dpart = nullptr;  // its partial sums
    int device = 0;
    std::vector<Lev> lev;  // 1..L
    double* G = nullptr;   // coarsest solution operator
    int *mfp = nullptr, *mfc = nullptr;
    double* mfv = nullptr;
    double *part = nullptr, *red = nullptr, *means = nullptr, *h_red = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t cycle_exec = nullptr;
    long long launches = 0, launches_per_cycle = 0;
    std::vector<void*> allocs;
};

namespace {

template <typename T>
int dev_upload(ms_ctx* H, T*& d, const T* src, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)&d, n * sizeof(T));
    if (e != cudaSuccess) return set_error(AAOMG_ERR_OOM, std::string("stokes workspace: ") + cudaGetErrorString(e));
    H->allocs.push_back(d);
    if (src) SCK(cudaMemcpy(d, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return AAOMG_OK;
}

template <typename T>
int dev_alloc(ms_ctx* H, T*& d, size_t n) {
    int rc = dev_upload<T>(H, d, nullptr, n);
    if (rc) return rc;
    SCK(cudaMemset(d, 0, (n ? n : 1) * sizeof(T)));
    return AAOMG_OK;
}

int upload_csr(ms_ctx* H, const Csr& P, int*& ptr, int*& col, double*& val) {
    int rc;
    if ((rc = dev_upload(H, ptr, P.ptr.data(), P.ptr.size())) || (rc = dev_upload(H, col, P.col.data(), P.col.size())) ||
        (rc = dev_upload(H, val, P.val.data(), P.val.size())))
        return rc;
    return AAOMG_OK;
}

Csr rows_to_csr(const Rows& R, int ncols) {
    Csr C;
    C.nrows = R.nrows();
    C.ncols = ncols;
    C.ptr.push_back(0);
    for (int r = 0; r < R.nrows(); ++r) {
        for (int k = 0; k < R.cnt[r]; ++k) {
            C.col.push_back(R.col[(size_t)r * R.cap + k]);
            C.val.push_back(R.val[(size_t)r * R.cap + k]);
        }
        C.ptr.push_back((int)C.col.size());
    }
    return C;
}

// the level's operator in sliced ELL, rows in the visiting order
int build_level(ms_ctx* H, const HostLevel& HL, ms_ctx::Lev& D) {
    D.n = HL.n;
    D.nv = HL.nv;
    D.np = HL.np;
    D.m = HL.m;
    // rows of A are generated on demand (a_row) rather than stored: the
    // finest levels have millions of them
    std::vector<int> rc;
    std::vector<double> rv;
    std::vector<int> rowlen(HL.m);
    std::vector<double> Nd(HL.m, 0.0), invL(HL.m);
    for (int u = 0; u < HL.m; ++u) {
        a_row(HL, H->alpha, u, rc, rv);
        rowlen[u] = (int)rc.size();
        invL[u] = 1.0 / HL.Ld[u];
        double s = 0.0;
        for (size_t k = 0; k < rc.size(); ++k) s += rv[k] * rv[k] / HL.Ld[rc[k]];
        Nd[u] = s;
    }
    const auto cls = colour_classes(HL, rowlen);
    std::vector<int> rowid;
    D.poff.assign(1, 0);
    for (const auto& c : cls) {
        for (int u : c) rowid.push_back(u);
        while (rowid.size() % 4) rowid.push_back(-1);  // four rows of kGroup lanes per warp
        D.poff.push_back((int)rowid.size());
    }
    D.nph = (int)cls.size();
    D.nrows = (int)rowid.size();
    std::vector<int> len(D.nrows, 0);
    std::vector<long long> start(D.nrows + 1, 0);
    for (int row = 0; row < D.nrows; ++row) {
        const int u = rowid[row];
        len[row] = u < 0 ? 0 : (rowlen[u] + kGroup - 1) / kGroup * kGroup;
        start[row + 1] = start[row] + len[row];
    }
    const size_t ne = (size_t)start[D.nrows];
    D.stored = (long long)ne;
    D.nnz = 0;
    for (int u = 0; u < HL.m; ++u) D.nnz += rowlen[u];
    std::vector<int> col(ne, 0);
    std::vector<double> a(ne, 0.0), al(ne, 0.0), invN(D.nrows, 0.0);
    for (int row = 0; row < D.nrows; ++row) {
        const int u = rowid[row];
        if (u < 0) continue;
        invN[row] = 1.0 / Nd[u];
        a_row(HL, H->alpha, u, rc, rv);
        for (int k = 0; k < rowlen[u]; ++k) {
            col[start[row] + k] = rc[k];
            a[start[row] + k] = rv[k];
            al[start[row] + k] = rv[k] / HL.Ld[rc[k]];
        }
    }
    int rc_;
    if ((rc_ = dev_upload(H, D.rowid, rowid.data(), rowid.size())) || (rc_ = dev_upload(H, D.len, len.data(), len.size())) ||
        (rc_ = dev_upload(H, D.start, start.data(), start.size())) || (rc_ = dev_upload(H, D.col, col.data(), col.size())) ||
        (rc_ = dev_upload(H, D.a, a.data(), a.size())) || (rc_ = dev_upload(H, D.al, al.data(), al.size())) ||
        (rc_ = dev_upload(H, D.invN, invN.data(), invN.size())) ||
        (rc_ = dev_upload(H, D.invL, invL.data(), invL.size())) ||
        (rc_ = dev_upload(H, D.poff_d, D.poff.data(), D.poff.size())) ||
        (rc_ = dev_upload(H, D.w, HL.w.data(), HL.w.size())) || (rc_ = dev_alloc(H, D.x, HL.m)) ||
        (rc_ = dev_alloc(H, D.f, HL.m)) || (rc_ = dev_alloc(H, D.r, HL.m)) || (rc_ = dev_alloc(H, D.p, HL.m)))
        return rc_;
    return AAOMG_OK;
}

// the coarsest solution operator G: x = G f solves A x = f with int p =
// int mu = 0, from the bordered system [[S A S, S C], [C^T S, 0]] (S =
// L^{-1/2}, C the two mean functionals) inverted in FP64: G = S B^-1 S
int build_coarse(ms_ctx* H, const HostLevel& HL) {
    const int m = HL.m, cm = m + 2;
    std::vector<double> B((size_t)cm * cm, 0.0);
    std::vector<int> c;
    std::vector<double> v;
    std::vector<double> s(m);
    for (int u = 0; u < m; ++u) s[u] = 1.0 / std::sqrt(HL.Ld[u]);
    for (int u = 0; u < m; ++u) {
        a_row(HL, H->alpha, u, c, v);
        for (size_t k = 0; k < c.size(); ++k) B[(size_t)u * cm + c[k]] += s[u] * v[k] * s[c[k]];
    }
    const Blocks Bk = HL.blocks();
    for (int q = 0; q < HL.np; ++q) {
        const int ip = Bk.off(2) + q, im = Bk.off(5) + q;
        B[(size_t)ip * cm + m] = B[(size_t)m * cm + ip] = HL.w[q] * s[ip];
        B[(size_t)im * cm + m + 1] = B[(size_t)(m + 1) * cm + im] = HL.w[q] * s[im];
    }
    if (!invert(cm, B)) return set_error(AAOMG_ERR_CUDA, "stokes: singular coarsest system");
    std::vector<double> G((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) G[(size_t)i * m + j] = s[i] * B[(size_t)i * cm + j] * s[j];
    return dev_upload(H, H->G, G.data(), G.size());
}

// ----------------------------------------------------------- launches --

int grid_of(long long n, int t = 256) { return (int)((n + t - 1) / t); }

void launch_smooth(ms_ctx* H, int k, const double* f, double* x, int steps, cudaStream_t s) {
    ms_ctx::Lev& D = H->lev[k];
    const RowsDev S = D.rows();
    const int sm = H->o.smoother;
    if (D.small) {
        launch_pdl(k_st_small, dim3(1), dim3(kSmallThreads), 3 * (size_t)D.m * sizeof(double), s, S,
                   (const int*)D.poff_d, D.nph, sm, steps, H->o.tau, f, x);
        ++H->launches;
        return;
    }
    const int gr = grid_of((long long)D.nrows * kGroup);
    launch_pdl(k_st_resid, dim3(gr), dim3(256), 0, s, S, f, (const double*)x, D.r);
    ++H->launches;
    for (int m = 0; m < steps; ++m) {
        if (sm == MS_SMOOTHER_NE) {
            launch_pdl(k_st_ne_p, dim3(gr), dim3(256), 0, s, S, H->o.tau, (const double*)D.r, D.p);
            launch_pdl(k_st_ne_update, dim3(gr), dim3(256), 0, s, S, (const double*)D.p, x, D.r);
            H->launches += 2;
            continue;
        }
        for (int pass = 0; pass < (sm == MS_SMOOTHER_SLSGS ? 2 : 1); ++pass)
            for (int q = 0; q < D.nph; ++q) {
                const int ph = pass == 0 ? q : D.nph - 1 - q;
                const int r0 = D.poff[ph], cnt = D.poff[ph + 1] - r0;
                if (cnt == 0) continue;
                launch_pdl(k_st_phase, dim3(grid_of((long long)cnt * kGroup)), dim3(256), 0, s, S, r0, cnt, x, D.r);
                ++H->launches;
            }
    }
}

void launch_resid(ms_ctx* H, int k, const double* f, const double* x, double* r, cudaStream_t s) {
    ms_ctx::Lev& D = H->lev[k];
    launch_pdl(k_st_resid, dim3(grid_of((long long)D.nrows * kGroup)), dim3(256), 0, s, D.rows(), f, x, r);
    ++H->launches;
}

void cycle_rec(ms_ctx* H, int k, const double* f, double* x, cudaStream_t s) {
    if (k == 1) {
        launch_pdl(k_st_coarse, dim3(1), dim3(256), 0, s, H->lev[1].m, (const double*)H->G, f, x);
        ++H->launches;
        return;
    }
    ms_ctx::Lev& D = H->lev[k];
    ms_ctx::Lev& C = H->lev[k - 1];
    if (H->o.nu_pre > 0) launch_smooth(H, k, f, x, H->o.nu_pre, s);
    launch_resid(H, k, f, x, D.r, s);
    launch_pdl(k_st_restrict, dim3(grid_of(C.m)), dim3(256), 0, s, D.blocks(), C.blocks(),
               CsrDev{D.r2p, D.r2c, D.r2v}, CsrDev{D.r1p, D.r1c, D.r1v}, (const double*)D.r, C.f, C.x);
    ++H->launches;
    if (k - 1 == H->kd) {
        // the gamma coarse-grid iterations of levels <= kd from x = 0 are a
        // fixed linear map of the restricted defect: x_c = B f_c
        launch_pdl(k_st_dense, dim3(grid_of(C.m, 128), kDenseChunks), dim3(128), 0, s, C.m,
                   (C.m + kDenseChunks - 1) / kDenseChunks, (const double*)H->B, (const double*)C.f, H->dpart);
        launch_pdl(k_st_dense_sum, dim3(grid_of(C.m)), dim3(256), 0, s, C.m, (const double*)H->dpart, C.x);
        H->launches += 2;
    } else {
        for (int g = 0; g < H->o.cycle; ++g) cycle_rec(H, k - 1, C.f, C.x, s);
    }
    launch_pdl(k_st_prolong, dim3(grid_of(D.m)), dim3(256), 0, s, D.blocks(), C.blocks(),
               CsrDev{D.p2p, D.p2c, D.p2v}, CsrDev{D.p1p, D.p1c, D.p1v}, (const double*)C.x, x);
    ++H->launches;
    if (H->o.nu_post > 0) launch_smooth(H, k, f, x, H->o.nu_post, s);
}

// The dense map of levels <= kd: the gamma iterations of level kd from x = 0
// applied to the unit vectors, a batch of them at a time (multi-vectors:
// vector j at offset j m_k; one grid row per vector, or one block per vector
// for whole smoothing calls on the small levels); the images are the map's
// columns.
struct Multi {
    std::vector<double*> f, x, r, p;
};

void smooth_multi(ms_ctx* H, int k, Multi& W, int nc, int steps, cudaStream_t s) {
    if (steps <= 0) return;
    ms_ctx::Lev& D = H->lev[k];
    const RowsDev S = D.rows();
    const int sm = H->o.smoother;
    const size_t smem = 3 * (size_t)D.m * sizeof(double);
    if (smem <= 200 * 1024) {
        launch_pdl(k_st_small, dim3(nc), dim3(kSmallThreads), smem, s, S, (const int*)D.poff_d, D.nph, sm, steps,
                   H->o.tau, (const double*)W.f[k], W.x[k]);
        return;
    }
    const int gr = grid_of((long long)D.nrows * kGroup);
    launch_pdl(k_st_resid, dim3(gr, nc), dim3(256), 0, s, S, (const double*)W.f[k], (const double*)W.x[k], W.r[k]);
    for (int m = 0; m < steps; ++m) {
        if (sm == MS_SMOOTHER_NE) {
            launch_pdl(k_st_ne_p, dim3(gr, nc), dim3(256), 0, s, S, H->o.tau, (const double*)W.r[k], W.p[k]);
            launch_pdl(k_st_ne_update, dim3(gr, nc), dim3(256), 0, s, S, (const double*)W.p[k], W.x[k], W.r[k]);
            continue;
        }
        for (int pass = 0; pass < (sm == MS_SMOOTHER_SLSGS ? 2 : 1); ++pass)
            for (int q = 0; q < D.nph; ++q) {
                const int ph = pass == 0 ? q : D.nph - 1 - q;
                const int r0 = D.poff[ph], cnt = D.poff[ph + 1] - r0;
                if (cnt > 0)
                    launch_pdl(k_st_phase, dim3(grid_of((long long)cnt * kGroup), nc), dim3(256), 0, s, S, r0, cnt,
                               W.x[k], W.r[k]);
            }
    }
}

void cycle_multi(ms_ctx* H, int k, Multi& W, int nc, cudaStream_t s) {
    if (k == 1) {
        launch_pdl(k_st_coarse, dim3(nc), dim3(256), 0, s, H->lev[1].m, (const double*)H->G, (const double*)W.f[1],
                   W.x[1]);
        return;
    }
    ms_ctx::Lev& D = H->lev[k];
    ms_ctx::Lev& C = H->lev[k - 1];
    smooth_multi(H, k, W, nc, H->o.nu_pre, s);
    launch_pdl(k_st_resid, dim3(grid_of((long long)D.nrows * kGroup), nc), dim3(256), 0, s, D.rows(),
               (const double*)W.f[k], (const double*)W.x[k], W.r[k]);
    launch_pdl(k_st_restrict, dim3(grid_of(C.m), nc), dim3(256), 0, s, D.blocks(), C.blocks(),
               CsrDev{D.r2p, D.r2c, D.r2v}, CsrDev{D.r1p, D.r1c, D.r1v}, (const double*)W.r[k], W.f[k - 1],
               W.x[k - 1]);
    for (int g = 0; g < H->o.cycle; ++g) cycle_multi(H, k - 1, W, nc, s);
    launch_pdl(k_st_prolong, dim3(grid_of(D.m), nc), dim3(256), 0, s, D.blocks(), C.blocks(),
               CsrDev{D.p2p, D.p2c, D.p2v}, CsrDev{D.p1p, D.p1c, D.p1v}, (const double*)W.x[k - 1], W.x[k]);
    smooth_multi(H, k, W, nc, H->o.nu_post, s);
}

constexpr int kDenseBatch = 4096;  // unit vectors per pass of the dense map build

int build_dense(ms_ctx* H) {
    TraceRange tr("stokes: dense map of levels <= %d", H->kd);
    const int kd = H->kd, m = H->lev[kd].m;
    const int nb = std::min(m, kDenseBatch);
    Multi W;
    W.f.assign(kd + 1, nullptr);
    W.x.assign(kd + 1, nullptr);
    W.r.assign(kd + 1, nullptr);
    W.p.assign(kd + 1, nullptr);
    int rc = dev_upload<double>(H, H->B, nullptr, (size_t)m * m);
    for (int k = 1; k <= kd && !rc; ++k) {
        const size_t n = (size_t)H->lev[k].m * nb * sizeof(double);
        if (cudaMalloc((void**)&W.f[k], n) != cudaSuccess || cudaMalloc((void**)&W.x[k], n) != cudaSuccess ||
            cudaMalloc((void**)&W.r[k], n) != cudaSuccess || cudaMalloc((void**)&W.p[k], n) != cudaSuccess)
            rc = set_error(AAOMG_ERR_OOM, "stokes dense map workspace");
    }
    cudaStream_t s = H->cap;
    for (int j0 = 0; j0 < m && !rc; j0 += nb) {
        const int nc = std::min(nb, m - j0);
        const size_t n = (size_t)nc * m;
        launch_pdl(k_st_identity, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, m, j0, nc, W.f[kd]);
        cudaMemsetAsync(W.x[kd], 0, n * sizeof(double), s);
        for (int g = 0; g < H->o.cycle; ++g) cycle_multi(H, kd, W, nc, s);
        cudaMemcpyAsync(H->B + (size_t)j0 * m, W.x[kd], n * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) rc = set_error(AAOMG_ERR_CUDA, std::string("stokes dense map: ") + cudaGetErrorString(e));
    }
    for (int k = 1; k <= kd; ++k) {
        cudaFree(W.f[k]);
        cudaFree(W.x[k]);
        cudaFree(W.r[k]);
        cudaFree(W.p[k]);
    }
    if (!rc) rc = dev_alloc(H, H->dpart, (size_t)kDenseChunks * m);
    return rc;
}

int record_cycle(ms_ctx* H) {
    TraceRange tr("stokes: record cycle L=%d", H->L);
    ms_ctx::Lev& T = H->lev[H->L];
    cudaGraph_t g = nullptr;
    SCK(cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal));
    const long long before = H->launches;
    cycle_rec(H, H->L, T.f, T.x, H->cap);
    H->launches_per_cycle = H->launches - before;
    H->launches = before;
    cudaError_t e = cudaStreamEndCapture(H->cap, &g);
    if (e != cudaSuccess) return set_error(AAOMG_ERR_CUDA, std::string("stokes cycle capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&H->cycle_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return set_error(AAOMG_ERR_CUDA, std::string("stokes cycle instantiation: ") + cudaGetErrorString(e));
    return AAOMG_OK;
}

// out[0], out[1] (device) from the partial sums
void launch_norms(ms_ctx* H, int mode, const double* v, const double* g, const double* means, double* out,
                  cudaStream_t s) {
    ms_ctx::Lev& T = H->lev[H->L];
    launch_pdl(k_st_norm_part, dim3(kNormBlocks), dim3(256), 0, s, T.blocks(), mode, T.invL, v, g, means, H->part);
    launch_pdl(k_st_norm_final, dim3(1), dim3(256), 0, s, H->part, kNormBlocks, out);
    H->launches += 2;
}

void launch_means(ms_ctx* H, const double* x, cudaStream_t s) {
    ms_ctx::Lev& T = H->lev[H->L];
    launch_pdl(k_st_means, dim3(1), dim3(1024), 0, s, T.blocks(), T.w, x, H->means);
    ++H->launches;
}

int check_handle(ms_ctx* h) {
    if (!h) return set_error(AAOMG_ERR_BAD_ARG, "null handle");
    SCK(cudaSetDevice(h->device));
    return AAOMG_OK;
}

int run_cycle(ms_ctx* H, cudaStream_t s) {
    SCK(cudaGraphLaunch(H->cycle_exec, s));
    H->launches += H->launches_per_cycle;
    return AAOMG_OK;
}

int read_norms(ms_ctx* H, cudaStream_t s, double out[2]) {
    SCK(cudaMemcpyAsync(H->h_red, H->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    out[0] = H->h_red[0];
    out[1] = H->h_red[1];
    return AAOMG_OK;
}

}  // namespace

// ================================================================ ABI ==

extern "C" {

int ms_setup(int levels, double alpha, const ms_options* opt, ms_handle* out) {
    TraceRange tr("stokes setup L=%d alpha=%g", levels, alpha);
    if (!out) return set_error(AAOMG_ERR_BAD_ARG, "out is null");
    *out = nullptr;
    if (levels < 1 || levels > 9) return set_error(AAOMG_ERR_BAD_ARG, "levels must be in [1, 9]");
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return set_error(AAOMG_ERR_BAD_ARG, "alpha must be positive and finite");
    ms_options o{};
    o.smoother = MS_SMOOTHER_LSGS;
    o.cycle = 2;
    if (opt) o = *opt;
    if (o.smoother < 0 || o.smoother > MS_SMOOTHER_SLSGS) return set_error(AAOMG_ERR_BAD_ARG, "unknown smoother");
    if (o.cycle == 0) o.cycle = 2;
    if (o.cycle < 1 || o.cycle > 2) return set_error(AAOMG_ERR_BAD_ARG, "cycle must be 1 (V) or 2 (W)");
    const int nu = o.smoother == MS_SMOOTHER_SLSGS ? 1 : 2;
    if (o.nu_pre <= 0) o.nu_pre = nu;
    if (o.nu_post <= 0) o.nu_post = nu;
    if (!(o.tau > 0.0)) o.tau = 0.35;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.block_max == 0) o.block_max = 4;
    if (o.block_max > 4) return set_error(AAOMG_ERR_BAD_ARG, "block_max must be at most 4");
    if (o.dense_level > 5 || (o.dense_level > 0 && o.dense_level >= levels))
        return set_error(AAOMG_ERR_BAD_ARG, "dense_level must be below levels and at most 5");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(AAOMG_ERR_NO_DEVICE, "no CUDA device");
    }
    ms_ctx* H = new (std::nothrow) ms_ctx;
    if (!H) return set_error(AAOMG_ERR_OOM, "host allocation");
    H->L = levels;
    H->alpha = alpha;
    H->o = o;
    H->kd = o.dense_level > 0 ? o.dense_level : (o.dense_level == 0 && levels >= 5 ? (levels >= 7 ? 5 : 4) : 0);
    cudaGetDevice(&H->device);
    H->lev.resize(levels + 1);
    int rc = AAOMG_OK;
    std::vector<HostLevel> hl(levels + 1);
    for (int k = 1; k <= levels && !rc; ++k) {
        if (!assemble(1 << k, alpha, hl[k])) rc = set_error(AAOMG_ERR_BAD_ARG, "stokes assembly: row capacity exceeded");
        if (!rc) rc = build_level(H, hl[k], H->lev[k]);
        if (!rc) H->lev[k].small = k <= o.block_max && 3 * (size_t)hl[k].m * sizeof(double) <= 200 * 1024;
        if (!rc && k > 1) {
            const Csr P2 = embed_p2(hl[k], hl[k - 1]), P1 = embed_p1(hl[k], hl[k - 1]);
            const Csr R2 = transpose(P2), R1 = transpose(P1);
            ms_ctx::Lev& D = H->lev[k];
            if (!rc) rc = upload_csr(H, P2, D.p2p, D.p2c, D.p2v);
            if (!rc) rc = upload_csr(H, P1, D.p1p, D.p1c, D.p1v);
            if (!rc) rc = upload_csr(H, R2, D.r2p, D.r2c, D.r2v);
            if (!rc) rc = upload_csr(H, R1, D.r1p, D.r1c, D.r1v);
        }
        if (!rc && k == 1) rc = build_coarse(H, hl[1]);
    }
    if (!rc) {
        const Csr Mf = rows_to_csr(hl[levels].Mf, hl[levels].ng * hl[levels].ng);
        rc = upload_csr(H, Mf, H->mfp, H->mfc, H->mfv);
    }
    if (!rc) rc = dev_alloc(H, H->part, 2 * kNormBlocks);
    if (!rc) rc = dev_alloc(H, H->red, 2);
    if (!rc) rc = dev_alloc(H, H->means, 2);
    if (!rc && cudaMallocHost((void**)&H->h_red, 2 * sizeof(double)) != cudaSuccess)
        rc = set_error(AAOMG_ERR_OOM, "pinned host allocation");
    if (!rc && cudaFuncSetAttribute(k_st_small, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
        rc = set_error(AAOMG_ERR_CUDA, "stokes small-level kernel attributes");
    if (!rc && cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_error(AAOMG_ERR_CUDA, "stream creation");
    if (!rc && H->kd > 0) rc = build_dense(H);
    if (!rc) rc = record_cycle(H);
    if (rc) {
        ms_destroy(H);
        return rc;
    }
    *out = H;
    return AAOMG_OK;
}

void ms_destroy(ms_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->cycle_exec) cudaGraphExecDestroy(h->cycle_exec);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (void* p : h->allocs) cudaFree(p);
    if (h->h_red) cudaFreeHost(h->h_red);
    delete h;
}

int ms_sizes(ms_handle h, int level, int* out) {
    if (!h || !out) return set_error(AAOMG_ERR_BAD_ARG, "null argument");
    if (level < 1 || level > h->L) return set_error(AAOMG_ERR_BAD_ARG, "level out of range");
    const auto& D = h->lev[level];
    out[0] = D.n;
    out[1] = D.nv;
    out[2] = D.np;
    out[3] = D.m;
    return AAOMG_OK;
}

int ms_rhs_from_vd(ms_handle h, const double* vD, double* f, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!vD || !f) return set_error(AAOMG_ERR_BAD_ARG, "null vector");
    auto& T = h->lev[h->L];
    const int ng = 2 * T.n + 1;
    launch_pdl(k_st_rhs, dim3(grid_of(T.m)), dim3(256), 0, (cudaStream_t)stream, T.blocks(), ng * ng, CsrDev{h->mfp, h->mfc, h->mfv}, vD, f);
    ++h->launches;
    SCK(cudaGetLastError());
    return AAOMG_OK;
}

int ms_residual(ms_handle h, const double* f, const double* x, double* r, double* relres, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x) return set_error(AAOMG_ERR_BAD_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    auto& T = h->lev[h->L];
    double* rr = r ? r : T.r;
    launch_resid(h, h->L, f, x, rr, s);
    if (relres) {
        launch_norms(h, 0, rr, f, nullptr, h->red, s);
        double nr[2];
        if ((rc = read_norms(h, s, nr))) return rc;
        *relres = std::sqrt(nr[0] / (nr[1] > 0.0 ? nr[1] : 1.0));
    }
    SCK(cudaGetLastError());
    return AAOMG_OK;
}

int ms_smooth(ms_handle h, const double* f, double* x, int steps, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x || steps < 0) return set_error(AAOMG_ERR_BAD_ARG, "null vector or negative steps");
    if (steps > 0) launch_smooth(h, h->L, f, x, steps, (cudaStream_t)stream);
    SCK(cudaGetLastError());
    return AAOMG_OK;
}

int ms_cycle(ms_handle h, const double* f, double* x, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x) return set_error(AAOMG_ERR_BAD_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    auto& T = h->lev[h->L];
    const size_t bytes = (size_t)T.m * sizeof(double);
    SCK(cudaMemcpyAsync(T.f, f, bytes, cudaMemcpyDeviceToDevice, s));
    SCK(cudaMemcpyAsync(T.x, x, bytes, cudaMemcpyDeviceToDevice, s));
    if ((rc = run_cycle(h, s))) return rc;
    SCK(cudaMemcpyAsync(x, T.x, bytes, cudaMemcpyDeviceToDevice, s));
    return AAOMG_OK;
}

int ms_solve(ms_handle h, const double* f, double* x, double tol, int* iters, double* relres, void* stream) {
    TraceRange tr("stokes solve");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x || !(tol > 0.0)) return set_error(AAOMG_ERR_BAD_ARG, "null vector or tol <= 0");
    cudaStream_t s = (cudaStream_t)stream;
    auto& T = h->lev[h->L];
    const size_t bytes = (size_t)T.m * sizeof(double);
    SCK(cudaMemcpyAsync(T.f, f, bytes, cudaMemcpyDeviceToDevice, s));
    SCK(cudaMemcpyAsync(T.x, x, bytes, cudaMemcpyDeviceToDevice, s));
    int it = 0;
    double rr = 0.0, r0 = 0.0;
    int status = AAOMG_OK;
    for (;;) {
        launch_resid(h, h->L, T.f, T.x, T.r, s);
        launch_norms(h, 0, T.r, T.f, nullptr, h->red, s);
        double nr[2];
        if ((rc = read_norms(h, s, nr))) return rc;
        rr = std::sqrt(nr[0] / (nr[1] > 0.0 ? nr[1] : 1.0));
        if (it == 0) r0 = rr;
        if (!std::isfinite(rr) || rr > 1e6 * (r0 > 0.0 ? r0 : 1.0)) {
            status = set_error(AAOMG_ERR_DIVERGED, "residual diverged");
            break;
        }
        if (rr <= tol) break;
        if (it >= h->o.max_iter) {
            status = set_error(AAOMG_ERR_NOT_CONVERGED, "max_iter reached");
            break;
        }
        if ((rc = run_cycle(h, s))) return rc;
        ++it;
    }
    SCK(cudaMemcpyAsync(x, T.x, bytes, cudaMemcpyDeviceToDevice, s));
    SCK(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return status;
}

int ms_normalize(ms_handle h, double* x, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x) return set_error(AAOMG_ERR_BAD_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    auto& T = h->lev[h->L];
    launch_means(h, x, s);
    launch_pdl(k_st_shift, dim3(grid_of(T.np)), dim3(256), 0, s, T.blocks(), h->means, x);
    ++h->launches;
    SCK(cudaGetLastError());
    return AAOMG_OK;
}

int ms_control(ms_handle h, const double* x, double* u, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x || !u) return set_error(AAOMG_ERR_BAD_ARG, "null vector");
    auto& T = h->lev[h->L];
    launch_pdl(k_st_control, dim3(grid_of(2LL * T.nv)), dim3(256), 0, (cudaStream_t)stream, T.blocks(),
               1.0 / h->alpha, x, u);
    ++h->launches;
    SCK(cudaGetLastError());
    return AAOMG_OK;
}

int ms_norms(ms_handle h, const double* x, double* norm_L, double* norm_Linv, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x) return set_error(AAOMG_ERR_BAD_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    launch_norms(h, 1, x, nullptr, nullptr, h->red, s);
    double nr[2];
    if ((rc = read_norms(h, s, nr))) return rc;
    if (norm_L) *norm_L = std::sqrt(nr[0]);
    if (norm_Linv) *norm_Linv = std::sqrt(nr[1]);
    return AAOMG_OK;
}

int ms_protocol_iterations(ms_handle h, const double* x0, double reduction, int max_iter, int* iters, void* stream) {
    TraceRange tr("stokes protocol");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x0 || !iters || !(reduction > 0.0) || max_iter < 0) return set_error(AAOMG_ERR_BAD_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    auto& T = h->lev[h->L];
    const size_t bytes = (size_t)T.m * sizeof(double);
    SCK(cudaMemsetAsync(T.f, 0, bytes, s));
    SCK(cudaMemcpyAsync(T.x, x0, bytes, cudaMemcpyDeviceToDevice, s));
    double e0 = 0.0;
    int it = 0;
    for (;;) {
        launch_means(h, T.x, s);
        launch_norms(h, 1, T.x, nullptr, h->means, h->red, s);
        double nr[2];
        if ((rc = read_norms(h, s, nr))) return rc;
        const double e = std::sqrt(nr[0]);
        if (it == 0) e0 = e;
        if (e <= reduction * e0) break;
        if (it >= max_iter || !std::isfinite(e)) {
            it = -1;
            break;
        }
        if ((rc = run_cycle(h, s))) return rc;
        ++it;
    }
    *iters = it;
    return AAOMG_OK;
}

long long ms_kernel_launches(ms_handle h) { return h ? h->launches : -1; }

int ms_operator_entries(ms_handle h, int level, long long* nnz, long long* stored) {
    if (!h || !nnz || !stored) return set_error(AAOMG_ERR_BAD_ARG, "null argument");
    if (level < 1 || level > h->L) return set_error(AAOMG_ERR_BAD_ARG, "level out of range");
    *nnz = h->lev[level].nnz;
    *stored = h->lev[level].stored;
    return AAOMG_OK;
}

}  // extern "C"
