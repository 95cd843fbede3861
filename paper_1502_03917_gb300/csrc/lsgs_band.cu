// lsgs_band.cu -- one complete LSGS step (Algorithm 2: all 14 colour phases,
// fields y then lambda, colours 0,6,5,4,3,2,1 of (i + 2j) mod 7) in one launch.
//
// Wavefront schedule.  A block owns a band of columns and a segment of rows
// and marches up its rows with one thread per column.  At step tau it
//   * prefetches x and f of row tau + kPre into shared-memory rings (cp.async),
//   * forms rh = L^{-1}(f - A x) on row tau - 2 from the original iterate,
//   * applies colour phase t on row tau - 4 - 2t for t = 0..13,
//   * writes row tau - 31, on which all phases are done, to the output.
// With this colour sequence a phase-t update at row j depends only on phase
// t-1 updates up to row j+1 (and on earlier phases up to row j+2), so a lag of
// two rows per phase satisfies every dependency; and no two updates of one
// step touch a common unknown or residual entry, so a step needs one barrier.
// Within a colour the updates commute exactly (each residual entry receives one
// update per phase), so the result equals the sequential multicolour sweep.
//
// Halos.  The final iterate at node (i,j) depends only on the initial data in
// columns i-28..i+15 and rows j-28..j+15, so a block computes columns
// [i0-28, i0+W+15) and rows [j0-28, j1+15) and keeps columns [i0, i0+W) and
// rows [j0, j1); everything outside is recomputed by the neighbouring blocks.
// The step is out of place (x_in -> x_out) because halos overlap.
#include <cuda_runtime.h>

#include "band.h"
#include "stencil.cuh"

namespace aaomg {

namespace {

constexpr int kRing = 40;   // rows of x kept: 32 in use + prefetch distance
constexpr int kRRing = 32;  // rows of rh in use: tau-31 .. tau-2
constexpr int kFRing = 16;  // rows of f: prefetched at tau-kPre, used at tau+2
constexpr int kPre = 8;     // prefetch distance in rows
constexpr int kLag = 31;    // output row = tau - kLag

template <typename T, int WT>
struct BandSmem {
    T xy[kRing][WT];
    T xl[kRing][WT];
    T ry[kRRing][WT];
    T rl[kRRing][WT];
    T fy[kFRing][WT];
    T fl[kFRing][WT];
};

template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// shared-memory window of the band: columns [c0, c0+WT), rows [jl, jh]
template <typename T, int WT>
struct View {
    BandSmem<T, WT>* S;
    int c0, jl, jh, n;
    __device__ __forceinline__ bool has(int c, int j) const {
        unsigned t = (unsigned)(c - c0);
        return t < (unsigned)WT && j >= jl && j <= jh && c >= 0 && c <= n;
    }
    __device__ __forceinline__ T& x(int field, int c, int j) const {
        return field ? S->xl[j % kRing][c - c0] : S->xy[j % kRing][c - c0];
    }
    __device__ __forceinline__ T& r(int field, int c, int j) const {
        return field ? S->rl[j % kRRing][c - c0] : S->ry[j % kRRing][c - c0];
    }
};

// rh = L^{-1}(f - A x) at node (i,j), from the window
template <typename T, int WT>
__device__ __forceinline__ void band_resid(const LevelP<T>& P, const View<T, WT>& V, int i, int j) {
    T m[7], kd[7], y[7], l[7];
    row_coeffs(P, i, j, m, kd);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        bool ok = V.has(ii, jj);
        y[o] = ok ? V.x(0, ii, jj) : T(0);
        l[o] = ok ? V.x(1, ii, jj) : T(0);
    }
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, ay, al;
    dots(in, m, kd, y, My, Ky);
    dots(in, m, kd, l, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    T il = inv_ly(P, i, j);
    T fy = V.S->fy[j % kFRing][i - V.c0], fl = V.S->fl[j % kFRing][i - V.c0];
    V.r(0, i, j) = (fy - ay) * il;
    V.r(1, i, j) = (fl - al) * (il * P.invd);
}

// Algorithm 2 update of unknown (field, (i,j)) inside the window
template <typename T, int WT>
__device__ __forceinline__ void band_update(const LevelP<T>& P, const View<T, WT>& V, int field, int i, int j) {
    T m[7], kd[7], ry[7], rl[7];
    bool ok[7];
    row_coeffs(P, i, j, m, kd);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        ok[o] = V.has(ii, jj);
        ry[o] = ok[o] ? V.r(0, ii, jj) : T(0);
        rl[o] = ok[o] ? V.r(1, ii, jj) : T(0);
    }
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, qy, ql;
    dots(in, m, kd, ry, My, Ky);
    dots(in, m, kd, rl, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    T p = (field == 0 ? qy : ql) * inv_n(P, field, i, j);
    V.x(field, i, j) += p;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        if (!ok[o]) continue;
        int ii = i + DI(o), jj = j + DJ(o);
        T il = inv_ly(P, ii, jj);
        T mp = m[o] * p;
        T kp = P.c * (kd[o] * p + P.km * mp);
        if (field == 0) {
            V.r(0, ii, jj) = ry[o] - mp * il;
            V.r(1, ii, jj) = rl[o] - kp * (il * P.invd);
        } else {
            V.r(0, ii, jj) = ry[o] - kp * il;
            V.r(1, ii, jj) = rl[o] + mp * il;
        }
    }
}

template <typename T, int WT>
__global__ void __launch_bounds__(WT) k_lsgs_band(LevelP<T> P, const T* __restrict__ f, const T* __restrict__ xin,
                                                  T* __restrict__ xout, int W, int Hs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BandSmem<T, WT>* S = reinterpret_cast<BandSmem<T, WT>*>(smem_raw);
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * W;
    const int i1 = min(i0 + W, P.n + 1);
    const int c0 = i0 - kBandHL;
    const int c = c0 + tid;
    const bool col_in = c >= 0 && c <= P.n;
    const int j0 = blockIdx.y * Hs;
    const int j1 = min(j0 + Hs, P.n + 1);
    const int jl = max(0, j0 - kBandHL);
    const int jh = min(P.n, j1 - 1 + kBandHR);
    View<T, WT> V{S, c0, jl, jh, P.n};

    for (int r = 0; r < kRing; ++r) S->xy[r][tid] = S->xl[r][tid] = T(0);
    for (int r = 0; r < kRRing; ++r) S->ry[r][tid] = S->rl[r][tid] = T(0);
    for (int r = 0; r < kFRing; ++r) S->fy[r][tid] = S->fl[r][tid] = T(0);
    __syncthreads();

    // one commit group per row, also when the row is outside the window
    auto issue = [&](int row) {
        if (col_in && row >= jl && row <= jh) {
            int64_t g = (int64_t)row * P.ld + c;
            cp_async(&S->xy[row % kRing][tid], xin + g);
            cp_async(&S->xl[row % kRing][tid], xin + g + P.fs);
            cp_async(&S->fy[row % kFRing][tid], f + g);
            cp_async(&S->fl[row % kFRing][tid], f + g + P.fs);
        }
        cp_async_commit();
    };
    for (int row = jl; row < jl + kPre; ++row) issue(row);
    cp_async_wait<kPre - 1>();  // row jl is in
    __syncthreads();

    const int cm7 = ((c % 7) + 7) % 7;
    for (int tau = jl; tau <= j1 - 1 + kLag; ++tau) {
        issue(tau + kPre);
        const int rho = tau - 2;
        if (col_in && rho >= jl && rho <= jh) band_resid<T, WT>(P, V, c, rho);
        // the y phase and the lambda phase that meet this column at this step
        const int ts = (5 * ((cm7 + 2 * (tau % 7) + 6) % 7)) % 7;
        const int jy = tau - 4 - 2 * ts, jlam = tau - 18 - 2 * ts;
        if (col_in && jy >= jl && jy <= jh) band_update<T, WT>(P, V, 0, c, jy);
        if (col_in && jlam >= jl && jlam <= jh) band_update<T, WT>(P, V, 1, c, jlam);
        const int ro = tau - kLag;
        if (ro >= j0 && ro < j1 && c >= i0 && c < i1) {
            int64_t g = (int64_t)ro * P.ld + c;
            xout[g] = S->xy[ro % kRing][tid];
            xout[g + P.fs] = S->xl[ro % kRing][tid];
        }
        cp_async_wait<kPre - 1>();  // row tau + 1 has landed
        __syncthreads();
    }
    cp_async_wait<0>();
}

}  // namespace

template <typename T>
size_t band_smem_bytes() {
    return sizeof(BandSmem<T, band_threads<T>()>);
}

template <typename T>
cudaError_t band_prepare() {
    return cudaFuncSetAttribute(k_lsgs_band<T, band_threads<T>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)band_smem_bytes<T>());
}

template <typename T>
void launch_lsgs_band(const LevelP<T>& P, const T* f, const T* xin, T* xout, const BandGrid& g, cudaStream_t s) {
    constexpr int WT = band_threads<T>();
    k_lsgs_band<T, WT><<<dim3(g.nb, g.ns), WT, band_smem_bytes<T>(), s>>>(P, f, xin, xout, g.W, g.Hs);
}

template size_t band_smem_bytes<float>();
template size_t band_smem_bytes<double>();
template cudaError_t band_prepare<float>();
template cudaError_t band_prepare<double>();
template void launch_lsgs_band<float>(const LevelP<float>&, const float*, const float*, float*, const BandGrid&,
                                      cudaStream_t);
template void launch_lsgs_band<double>(const LevelP<double>&, const double*, const double*, double*,
                                       const BandGrid&, cudaStream_t);

}  // namespace aaomg
