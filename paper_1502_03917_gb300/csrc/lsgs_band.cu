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
// Each column meets exactly one y phase and one lambda phase per step; four
// threads share a column, one per task of the step (prefetch and output, y
// update, residual, lambda update), so that 32 warps per SM hide each
// other's latencies (measured against two threads per column: 6% faster).
//
// Halos.  The final iterate at node (i,j) depends only on the initial data in
// columns i-28..i+15 and rows j-28..j+15, so a block computes columns
// [i0-28, i0+W+15) and rows [j0-28, j1+15) and keeps columns [i0, i0+W) and
// rows [j0, j1); everything outside is recomputed by the neighbouring blocks.
// The step is out of place (x_in -> x_out) because halos overlap.
//
// Storage.  The two fields of a node sit side by side (float2 / double2) in
// power-of-two row rings, so one shared-memory access moves both fields and a
// ring slot is a mask.  Nodes whose whole neighbourhood is interior to the grid
// and to the window take a branch-free path with the constant interior stencil;
// a warp holding a column within two of the left or right boundary takes the
// same path with its columns' stencils from a small table instead (otherwise
// that one warp would run two paths per step and hold up its whole block).
#include <cuda_runtime.h>

#include "band.h"
#include "lean.cuh"
#include "pdl.h"
#include "pair.cuh"
#include "stencil.cuh"

namespace aaomg {

namespace {

constexpr int kRing = 64;   // rows of x: tau-31 .. tau+kPre in use
constexpr int kRRing = 32;  // rows of rh: tau-31 .. tau-2 in use
constexpr int kFRing = 16;  // rows of f: prefetched at rho-kPre, used at rho+2
constexpr int kPre = 8;     // prefetch distance in rows
constexpr int kLag = 31;    // output row = tau - kLag

template <typename T>
struct V2;
template <>
struct V2<float> {
    using type = float2;
};
template <>
struct V2<double> {
    using type = double2;
};

// Stencils of a node in a row with 2 <= j <= n-2, by the class cls5(i) of its
// column (0, 1, interior, n-1, n): mass and bare stiffness weights (0 for a
// neighbour outside the grid), L_y^-1 of the node, N_ii^-1 of both fields, and
// the scatter weights of both fields' updates (the column of A scaled by the
// neighbours' L^-1, as in the interior constants sc of LevelP).
template <typename T>
struct ColClass {
    T m[7], kd[7], il0, iny, inl;
    T sc[2][7][2];
};

template <typename T, int WT>
struct BandSmem {
    typename V2<T>::type X[kRing][WT];
    typename V2<T>::type R[kRRing][WT];
    typename V2<T>::type F[kFRing][WT];
    ColClass<T> cls[5];
};

template <typename T>
__device__ void col_class_init(const LevelP<T>& P, int k, ColClass<T>& C) {
    const int n = P.n;
    const int i = k <= 2 ? k : n - 4 + k, j = 2;  // representative node of the class
    double m[7], kd[7];
    row_coeffs_general<double>(i, j, n, (double)P.h2, m, kd);
    C.il0 = inv_ly(P, i, j);
    C.iny = inv_n(P, 0, i, j);
    C.inl = inv_n(P, 1, i, j);
    for (int o = 0; o < 7; ++o) {
        const int ii = i + DI(o), jj = j + DJ(o);
        const double il = in_grid(ii, jj, n) ? (double)inv_ly(P, ii, jj) : 0.0;
        const double ko = (double)P.c * (kd[o] + (double)P.km * m[o]);
        C.m[o] = (T)m[o];
        C.kd[o] = (T)kd[o];
        C.sc[0][o][0] = (T)(m[o] * il);  // y update: rh_y -= m p/L, rh_l -= cK p/L_l
        C.sc[0][o][1] = (T)(ko * il * (double)P.invd);
        C.sc[1][o][0] = (T)(ko * il);  // lambda update: rh_y -= cK p/L, rh_l += m p/L
        C.sc[1][o][1] = (T)(-m[o] * il);
    }
}

// the block barrier, taken by the task roles from their own loops (each
// thread passes it once per step)
__device__ __forceinline__ void block_bar() { asm volatile("bar.sync 0;\n" ::: "memory"); }

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

// ------------------------------------------------ general (boundary) path --
template <typename T, int WT>
struct View {
    BandSmem<T, WT>* S;
    int c0, jl, jh, n;
    __device__ __forceinline__ bool has(int c, int j) const {
        unsigned t = (unsigned)(c - c0);
        return t < (unsigned)WT && j >= jl && j <= jh && c >= 0 && c <= n;
    }
    __device__ __forceinline__ typename V2<T>::type& x(int c, int j) const { return S->X[j & (kRing - 1)][c - c0]; }
    __device__ __forceinline__ typename V2<T>::type& r(int c, int j) const { return S->R[j & (kRRing - 1)][c - c0]; }
};

template <typename T, int WT>
__device__ void band_resid_general(const LevelP<T>& P, const View<T, WT>& V, int i, int j) {
    T m[7], kd[7], y[7], l[7];
    row_coeffs(P, i, j, m, kd);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        bool ok = V.has(ii, jj);
        typename V2<T>::type v = ok ? V.x(ii, jj) : typename V2<T>::type{T(0), T(0)};
        y[o] = v.x;
        l[o] = v.y;
    }
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, ay, al;
    dots(in, m, kd, y, My, Ky);
    dots(in, m, kd, l, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    T il = inv_ly(P, i, j);
    typename V2<T>::type fv = V.S->F[j & (kFRing - 1)][i - V.c0];
    V.r(i, j) = {(fv.x - ay) * il, (fv.y - al) * (il * P.invd)};
}

template <typename T, int WT>
__device__ void band_update_general(const LevelP<T>& P, const View<T, WT>& V, int field, int i, int j) {
    T m[7], kd[7], ry[7], rl[7];
    bool ok[7];
    row_coeffs(P, i, j, m, kd);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        ok[o] = V.has(ii, jj);
        typename V2<T>::type v = ok[o] ? V.r(ii, jj) : typename V2<T>::type{T(0), T(0)};
        ry[o] = v.x;
        rl[o] = v.y;
    }
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, qy, ql;
    dots(in, m, kd, ry, My, Ky);
    dots(in, m, kd, rl, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    T p = (field == 0 ? qy : ql) * inv_n(P, field, i, j);
    if (field == 0) V.x(i, j).x += p;
    else V.x(i, j).y += p;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        if (!ok[o]) continue;
        int ii = i + DI(o), jj = j + DJ(o);
        T il = inv_ly(P, ii, jj);
        T mp = m[o] * p;
        T kp = P.c * (kd[o] * p + P.km * mp);
        if (field == 0) V.r(ii, jj) = {ry[o] - mp * il, rl[o] - kp * (il * P.invd)};
        else V.r(ii, jj) = {ry[o] - kp * il, rl[o] + mp * il};
    }
}

// ------------------------------------------------------ interior fast path --
// constant stencil (lean.cuh); in the ring, row offsets select the slots sm/s/sp
template <typename T, int WT>
__device__ __forceinline__ void band_resid_fast(const LevelP<T>& P, BandSmem<T, WT>* S, int t, int sxm, int sx,
                                                int sxp, int sr, int sf) {
    const typename V2<T>::type fv = S->F[sf][t];
    S->R[sr][t] = rows_resid_fast<T>(P, S->X[sx], S->X[sxp], S->X[sxm], t, fv.x, fv.y);
}

template <typename T, int WT, typename C>
__device__ __forceinline__ void band_update_fast(const LevelP<T>& P, const C& c, BandSmem<T, WT>* S, int field,
                                                 int t, int sm, int s, int sp, int sx) {
    rows_lsgs_fast_c<T>(P, c, field, S->X[sx], S->R[s], S->R[sp], S->R[sm], t);
}

// ---------------------------------------------- boundary-column path ----
// The rows 2..n-2 of a column near the left or right boundary: the stencils of
// the column's class from the table, neighbours outside the grid weighted 0
// (their ring slots hold zeros).  A warp that holds such a column runs this
// path on all its lanes, so it never executes two paths per step.
template <typename T, typename V2>
__device__ __forceinline__ void class_dots(const ColClass<T>& C, const V2 (&nb)[7], V2& M, V2& K) {
    M = pmul(psplat(C.m[0]), nb[0]);
    K = pmul(psplat(C.kd[0]), nb[0]);
#pragma unroll
    for (int o = 1; o < 7; ++o) {
        M = pfma(psplat(C.m[o]), nb[o], M);
        K = pfma(psplat(C.kd[o]), nb[o], K);
    }
}

template <typename V2>
__device__ __forceinline__ void ring_load7(const V2* rs, const V2* rsp, const V2* rsm, int t, V2 (&nb)[7]) {
    nb[0] = rs[t];
    nb[1] = rs[t + 1];
    nb[2] = rs[t - 1];
    nb[3] = rsp[t];
    nb[4] = rsm[t];
    nb[5] = rsp[t + 1];
    nb[6] = rsm[t - 1];
}

template <typename T, int WT>
__device__ __forceinline__ void band_resid_col(const LevelP<T>& P, const ColClass<T>& C, BandSmem<T, WT>* S, int t,
                                               int sxm, int sx, int sxp, int sr, int sf) {
    using V2 = typename V2<T>::type;
    V2 nb[7], M, K;
    ring_load7(S->X[sx], S->X[sxp], S->X[sxm], t, nb);
    class_dots(C, nb, M, K);
    T ay, al;
    rows_from_dots(P, M.x, K.x, M.y, K.y, ay, al);
    const V2 fv = S->F[sf][t];
    const T il = C.il0;
    S->R[sr][t] = pmake<T>((fv.x - ay) * il, (fv.y - al) * (il * P.invd));
}

template <typename T, int WT>
__device__ __forceinline__ void band_update_col(const LevelP<T>& P, const ColClass<T>& C, BandSmem<T, WT>* S,
                                                int field, int t, int sm, int s, int sp, int sx) {
    using V2 = typename V2<T>::type;
    V2 sc[7];  // read before the first store
#pragma unroll
    for (int o = 0; o < 7; ++o) sc[o] = pmake<T>(C.sc[field][o][0], C.sc[field][o][1]);
    const T inv_nd = field == 0 ? C.iny : C.inl;
    V2* rs = S->R[s];
    V2* rsp = S->R[sp];
    V2* rsm = S->R[sm];
    V2 nb[7], M, K;
    ring_load7(rs, rsp, rsm, t, nb);
    class_dots(C, nb, M, K);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T pv = (field == 0 ? qy : ql) * inv_nd;
    if (field == 0) S->X[sx][t].x += pv;
    else S->X[sx][t].y += pv;
    const V2 mp = psplat(-pv);
    rs[t] = pfma(mp, sc[0], nb[0]);
    rs[t + 1] = pfma(mp, sc[1], nb[1]);
    rs[t - 1] = pfma(mp, sc[2], nb[2]);
    rsp[t] = pfma(mp, sc[3], nb[3]);
    rsm[t] = pfma(mp, sc[4], nb[4]);
    rsp[t + 1] = pfma(mp, sc[5], nb[5]);
    rsm[t - 1] = pfma(mp, sc[6], nb[6]);
}

template <typename T, int WT>
__global__ void __launch_bounds__(4 * WT) k_lsgs_band(LevelP<T> P, const T* __restrict__ f,
                                                      const T* __restrict__ xin, T* __restrict__ xout, int W, int Hs) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BandSmem<T, WT>* S = reinterpret_cast<BandSmem<T, WT>*>(smem_raw);
    // four threads per column, one per task
    const int tid = threadIdx.x % WT;
    const int role = threadIdx.x / WT;  // 0: prefetch and output, 1: y update, 2: residual, 3: lambda update
    const int i0 = blockIdx.x * W;
    const int i1 = min(i0 + W, P.n + 1);
    const int c0 = i0 - kBandHL;
    const int c = c0 + tid;
    const bool col_in = c >= 0 && c <= P.n;
    // The outermost window columns only supply data: by the dependency reach
    // no kept node uses an update or a residual formed on them, so they are
    // not computed (which keeps every warp on the same path).
    const bool col_work = col_in && tid >= 1 && tid <= WT - 2;
    const int j0 = blockIdx.y * Hs;
    const int j1 = min(j0 + Hs, P.n + 1);
    const int jl = max(0, j0 - kBandHL);
    const int jh = min(P.n, j1 - 1 + kBandHR);
    const View<T, WT> V{S, c0, jl, jh, P.n};
    // this column (and its neighbours) interior to the grid and the window
    const bool col_fast = c >= 2 && c <= P.n - 2;
    const int jfl = max(2, jl + 1), jfh = min(P.n - 2, jh - 1);  // rows whose neighbourhood is fast
    // a warp with a working column near the left or right boundary takes the
    // table path on all its lanes (rows jfl..jfh)
    const bool warp_fast = !__any_sync(0xffffffffu, col_work && !col_fast);
    const ColClass<T>& C = S->cls[cls5(min(max(c, 0), P.n), P.n)];

    using V2T = typename V2<T>::type;
    if (threadIdx.x < 5) col_class_init<T>(P, threadIdx.x, S->cls[threadIdx.x]);
    if (role == 0) {
        for (int r = 0; r < kRing; ++r) S->X[r][tid] = V2T{T(0), T(0)};
    } else if (role == 1) {
        for (int r = 0; r < kRRing; ++r) S->R[r][tid] = V2T{T(0), T(0)};
    } else if (role == 2) {
        for (int r = 0; r < kFRing; ++r) S->F[r][tid] = V2T{T(0), T(0)};
    }
    __syncthreads();

    // one commit group per row, also for rows outside the window
    const T* xin_c = xin + c;
    const T* f_c = f + c;
    auto issue = [&](int row) {
        if (col_in && row >= jl && row <= jh) {
            int64_t g = (int64_t)row * P.ld;
            T* xs = reinterpret_cast<T*>(&S->X[row & (kRing - 1)][tid]);
            T* fs = reinterpret_cast<T*>(&S->F[row & (kFRing - 1)][tid]);
            cp_async(xs, xin_c + g);
            cp_async(xs + 1, xin_c + g + P.fs);
            cp_async(fs, f_c + g);
            cp_async(fs + 1, f_c + g + P.fs);
        }
        cp_async_commit();
    };
    if (role == 0) {
        for (int row = jl; row < jl + kPre; ++row) issue(row);
        cp_async_wait<kPre - 1>();  // row jl has landed
    }
    __syncthreads();

    // Each role runs its own loop over the steps; every thread passes the
    // block barrier once per step.  A role's rows lie in the fast range for
    // every lane in a warp-uniform interval of steps [ta, tb], where only the
    // lane's column decides whether it works.
    const int tau_end = j1 - 1 + kLag;
    if (role == 0) {
        const bool out_col = c >= i0 && c < i1;
        const int64_t ld = P.ld, fsz = P.fs;
        int64_t gi = (int64_t)(jl + kPre) * ld;      // element offset of row tau + kPre
        int64_t go = (int64_t)(jl - kLag) * ld + c;  // element offset of (c, tau - kLag)
        for (int tau = jl; tau <= tau_end; ++tau, gi += ld, go += ld) {
            const int row = tau + kPre;
            if (col_in && row <= jh) {
                T* xs = reinterpret_cast<T*>(&S->X[row & (kRing - 1)][tid]);
                T* fs = reinterpret_cast<T*>(&S->F[row & (kFRing - 1)][tid]);
                cp_async(xs, xin_c + gi);
                cp_async(xs + 1, xin_c + gi + fsz);
                cp_async(fs, f_c + gi);
                cp_async(fs + 1, f_c + gi + fsz);
            }
            cp_async_commit();
            // row tau - kLag has all its phases: to the output
            const int ro = tau - kLag;
            if (out_col && ro >= j0 && ro < j1) {
                V2T v = S->X[ro & (kRing - 1)][tid];
                xout[go] = v.x;
                xout[go + fsz] = v.y;
            }
            cp_async_wait<kPre - 1>();  // row tau + 1 has landed
            block_bar();
        }
        cp_async_wait<0>();
    } else if (role == 2) {
        // rh of row rho = tau - 2 from the original iterate
        const int ta = jfl + 2, tb = jfh + 2;
        for (int tau = jl; tau <= tau_end; ++tau) {
            const int rho = tau - 2;
            if (tau >= ta && tau <= tb) {
                if (col_work) {
                    if (warp_fast)
                        band_resid_fast<T, WT>(P, S, tid, (rho - 1) & (kRing - 1), rho & (kRing - 1),
                                               (rho + 1) & (kRing - 1), rho & (kRRing - 1), rho & (kFRing - 1));
                    else
                        band_resid_col<T, WT>(P, C, S, tid, (rho - 1) & (kRing - 1), rho & (kRing - 1),
                                              (rho + 1) & (kRing - 1), rho & (kRRing - 1), rho & (kFRing - 1));
                }
            } else if (col_work && rho >= jl && rho <= jh) {
                band_resid_general<T, WT>(P, V, c, rho);
            }
            block_bar();
        }
    } else {
        // the y phase (role 1) or the lambda phase (role 3) that meets this
        // column: phase index t* = 5 (c + 2 tau + 6) mod 7 of the y update,
        // advancing by 3 (mod 7) per step; the lambda phase runs 14 rows below
        auto run = [&](auto fc) {
            constexpr int field = decltype(fc)::value;
            const auto lc = lsgs_consts<T, V2T>(P, field);
            int ts = (5 * ((((c % 7) + 7) % 7 + 2 * (jl % 7) + 6) % 7)) % 7;
            // j = tau - 4 - 2 t* - 14 field lies in [jfl, jfh] for every t* in 0..6
            const int ta = jfl + 16 + 14 * field, tb = jfh + 4 + 14 * field;
            for (int tau = jl; tau <= tau_end; ++tau) {
                const int j = tau - 4 - 2 * ts - 14 * field;
                if (tau >= ta && tau <= tb) {
                    if (col_work) {
                        if (warp_fast)
                            band_update_fast<T, WT>(P, lc, S, field, tid, (j - 1) & (kRRing - 1), j & (kRRing - 1),
                                                    (j + 1) & (kRRing - 1), j & (kRing - 1));
                        else
                            band_update_col<T, WT>(P, C, S, field, tid, (j - 1) & (kRRing - 1), j & (kRRing - 1),
                                                   (j + 1) & (kRRing - 1), j & (kRing - 1));
                    }
                } else if (col_work && j >= jl && j <= jh) {
                    if (j >= jfl && j <= jfh) {
                        if (warp_fast)
                            band_update_fast<T, WT>(P, lc, S, field, tid, (j - 1) & (kRRing - 1), j & (kRRing - 1),
                                                    (j + 1) & (kRRing - 1), j & (kRing - 1));
                        else
                            band_update_col<T, WT>(P, C, S, field, tid, (j - 1) & (kRRing - 1), j & (kRRing - 1),
                                                   (j + 1) & (kRRing - 1), j & (kRing - 1));
                    } else
                        band_update_general<T, WT>(P, V, field, c, j);
                }
                ts = ts >= 4 ? ts - 4 : ts + 3;
                block_bar();
            }
        };
        if (role == 1) run(FieldC<0>{});
        else run(FieldC<1>{});
    }
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
int band_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lsgs_band<T, band_threads<T>()>, 4 * band_threads<T>(),
                                                      band_smem_bytes<T>()) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

template <typename T>
void launch_lsgs_band(const LevelP<T>& P, const T* f, const T* xin, T* xout, const BandGrid& g, cudaStream_t s) {
    constexpr int WT = band_threads<T>();
    launch_pdl(k_lsgs_band<T, WT>, dim3(g.nb, g.ns), 4 * WT, band_smem_bytes<T>(), s, P, f, xin, xout, g.W, g.Hs);
}

template size_t band_smem_bytes<float>();
template size_t band_smem_bytes<double>();
template cudaError_t band_prepare<float>();
template cudaError_t band_prepare<double>();
template int band_blocks_per_sm<float>();
template int band_blocks_per_sm<double>();
template void launch_lsgs_band<float>(const LevelP<float>&, const float*, const float*, float*, const BandGrid&,
                                      cudaStream_t);
template void launch_lsgs_band<double>(const LevelP<double>&, const double*, const double*, double*,
                                       const BandGrid&, cudaStream_t);

}  // namespace aaomg
