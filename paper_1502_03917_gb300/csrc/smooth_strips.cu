// smooth_strips.cu -- a whole smoothing call (nu steps of Algorithm 1 or 2) on
// one small or mid-size level in ONE launch: of one thread block (levels up to
// 65 x 65 nodes) or of one thread-block cluster (65 to 257 nodes per side).
//
// On these levels a colour phase of Algorithm 2 has a few dozen to a few
// thousand independent updates: too few to fill the GPU, and a launch per phase
// costs more than the phase.  The kernel loops over the phases with a barrier
// between dependent ones instead.  The level's grid rows are split into cs
// strips, one per block (cs = 1 for a single block, up to 16 blocks of a
// cluster).  Each block keeps the iterate x and the scaled residual
// rh = L^{-1}(f - Ax) of its strip in its own shared memory as (y, lambda)
// pairs for the whole call; x is read from global memory once at the start and
// written back once at the end.  In a cluster, a node in the first or last row
// of a strip reaches one row into the neighbouring strip: those loads and, for
// Algorithm 2, the residual updates of the scatter go to the neighbouring
// block's shared memory (distributed shared memory), and the phases are
// separated by cluster barriers (release / acquire), which also make those
// remote stores visible.  Within a colour phase no two updates touch a common
// unknown or residual entry (distance-2 colouring), so the result is the
// sequential multicolour sweep's whatever the strips.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "lean.cuh"
#include "pdl.h"
#include "stencil.cuh"
#include "strips.h"

namespace cg = cooperative_groups;

namespace aaomg {

namespace {

__device__ __forceinline__ void cluster_barrier() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;\n" ::
            : "memory");
}

// The strip of this block: own rows [r0, r1) in shared memory, and in a
// cluster the boundary rows of the neighbouring strips (null at the grid's
// bottom / top).  A single block (CL = false) owns every row, so all row
// pointers point into its own shared memory.
template <typename T, int N, bool CL>
struct Strip {
    using V2 = typename P2<T>::t;
    static constexpr int LD = N + 1;
    int r0, r1;
    V2 *X, *R;    // own rows
    V2 *Xb, *Rb;  // row r0 - 1 (last row of the block below)
    V2 *Xa, *Ra;  // row r1 (first row of the block above)
    // rows j in [r0 - 1, r1]
    __device__ __forceinline__ V2* xrow(int j) const {
        if constexpr (!CL) return X + j * LD;
        else return j < r0 ? Xb : (j >= r1 ? Xa : X + (j - r0) * LD);
    }
    __device__ __forceinline__ V2* rrow(int j) const {
        if constexpr (!CL) return R + j * LD;
        else return j < r0 ? Rb : (j >= r1 ? Ra : R + (j - r0) * LD);
    }
};

// ------------------------------------------------------- edge nodes --
// Nodes within two rows or columns of the boundary.  Their stencils, the L_y^-1
// of their neighbours and their N_ii^-1 depend only on the node's boundary
// class cls5(i) + 5 cls5(j); each block copies the level's 25-class table
// (EdgeClass, built on the host) into shared memory at the start, so a phase
// sees no global-memory latency.  An LSGS
// update reads the table entries its scatter needs before its first store, so
// that no table load waits behind a store it might alias.
template <typename T, int N, typename RowPtr, typename V2>
__device__ __forceinline__ void cl_gather(const RowPtr (&rows)[3], int i, int j, const EdgeClass<T>& C, V2 (&v)[7],
                                          T& My, T& Ky, T& Ml, T& Kl) {
    My = Ky = Ml = Kl = T(0);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        const int ii = i + DI(o), jj = j + DJ(o);
        v[o] = in_grid(ii, jj, N) ? rows[DJ(o) + 1][ii] : pmake<T>(T(0), T(0));
        My += C.m[o] * v[o].x;
        Ky += C.kd[o] * v[o].x;
        Ml += C.m[o] * v[o].y;
        Kl += C.kd[o] * v[o].y;
    }
}

template <typename T, int N, class S_>
__device__ __forceinline__ void cl_resid_edge(const LevelP<T>& P, const EdgeClass<T>& C,
                                              typename P2<T>::t fv, const S_& S, int i, int j) {
    using V2 = typename P2<T>::t;
    const V2* const rows[3] = {S.xrow(j - 1), S.xrow(j), S.xrow(j + 1)};
    V2 v[7];
    T My, Ky, Ml, Kl, ay, al;
    cl_gather<T, N>(rows, i, j, C, v, My, Ky, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    const T il = C.il[0];
    S.rrow(j)[i] = pmake<T>((fv.x - ay) * il, (fv.y - al) * (il * P.invd));
}

template <typename T, int N, class S_>
__device__ __forceinline__ void cl_ne_edge(const LevelP<T>& P, const EdgeClass<T>& C, const S_& S, int i, int j) {
    using V2 = typename P2<T>::t;
    const V2* const rows[3] = {S.rrow(j - 1), S.rrow(j), S.rrow(j + 1)};
    V2 v[7];
    T My, Ky, Ml, Kl, qy, ql;
    cl_gather<T, N>(rows, i, j, C, v, My, Ky, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T il = C.il[0];
    V2* xr = S.xrow(j);
    V2 u = xr[i];
    u.x += P.tau * il * qy;
    u.y += P.tau * (il * P.invd) * ql;
    xr[i] = u;
}

template <typename T, int N, class S_>
__device__ __forceinline__ void cl_lsgs_edge(const LevelP<T>& P, const EdgeClass<T>& C, int field, const S_& S,
                                             int i, int j) {
    using V2 = typename P2<T>::t;
    V2 sc[7];  // read before the first store
#pragma unroll
    for (int o = 0; o < 7; ++o) sc[o] = pmake<T>(C.sc[field][o][0], C.sc[field][o][1]);
    const T inv_nd = field == 0 ? C.iny : C.inl;
    V2* const rows[3] = {S.rrow(j - 1), S.rrow(j), S.rrow(j + 1)};
    V2 v[7];
    T My, Ky, Ml, Kl, qy, ql;
    cl_gather<T, N>(rows, i, j, C, v, My, Ky, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T p = (field == 0 ? qy : ql) * inv_nd;
    V2* xr = S.xrow(j);
    if (field == 0) xr[i].x += p;
    else xr[i].y += p;
    const V2 mp = psplat(-p);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        const int ii = i + DI(o), jj = j + DJ(o);
        if (in_grid(ii, jj, N)) rows[DJ(o) + 1][ii] = pfma(mp, sc[o], v[o]);
    }
}

// Edge nodes of a strip, enumerated per pass: the strip's full boundary rows
// (rows 0, 1 in the first block, n-1, n in the last) slot by slot, then the
// columns 0, 1, n-1, n of its other rows.  Colour c of node (i, j) is
// (i + A j) mod K (LSGS: A = 2, K = 7; CGS: A = 1, K = 3); in column i the
// nodes of colour c sit in the rows j = AINV (c - i) mod K (AINV = A^-1 mod K),
// every K-th row, so each column gets ceil(rows / K) slots; c < 0 (every
// colour): every row.
template <int N, int K = 7, int A = 2, int AINV = 4>
struct StripEdges {
    static constexpr int FPR = (N + 1 + K - 1) / K;  // slots of one colour per full row
    int nfull, first_full_hi, ja, nrows;
    __device__ __forceinline__ int per_col(int c) const { return c < 0 ? nrows : (nrows + K - 1) / K; }
    __device__ __forceinline__ int count(int c) const { return nfull * (c < 0 ? N + 1 : FPR) + 4 * per_col(c); }
    __device__ __forceinline__ bool node(int t, int c, int& i, int& j) const {
        return c < 0 ? node_any<N + 1, true>(t, c, i, j) : node_any<FPR, false>(t, c, i, j);
    }
    template <int PER, bool ALL>
    __device__ __forceinline__ bool node_any(int t, int c, int& i, int& j) const {
        if (t < nfull * PER) {
            const int r = t / PER, k = t - r * PER;
            j = r < first_full_hi ? r : N - 1 + (r - first_full_hi);
            i = ALL ? k : ((c - A * j) % K + K) % K + K * k;
            return i <= N;
        }
        t -= nfull * PER;
        const int pc = ALL ? nrows : (nrows + K - 1) / K;
        int q = 0, k = t;
        while (k >= pc && q < 3) {  // q = t / pc for t < 4 pc
            k -= pc;
            ++q;
        }
        i = q < 2 ? q : N - 3 + q;
        j = ALL ? ja + k : ja + ((AINV * (c - i) - ja) % K + K) % K + K * k;
        return j < ja + nrows;
    }
};

// A thread's slot of the LSGS colour phases, resolved once per call.  The
// slot index t of a phase enumerates the same kind of node for every colour:
// a deep-interior node of row j, a node of a full edge row j, or a node of an
// edge column i; only the position along that row or column depends on the
// colour, through a residue mod 7:
//   interior:  i = 2 + (c + m) mod 7 + 7k,  m = (-2 j - 2) mod 7
//   edge row:  i =     (c + m) mod 7 + 7k,  m = (-2 j) mod 7
//   edge col:  j = ja + (4c + m) mod 7 + 7k,  m = (-4 i - ja) mod 7
// (colour of (i, j) = (i + 2j) mod 7, 4 = 2^-1 mod 7), so a phase costs a
// few integer operations per slot instead of the enumeration (used by the
// 513^2 kernel, whose threads have five slots per phase; in the one-slot
// phases of the smaller levels it measured slower than the enumeration).
// Packed into one int: kind (2 bits: 0 none, 1 interior, 2 edge row, 3 edge
// column), m (3 bits), the fixed coordinate (11 bits: j for kinds 1, 2, i for
// kind 3) and the base of the varying one (16 bits: 2 + 7k, 7k, ja + 7k).
using SlotDesc = int;

__device__ __forceinline__ int mod7(int v) { return ((v % 7) + 7) % 7; }

__device__ __forceinline__ SlotDesc slot_pack(int kind, int m, int fixed, int base) {
    return kind | (m << 2) | (fixed << 5) | (base << 16);
}

template <int N, int CPR>
__device__ __forceinline__ SlotDesc slot_desc(int t, int ni, int nip, const StripEdges<N>& SE) {
    if (t < nip) {
        if (t >= ni) return 0;
        const int r = t / CPR, k = t - r * CPR, j = SE.ja + r;
        return slot_pack(1, mod7(-2 * j - 2), j, 2 + 7 * k);
    }
    t -= nip;
    constexpr int FPR = StripEdges<N>::FPR;
    if (t < SE.nfull * FPR) {
        const int r = t / FPR, k = t - r * FPR;
        const int j = r < SE.first_full_hi ? r : N - 1 + (r - SE.first_full_hi);
        return slot_pack(2, mod7(-2 * j), j, 7 * k);
    }
    t -= SE.nfull * FPR;
    const int pc = (SE.nrows + 6) / 7;
    if (pc <= 0 || t >= 4 * pc) return 0;
    const int q = t / pc, k = t - q * pc;
    const int i = q < 2 ? q : N - 3 + q;
    return slot_pack(3, mod7(-4 * i - SE.ja), i, SE.ja + 7 * k);
}

// the node of a slot in colour c; false if the slot is empty in this colour
// (jmax: the last row of the strip's edge-column range)
template <int N>
__device__ __forceinline__ bool slot_node(SlotDesc d, int c, int jmax, int& i, int& j) {
    const int kind = d & 3;
    if (!kind) return false;
    const int m = (d >> 2) & 7, fixed = (d >> 5) & 2047, base = d >> 16;
    int r = (kind == 3 ? ((4 * c) % 7) : c) + m;
    r -= r >= 7 ? 7 : 0;
    const int pos = base + r;
    if (kind == 3) {
        i = fixed;
        j = pos;
        return pos <= jmax;
    }
    i = pos;
    j = fixed;
    return pos <= (kind == 1 ? N - 2 : N);
}

// ----------------------------------------------------------------- CGS --
// Collective Gauss-Seidel update of node (i,j): the residual of its two rows
// from the current iterate (x rows) and its (f_y, f_lambda), then the 2x2
// diagonal block solve; the deep-interior block is constant.
template <typename T, typename V2>
__device__ __forceinline__ void rows_cgs_fast(const LevelP<T>& P, V2* xs, const V2* xsp, const V2* xsm, int i,
                                              V2 fv) {
    V2 M, K, nb[7];
    rows_stencil(xs, xsp, xsm, i, psplat(P.mC), psplat(P.mO), M, K, nb);
    T ay, al, dy, dl;
    rows_from_dots(P, M.x, K.x, M.y, K.y, ay, al);
    cgs_block(P, P.mC, T(4) + P.km * P.mC, fv.x - ay, fv.y - al, dy, dl);
    xs[i] = pmake<T>(nb[0].x + dy, nb[0].y + dl);
}

template <typename T, int N, class S_>
__device__ __forceinline__ void cl_cgs_edge(const LevelP<T>& P, const EdgeClass<T>& C, const S_& S,
                                            const typename P2<T>::t* F, int i, int j) {
    using V2 = typename P2<T>::t;
    V2* const rows[3] = {S.xrow(j - 1), S.xrow(j), S.xrow(j + 1)};
    V2 v[7];
    T My, Ky, Ml, Kl, ay, al, dy, dl;
    cl_gather<T, N>(rows, i, j, C, v, My, Ky, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    const V2 fv = F[(j - S.r0) * (N + 1) + i];
    cgs_block(P, C.m[0], C.kd[0] + P.km * C.m[0], fv.x - ay, fv.y - al, dy, dl);
    rows[1][i] = pmake<T>(v[0].x + dy, v[0].y + dl);
}

// ------------------------------------------------------------- kernel --
// Deep-interior nodes of the strip (rows and columns 2..N-2; warp-rounded
// count) come first in every pass, then the strip's edge nodes, so that no warp
// mixes the two paths.
template <typename T, int N, bool CL>
__global__ void __launch_bounds__(strip_threads<T>()) k_smooth_strips(LevelP<T> P,
                                                                      const EdgeClass<T>* __restrict__ ctab,
                                                                      int smoother, int steps, T* __restrict__ x,
                                                                      const T* __restrict__ f) {
    pdl_wait();
    using V2 = typename P2<T>::t;
    constexpr int LD = N + 1;
    constexpr int W = N - 3;             // deep-interior columns
    constexpr int CPR = (N - 3 + 6) / 7;  // slots per row of one colour
    int cs = 1, rank = 0;
    if constexpr (CL) {
        cs = (int)cg::this_cluster().num_blocks();
        rank = (int)cg::this_cluster().block_rank();
    }
    const int rmax = (N + 1 + cs - 1) / cs;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* X = reinterpret_cast<V2*>(smem_raw);
    V2* R = X + rmax * LD;  // same offset in every block of a cluster
    __shared__ EdgeClass<T> s_cls[25];

    Strip<T, N, CL> S;
    S.r0 = strip_row_lo(rank, N + 1, cs);
    S.r1 = strip_row_lo(rank + 1, N + 1, cs);
    S.X = X;
    S.R = R;
    S.Xb = S.Rb = S.Xa = S.Ra = nullptr;
    if constexpr (CL) {
        cg::cluster_group cl = cg::this_cluster();
        if (rank > 0) {
            const int lb = S.r0 - 1 - strip_row_lo(rank - 1, N + 1, cs);  // local index of row r0-1 below
            S.Xb = cl.map_shared_rank(X, rank - 1) + lb * LD;
            S.Rb = cl.map_shared_rank(R, rank - 1) + lb * LD;
        }
        if (rank < cs - 1) {
            S.Xa = cl.map_shared_rank(X, rank + 1);
            S.Ra = cl.map_shared_rank(R, rank + 1);
        }
    }
    // between dependent phases; in a cluster, also before the first remote
    // access (every block has loaded its strip and is running)
    auto barrier = [&]() {
        if constexpr (CL) cluster_barrier();
        else __syncthreads();
    };

    const int g = threadIdx.x, G = blockDim.x;
    {
        constexpr int words = 25 * sizeof(EdgeClass<T>) / sizeof(T);
        T* dst = reinterpret_cast<T*>(s_cls);
        const T* src = reinterpret_cast<const T*>(ctab);
        for (int t = g; t < words; t += G) dst[t] = src[t];
    }
    const int nown = (S.r1 - S.r0) * LD;
    const int64_t base = (int64_t)S.r0 * LD;
    // x, and for LSGS, sLSGS and CGS also f into R (one global round trip;
    // the residual then overwrites each node's f in place)
    for (int t = g; t < nown; t += G) {
        X[t] = pmake<T>(x[base + t], x[base + t + P.fs]);
        if (smoother != 0) R[t] = pmake<T>(f[base + t], f[base + t + P.fs]);
    }
    barrier();

    const int ja = max(S.r0, 2), jb = min(S.r1, N - 1);
    const int nrows = jb > ja ? jb - ja : 0;
    const int nia = nrows * W, niap = (nia + 31) & ~31;
    StripEdges<N> SE;
    SE.first_full_hi = rank == 0 ? 2 : 0;
    SE.nfull = SE.first_full_hi + (rank == cs - 1 ? 2 : 0);
    SE.ja = ja;
    SE.nrows = nrows;
    const int nea = SE.count(-1);

    auto resid_all = [&]() {
        for (int t = g; t < niap + nea; t += G) {
            if (t < niap) {
                if (t < nia) {
                    const int r = t / W, i = 2 + t - r * W, j = ja + r;
                    const int64_t p = (int64_t)j * LD + i;
                    const V2 fv = smoother == 0 ? pmake<T>(f[p], f[p + P.fs]) : S.rrow(j)[i];
                    S.rrow(j)[i] = rows_resid_fast<T>(P, S.xrow(j), S.xrow(j + 1), S.xrow(j - 1), i, fv.x, fv.y);
                }
            } else {
                int i, j;
                if (SE.node(t - niap, -1, i, j)) {
                    const int64_t p = (int64_t)j * LD + i;
                    const V2 fv = smoother == 0 ? pmake<T>(f[p], f[p + P.fs]) : S.rrow(j)[i];
                    cl_resid_edge<T, N>(P, s_cls[cls5(i, N) + 5 * cls5(j, N)], fv, S, i, j);
                }
            }
        }
        barrier();
    };
    auto phase = [&](auto fc, int c) {
        constexpr int field = decltype(fc)::value;
        const int ni = nrows * CPR, nip = (ni + 31) & ~31;
        const int ne = SE.count(c);
        for (int t = g; t < nip + ne; t += G) {
            if (t < nip) {
                if (t < ni) {
                    const int r = t / CPR, k = t - r * CPR, j = ja + r;
                    const int i = 2 + ((c - 2 * j - 2) % 7 + 7) % 7 + 7 * k;
                    if (i <= N - 2) rows_lsgs_fast<T>(P, field, S.xrow(j), S.rrow(j), S.rrow(j + 1), S.rrow(j - 1), i);
                }
            } else {
                int i, j;
                if (SE.node(t - nip, c, i, j))
                    cl_lsgs_edge<T, N>(P, s_cls[cls5(i, N) + 5 * cls5(j, N)], field, S, i, j);
            }
        }
        barrier();
    };

    if (smoother == 3) {
        // CGS keeps no residual: R holds the strip's (f_y, f_lambda) pairs
        constexpr int CPR3 = (N - 3 + 2) / 3;  // deep-interior slots per row of one colour
        StripEdges<N, 3, 1, 1> SE3;
        SE3.first_full_hi = SE.first_full_hi;
        SE3.nfull = SE.nfull;
        SE3.ja = ja;
        SE3.nrows = nrows;
        for (int m = 0; m < steps; ++m)
            for (int c = 0; c < 3; ++c) {
                const int ni = nrows * CPR3, nip = (ni + 31) & ~31;
                const int ne = SE3.count(c);
                for (int t = g; t < nip + ne; t += G) {
                    if (t < nip) {
                        if (t < ni) {
                            const int r = t / CPR3, k = t - r * CPR3, j = ja + r;
                            const int i = 2 + ((c - j - 2) % 3 + 3) % 3 + 3 * k;
                            if (i <= N - 2)
                                rows_cgs_fast<T>(P, S.xrow(j), S.xrow(j + 1), S.xrow(j - 1), i, R[(j - S.r0) * LD + i]);
                        }
                    } else {
                        int i, j;
                        if (SE3.node(t - nip, c, i, j)) cl_cgs_edge<T, N>(P, s_cls[cls5(i, N) + 5 * cls5(j, N)], S, R, i, j);
                    }
                }
                barrier();
            }
    } else if (smoother == 0) {
        for (int m = 0; m < steps; ++m) {
            resid_all();
            for (int t = g; t < niap + nea; t += G) {
                if (t < niap) {
                    if (t < nia) {
                        const int r = t / W, i = 2 + t - r * W, j = ja + r;
                        rows_ne_fast<T>(P, S.xrow(j), S.rrow(j), S.rrow(j + 1), S.rrow(j - 1), i);
                    }
                } else {
                    int i, j;
                    if (SE.node(t - niap, -1, i, j)) cl_ne_edge<T, N>(P, s_cls[cls5(i, N) + 5 * cls5(j, N)], S, i, j);
                }
            }
            barrier();
        }
    } else {
        resid_all();
        for (int m = 0; m < steps; ++m) {
            for (int c = 0; c < 7; ++c) phase(FieldC<0>{}, colour_seq(c));
            for (int c = 0; c < 7; ++c) phase(FieldC<1>{}, colour_seq(c));
            if (smoother == 2) {
                for (int c = 6; c >= 0; --c) phase(FieldC<1>{}, colour_seq(c));
                for (int c = 6; c >= 0; --c) phase(FieldC<0>{}, colour_seq(c));
            }
        }
    }
    // after the last barrier no block touches another's shared memory
    for (int t = g; t < nown; t += G) {
        const V2 v = X[t];
        x[base + t] = v.x;
        x[base + t + P.fs] = v.y;
    }
}

// ------------------------------------ level 513^2: residual on chip only --
// On the level with 513 x 513 nodes the iterate and the residual of a 16-block
// cluster's strips (4.2 MB in FP32) do not fit in shared memory, the residual
// alone does (33 rows of (y, lambda) pairs, 135 KB per block).  This kernel
// keeps the scaled residual on chip for the whole smoothing call and updates
// the iterate in place in global memory (L2-resident): in an LSGS phase each
// update writes one field of one node, which only the updating thread touches,
// and the residual at the start of the call is the only place that reads a
// node's neighbours' x.  LSGS and sLSGS only (NE recomputes the residual from
// x every step, CGS reads its neighbours' x in every phase).
template <typename T>
struct RhLocal {  // the strip's residual pairs addressed by global node index
    typename P2<T>::t* r;
    int64_t off;
    __device__ __forceinline__ T& y(int64_t p) const { return r[p - off].x; }
    __device__ __forceinline__ T& l(int64_t p) const { return r[p - off].y; }
};

// Algorithm 2 update of (field, node (i, j)) on the residual rows: gather,
// p = q / N_ii, scatter; returns p (the caller adds it to x)
template <typename T, typename V2>
__device__ __forceinline__ T rg_lsgs_fast(const LevelP<T>& P, int field, V2* rs, V2* rsp, V2* rsm, int i) {
    V2 M, K, nb[7];
    rows_stencil(rs, rsp, rsm, i, psplat(P.mC), psplat(P.mO), M, K, nb);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T pv = field == 0 ? qy * P.invNy_int : ql * P.invNl_int;
    const V2 mp = psplat(-pv);
    const V2 cC = pmake<T>(P.sc[field][0][0], P.sc[field][0][1]);
    const V2 cE = pmake<T>(P.sc[field][1][0], P.sc[field][1][1]);
    const V2 cD = pmake<T>(P.sc[field][2][0], P.sc[field][2][1]);
    rs[i] = pfma(mp, cC, nb[0]);
    rs[i + 1] = pfma(mp, cE, nb[1]);
    rs[i - 1] = pfma(mp, cE, nb[2]);
    rsp[i] = pfma(mp, cE, nb[3]);
    rsm[i] = pfma(mp, cE, nb[4]);
    rsp[i + 1] = pfma(mp, cD, nb[5]);
    rsm[i - 1] = pfma(mp, cD, nb[6]);
    return pv;
}

template <typename T, int N, class S_>
__device__ __forceinline__ T rg_lsgs_edge(const LevelP<T>& P, const EdgeClass<T>& C, int field, const S_& S, int i,
                                          int j) {
    using V2 = typename P2<T>::t;
    V2 sc[7];  // read before the first store
#pragma unroll
    for (int o = 0; o < 7; ++o) sc[o] = pmake<T>(C.sc[field][o][0], C.sc[field][o][1]);
    const T inv_nd = field == 0 ? C.iny : C.inl;
    V2* const rows[3] = {S.rrow(j - 1), S.rrow(j), S.rrow(j + 1)};
    V2 v[7];
    T My, Ky, Ml, Kl, qy, ql;
    cl_gather<T, N>(rows, i, j, C, v, My, Ky, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T p = (field == 0 ? qy : ql) * inv_nd;
    const V2 mp = psplat(-p);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        const int ii = i + DI(o), jj = j + DJ(o);
        if (in_grid(ii, jj, N)) rows[DJ(o) + 1][ii] = pfma(mp, sc[o], v[o]);
    }
    return p;
}

constexpr int kRgThreads = 512;  // threads per block of the 513^2 cluster kernel

template <typename T, int N>
__global__ void __launch_bounds__(kRgThreads) k_smooth_rg(LevelP<T> P, const EdgeClass<T>* __restrict__ ctab,
                                                                  int smoother, int steps, T* __restrict__ x,
                                                                  const T* __restrict__ f) {
    pdl_wait();
    using V2 = typename P2<T>::t;
    constexpr int LD = N + 1;
    constexpr int W = N - 3;              // deep-interior columns
    constexpr int CPR = (N - 3 + 6) / 7;  // slots per row of one colour
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* R = reinterpret_cast<V2*>(smem_raw);
    __shared__ EdgeClass<T> s_cls[25];

    Strip<T, N, true> S;
    S.r0 = strip_row_lo(rank, N + 1, cs);
    S.r1 = strip_row_lo(rank + 1, N + 1, cs);
    S.X = S.Xb = S.Xa = nullptr;  // the iterate stays in global memory
    S.R = R;
    S.Rb = S.Ra = nullptr;
    if (rank > 0) {
        const int lb = S.r0 - 1 - strip_row_lo(rank - 1, N + 1, cs);  // local index of row r0-1 below
        S.Rb = cl.map_shared_rank(R, rank - 1) + lb * LD;
    }
    if (rank < cs - 1) S.Ra = cl.map_shared_rank(R, rank + 1);

    const int g = threadIdx.x, G = blockDim.x;
    {
        constexpr int words = 25 * sizeof(EdgeClass<T>) / sizeof(T);
        T* dst = reinterpret_cast<T*>(s_cls);
        const T* src = reinterpret_cast<const T*>(ctab);
        for (int t = g; t < words; t += G) dst[t] = src[t];
    }
    // the residual L^{-1}(f - A x) of the strip's nodes from global x and f:
    // the constant interior stencil where the whole neighbourhood is interior,
    // the general stencil on the two rows and columns along the boundary
    const RhLocal<T> rl{R, (int64_t)S.r0 * LD};
    for (int t = g; t < (S.r1 - S.r0) * LD; t += G) {
        const int j = S.r0 + t / LD, i = t - (j - S.r0) * LD;
        if (i >= 2 && i <= N - 2 && j >= 2 && j <= N - 2) {
            const int64_t p = (int64_t)j * LD + i;
            const T* xl = x + P.fs;
            const T y4 = (x[p + 1] + x[p - 1]) + (x[p + LD] + x[p - LD]);
            const T l4 = (xl[p + 1] + xl[p - 1]) + (xl[p + LD] + xl[p - LD]);
            const T y6 = y4 + (x[p + LD + 1] + x[p - LD - 1]);
            const T l6 = l4 + (xl[p + LD + 1] + xl[p - LD - 1]);
            const T My = P.mC * x[p] + P.mO * y6, Ml = P.mC * xl[p] + P.mO * l6;
            const T Ky = T(4) * x[p] - y4, Kl = T(4) * xl[p] - l4;
            T ay, al;
            rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
            const T il = P.invLy_int;
            R[t] = pmake<T>((f[p] - ay) * il, (f[p + P.fs] - al) * (il * P.invd));
        } else {
            resid_hat_acc(P, f, x, rl, i, j);
        }
    }
    // every block has its residual and is running before any remote access
    cluster_barrier();

    const int ja = max(S.r0, 2), jb = min(S.r1, N - 1);
    const int nrows = jb > ja ? jb - ja : 0;
    StripEdges<N> SE;
    SE.first_full_hi = rank == 0 ? 2 : 0;
    SE.nfull = SE.first_full_hi + (rank == cs - 1 ? 2 : 0);
    SE.ja = ja;
    SE.nrows = nrows;
    (void)W;

    // A thread's first kSlots slots of a phase are resolved once per call
    // (SlotDesc); in a phase every slot's node and its x value come first (one
    // round of L2 loads in flight together), then the updates.  Further slots
    // (none at 513^2 with 16 blocks of 512 threads) by the enumeration.
    constexpr int kSlots = 5;
    const int ni = nrows * CPR, nip = (ni + 31) & ~31, ne = SE.count(0);
    SlotDesc sd[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; ++q) sd[q] = slot_desc<N, CPR>(g + q * G, ni, nip, SE);
    const int jmax = ja + nrows - 1;
    auto phase = [&](auto fc, int c) {
        constexpr int field = decltype(fc)::value;
        const int64_t foff = field ? P.fs : 0;
        int si[kSlots], sj[kSlots];
        bool on[kSlots];
        T xv[kSlots];
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            on[q] = slot_node<N>(sd[q], c, jmax, si[q], sj[q]);
            xv[q] = on[q] ? x[(int64_t)sj[q] * LD + si[q] + foff] : T(0);
        }
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            if (!on[q]) continue;
            const int i = si[q], j = sj[q];
            const T pv = (sd[q] & 3) == 1
                             ? rg_lsgs_fast<T>(P, field, S.rrow(j), S.rrow(j + 1), S.rrow(j - 1), i)
                             : rg_lsgs_edge<T, N>(P, s_cls[cls5(i, N) + 5 * cls5(j, N)], field, S, i, j);
            x[(int64_t)j * LD + i + foff] = xv[q] + pv;
        }
        for (int t = g + kSlots * G; t < nip + ne; t += G) {
            int i, j;
            T pv;
            if (t < nip) {
                if (t >= ni) continue;
                const int r = t / CPR, k = t - r * CPR;
                j = ja + r;
                i = 2 + ((c - 2 * j - 2) % 7 + 7) % 7 + 7 * k;
                if (i > N - 2) continue;
                pv = rg_lsgs_fast<T>(P, field, S.rrow(j), S.rrow(j + 1), S.rrow(j - 1), i);
            } else {
                if (!SE.node(t - nip, c, i, j)) continue;
                pv = rg_lsgs_edge<T, N>(P, s_cls[cls5(i, N) + 5 * cls5(j, N)], field, S, i, j);
            }
            x[(int64_t)j * LD + i + foff] += pv;
        }
        cluster_barrier();
    };
    for (int m = 0; m < steps; ++m) {
        for (int c = 0; c < 7; ++c) phase(FieldC<0>{}, colour_seq(c));
        for (int c = 0; c < 7; ++c) phase(FieldC<1>{}, colour_seq(c));
        if (smoother == 2) {
            for (int c = 6; c >= 0; --c) phase(FieldC<1>{}, colour_seq(c));
            for (int c = 6; c >= 0; --c) phase(FieldC<0>{}, colour_seq(c));
        }
    }
}

template <typename T, int N, bool CL>
cudaLaunchConfig_t strips_config(int cs, cudaStream_t s, cudaLaunchAttribute* at, bool pdl = true) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(strip_threads<T>(), 1, 1);
    cfg.dynamicSmemBytes = strips_smem<T>(N, cs);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 0;
    if (pdl && !g_pdl_off) {
        at[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see pdl.h
        at[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
        ++cfg.numAttrs;
    }
    if (CL) {
        at[cfg.numAttrs].id = cudaLaunchAttributeClusterDimension;
        at[cfg.numAttrs].val.clusterDim.x = cs;
        at[cfg.numAttrs].val.clusterDim.y = 1;
        at[cfg.numAttrs].val.clusterDim.z = 1;
        ++cfg.numAttrs;
    }
    return cfg;
}

}  // namespace

// instantiated level sizes: single block for n = 4 .. 64, cluster for 64 .. 256
#define AAOMG_BLOCK_N(CALL) CALL(4) CALL(8) CALL(16) CALL(32) CALL(64)
#define AAOMG_CLUSTER_N(CALL) CALL(64) CALL(128) CALL(256)

template <typename T>
size_t strips_smem(int n, int cs) {
    const size_t rmax = (size_t)(n + 1 + cs - 1) / cs;
    return 2 * rmax * (n + 1) * sizeof(typename P2<T>::t);
}

template <typename T>
cudaError_t strips_prepare() {
    cudaError_t e = cudaSuccess;
#define B_(N)                                                                                            \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_smooth_strips<T, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 kStripSmemMax);
#define C_(N)                                                                                           \
    if (e == cudaSuccess)                                                                               \
        e = cudaFuncSetAttribute(k_smooth_strips<T, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 kStripSmemMax);                                                        \
    if (e == cudaSuccess)                                                                               \
        e = cudaFuncSetAttribute(k_smooth_strips<T, N, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    AAOMG_BLOCK_N(B_)
    AAOMG_CLUSTER_N(C_)
#undef B_
#undef C_
    return e;
}

template <typename T>
bool strips_fit(int n, int cs) {
    if (cs < 1 || cs > kClusterMax || (cs > 1 && (n + 1) / cs < 2)) return false;
    if (cs == 1 ? !block_level(n) : !cluster_level(n)) return false;
    return strips_smem<T>(n, cs) <= (size_t)kStripSmemMax;
}

template <typename T>
int strips_max_active(int n, int cs) {
    if (!strips_fit<T>(n, cs)) return 0;
    if (cs == 1) return 1;
    cudaLaunchAttribute at[2];
    int num = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (n) {
#define C_(N)                                                                                  \
    case N: {                                                                                  \
        cudaLaunchConfig_t cfg = strips_config<T, N, true>(cs, 0, at, false);                  \
        e = cudaOccupancyMaxActiveClusters(&num, (void*)k_smooth_strips<T, N, true>, &cfg);    \
        break;                                                                                 \
    }
        AAOMG_CLUSTER_N(C_)
#undef C_
    default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();  // a refused size is an answer, not a sticky error
        return 0;
    }
    return num;
}

template <typename T>
cudaError_t launch_smooth_strips(const LevelP<T>& P, const EdgeClass<T>* ctab, int smoother, int steps, T* x,
                                 const T* f, int cs, cudaStream_t s) {
    cudaLaunchAttribute at[2];
    if (cs == 1) {
        switch (P.n) {
#define B_(N)                                                                                        \
    case N: {                                                                                        \
        cudaLaunchConfig_t cfg = strips_config<T, N, false>(1, s, at);                               \
        return cudaLaunchKernelEx(&cfg, k_smooth_strips<T, N, false>, P, ctab, smoother, steps, x, f);     \
    }
            AAOMG_BLOCK_N(B_)
#undef B_
        default: return cudaErrorInvalidValue;
        }
    }
    switch (P.n) {
#define C_(N)                                                                                       \
    case N: {                                                                                       \
        cudaLaunchConfig_t cfg = strips_config<T, N, true>(cs, s, at);                              \
        return cudaLaunchKernelEx(&cfg, k_smooth_strips<T, N, true>, P, ctab, smoother, steps, x, f);     \
    }
        AAOMG_CLUSTER_N(C_)
#undef C_
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------- the 513^2 cluster kernel --
constexpr int kRgN = 512;    // cells per side of the level it serves
constexpr int kRgBlocks = 16;

template <typename T>
size_t rg_smem() {
    const size_t rmax = (size_t)(kRgN + 1 + kRgBlocks - 1) / kRgBlocks;
    return rmax * (kRgN + 1) * sizeof(typename P2<T>::t);
}

namespace {
template <typename T>
cudaLaunchConfig_t rg_config(cudaStream_t s, cudaLaunchAttribute* at, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kRgBlocks, 1, 1);
    cfg.blockDim = dim3(kRgThreads, 1, 1);
    cfg.dynamicSmemBytes = rg_smem<T>();
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 0;
    if (pdl && !g_pdl_off) {
        at[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see pdl.h
        at[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
        ++cfg.numAttrs;
    }
    at[cfg.numAttrs].id = cudaLaunchAttributeClusterDimension;
    at[cfg.numAttrs].val.clusterDim.x = kRgBlocks;
    at[cfg.numAttrs].val.clusterDim.y = 1;
    at[cfg.numAttrs].val.clusterDim.z = 1;
    ++cfg.numAttrs;
    return cfg;
}
}  // namespace

template <typename T>
int rg_max_active(int n) {
    if (sizeof(T) != 4 || n != kRgN || rg_smem<T>() > (size_t)kStripSmemMax) return 0;
    if (cudaFuncSetAttribute(k_smooth_rg<T, kRgN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStripSmemMax) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_smooth_rg<T, kRgN>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = rg_config<T>(0, at, false);
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, (void*)k_smooth_rg<T, kRgN>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return num;
}

template <typename T>
cudaError_t launch_smooth_rg(const LevelP<T>& P, const EdgeClass<T>* ctab, int smoother, int steps, T* x, const T* f,
                             cudaStream_t s) {
    if (sizeof(T) != 4 || P.n != kRgN || (smoother != 1 && smoother != 2)) return cudaErrorInvalidValue;
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = rg_config<T>(s, at, true);
    return cudaLaunchKernelEx(&cfg, k_smooth_rg<T, kRgN>, P, ctab, smoother, steps, x, f);
}

#define AAOMG_STRIPS_INST(T)                                                                                    \
    template size_t strips_smem<T>(int, int);                                                                   \
    template cudaError_t strips_prepare<T>();                                                                   \
    template bool strips_fit<T>(int, int);                                                                      \
    template int strips_max_active<T>(int, int);                                                                \
    template cudaError_t launch_smooth_strips<T>(const LevelP<T>&, const EdgeClass<T>*, int, int, T*, const T*, int, \
                                                 cudaStream_t);                                                 \
    template int rg_max_active<T>(int);                                                                         \
    template cudaError_t launch_smooth_rg<T>(const LevelP<T>&, const EdgeClass<T>*, int, int, T*, const T*,     \
                                             cudaStream_t);
AAOMG_STRIPS_INST(float)
AAOMG_STRIPS_INST(double)

}  // namespace aaomg
