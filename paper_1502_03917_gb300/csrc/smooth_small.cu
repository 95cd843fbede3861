// smooth_small.cu -- a whole smoothing call (nu steps of Algorithm 1 or 2) on
// one grid level in ONE launch, for the small and middle levels of the cycle.
//
// On small levels a smoothing step is a chain of short dependent phases (the
// residual, then for LSGS the 14 colour phases y 0,6,5,4,3,2,1 then lambda
// 0,6,5,4,3,2,1 of (i + 2j) mod 7; for NE the residual and the update); a
// launch per phase costs more than the phase.  These kernels loop over the
// phases with a barrier between them instead:
//   * k_smooth_block: one thread block; the scaled residual rh = L^{-1}(f - Ax)
//     lives in shared memory (every gather and scatter of Algorithm 2 hits it),
//     x and f stay in global memory (each is touched once per unknown).
//   * k_smooth_cluster: one thread-block cluster; x, f and rh stay in global
//     memory, resident in L2, and are read past L1 (the blocks of a cluster run
//     on different SMs); phases are separated by the hardware cluster barrier.
// The updates inside one colour phase are independent (distance-2 colouring),
// so any assignment of nodes to threads gives the sequential sweep's result.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "edge.h"
#include "lean.cuh"
#include "small.h"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace aaomg {

namespace {

struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct ClusterSync {
    __device__ __forceinline__ void operator()() const { cg::this_cluster().sync(); }
};

// ----------------------------------------------- tabulated edge updates --
template <typename T>
struct EdgeRow {
    int p, mask;
    T m[7], kd[7];
};

template <typename T>
__device__ __forceinline__ void edge_load(const EdgeTable<T>& E, int e, EdgeRow<T>& r) {
    r.p = E.node[e];
    r.mask = E.mask[e];
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        r.m[o] = E.m[o * E.total + e];
        r.kd[o] = E.kd[o * E.total + e];
    }
}

__device__ __forceinline__ int edge_off(int o, int ld) {
    return DI(o) + DJ(o) * ld;
}

template <typename T>
__device__ __forceinline__ void edge_gather(const EdgeRow<T>& r, const T* v, int ld, T& Mv, T& Kv) {
    Mv = T(0);
    Kv = T(0);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        T a = ((r.mask >> o) & 1) ? v[r.p + edge_off(o, ld)] : T(0);
        Mv += r.m[o] * a;
        Kv += r.kd[o] * a;
    }
}

template <typename T>
__device__ __forceinline__ void resid_edge(const LevelP<T>& P, const EdgeTable<T>& E, int e, const T* f, const T* x,
                                           T* rh) {
    EdgeRow<T> r;
    edge_load(E, e, r);
    T My, Ky, Ml, Kl, ay, al;
    edge_gather(r, x, P.ld, My, Ky);
    edge_gather(r, x + P.fs, P.ld, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    const T il = E.il[e];  // offset 0 is the node itself
    rh[r.p] = (f[r.p] - ay) * il;
    rh[r.p + P.fs] = (f[r.p + P.fs] - al) * (il * P.invd);
}

template <typename T>
__device__ __forceinline__ void ne_edge(const LevelP<T>& P, const EdgeTable<T>& E, int e, T* x, const T* rh) {
    EdgeRow<T> r;
    edge_load(E, e, r);
    T My, Ky, Ml, Kl, qy, ql;
    edge_gather(r, rh, P.ld, My, Ky);
    edge_gather(r, rh + P.fs, P.ld, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T il = E.il[e];
    x[r.p] += P.tau * il * qy;
    x[r.p + P.fs] += P.tau * (il * P.invd) * ql;
}

template <typename T>
__device__ __forceinline__ void lsgs_edge(const LevelP<T>& P, const EdgeTable<T>& E, int e, int field, T* x,
                                          T* rh) {
    EdgeRow<T> r;
    edge_load(E, e, r);
    T ry[7], rl[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        bool v = (r.mask >> o) & 1;
        ry[o] = v ? rh[r.p + edge_off(o, P.ld)] : T(0);
        rl[o] = v ? rh[r.p + edge_off(o, P.ld) + P.fs] : T(0);
    }
    T My = T(0), Ky = T(0), Ml = T(0), Kl = T(0);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        My += r.m[o] * ry[o];
        Ky += r.kd[o] * ry[o];
        Ml += r.m[o] * rl[o];
        Kl += r.kd[o] * rl[o];
    }
    T qy, ql;
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    T p = field == 0 ? qy * E.inv_ny[e] : ql * E.inv_nl[e];
    x[r.p + (field ? P.fs : 0)] += p;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        if (!((r.mask >> o) & 1)) continue;
        const int q = r.p + edge_off(o, P.ld);
        const T il = E.il[o * E.total + e];
        T mp = r.m[o] * p;
        T kp = P.c * (r.kd[o] * p + P.km * mp);
        if (field == 0) {
            rh[q] = ry[o] - mp * il;
            rh[q + P.fs] = rl[o] - kp * (il * P.invd);
        } else {
            rh[q] = ry[o] - kp * il;
            rh[q + P.fs] = rl[o] + mp * il;
        }
    }
}

// Gather of v at the 7 offsets through an L2 load (cluster variant).
template <typename T>
__device__ __forceinline__ void load7_l2(const LevelP<T>& P, const T* v, int i, int j, T out[7]) {
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        out[o] = in_grid(ii, jj, P.n) ? __ldcg(v + (int64_t)jj * P.ld + ii) : T(0);
    }
}

// rh = L^{-1}(f - A x) at (i,j) with x, f read through L2
template <typename T>
__device__ __forceinline__ void resid_hat_l2(const LevelP<T>& P, const T* f, const T* x, T* rh, int i, int j) {
    T m[7], kd[7], y[7], l[7];
    row_coeffs(P, i, j, m, kd);
    load7_l2(P, x, i, j, y);
    load7_l2(P, x + P.fs, i, j, l);
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, ay, al;
    dots(in, m, kd, y, My, Ky);
    dots(in, m, kd, l, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    int64_t p = nidx(P, i, j);
    T il = inv_ly(P, i, j);
    __stcg(rh + p, (__ldcg(f + p) - ay) * il);
    __stcg(rh + p + P.fs, (__ldcg(f + p + P.fs) - al) * (il * P.invd));
}

template <typename T>
__device__ __forceinline__ void ne_update_l2(const LevelP<T>& P, T* x, const T* rh, int i, int j) {
    T m[7], kd[7], y[7], l[7];
    row_coeffs(P, i, j, m, kd);
    load7_l2(P, rh, i, j, y);
    load7_l2(P, rh + P.fs, i, j, l);
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, qy, ql;
    dots(in, m, kd, y, My, Ky);
    dots(in, m, kd, l, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    int64_t p = nidx(P, i, j);
    T il = inv_ly(P, i, j);
    __stcg(x + p, __ldcg(x + p) + P.tau * il * qy);
    __stcg(x + p + P.fs, __ldcg(x + p + P.fs) + P.tau * (il * P.invd) * ql);
}

template <typename T>
__device__ __forceinline__ void lsgs_update_l2(const LevelP<T>& P, int field, T* x, T* rh, int i, int j) {
    T m[7], kd[7], ry[7], rl[7];
    row_coeffs(P, i, j, m, kd);
    load7_l2(P, rh, i, j, ry);
    load7_l2(P, rh + P.fs, i, j, rl);
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, qy, ql;
    dots(in, m, kd, ry, My, Ky);
    dots(in, m, kd, rl, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    T p = (field == 0 ? qy : ql) * inv_n(P, field, i, j);
    int64_t q0 = nidx(P, i, j) + (field ? P.fs : 0);
    __stcg(x + q0, __ldcg(x + q0) + p);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        if (!in && !in_grid(ii, jj, P.n)) continue;
        T il = inv_ly(P, ii, jj);
        int64_t q = nidx(P, ii, jj);
        T mp = m[o] * p;
        T kp = P.c * (kd[o] * p + P.km * mp);
        if (field == 0) {
            __stcg(rh + q, ry[o] - mp * il);
            __stcg(rh + q + P.fs, rl[o] - kp * (il * P.invd));
        } else {
            __stcg(rh + q, ry[o] - kp * il);
            __stcg(rh + q + P.fs, rl[o] + mp * il);
        }
    }
}

// phase loops shared by both kernels; `sync` separates dependent phases,
// `g`/`G` are the thread's rank and the thread count of the group
template <typename T, bool L2, typename Sync>
__device__ void smooth_loop(const LevelP<T>& P, const EdgeTable<T>& E, int smoother, int steps, T* x, const T* f,
                            T* rh, int g, int G, Sync sync) {
    const int n1 = P.n + 1, nn = n1 * n1;
    // the deep-interior nodes (warp-rounded) first, then the edge nodes: a warp
    // never mixes the constant-stencil path with the general one (L1 variant)
    const InteriorAll ia(P.n);
    const int nia = ia.count(), niap = (nia + 31) & ~31, nea = E.total;
    auto resid_all = [&]() {
        if (L2) {
            for (int t = g; t < nn; t += G) resid_hat_l2(P, f, x, rh, t % n1, t / n1);
        } else {
            for (int t = g; t < niap + nea; t += G) {
                int i, j;
                if (t < niap) {
                    if (t < nia) {
                        ia.node(t, i, j);
                        resid_fast(P, f, x, rh, i, j);
                    }
                } else {
                    resid_edge(P, E, t - niap, f, x, rh);
                }
            }
        }
        sync();
    };
    auto phase = [&](int field, int colour) {
        if (L2) {
            const int cpr = (n1 + 6) / 7;
            for (int t = g; t < n1 * cpr; t += G) {
                int j = t / cpr, k = t - j * cpr;
                int i = ((colour - 2 * j) % 7 + 7) % 7 + 7 * k;
                if (i <= P.n) lsgs_update_l2(P, field, x, rh, i, j);
            }
        } else {
            const InteriorColour ic(P.n, colour);
            const int ni = ic.count(), nip = (ni + 31) & ~31, ne = E.count[colour], e0 = E.start[colour];
            for (int t = g; t < nip + ne; t += G) {
                int i, j;
                if (t < nip) {
                    if (t < ni && ic.node(t, i, j)) lsgs_fast(P, field, x, rh, i, j);
                } else {
                    lsgs_edge(P, E, e0 + t - nip, field, x, rh);
                }
            }
        }
        sync();
    };
    if (smoother == 0) {
        for (int m = 0; m < steps; ++m) {
            resid_all();
            if (L2) {
                for (int t = g; t < nn; t += G) ne_update_l2(P, x, rh, t % n1, t / n1);
            } else {
                for (int t = g; t < niap + nea; t += G) {
                    int i, j;
                    if (t < niap) {
                        if (t < nia) {
                            ia.node(t, i, j);
                            ne_fast(P, x, rh, i, j);
                        }
                    } else {
                        ne_edge(P, E, t - niap, x, rh);
                    }
                }
            }
            sync();
        }
        return;
    }
    resid_all();
    for (int m = 0; m < steps; ++m) {
        for (int field = 0; field < 2; ++field)
            for (int c = 0; c < 7; ++c) phase(field, colour_seq(c));
        if (smoother == 2)
            for (int field = 1; field >= 0; --field)
                for (int c = 6; c >= 0; --c) phase(field, colour_seq(c));
    }
}

template <typename T>
__global__ void __launch_bounds__(small_threads<T>()) k_smooth_block(LevelP<T> P, EdgeTable<T> E, int smoother,
                                                                     int steps, T* x, const T* __restrict__ f) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* rh = reinterpret_cast<T*>(smem_raw);  // layout of P (ld = n+1, fs = (n+1)^2)
    smooth_loop<T, false>(P, E, smoother, steps, x, f, rh, threadIdx.x, blockDim.x, BlockSync{});
}

template <typename T>
__global__ void __launch_bounds__(small_threads<T>()) k_smooth_cluster(LevelP<T> P, int smoother, int steps, T* x,
                                                                       const T* __restrict__ f, T* rh) {
    cg::cluster_group cl = cg::this_cluster();
    int g = (int)(cl.block_rank() * blockDim.x + threadIdx.x);
    int G = (int)(cl.num_blocks() * blockDim.x);
    smooth_loop<T, true>(P, EdgeTable<T>{}, smoother, steps, x, f, rh, g, G, ClusterSync{});
}

}  // namespace

template <typename T>
size_t block_smooth_smem(int n) {
    return sizeof(T) * 2 * (size_t)(n + 1) * (n + 1);
}

template <typename T>
cudaError_t small_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_smooth_block<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlockSmemMax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_smooth_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename T>
void launch_smooth_block(const LevelP<T>& P, const EdgeTable<T>& E, int smoother, int steps, T* x, const T* f,
                         cudaStream_t s) {
    k_smooth_block<T><<<1, small_threads<T>(), block_smooth_smem<T>(P.n), s>>>(P, E, smoother, steps, x, f);
}

template <typename T>
cudaError_t launch_smooth_cluster(const LevelP<T>& P, int smoother, int steps, T* x, const T* f, T* rh, int csize,
                                  cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    cfg.blockDim = dim3(small_threads<T>(), 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_smooth_cluster<T>, P, smoother, steps, x, f, rh);
}

template <typename T>
int max_cluster_size() {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(small_threads<T>(), 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int cs = 16; cs >= 2; cs /= 2) {
        cfg.gridDim.x = cs;
        attr[0].val.clusterDim.x = cs;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_smooth_cluster<T>, &cfg) == cudaSuccess && ncl > 0) return cs;
        cudaGetLastError();
    }
    return 1;
}

#define AAOMG_SMALL_INST(T)                                                                                       \
    template size_t block_smooth_smem<T>(int);                                                                    \
    template cudaError_t small_prepare<T>();                                                                      \
    template void launch_smooth_block<T>(const LevelP<T>&, const EdgeTable<T>&, int, int, T*, const T*,           \
                                         cudaStream_t);                                                           \
    template cudaError_t launch_smooth_cluster<T>(const LevelP<T>&, int, int, T*, const T*, T*, int, cudaStream_t); \
    template int max_cluster_size<T>();
AAOMG_SMALL_INST(float)
AAOMG_SMALL_INST(double)

}  // namespace aaomg
