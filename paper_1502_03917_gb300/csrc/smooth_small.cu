// smooth_small.cu -- a whole smoothing call (nu steps of Algorithm 1 or 2) on
// one small grid level in ONE launch of ONE thread block.
//
// On small levels a smoothing step is a chain of short dependent phases (the
// residual, then for LSGS the 14 colour phases y 0,6,5,4,3,2,1 then lambda
// 0,6,5,4,3,2,1 of (i + 2j) mod 7; for NE the residual and the update); a
// launch per phase costs more than the phase.  This kernel loops over the
// phases with a block barrier between them instead.  The scaled residual
// rh = L^{-1}(f - Ax) lives in shared memory as (y, lambda) pairs (every gather
// and scatter of Algorithm 2 hits it); x and f stay in global memory (each is
// touched once per unknown).
// The updates inside one colour phase are independent (distance-2 colouring),
// so any assignment of nodes to threads gives the sequential sweep's result.
#include <cuda_runtime.h>

#include "edge.h"
#include "lean.cuh"
#include "small.h"
#include "stencil.cuh"


namespace aaomg {

namespace {


// ----------------------------------------------- tabulated edge updates --
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
                                           typename P2<T>::t* rh, int ld, int fs) {
    EdgeRow<T> r;
    edge_load(E, e, r);
    T My, Ky, Ml, Kl, ay, al;
    edge_gather(r, x, ld, My, Ky);
    edge_gather(r, x + fs, ld, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    const T il = E.il[e];  // offset 0 is the node itself
    rh[r.p] = pmake<T>((f[r.p] - ay) * il, (f[r.p + fs] - al) * (il * P.invd));
}

template <typename T>
__device__ __forceinline__ void ne_edge(const LevelP<T>& P, const EdgeTable<T>& E, int e, T* x,
                                        const typename P2<T>::t* rh, int ld, int fs) {
    EdgeRow<T> r;
    edge_load(E, e, r);
    T My = T(0), Ky = T(0), Ml = T(0), Kl = T(0), qy, ql;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        typename P2<T>::t a = ((r.mask >> o) & 1) ? rh[r.p + edge_off(o, ld)] : pmake<T>(T(0), T(0));
        My += r.m[o] * a.x;
        Ky += r.kd[o] * a.x;
        Ml += r.m[o] * a.y;
        Kl += r.kd[o] * a.y;
    }
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T il = E.il[e];
    x[r.p] += P.tau * il * qy;
    x[r.p + fs] += P.tau * (il * P.invd) * ql;
}

template <typename T>
__device__ __forceinline__ void lsgs_edge(const LevelP<T>& P, const EdgeTable<T>& E, int e, int field, T* x,
                                          typename P2<T>::t* rh, int ld, int fs) {
    EdgeRow<T> r;
    edge_load(E, e, r);
    T ry[7], rl[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        typename P2<T>::t a = ((r.mask >> o) & 1) ? rh[r.p + edge_off(o, ld)] : pmake<T>(T(0), T(0));
        ry[o] = a.x;
        rl[o] = a.y;
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
    x[r.p + (field ? fs : 0)] += p;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        if (!((r.mask >> o) & 1)) continue;
        const int q = r.p + edge_off(o, ld);
        const T il = E.il[o * E.total + e];
        T mp = r.m[o] * p;
        T kp = P.c * (r.kd[o] * p + P.km * mp);
        if (field == 0) rh[q] = pmake<T>(ry[o] - mp * il, rl[o] - kp * (il * P.invd));
        else rh[q] = pmake<T>(ry[o] - kp * il, rl[o] + mp * il);
    }
}

// The phases of `steps` smoothing steps, one barrier between dependent phases.
// Deep-interior nodes (warp-rounded count) come first, then the tabulated edge
// nodes, so that no warp mixes the two paths.
template <typename T, int N>
__device__ void smooth_loop(const LevelP<T>& P, const EdgeTable<T>& E, int smoother, int steps, T* x, const T* f,
                            typename P2<T>::t* rh) {
    const int g = threadIdx.x, G = blockDim.x;
    constexpr int ld = N + 1, fs = ld * ld;
    const InteriorAll ia(N);
    const int nia = ia.count(), niap = (nia + 31) & ~31, nea = E.total;
    auto resid_all = [&]() {
        for (int t = g; t < niap + nea; t += G) {
            int i, j;
            if (t < niap) {
                if (t < nia) {
                    ia.node(t, i, j);
                    resid_fast(P, f, x, rh, i, j, ld, fs);
                }
            } else {
                resid_edge(P, E, t - niap, f, x, rh, ld, fs);
            }
        }
        __syncthreads();
    };
    auto phase = [&](int field, int colour) {
        const InteriorColour ic(N, colour);
        const int ni = ic.count(), nip = (ni + 31) & ~31, ne = E.count[colour], e0 = E.start[colour];
        for (int t = g; t < nip + ne; t += G) {
            int i, j;
            if (t < nip) {
                if (t < ni && ic.node(t, i, j)) lsgs_fast(P, field, x, rh, i, j, ld, fs);
            } else {
                lsgs_edge(P, E, e0 + t - nip, field, x, rh, ld, fs);
            }
        }
        __syncthreads();
    };
    if (smoother == 0) {
        for (int m = 0; m < steps; ++m) {
            resid_all();
            for (int t = g; t < niap + nea; t += G) {
                int i, j;
                if (t < niap) {
                    if (t < nia) {
                        ia.node(t, i, j);
                        ne_fast(P, x, rh, i, j, ld, fs);
                    }
                } else {
                    ne_edge(P, E, t - niap, x, rh, ld, fs);
                }
            }
            __syncthreads();
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

template <typename T, int N>
__global__ void __launch_bounds__(small_threads<T>()) k_smooth_block(LevelP<T> P, EdgeTable<T> E, int smoother,
                                                                     int steps, T* x, const T* __restrict__ f) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto* rh = reinterpret_cast<typename P2<T>::t*>(smem_raw);  // (y, lambda) pairs, row stride n+1
    smooth_loop<T, N>(P, E, smoother, steps, x, f, rh);
}

}  // namespace

template <typename T>
size_t block_smooth_smem(int n) {
    return sizeof(T) * 2 * (size_t)(n + 1) * (n + 1);
}

// instantiated for n = 4 .. 128 (levels 2 .. 7)
#define AAOMG_SMALL_N(CALL) CALL(4) CALL(8) CALL(16) CALL(32) CALL(64) CALL(128)

template <typename T>
cudaError_t small_prepare() {
    cudaError_t e = cudaSuccess;
#define P_(N)                                                                                                 \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(k_smooth_block<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlockSmemMax);
    AAOMG_SMALL_N(P_)
#undef P_
    return e;
}

template <typename T>
void launch_smooth_block(const LevelP<T>& P, const EdgeTable<T>& E, int smoother, int steps, T* x, const T* f,
                         cudaStream_t s) {
    const size_t sm = block_smooth_smem<T>(P.n);
    switch (P.n) {
#define C_(N)                                                                                   \
    case N: k_smooth_block<T, N><<<1, small_threads<T>(), sm, s>>>(P, E, smoother, steps, x, f); break;
        AAOMG_SMALL_N(C_)
#undef C_
    default: break;
    }
}

#define AAOMG_SMALL_INST(T)                                                                                       \
    template size_t block_smooth_smem<T>(int);                                                                    \
    template cudaError_t small_prepare<T>();                                                                      \
    template void launch_smooth_block<T>(const LevelP<T>&, const EdgeTable<T>&, int, int, T*, const T*,           \
                                         cudaStream_t);
AAOMG_SMALL_INST(float)
AAOMG_SMALL_INST(double)

}  // namespace aaomg
