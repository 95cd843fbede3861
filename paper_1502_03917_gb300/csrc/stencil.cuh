// stencil.cuh -- device-side pieces of the operator shared by the level kernels
// and the single-block coarse-grid kernel: the stencil of a node, the
// diagonals L and N, the action of A at a node, and one NE / LSGS update
// (Algorithms 1 and 2).  Vectors are addressed through plain pointers with the
// layout of a LevelP (row stride ld, field stride fs), so the same code works on
// global memory and on shared memory.
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace aaomg {

template <typename T>
__device__ __forceinline__ bool node_interior(const LevelP<T>& P, int i, int j) {
    return i > 0 && i < P.n && j > 0 && j < P.n;
}

template <typename T>
__device__ __forceinline__ bool all_interior(const LevelP<T>& P, int i, int j) {
    return i >= 2 && i <= P.n - 2 && j >= 2 && j <= P.n - 2;
}

// mass stencil m and bare stiffness stencil kd of node (i,j)
template <typename T>
__device__ __forceinline__ void row_coeffs(const LevelP<T>& P, int i, int j, T m[7], T kd[7]) {
    if (node_interior(P, i, j)) {
        m[0] = P.mC;
        kd[0] = T(4);
#pragma unroll
        for (int o = 1; o < 7; ++o) {
            m[o] = P.mO;
            kd[o] = o <= 4 ? T(-1) : T(0);
        }
    } else {
        row_coeffs_general<T>(i, j, P.n, P.h2, m, kd);
    }
}

template <typename T>
__device__ __forceinline__ T inv_ly(const LevelP<T>& P, int i, int j) {
    return node_interior(P, i, j) ? P.invLy_int : P.invLy[cls3(i, P.n) + 3 * cls3(j, P.n)];
}

template <typename T>
__device__ __forceinline__ T inv_n(const LevelP<T>& P, int field, int i, int j) {
    if (all_interior(P, i, j)) return field == 0 ? P.invNy_int : P.invNl_int;
    int c = cls5(i, P.n) + 5 * cls5(j, P.n);
    return field == 0 ? P.invNy[c] : P.invNl[c];
}

template <typename T>
__device__ __forceinline__ int64_t nidx(const LevelP<T>& P, int i, int j) {
    return (int64_t)j * P.ld + i;
}

// v at the 7 offsets of node (i,j); 0 where the offset leaves the grid
template <typename T>
__device__ __forceinline__ void load7(const LevelP<T>& P, const T* v, int i, int j, T out[7]) {
    if (node_interior(P, i, j)) {
        const T* p = v + (int64_t)j * P.ld + i;
#pragma unroll
        for (int o = 0; o < 7; ++o) out[o] = p[DJ(o) * P.ld + DI(o)];
    } else {
#pragma unroll
        for (int o = 0; o < 7; ++o) {
            int ii = i + DI(o), jj = j + DJ(o);
            out[o] = in_grid(ii, jj, P.n) ? v[(int64_t)jj * P.ld + ii] : T(0);
        }
    }
}

// Mv = m . v and Kv = kd . v; on interior nodes with the neighbour sums grouped
// so that the stiffness sum cancels exactly for smooth v
template <typename T>
__device__ __forceinline__ void dots(bool interior, const T m[7], const T kd[7], const T v[7], T& Mv, T& Kv) {
    if (interior) {
        T s4 = (v[1] + v[2]) + (v[3] + v[4]);
        Mv = m[0] * v[0] + m[1] * (s4 + (v[5] + v[6]));
        Kv = T(4) * v[0] - s4;
    } else {
        Mv = T(0);
        Kv = T(0);
#pragma unroll
        for (int o = 0; o < 7; ++o) {
            Mv += m[o] * v[o];
            Kv += kd[o] * v[o];
        }
    }
}

// rows of A = [[M, cK], [cK, -dM]] with K = Kd + km M, from the four products
template <typename T>
__device__ __forceinline__ void rows_from_dots(const LevelP<T>& P, T My, T Ky, T Ml, T Kl, T& ay, T& al) {
    ay = My + P.c * (Kl + P.km * Ml);
    al = P.c * (Ky + P.km * My) - P.d * Ml;
}

// (A x) at node (i,j)
template <typename T>
__device__ __forceinline__ void apply_A(const LevelP<T>& P, const T* x, int i, int j, T& ay, T& al) {
    T m[7], kd[7], y[7], l[7];
    row_coeffs(P, i, j, m, kd);
    load7(P, x, i, j, y);
    load7(P, x + P.fs, i, j, l);
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl;
    dots(in, m, kd, y, My, Ky);
    dots(in, m, kd, l, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
}

// The scaled residual rh = L^{-1}(f - A x) is addressed through an accessor:
// RhSep keeps the two fields apart (field stride fs), RhPair interleaves them.
template <typename T>
struct RhSep {
    T* r;
    int64_t fs;
    __device__ __forceinline__ T& y(int64_t p) const { return r[p]; }
    __device__ __forceinline__ T& l(int64_t p) const { return r[p + fs]; }
};
template <typename T>
struct RhPair {
    typename P2<T>::t* r;
    __device__ __forceinline__ T& y(int64_t p) const { return r[p].x; }
    __device__ __forceinline__ T& l(int64_t p) const { return r[p].y; }
};

// rh at the 7 offsets of node (i,j) for both fields; 0 where the offset leaves the grid
template <typename T, typename R>
__device__ __forceinline__ void load7_rh(const LevelP<T>& P, const R& rh, int i, int j, T ry[7], T rl[7]) {
    const bool in = node_interior(P, i, j);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        bool ok = in || in_grid(ii, jj, P.n);
        int64_t q = ok ? nidx(P, ii, jj) : 0;
        ry[o] = ok ? rh.y(q) : T(0);
        rl[o] = ok ? rh.l(q) : T(0);
    }
}

// rh = L^{-1}(f - A x) at node (i,j)
template <typename T, typename R>
__device__ __forceinline__ void resid_hat_acc(const LevelP<T>& P, const T* f, const T* x, const R& rh, int i, int j) {
    T ay, al;
    apply_A(P, x, i, j, ay, al);
    int64_t p = nidx(P, i, j);
    T il = inv_ly(P, i, j);
    rh.y(p) = (f[p] - ay) * il;
    rh.l(p) = (f[p + P.fs] - al) * (il * P.invd);
}

// Algorithm 1 update at node (i,j): x += tau L^{-1} A rh (A symmetric)
template <typename T, typename R>
__device__ __forceinline__ void ne_update_acc(const LevelP<T>& P, T* x, const R& rh, int i, int j) {
    T m[7], kd[7], ry[7], rl[7];
    row_coeffs(P, i, j, m, kd);
    load7_rh(P, rh, i, j, ry, rl);
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl, qy, ql;
    dots(in, m, kd, ry, My, Ky);
    dots(in, m, kd, rl, Ml, Kl);
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    int64_t p = nidx(P, i, j);
    T il = inv_ly(P, i, j);
    x[p] += P.tau * il * qy;
    x[p + P.fs] += P.tau * (il * P.invd) * ql;
}

// Algorithm 2 update of unknown (field, node (i,j)): q = sum_j A_ij rh_j,
// p = q / N_ii, x_i += p, rh_j -= A_ji p / L_jj over the neighbourhood.
template <typename T, typename R>
__device__ __forceinline__ void lsgs_update_acc(const LevelP<T>& P, int field, T* x, const R& rh, int i, int j) {
    T m[7], kd[7], ry[7], rl[7];
    row_coeffs(P, i, j, m, kd);
    load7_rh(P, rh, i, j, ry, rl);
    bool in = node_interior(P, i, j);
    T My, Ky, Ml, Kl;
    dots(in, m, kd, ry, My, Ky);
    dots(in, m, kd, rl, Ml, Kl);
    T qy, ql;
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    T p = (field == 0 ? qy : ql) * inv_n(P, field, i, j);
    x[nidx(P, i, j) + (field ? P.fs : 0)] += p;
    // column of A for this unknown: field y -> (m, cK) ; field lambda -> (cK, -dm)
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        if (!in && !in_grid(ii, jj, P.n)) continue;
        T il = inv_ly(P, ii, jj);
        int64_t q = nidx(P, ii, jj);
        T mp = m[o] * p;
        T kp = P.c * (kd[o] * p + P.km * mp);
        if (field == 0) {
            rh.y(q) = ry[o] - mp * il;
            rh.l(q) = rl[o] - kp * (il * P.invd);
        } else {
            rh.y(q) = ry[o] - kp * il;
            rh.l(q) = rl[o] + mp * il;
        }
    }
}

// Collective Gauss-Seidel (section 2, the point block smoother): solve the 2x2
// diagonal block [[m, c k], [c k, -d m]] of node i (m = M_ii, k = K_ii) for the
// residual (ry, rl) of its two rows and return the correction.
template <typename T>
__device__ __forceinline__ void cgs_block(const LevelP<T>& P, T m, T k, T ry, T rl, T& dy, T& dl) {
    const T ck = P.c * k;
    const T det = -(P.d * m * m + ck * ck);
    dy = (-P.d * m * ry - ck * rl) / det;
    dl = (m * rl - ck * ry) / det;
}

// one CGS update of node (i,j): the residual of its two rows from the current
// iterate (nodes of one colour of (i + j) mod 3 are not coupled, so the
// updates of a colour are independent), then the block solve
template <typename T>
__device__ __forceinline__ void cgs_update_at(const LevelP<T>& P, const T* f, T* x, int i, int j) {
    T ay, al, m[7], kd[7];
    apply_A(P, x, i, j, ay, al);
    row_coeffs(P, i, j, m, kd);
    const int64_t p = nidx(P, i, j);
    T dy, dl;
    cgs_block(P, m[0], kd[0] + P.km * m[0], f[p] - ay, f[p + P.fs] - al, dy, dl);
    x[p] += dy;
    x[p + P.fs] += dl;
}

// the same with the two fields of rh apart (field stride P.fs)
template <typename T>
__device__ __forceinline__ void resid_hat_at(const LevelP<T>& P, const T* f, const T* x, T* rh, int i, int j) {
    resid_hat_acc(P, f, x, RhSep<T>{rh, P.fs}, i, j);
}
template <typename T>
__device__ __forceinline__ void ne_update_at(const LevelP<T>& P, T* x, const T* rh, int i, int j) {
    ne_update_acc(P, x, RhSep<T>{const_cast<T*>(rh), P.fs}, i, j);
}
template <typename T>
__device__ __forceinline__ void lsgs_update_at(const LevelP<T>& P, int field, T* x, T* rh, int i, int j) {
    lsgs_update_acc(P, field, x, RhSep<T>{rh, P.fs}, i, j);
}

// defect restricted to coarse node (I,J): P^T (f - A x), weight 1 at (2I,2J)
// and 1/2 at its six neighbours (the midpoints of the coarse edges)
template <typename T>
__device__ __forceinline__ void restrict_at(const LevelP<T>& Pf, const T* f, const T* x, int I, int J, T& sy,
                                            T& sl) {
    sy = T(0);
    sl = T(0);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        int i = 2 * I + DI(o), j = 2 * J + DJ(o);
        if (!in_grid(i, j, Pf.n)) continue;
        T ay, al;
        apply_A(Pf, x, i, j, ay, al);
        int64_t p = nidx(Pf, i, j);
        T w = o == 0 ? T(1) : T(0.5);
        sy += w * (f[p] - ay);
        sl += w * (f[p + Pf.fs] - al);
    }
}

// (P xc) at fine node (i,j): nodal interpolation of the coarse P1 function
template <typename T>
__device__ __forceinline__ void prolong_at(const LevelP<T>& Pf, const LevelP<T>& Pc, const T* xc, int i, int j,
                                           T& vy, T& vl) {
    int I = i >> 1, J = j >> 1;
    int64_t a = nidx(Pc, I, J);
    int64_t b = a;
    if ((i & 1) && (j & 1)) b = nidx(Pc, I + 1, J + 1);
    else if (i & 1) b = nidx(Pc, I + 1, J);
    else if (j & 1) b = nidx(Pc, I, J + 1);
    if (a == b) {
        vy = xc[a];
        vl = xc[a + Pc.fs];
    } else {
        vy = T(0.5) * (xc[a] + xc[b]);
        vl = T(0.5) * (xc[a + Pc.fs] + xc[b + Pc.fs]);
    }
}

}  // namespace aaomg
