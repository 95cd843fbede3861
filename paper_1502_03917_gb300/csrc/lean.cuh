// lean.cuh -- warp-uniform node enumeration and the constant-stencil updates.
//
// Nodes with 2 <= i, j <= n-2 ("deep interior") see the interior stencil at
// themselves and at all six neighbours, so their residual and their NE / LSGS
// updates need no boundary logic at all.  The remaining nodes (two rows or
// columns at each edge) take the general path of stencil.cuh.  The kernels
// enumerate the two sets as separate index ranges so that a warp never mixes
// them.
#pragma once
#include "stencil.cuh"

namespace aaomg {

// ---------------------------------------------------------- enumeration --
// deep-interior nodes of colour c: rows 2..n-2, columns 2..n-2
struct InteriorColour {
    int n, c, cpr;  // cpr: slots per row
    __device__ __forceinline__ InteriorColour(int n_, int c_) : n(n_), c(c_), cpr((n_ - 3 + 6) / 7) {}
    __device__ __forceinline__ int count() const { return n >= 4 ? (n - 3) * cpr : 0; }
    // slot t -> node (i, j); false if the slot is empty
    __device__ __forceinline__ bool node(int t, int& i, int& j) const {
        int r = t / cpr, k = t - r * cpr;
        j = 2 + r;
        i = 2 + ((c - 2 * j - 2) % 7 + 7) % 7 + 7 * k;
        return i <= n - 2;
    }
};

// all deep-interior nodes
struct InteriorAll {
    int n, w;
    __device__ __forceinline__ InteriorAll(int n_) : n(n_), w(n_ - 3) {}
    __device__ __forceinline__ int count() const { return n >= 4 ? w * w : 0; }
    __device__ __forceinline__ void node(int t, int& i, int& j) const {
        j = 2 + t / w;
        i = 2 + t - (j - 2) * w;
    }
};

// edge nodes (rows 0, 1, n-1, n and columns 0, 1, n-1, n) of colour c, or of
// every colour when c < 0
struct EdgeNodes {
    int n, c, full;  // full: slots per edge row
    __device__ __forceinline__ EdgeNodes(int n_, int c_) : n(n_), c(c_), full(c_ < 0 ? n_ + 1 : (n_ + 7) / 7) {}
    __device__ __forceinline__ int rows() const { return n >= 4 ? 4 : n + 1; }
    __device__ __forceinline__ int count() const { return rows() * full + (n >= 4 ? 4 * (n - 3) : 0); }
    __device__ __forceinline__ bool node(int t, int& i, int& j) const {
        int nr = rows();
        if (t < nr * full) {
            int r = t / full, k = t - r * full;
            j = n >= 4 ? (r < 2 ? r : n - 3 + r) : r;
            i = c < 0 ? k : ((c - 2 * j) % 7 + 7) % 7 + 7 * k;
            return i <= n;
        }
        t -= nr * full;
        int q = t / (n - 3);
        i = q < 2 ? q : n - 3 + q;
        j = 2 + t - q * (n - 3);
        return c < 0 || (i + 2 * j) % 7 == c;
    }
};

// ------------------------------------------------------- fast updates ----
// Vectors in the layout of P (row stride P.ld, field stride P.fs); the node
// (i,j) satisfies 2 <= i, j <= n-2.

template <typename T>
__device__ __forceinline__ void sums7(const T* v, int64_t p, int ld, T& s4, T& s6, T& v0) {
    v0 = v[p];
    s4 = (v[p + 1] + v[p - 1]) + (v[p + ld] + v[p - ld]);
    s6 = s4 + (v[p + ld + 1] + v[p - ld - 1]);
}

template <typename T>
__device__ __forceinline__ void resid_fast(const LevelP<T>& P, const T* f, const T* x, T* rh, int i, int j) {
    const int64_t p = (int64_t)j * P.ld + i;
    T y0, y4, y6, l0, l4, l6;
    sums7(x, p, P.ld, y4, y6, y0);
    sums7(x + P.fs, p, P.ld, l4, l6, l0);
    T My = P.mC * y0 + P.mO * y6, Ml = P.mC * l0 + P.mO * l6;
    T Ky = T(4) * y0 - y4, Kl = T(4) * l0 - l4;
    T ay, al;
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    const T il = P.invLy_int;
    rh[p] = (f[p] - ay) * il;
    rh[p + P.fs] = (f[p + P.fs] - al) * (il * P.invd);
}

template <typename T>
__device__ __forceinline__ void ne_fast(const LevelP<T>& P, T* x, const T* rh, int i, int j) {
    const int64_t p = (int64_t)j * P.ld + i;
    T y0, y4, y6, l0, l4, l6;
    sums7(rh, p, P.ld, y4, y6, y0);
    sums7(rh + P.fs, p, P.ld, l4, l6, l0);
    T My = P.mC * y0 + P.mO * y6, Ml = P.mC * l0 + P.mO * l6;
    T Ky = T(4) * y0 - y4, Kl = T(4) * l0 - l4;
    T qy, ql;
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T il = P.invLy_int;
    x[p] += P.tau * il * qy;
    x[p + P.fs] += P.tau * (il * P.invd) * ql;
}

template <typename T>
__device__ __forceinline__ void lsgs_fast(const LevelP<T>& P, int field, T* x, T* rh, int i, int j) {
    const int ld = P.ld;
    const int64_t p = (int64_t)j * ld + i;
    T* ry = rh;
    T* rl = rh + P.fs;
    const T r0 = ry[p], e = ry[p + 1], w = ry[p - 1], nn = ry[p + ld], so = ry[p - ld], ne = ry[p + ld + 1],
            sw = ry[p - ld - 1];
    const T l0 = rl[p], le = rl[p + 1], lw = rl[p - 1], ln = rl[p + ld], ls = rl[p - ld], lne = rl[p + ld + 1],
            lsw = rl[p - ld - 1];
    T y4 = (e + w) + (nn + so), l4 = (le + lw) + (ln + ls);
    T My = P.mC * r0 + P.mO * (y4 + (ne + sw));
    T Ml = P.mC * l0 + P.mO * (l4 + (lne + lsw));
    T Ky = T(4) * r0 - y4, Kl = T(4) * l0 - l4;
    T qy, ql;
    rows_from_dots(P, My, Ky, Ml, Kl, qy, ql);
    const T il = P.invLy_int, ill = P.invLy_int * P.invd;
    T p_, dCy, dCl, dEy, dEl, dDy, dDl;
    if (field == 0) {
        p_ = qy * P.invNy_int;
        x[p] += p_;
        T mCp = P.mC * p_, mOp = P.mO * p_;
        dCy = mCp * il;
        dEy = mOp * il;
        dDy = dEy;
        dCl = P.c * (T(4) * p_ + P.km * mCp) * ill;
        dEl = P.c * (-p_ + P.km * mOp) * ill;
        dDl = P.c * (P.km * mOp) * ill;
    } else {
        p_ = ql * P.invNl_int;
        x[p + P.fs] += p_;
        T mCp = P.mC * p_, mOp = P.mO * p_;
        dCy = P.c * (T(4) * p_ + P.km * mCp) * il;
        dEy = P.c * (-p_ + P.km * mOp) * il;
        dDy = P.c * (P.km * mOp) * il;
        dCl = -mCp * il;
        dEl = -mOp * il;
        dDl = dEl;
    }
    ry[p] = r0 - dCy;
    rl[p] = l0 - dCl;
    ry[p + 1] = e - dEy;
    rl[p + 1] = le - dEl;
    ry[p - 1] = w - dEy;
    rl[p - 1] = lw - dEl;
    ry[p + ld] = nn - dEy;
    rl[p + ld] = ln - dEl;
    ry[p - ld] = so - dEy;
    rl[p - ld] = ls - dEl;
    ry[p + ld + 1] = ne - dDy;
    rl[p + ld + 1] = lne - dDl;
    ry[p - ld - 1] = sw - dDy;
    rl[p - ld - 1] = lsw - dDl;
}

}  // namespace aaomg
