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

// a field index as a type, for loops compiled per field (the field-dependent
// constants and selections then fold at compile time)
template <int F>
struct FieldC {
    static constexpr int value = F;
};

// ------------------------------------------------------- fast updates ----
// The node (i,j) satisfies 2 <= i, j <= n-2.  x and f keep their two fields
// apart (layout of P); the scaled residual rh is an array of (y, lambda) pairs
// with row stride P.ld.  Pair arithmetic: the sums over the neighbours give
// (M rh_y, M rh_l) and (Kd rh_y, Kd rh_l) at once.

// (M v, Kd v) for both fields of a pair field v around linear index p
template <typename V2>
__device__ __forceinline__ void pair_stencil(const V2* v, int p, int ld, V2 mC2, V2 mO2, V2& Mv, V2& Kv,
                                             V2 (&nb)[7]) {
    nb[0] = v[p];
    nb[1] = v[p + 1];
    nb[2] = v[p - 1];
    nb[3] = v[p + ld];
    nb[4] = v[p - ld];
    nb[5] = v[p + ld + 1];
    nb[6] = v[p - ld - 1];
    V2 s4 = padd(padd(nb[1], nb[2]), padd(nb[3], nb[4]));
    V2 s6 = padd(s4, padd(nb[5], nb[6]));
    Mv = pfma(mC2, nb[0], pmul(mO2, s6));
    using T = decltype(s4.x);
    Kv = pfma(psplat(T(4)), nb[0], pmul(psplat(T(-1)), s4));
}

// `ld` and `fs` are the row and field strides (compile-time constants in the
// kernels instantiated per level size)
template <typename T>
__device__ __forceinline__ void resid_fast(const LevelP<T>& P, const T* f, const T* x,
                                           typename P2<T>::t* __restrict__ rh, int i, int j, int ld, int fs) {
    const int p = j * ld + i;
    const T* xl = x + fs;
    T y4 = (x[p + 1] + x[p - 1]) + (x[p + ld] + x[p - ld]);
    T l4 = (xl[p + 1] + xl[p - 1]) + (xl[p + ld] + xl[p - ld]);
    T y6 = y4 + (x[p + ld + 1] + x[p - ld - 1]);
    T l6 = l4 + (xl[p + ld + 1] + xl[p - ld - 1]);
    T My = P.mC * x[p] + P.mO * y6, Ml = P.mC * xl[p] + P.mO * l6;
    T Ky = T(4) * x[p] - y4, Kl = T(4) * xl[p] - l4;
    T ay, al;
    rows_from_dots(P, My, Ky, Ml, Kl, ay, al);
    const T il = P.invLy_int;
    rh[p] = pmake<T>((f[p] - ay) * il, (f[p + fs] - al) * (il * P.invd));
}

template <typename T>
__device__ __forceinline__ void ne_fast(const LevelP<T>& P, T* x, const typename P2<T>::t* __restrict__ rh, int i,
                                        int j, int ld, int fs) {
    using V2 = typename P2<T>::t;
    const int p = j * ld + i;
    V2 M, K, nb[7];
    pair_stencil(rh, p, ld, psplat(P.mC), psplat(P.mO), M, K, nb);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T il = P.invLy_int;
    x[p] += P.tau * il * qy;
    x[p + fs] += P.tau * (il * P.invd) * ql;
}

template <typename T>
__device__ __forceinline__ void lsgs_fast(const LevelP<T>& P, int field, T* x, typename P2<T>::t* __restrict__ rh,
                                          int i, int j, int ld, int fs) {
    using V2 = typename P2<T>::t;
    const int p = j * ld + i;
    V2 M, K, nb[7];
    pair_stencil(rh, p, ld, psplat(P.mC), psplat(P.mO), M, K, nb);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T pv = field == 0 ? qy * P.invNy_int : ql * P.invNl_int;
    x[p + (field ? fs : 0)] += pv;
    const V2 mp = psplat(-pv);
    const V2 cC = pmake<T>(P.sc[field][0][0], P.sc[field][0][1]);
    const V2 cE = pmake<T>(P.sc[field][1][0], P.sc[field][1][1]);
    const V2 cD = pmake<T>(P.sc[field][2][0], P.sc[field][2][1]);
    rh[p] = pfma(mp, cC, nb[0]);
    rh[p + 1] = pfma(mp, cE, nb[1]);
    rh[p - 1] = pfma(mp, cE, nb[2]);
    rh[p + ld] = pfma(mp, cE, nb[3]);
    rh[p - ld] = pfma(mp, cE, nb[4]);
    rh[p + ld + 1] = pfma(mp, cD, nb[5]);
    rh[p - ld - 1] = pfma(mp, cD, nb[6]);
}

// ------------------------------------------------ row-pointer variants ----
// The same updates with the three rows j-1, j, j+1 of a pair field given as
// separate pointers (rows of a ring buffer, or rows that live in the shared
// memory of another block of a cluster); i is the index within the row.

template <typename V2>
__device__ __forceinline__ void rows_stencil(const V2* rs, const V2* rsp, const V2* rsm, int i, V2 mC2, V2 mO2,
                                             V2& M, V2& K, V2 (&nb)[7]) {
    nb[0] = rs[i];
    nb[1] = rs[i + 1];
    nb[2] = rs[i - 1];
    nb[3] = rsp[i];
    nb[4] = rsm[i];
    nb[5] = rsp[i + 1];
    nb[6] = rsm[i - 1];
    V2 s4 = padd(padd(nb[1], nb[2]), padd(nb[3], nb[4]));
    V2 s6 = padd(s4, padd(nb[5], nb[6]));
    using T = decltype(s4.x);
    M = pfma(mC2, nb[0], pmul(mO2, s6));
    K = pfma(psplat(T(4)), nb[0], pmul(psplat(T(-1)), s4));
}

// rh pair L^{-1}(f - A x) of a node from the x rows and its (f_y, f_lambda)
template <typename T, typename V2>
__device__ __forceinline__ V2 rows_resid_fast(const LevelP<T>& P, const V2* xs, const V2* xsp, const V2* xsm, int i,
                                              T fy, T fl) {
    V2 M, K, nb[7];
    rows_stencil(xs, xsp, xsm, i, psplat(P.mC), psplat(P.mO), M, K, nb);
    T ay, al;
    rows_from_dots(P, M.x, K.x, M.y, K.y, ay, al);
    const T il = P.invLy_int;
    return pmake<T>((fy - ay) * il, (fl - al) * (il * P.invd));
}

// Algorithm 1 update of the x pair xr[i] from the rh rows
template <typename T, typename V2>
__device__ __forceinline__ void rows_ne_fast(const LevelP<T>& P, V2* xr, const V2* rs, const V2* rsp, const V2* rsm,
                                             int i) {
    V2 M, K, nb[7];
    rows_stencil(rs, rsp, rsm, i, psplat(P.mC), psplat(P.mO), M, K, nb);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T il = P.invLy_int;
    V2 v = xr[i];
    v.x += P.tau * il * qy;
    v.y += P.tau * (il * P.invd) * ql;
    xr[i] = v;
}

// The field-dependent constants of an interior update: the scatter weights of
// the centre, edge and diagonal neighbours and N_ii^-1.  A thread whose field
// is fixed loads them once (a run-time field index would otherwise turn every
// update's reads of them into indexed constant loads).
template <typename V2, typename T>
struct LsgsConsts {
    V2 cC, cE, cD;
    T invN;
};

template <typename T, typename V2>
__device__ __forceinline__ LsgsConsts<V2, T> lsgs_consts(const LevelP<T>& P, int field) {
    LsgsConsts<V2, T> c;
    c.cC = pmake<T>(P.sc[field][0][0], P.sc[field][0][1]);
    c.cE = pmake<T>(P.sc[field][1][0], P.sc[field][1][1]);
    c.cD = pmake<T>(P.sc[field][2][0], P.sc[field][2][1]);
    c.invN = field == 0 ? P.invNy_int : P.invNl_int;
    return c;
}

// rows_lsgs_fast with the constants preloaded
template <typename T, typename V2>
__device__ __forceinline__ void rows_lsgs_fast_c(const LevelP<T>& P, const LsgsConsts<V2, T>& c, int field, V2* xr,
                                                 V2* rs, V2* rsp, V2* rsm, int i) {
    V2 M, K, nb[7];
    rows_stencil(rs, rsp, rsm, i, psplat(P.mC), psplat(P.mO), M, K, nb);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T pv = (field == 0 ? qy : ql) * c.invN;
    if (field == 0) xr[i].x += pv;
    else xr[i].y += pv;
    const V2 mp = psplat(-pv);
    rs[i] = pfma(mp, c.cC, nb[0]);
    rs[i + 1] = pfma(mp, c.cE, nb[1]);
    rs[i - 1] = pfma(mp, c.cE, nb[2]);
    rsp[i] = pfma(mp, c.cE, nb[3]);
    rsm[i] = pfma(mp, c.cE, nb[4]);
    rsp[i + 1] = pfma(mp, c.cD, nb[5]);
    rsm[i - 1] = pfma(mp, c.cD, nb[6]);
}

// Algorithm 2 update of one field of the x pair xr[i], with the scatter into
// the rh rows
template <typename T, typename V2>
__device__ __forceinline__ void rows_lsgs_fast(const LevelP<T>& P, int field, V2* xr, V2* rs, V2* rsp, V2* rsm,
                                               int i) {
    V2 M, K, nb[7];
    rows_stencil(rs, rsp, rsm, i, psplat(P.mC), psplat(P.mO), M, K, nb);
    T qy, ql;
    rows_from_dots(P, M.x, K.x, M.y, K.y, qy, ql);
    const T pv = field == 0 ? qy * P.invNy_int : ql * P.invNl_int;
    if (field == 0) xr[i].x += pv;
    else xr[i].y += pv;
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
}

}  // namespace aaomg
