// common.cuh -- operator description shared by every kernel of the library.
//
// Discretisation (section 1, eq. (mp2)): P1 elements on the uniform mesh of the
// unit square, n = 2^k cells per side, cells split by the SW-NE diagonal.  Node
// (i, j) is coupled to itself and to its six mesh neighbours, taken in the
// fixed offset order
//     0: C (0,0)  1: E (+1,0)  2: W (-1,0)  3: N (0,+1)  4: S (0,-1)
//     5: NE (+1,+1)  6: SW (-1,-1).
// With cnt_o the number of mesh triangles containing both the node and its
// neighbour o (cnt_0 = triangles at the node), the element matrices give
//     M_o = cnt_o h^2/24 (o > 0),  M_0 = cnt_0 h^2/12,
//     Kd_o = -cnt_o/2 for E, W, N, S;  Kd_o = 0 for NE, SW;  Kd_0 = -sum_o Kd_o
// (right isosceles triangles: no stiffness coupling across the hypotenuse),
// and K = Kd + km M (km = 1: the bilinear form of -Lap + id; km = 0: bare Kd).
//
// One parametrised operator covers both the paper's system and its symmetric
// rescaling:
//     A = [[M, c K], [c K, -d M]],  L_y = diag(M + beta K),  L_lambda = d L_y.
// The paper's system is c = 1, d = 1/alpha, beta = alpha^{1/2}; scaling lambda
// by alpha^{-1/2} (and its rows by alpha^{1/2}) gives c = beta, d = 1, where
// both fields are O(1) for every alpha -- the form the FP32 cycles use.  Both
// smoothers and the whole cycle are invariant under that diagonal scaling.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define AAOMG_HD __host__ __device__ __forceinline__
#else
#define AAOMG_HD inline
#endif

namespace aaomg {

AAOMG_HD constexpr int DI(int o) { return (o == 1 || o == 5) ? 1 : ((o == 2 || o == 6) ? -1 : 0); }
AAOMG_HD constexpr int DJ(int o) { return (o == 3 || o == 5) ? 1 : ((o == 4 || o == 6) ? -1 : 0); }

// Multicolour order of the LSGS sweep: colour(i,j) = (i + 2 j) mod 7 (a
// distance-2 colouring: equal colours never share a neighbour), visited field
// by field (y, then lambda) in the colour sequence 0,6,5,4,3,2,1.
AAOMG_HD constexpr int colour_seq(int s) { return s == 0 ? 0 : 7 - s; }

template <typename T>
struct LevelP {
    int n;       // cells per side; nodes 0..n in each direction
    int ld;      // row stride in elements
    int64_t fs;  // distance in elements between the y field and the lambda field
    T h2, c, d, invd, beta, km, tau;
    // interior node: mass stencil mC (centre), mO (six neighbours); the bare
    // stiffness stencil is 4 at the centre and -1 at E, W, N, S
    T mC, mO;
    T invLy_int, invNy_int, invNl_int;
    // interior LSGS residual update: rh_o -= p * sc[field][k] (k = 0 centre,
    // 1 E/W/N/S, 2 NE/SW), each a (y, lambda) pair of the column of A scaled by
    // L^{-1}; mass and stiffness parts are combined here, which only rounds the
    // smoother's carried residual (every defect is recomputed from x)
    T sc[2][3][2];
    // boundary classes: node class cls3(i)+3*cls3(j) (9) and cls5(i)+5*cls5(j) (25)
    T invLy[9];
    T invNy[25];
    T invNl[25];
};

AAOMG_HD int cls3(int i, int n) { return i == 0 ? 0 : (i == n ? 2 : 1); }
AAOMG_HD int cls5(int i, int n) { return i == 0 ? 0 : (i == n ? 4 : (i == 1 ? 1 : (i == n - 1 ? 3 : 2))); }

// triangle counts of node (i,j) for the 7 offsets
AAOMG_HD void tri_counts(int i, int j, int n, int cnt[7]) {
    int ip = i < n, im = i > 0, jp = j < n, jm = j > 0;
    cnt[1] = ip * (jp + jm);
    cnt[2] = im * (jp + jm);
    cnt[3] = jp * (ip + im);
    cnt[4] = jm * (ip + im);
    cnt[5] = 2 * ip * jp;
    cnt[6] = 2 * im * jm;
    cnt[0] = 2 * ip * jp + im * jp + ip * jm + 2 * im * jm;
}

// A-row coefficients of node (i,j) for the 7 offsets (zero for offsets that
// leave the domain): the mass stencil m and the bare stiffness stencil kd.
// K = kd + km m is never formed coefficient-wise: the mass part of K is about
// h^2/8 of its diagonal, below FP32 resolution on fine grids, so every kernel
// applies K v as (kd . v) + km (m . v).  The stiffness sum cancels exactly for
// smooth v (neighbouring values are close), which keeps the O(h^2) mass term.
template <typename T>
AAOMG_HD void row_coeffs_general(int i, int j, int n, T h2, T m[7], T kd[7]) {
    int cnt[7];
    tri_counts(i, j, n, cnt);
    const T q = h2 / T(24);
    m[0] = T(2 * cnt[0]) * q;
    T kd0 = T(0);
    for (int o = 1; o < 7; ++o) {
        m[o] = T(cnt[o]) * q;
        kd[o] = (o <= 4) ? T(-0.5) * T(cnt[o]) : T(0);
        kd0 -= kd[o];
    }
    kd[0] = kd0;
}

AAOMG_HD bool in_grid(int i, int j, int n) { return i >= 0 && i <= n && j >= 0 && j <= n; }

}  // namespace aaomg
