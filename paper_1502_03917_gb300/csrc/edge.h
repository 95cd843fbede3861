// edge.h -- tabulated coefficients of the edge nodes of one level (internal).
//
// The nodes within two rows or columns of the boundary see boundary stencils at
// themselves or at a neighbour.  For the single-block smoothing kernel their
// update data are tabulated once per level, per colour, in structure-of-arrays
// form: node index, a mask of the neighbours inside the grid, the mass and
// bare-stiffness stencils, the L_y^{-1} of each neighbour and the N_ii^{-1} of
// both fields.  An edge update then costs about as much as an interior one.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace aaomg {

template <typename T>
struct EdgeTable {
    int count[7];   // entries of colour c
    int start[7];   // first entry of colour c
    int total;
    int* node;      // j*(n+1)+i
    int* mask;      // bit o: neighbour o inside the grid
    T* m;           // [7][total]
    T* kd;          // [7][total]
    T* il;          // [7][total]  L_y^{-1} of neighbour o
    T* inv_ny;      // [total]
    T* inv_nl;      // [total]
};

#ifdef __CUDACC__
// one edge entry in registers
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
#endif

}  // namespace aaomg
