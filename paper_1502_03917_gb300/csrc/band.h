// band.h -- the one-launch LSGS step kernel (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace aaomg {

// dependency reach of one LSGS step in the colour sequence 0,6,5,4,3,2,1 of
// (i + 2j) mod 7: the new value at (i,j) depends on the old iterate in
// columns i-28..i+15 and rows j-28..j+15
constexpr int kBandHL = 28;
constexpr int kBandHR = 15;

// threads per block = columns held in shared memory
template <typename T>
constexpr int band_threads() {
    return sizeof(T) == 4 ? 256 : 128;
}

struct BandGrid {
    int nb, ns;  // blocks across (bands) and along (segments)
    int W, Hs;   // owned columns per band, owned rows per segment
};

// Tiling of a level with n cells: bands as wide as the block allows (or
// w_override), segments chosen so that about `target` blocks run at once.
template <typename T>
inline BandGrid band_grid(int n, int w_override, int h_override, int target) {
    BandGrid g{};
    int wmax = band_threads<T>() - kBandHL - kBandHR;
    g.W = (w_override > 0 && w_override < wmax) ? w_override : wmax;
    g.nb = (n + 1 + g.W - 1) / g.W;
    if (h_override > 0) {
        g.Hs = h_override;
    } else {
        int ns = target / g.nb;
        if (ns < 1) ns = 1;
        int nsmax = (n + 1 + 7) / 8;  // segments of at least 8 rows
        if (ns > nsmax) ns = nsmax;
        g.Hs = (n + 1 + ns - 1) / ns;
    }
    g.ns = (n + 1 + g.Hs - 1) / g.Hs;
    return g;
}

template <typename T>
size_t band_smem_bytes();
template <typename T>
cudaError_t band_prepare();
// blocks of the step kernel that can be resident on one SM
template <typename T>
int band_blocks_per_sm();
template <typename T>
void launch_lsgs_band(const LevelP<T>& P, const T* f, const T* xin, T* xout, const BandGrid& g, cudaStream_t s);

}  // namespace aaomg
