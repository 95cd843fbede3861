// aaomg.cu -- host side of the library: the handle, the grid hierarchy, the
// multigrid cycle of section 2 issued as kernel launches (recorded once into a
// CUDA graph), the solve loop with FP64 iterative refinement, and the C ABI
// declared in include/aaomg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "aaomg.h"
#include "band.h"
#include "coarse.h"
#include "common.cuh"
#include "launch.h"
#include "pdl.h"
#include "strips.h"
#include "trace.h"

using namespace aaomg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
}  // namespace

namespace aaomg {
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace aaomg

namespace {

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(AAOMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Lev {
    int n = 0, ld = 0;
    int64_t fs = 0;
    void* x = nullptr;
    void* x2 = nullptr;  // second iterate buffer for the out-of-place LSGS step
    void* f = nullptr;
    void* rh = nullptr;
    BandGrid bg{};
    int cs = 0;              // smoothing calls in one launch: of one block (1) or a cluster of cs blocks; 0: no
    bool band = false;       // LSGS steps by the one-launch band kernel (else one launch per colour phase)
    bool rg = false;         // whole smoothing calls by the 513^2 cluster kernel (residual on chip, x in global)
    void* ctab = nullptr;    // its boundary-class table (EdgeClass[25] in the cycles' precision)
    LevelP<float> pf{};
    LevelP<double> pd{};
};

template <typename T>
const LevelP<T>& lp(const Lev& v);
template <typename T>
const CtaParams<T>& ctap(const mg_ctx* H);
template <>
const LevelP<float>& lp<float>(const Lev& v) {
    return v.pf;
}
template <>
const LevelP<double>& lp<double>(const Lev& v) {
    return v.pd;
}

// Scalar coefficients of a level: L_y and N_ii of node (i,j) (FP64).
struct Coef {
    int n;
    double h2, beta, c, d, km;
};
Coef make_coef(int n, double alpha, bool scaled, double km) {
    double h = 1.0 / n, beta = std::sqrt(alpha);
    return Coef{n, h * h, beta, scaled ? beta : 1.0, scaled ? 1.0 : 1.0 / alpha, km};
}
void coef_row(const Coef& K, int i, int j, double m[7], double k[7]) {
    double kd[7];
    row_coeffs_general<double>(i, j, K.n, K.h2, m, kd);
    for (int o = 0; o < 7; ++o) k[o] = kd[o] + K.km * m[o];
}
double coef_ly(const Coef& K, int i, int j) {
    double m[7], k[7];
    coef_row(K, i, j, m, k);
    return m[0] + K.beta * k[0];
}
double coef_nd(const Coef& K, int i, int j, int field) {
    double m[7], k[7], s = 0.0;
    coef_row(K, i, j, m, k);
    for (int o = 0; o < 7; ++o) {
        int ii = i + DI(o), jj = j + DJ(o);
        if (!in_grid(ii, jj, K.n)) continue;
        double num = field == 0 ? m[o] * m[o] + K.c * K.c * k[o] * k[o] / K.d : K.c * K.c * k[o] * k[o] + K.d * m[o] * m[o];
        s += num / coef_ly(K, ii, jj);
    }
    return s;
}

// Coefficients of one level in the parametrised form A = [[M, cK], [cK, -dM]],
// L_y = diag(M + beta K), L_lambda = d L_y (see common.cuh), computed in FP64.
template <typename T>
LevelP<T> make_params(int n, int ld, int64_t fs, double alpha, bool scaled, double km, double tau) {
    LevelP<T> P{};
    P.n = n;
    P.ld = ld;
    P.fs = fs;
    const double h = 1.0 / n, h2 = h * h, beta = std::sqrt(alpha);
    const double c = scaled ? beta : 1.0, d = scaled ? 1.0 : 1.0 / alpha;
    P.h2 = (T)h2;
    P.c = (T)c;
    P.d = (T)d;
    P.invd = (T)(1.0 / d);
    P.beta = (T)beta;
    P.km = (T)km;
    P.tau = (T)tau;
    const Coef K = make_coef(n, alpha, scaled, km);
    auto Ly = [&](int i, int j) { return coef_ly(K, i, j); };
    auto Nd = [&](int i, int j, int field) { return coef_nd(K, i, j, field); };
    {
        double m[7], kd[7];
        row_coeffs_general<double>(1, 1, n, h2, m, kd);
        P.mC = (T)m[0];
        P.mO = (T)m[1];
        P.invLy_int = (T)(1.0 / Ly(1, 1));
    }
    const int rep3[3] = {0, 1, n};
    for (int cy = 0; cy < 3; ++cy)
        for (int cx = 0; cx < 3; ++cx) P.invLy[cx + 3 * cy] = (T)(1.0 / Ly(rep3[cx], rep3[cy]));
    if (n >= 4) {
        const int rep5[5] = {0, 1, 2, n - 1, n};
        for (int cy = 0; cy < 5; ++cy)
            for (int cx = 0; cx < 5; ++cx) {
                P.invNy[cx + 5 * cy] = (T)(1.0 / Nd(rep5[cx], rep5[cy], 0));
                P.invNl[cx + 5 * cy] = (T)(1.0 / Nd(rep5[cx], rep5[cy], 1));
            }
        P.invNy_int = (T)(1.0 / Nd(2, 2, 0));
        P.invNl_int = (T)(1.0 / Nd(2, 2, 1));
    }
    {
        // columns of A at an interior node, scaled by the interior L^{-1}
        double m[7], kd[7];
        row_coeffs_general<double>(1, 1, n, h2, m, kd);
        const double il = 1.0 / Ly(1, 1), ill = il / d;
        const int rep[3] = {0, 1, 5};  // centre, E (edge), NE (diagonal)
        for (int k = 0; k < 3; ++k) {
            double mo = m[rep[k]], ko = c * (kd[rep[k]] + km * m[rep[k]]);
            P.sc[0][k][0] = (T)(mo * il);   // y update: rh_y -= m p/L, rh_l -= cK p/L_l
            P.sc[0][k][1] = (T)(ko * ill);
            P.sc[1][k][0] = (T)(ko * il);   // lambda update: rh_y -= cK p/L, rh_l += m p/L
            P.sc[1][k][1] = (T)(-mo * il);
        }
    }
    return P;
}

// Dense inverse of the coarsest operator (n = 2, 18 unknowns) by Gauss-Jordan
// elimination with partial pivoting, in FP64.
bool coarse_inverse(double alpha, bool scaled, double km, double* inv) {
    const int n = 2, nn = 9, m = 18;
    const double h2 = 0.25, beta = std::sqrt(alpha);
    const double c = scaled ? beta : 1.0, d = scaled ? 1.0 : 1.0 / alpha;
    double a[18][36];
    std::memset(a, 0, sizeof(a));
    for (int j = 0; j <= n; ++j)
        for (int i = 0; i <= n; ++i) {
            double mm[7], kk[7];
            row_coeffs_general<double>(i, j, n, h2, mm, kk);
            for (int o = 0; o < 7; ++o) kk[o] += km * mm[o];
            int p = j * 3 + i;
            for (int o = 0; o < 7; ++o) {
                int ii = i + DI(o), jj = j + DJ(o);
                if (!in_grid(ii, jj, n)) continue;
                int q = jj * 3 + ii;
                a[p][q] += mm[o];
                a[p][nn + q] += c * kk[o];
                a[nn + p][q] += c * kk[o];
                a[nn + p][nn + q] += -d * mm[o];
            }
        }
    for (int i = 0; i < m; ++i) a[i][m + i] = 1.0;
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return false;
        if (piv != col)
            for (int t = 0; t < 2 * m; ++t) std::swap(a[piv][t], a[col][t]);
        double s = 1.0 / a[col][col];
        for (int t = 0; t < 2 * m; ++t) a[col][t] *= s;
        for (int r = 0; r < m; ++r)
            if (r != col && a[r][col] != 0.0) {
                double fct = a[r][col];
                for (int t = 0; t < 2 * m; ++t) a[r][t] -= fct * a[col][t];
            }
    }
    for (int r = 0; r < m; ++r)
        for (int t = 0; t < m; ++t) inv[r * m + t] = a[r][m + t];
    return true;
}

}  // namespace

struct mg_ctx {
    int L = 0;
    double alpha = 0.0, beta = 0.0;
    mg_options o{};
    int dev = 0;
    int nsm = 152;
    int band_min = 1025;      // FP32 levels with at least this many nodes per side use the one-launch LSGS step
    int small_max = 513;      // levels up to this many nodes per side: one launch per smoothing call
    bool fp32 = false;
    int in_batch = 0;         // instances of the batch graph being recorded (band steps use batch_grid when > 1)
    Lev lev[AAOMG_MAX_LEVELS + 1];
    int lc = 0;               // whole cycle inside the single-block kernel when L <= lc
    int ld = 0;               // level whose gamma coarse-grid steps are one dense map (0: none)
    void* bdense = nullptr;   // that map, (2 N_ld)^2 in the cycle's precision, row-major
    int bm = 0;
    CtaParams<float> cf{};
    CtaParams<double> cd{};
    LevelP<double> fine64{};  // the paper's system on the finest level, user layout
    double* x64 = nullptr;    // FP64 finest iterate and right-hand side (internal copies)
    double* f64 = nullptr;
    double* ainv = nullptr;   // coarsest inverse in the cycle's scaling
    double* part = nullptr;   // per-block partial sums
    double* red = nullptr;    // reduced norms (device)
    double* h_red = nullptr;  // pinned host copy
    cudaStream_t cap = nullptr;
    cudaStream_t own = nullptr;   // the handle's stream for mg_solve_batch
    cudaEvent_t norms_ready = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;
    long long launches = 0;
    long long rec_kernels = 0;
    std::vector<double> hist;
    std::vector<void*> allocs;
    // profiling: event pairs around the finest-level smoothing in the graph
    std::vector<cudaEvent_t> pev;
    int pev_used = 0;
    bool recording = false;
    bool pending = false;  // a graph launch whose events are not yet read
    double prof_ms = 0.0;
    long long prof_sweeps = 0, sweeps_per_iter = 0;
};

// The band tiling of a level inside a batch graph of `count` instances: the
// bands of the handle's own tiling with a quarter of the GPU's blocks, an
// eighth from 16 instances on.  There the instances run at once, and a step
// whose blocks hold every SM for its whole duration keeps the other
// instances' latency-bound coarse levels from starting; fewer blocks (taller
// segments, less recomputed halo and pipeline fill) leave SMs to them.
// Measured on the five concurrent h = 2^-11 solves (unknowns/s): every SM
// 2.06e8, a half 2.38e8, a quarter 2.45e8, a sixth 2.23e8; on 256 mixed
// instances: a half 2.09e8, a quarter 2.21e8, an eighth 2.26e8.
BandGrid batch_grid(const mg_ctx* H, const Lev& v, int count) {
    if (H->o.tile_w > 0 || H->o.tile_h > 0) return v.bg;
    const int part = H->nsm * (H->fp32 ? band_blocks_per_sm<float>() : band_blocks_per_sm<double>()) /
                     (count >= 16 ? 8 : 4);
    return H->fp32 ? band_grid<float>(v.n, v.bg.W, 0, part > 0 ? part : 1)
                   : band_grid<double>(v.n, v.bg.W, 0, part > 0 ? part : 1);
}

// State of one instance of a graph-captured batch solve (device memory).
struct BatchState {
    int it;      // iterations run
    int status;  // AAOMG_OK, NOT_CONVERGED or DIVERGED once the instance has stopped
    double rr;   // relative residual ||f - A x||_{L^-1} / ||f||_{L^-1} of the current iterate
    double r0;   // the initial one
};

struct mg_batch_ctx {
    int count = 0;
    int dev = 0;
    std::vector<mg_ctx*> H;
    std::vector<long long> body_kernels;  // kernels of one iteration of each instance
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    BatchState* d_state = nullptr;
    BatchState* h_state = nullptr;
    double* d_hist = nullptr;  // count x hcap residual histories
    double* h_hist = nullptr;
    int hcap = 0;
    double* d_tol = nullptr;
    double* h_tol = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};

namespace {

// The convergence test of the solve loop, on the device: reads the norms that
// the preceding residual kernels left in red, records the relative residual,
// decides as the host loop does (diverged, converged to tol, out of
// iterations, else one more iteration) and sets the condition of the
// instance's while node.  first: the test of the initial residual.
__global__ void k_batch_check(const double* __restrict__ red, BatchState* st, double* hist, int hcap,
                              const double* __restrict__ tol, int max_iter, cudaGraphConditionalHandle h, int first) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double fn = red[1] > 0.0 ? red[1] : 1.0;
    const double rr = sqrt(red[0] / fn);
    BatchState b;
    if (first) {
        b.it = 0;
        b.status = AAOMG_OK;
        b.r0 = rr;
    } else {
        b = *st;
    }
    if (b.it < hcap) hist[b.it] = rr;
    b.rr = rr;
    unsigned go = 0;
    if (!isfinite(rr) || rr > 1e6 * (b.r0 > 0.0 ? b.r0 : 1.0)) {
        b.status = AAOMG_ERR_DIVERGED;
    } else if (rr <= *tol) {
        b.status = AAOMG_OK;
    } else if (b.it >= max_iter) {
        b.status = AAOMG_ERR_NOT_CONVERGED;
    } else {
        go = 1;
        b.it += 1;
    }
    *st = b;
    cudaGraphSetConditional(h, go);
}

template <>
const CtaParams<float>& ctap<float>(const mg_ctx* H) {
    return H->cf;
}
template <>
const CtaParams<double>& ctap<double>(const mg_ctx* H) {
    return H->cd;
}

template <typename T>
CtaParams<T> make_cta(const mg_ctx* H, int lc, bool scaled, double km) {
    CtaParams<T> C{};
    C.lc = lc;
    for (int l = 1; l <= lc; ++l) {
        int n = 1 << l;
        C.P[l] = make_params<T>(n, n + 1, (int64_t)(n + 1) * (n + 1), H->alpha, scaled, km, H->o.tau);
    }
    C.smoother = H->o.smoother;
    C.nu_pre = H->o.nu_pre;
    C.nu_post = H->o.nu_post;
    C.gamma = H->o.cycle;
    C.g_ld = H->lev[lc].ld;
    C.g_fs = H->lev[lc].fs;
    return C;
}

int dalloc(mg_ctx* H, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? AAOMG_ERR_OOM : AAOMG_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    H->allocs.push_back(*p);
    return AAOMG_OK;
}

// ------------------------------------------------------------ the cycle --

const char* smoother_name(int sm) {
    switch (sm) {
    case MG_SMOOTHER_NE: return "NE";
    case MG_SMOOTHER_LSGS: return "LSGS";
    case MG_SMOOTHER_SLSGS: return "sLSGS";
    case MG_SMOOTHER_CGS: return "CGS";
    default: return "?";
    }
}

template <typename T>
void smooth(mg_ctx* H, int l, int steps, cudaStream_t s) {
    if (steps <= 0) return;
    TraceRange tr("level %d: %d %s steps", l, steps, smoother_name(H->o.smoother));
    Lev& v = H->lev[l];
    const LevelP<T>& P = lp<T>(v);
    T* x = (T*)v.x;
    T* f = (T*)v.f;
    T* rh = (T*)v.rh;
    if (v.rg) {
        // the whole LSGS / sLSGS smoothing call in one launch of a 16-block
        // cluster (rh in shared memory, x updated in global memory)
        launch_smooth_rg<T>(P, (const EdgeClass<T>*)v.ctab, H->o.smoother, steps, x, f, s);
        H->rec_kernels += 1;
        return;
    }
    if (v.cs > 0) {
        // the whole smoothing call in one launch of one block or one cluster
        // (x and rh, or for CGS x and f, in shared memory)
        launch_smooth_strips<T>(P, (const EdgeClass<T>*)v.ctab, H->o.smoother, steps, x, f, v.cs, s);
        H->rec_kernels += 1;
        return;
    }
    switch (H->o.smoother) {
    case MG_SMOOTHER_CGS:
        for (int m = 0; m < steps; ++m)
            for (int c = 0; c < 3; ++c) launch_cgs_phase<T>(P, c, f, x, s);
        H->rec_kernels += 3 * steps;
        break;
    case MG_SMOOTHER_NE:
        for (int m = 0; m < steps; ++m) {
            launch_resid_hat<T>(P, f, x, rh, s);
            launch_ne_update<T>(P, x, rh, s);
            H->rec_kernels += 2;
        }
        break;
    case MG_SMOOTHER_LSGS: {
        if (!v.band) goto phases;
        // one launch per step, ping-pong between x and x2
        T* a = x;
        T* b = (T*)v.x2;
        for (int m = 0; m < steps; ++m) {
            launch_lsgs_band<T>(P, f, a, b, H->in_batch > 1 ? batch_grid(H, v, H->in_batch) : v.bg, s);
            T* t = a;
            a = b;
            b = t;
        }
        H->rec_kernels += steps;
        if (a != x) {
            cudaMemcpyAsync(x, a, sizeof(T) * 2 * v.fs, cudaMemcpyDeviceToDevice, s);
        }
        break;
    }
    default:
    phases: {
        launch_resid_hat<T>(P, f, x, rh, s);
        H->rec_kernels += 1;
        for (int m = 0; m < steps; ++m) {
            for (int field = 0; field < 2; ++field)
                for (int c = 0; c < 7; ++c) launch_lsgs_phase<T>(P, field, colour_seq(c), x, rh, s);
            H->rec_kernels += 14;
            if (H->o.smoother == MG_SMOOTHER_SLSGS) {
                for (int field = 1; field >= 0; --field)
                    for (int c = 6; c >= 0; --c) launch_lsgs_phase<T>(P, field, colour_seq(c), x, rh, s);
                H->rec_kernels += 14;
            }
        }
    }
    }
}

// smoothing on the profiled level (the finest unless profile_level says
// otherwise), bracketed by profiling events while recording the graph
template <typename T>
void smooth_timed(mg_ctx* H, int l, int steps, cudaStream_t s) {
    const int pl = H->o.profile_level > 0 && H->o.profile_level < H->L ? H->o.profile_level : H->L;
    bool timed = H->recording && H->o.profile && l == pl && steps > 0;
    if (timed && H->pev_used + 2 <= (int)H->pev.size())
        cudaEventRecordWithFlags(H->pev[H->pev_used], s, cudaEventRecordExternal);
    smooth<T>(H, l, steps, s);
    if (timed && H->pev_used + 2 <= (int)H->pev.size()) {
        cudaEventRecordWithFlags(H->pev[H->pev_used + 1], s, cudaEventRecordExternal);
        H->pev_used += 2;
        H->sweeps_per_iter += steps;
    }
}

// `count` consecutive cycles on level l for the same right-hand side
template <typename T>
void cycle(mg_ctx* H, int l, int count, cudaStream_t s) {
    Lev& v = H->lev[l];
    const LevelP<T>& P = lp<T>(v);
    TraceRange tr("level %d: %d cycle(s)", l, count);
    if (l <= H->lc) {
        launch_coarse_cycle<T>(ctap<T>(H), (const T*)v.f, (T*)v.x, H->ainv, count, s);
        H->rec_kernels += 1;
        return;
    }
    if (l == H->ld && count == H->o.cycle) {
        // the gamma cycles from the zero initial guess set by the restriction:
        // x = Bd f with the precomputed dense map
        launch_dense_apply<T>((const T*)H->bdense, H->bm, (const T*)v.f, (T*)v.x, s);
        H->rec_kernels += 1;
        return;
    }
    for (int k = 0; k < count; ++k) {
        if (l == 1) {
            launch_coarsest<T>(H->ainv, (const T*)v.f, (T*)v.x, P.fs, s);
            H->rec_kernels += 1;
            continue;
        }
        Lev& c = H->lev[l - 1];
        smooth_timed<T>(H, l, H->o.nu_pre, s);
        launch_restrict<T>(P, lp<T>(c), (const T*)v.f, (const T*)v.x, (T*)c.f, (T*)c.x, s);
        H->rec_kernels += 1;
        cycle<T>(H, l - 1, H->o.cycle, s);
        launch_prolong<T>(P, lp<T>(c), (const T*)c.x, (T*)v.x, s);
        H->rec_kernels += 1;
        smooth_timed<T>(H, l, H->o.nu_post, s);
    }
}

// One iteration body (without the residual/norm launch):
//   FP64:        one cycle on lev[L] (x, f internal FP64 copies)
//   FP32_REFINE: x~ = 0; inner_cycles FP32 cycles on (lev[L].f = scaled defect);
//                x64 += S^{-1} x~
int record_iteration(mg_ctx* H, cudaStream_t s) {
    Lev& v = H->lev[H->L];
    if (!H->fp32) {
        cycle<double>(H, H->L, 1, s);
    } else {
        CK(cudaMemsetAsync(v.x, 0, sizeof(float) * 2 * v.fs, s));
        cycle<float>(H, H->L, H->o.inner_cycles, s);
        launch_refine_update(H->fine64, H->x64, (const float*)v.x, v.ld, v.fs, s);
        H->rec_kernels += 1;
    }
    return AAOMG_OK;
}

// The 25 boundary classes of level v for the one-launch smoothing kernel
// (EdgeClass, strips.h), from the FP64 coefficients, in the cycles' precision.
template <typename T>
int build_class_table(mg_ctx* H, Lev& v, double km) {
    const int n = v.n;
    const Coef K = make_coef(n, H->alpha, H->fp32, km);
    EdgeClass<T> tab[25];
    auto rep = [n](int a) { return a <= 2 ? a : n - 4 + a; };  // nodes 0, 1, 2, n-1, n
    for (int k = 0; k < 25; ++k) {
        const int i = rep(k % 5), j = rep(k / 5);
        double m[7], kd[7];
        row_coeffs_general<double>(i, j, n, K.h2, m, kd);
        EdgeClass<T>& C = tab[k];
        for (int o = 0; o < 7; ++o) {
            const int ii = i + DI(o), jj = j + DJ(o);
            const double il = in_grid(ii, jj, n) ? 1.0 / coef_ly(K, ii, jj) : 0.0;
            const double ko = K.c * (kd[o] + km * m[o]);
            C.m[o] = (T)m[o];
            C.kd[o] = (T)kd[o];
            C.il[o] = (T)il;
            C.sc[0][o][0] = (T)(m[o] * il);  // y update: rh_y -= m p/L, rh_l -= cK p/L_l
            C.sc[0][o][1] = (T)(ko * il / K.d);
            C.sc[1][o][0] = (T)(ko * il);  // lambda update: rh_y -= cK p/L, rh_l += m p/L
            C.sc[1][o][1] = (T)(-m[o] * il);
        }
        C.iny = (T)(1.0 / coef_nd(K, i, j, 0));
        C.inl = (T)(1.0 / coef_nd(K, i, j, 1));
    }
    int rc = dalloc(H, &v.ctab, sizeof(tab));
    if (rc) return rc;
    CK(cudaMemcpy(v.ctab, tab, sizeof(tab), cudaMemcpyHostToDevice));
    return AAOMG_OK;
}

// Autotuning: for every level, time the candidate smoothing kernels on the
// level's own vectors (zeroed at set-up) -- a single block and every cluster
// size that can run on levels up to small_max nodes per side; for LSGS above,
// one launch per colour phase against the band kernel in three tilings (the
// default segments of one full wave, segments twice as tall, and half as tall:
// two waves) -- and keep the fastest.  A candidate is a call of 2 steps, run
// once to warm up and then five times under CUDA events; the median counts,
// and a candidate replaces the level's default only if it is at least 5%
// faster, so that timing noise does not flip the choice between set-ups.
template <typename T>
int autotune_levels(mg_ctx* H, double km) {
    TraceRange tr("autotune level kernels");
    cudaStream_t s = nullptr;
    constexpr int kReps = 5;
    cudaEvent_t ev[kReps + 1] = {};
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (auto& e : ev) CK(cudaEventCreate(&e));
    int rc = AAOMG_OK;
    auto timed = [&](auto&& call) -> float {
        call();
        cudaEventRecord(ev[0], s);
        for (int r = 0; r < kReps; ++r) {
            call();
            cudaEventRecord(ev[r + 1], s);
        }
        float ms[kReps];
        if (cudaEventSynchronize(ev[kReps]) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.f;
        for (int r = 0; r < kReps; ++r)
            if (cudaEventElapsedTime(&ms[r], ev[r], ev[r + 1]) != cudaSuccess) return -1.f;
        std::sort(ms, ms + kReps);
        return ms[kReps / 2];
    };
    constexpr float kMargin = 0.95f;  // a challenger must beat the default by 5%
    for (int l = 2; l <= H->L && !rc; ++l) {
        Lev& v = H->lev[l];
        if (v.n + 1 <= H->small_max && H->o.cluster_size == 0 && !v.rg) {
            if (!v.ctab && (rc = build_class_table<T>(H, v, km))) break;
            const int dflt = v.cs;
            float best = dflt > 0 ? timed([&] { smooth<T>(H, l, 2, s); }) : -1.f;
            int best_cs = dflt;
            for (int cs : {1, 2, 4, 8, 16}) {
                if (cs == dflt || strips_max_active<T>(v.n, cs) <= 0) continue;
                v.cs = cs;
                const float ms = timed([&] { smooth<T>(H, l, 2, s); });
                if (ms >= 0.f && (best < 0.f || ms < kMargin * best)) {
                    best = ms;
                    best_cs = cs;
                }
            }
            v.cs = best_cs;
        } else if (v.cs == 0 && H->o.tile_w <= 0 && H->o.tile_h <= 0 &&
                   (H->o.smoother == MG_SMOOTHER_LSGS || (H->o.smoother == MG_SMOOTHER_SLSGS && v.rg))) {
            // candidates: one launch per colour phase (kind 0), the band
            // kernel in three tilings (kind 1, LSGS), the 513^2 cluster
            // kernel (kind 2, where it runs)
            const bool lsgs = H->o.smoother == MG_SMOOTHER_LSGS;
            const int dflt_kind = v.rg ? 2 : (v.band ? 1 : 0);
            const BandGrid g0 = v.bg;
            const int target = H->nsm * (H->fp32 ? band_blocks_per_sm<float>() : band_blocks_per_sm<double>());
            auto with_segments = [&](int ns) {
                ns = ns < 1 ? 1 : ns;
                const int hs = (v.n + 1 + ns - 1) / ns;
                return H->fp32 ? band_grid<float>(v.n, 0, hs, target) : band_grid<double>(v.n, 0, hs, target);
            };
            const BandGrid cand[3] = {g0, with_segments(g0.ns / 2), with_segments(g0.ns * 2)};
            auto set = [&](int kind, const BandGrid& g) {
                v.rg = kind == 2;
                v.band = kind == 1;
                v.bg = g;
            };
            set(dflt_kind, g0);
            float best = timed([&] { smooth<T>(H, l, 2, s); });
            int best_kind = dflt_kind;
            BandGrid best_g = g0;
            auto challenge = [&](int kind, const BandGrid& g) {
                if (kind == dflt_kind && (kind != 1 || (g.nb == g0.nb && g.ns == g0.ns))) return;
                set(kind, g);
                const float ms = timed([&] { smooth<T>(H, l, 2, s); });
                if (ms >= 0.f && (best < 0.f || ms < kMargin * best)) {
                    best = ms;
                    best_kind = kind;
                    best_g = g;
                }
            };
            challenge(0, g0);
            if (lsgs)
                for (const BandGrid& g : cand) challenge(1, g);
            if (dflt_kind == 2) challenge(2, g0);
            set(best_kind, best_g);
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    cudaStreamDestroy(s);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = fail(AAOMG_ERR_CUDA, "autotuning launch failed");
    return rc;
}

// blocks of the one-launch smoothing call by level size and precision,
// measured on GB300 (1: a single block)
int default_cluster(int n, bool fp32) {
    if (n <= 32) return 1;
    if (n <= 64) return fp32 ? 1 : 8;
    return 16;
}

// Dense map of the gamma coarse-grid steps on level ld (from a zero initial
// guess, the steps are linear in the right-hand side): computed column by column
// by the single-block kernel, one block per unit vector, in the cycles'
// precision and with the operator scaled as the cycles use it.
int build_dense_coarse(mg_ctx* H, double km) {
    TraceRange tr("dense map of level %d", H->ld);
    int ld = H->ld;
    int64_t m = 2 * (int64_t)((1 << ld) + 1) * ((1 << ld) + 1);
    H->bm = (int)m;
    double* tmp = nullptr;
    double* ainv64 = nullptr;
    CK(cudaMalloc(&tmp, sizeof(double) * m * m));
    CK(cudaMalloc(&ainv64, sizeof(double) * 18 * 18));
    double inv[18 * 18];
    coarse_inverse(H->alpha, H->fp32, km, inv);
    CK(cudaMemcpy(ainv64, inv, sizeof(inv), cudaMemcpyHostToDevice));
    // the columns in the precision of the cycles they replace (FP32 cycles run
    // about 64x faster than FP64 on GB300; the coarsest solve stays FP64)
    cudaError_t e = H->fp32 ? launch_coarse_basis<float>(make_cta<float>(H, ld, true, km), ainv64, H->o.cycle, tmp, 0)
                            : launch_coarse_basis<double>(make_cta<double>(H, ld, false, km), ainv64, H->o.cycle,
                                                          tmp, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int rc = AAOMG_OK;
    if (e != cudaSuccess) rc = fail(AAOMG_ERR_CUDA, std::string("dense coarse map: ") + cudaGetErrorString(e));
    if (!rc) {
        size_t es = H->fp32 ? sizeof(float) : sizeof(double);
        if ((rc = dalloc(H, &H->bdense, es * m * m)) == AAOMG_OK) {
            if (H->fp32) launch_f64_to_f32(tmp, (float*)H->bdense, m * m, 0);
            else e = cudaMemcpy(H->bdense, tmp, sizeof(double) * m * m, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) rc = fail(AAOMG_ERR_CUDA, std::string("dense coarse map: ") + cudaGetErrorString(e));
        }
    }
    cudaFree(tmp);
    cudaFree(ainv64);
    return rc;
}

int build_graph(mg_ctx* H) {
    TraceRange tr("record iteration graph");
    CK(cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking));
    if (H->o.profile) {
        // two smoothing calls per visit of the profiled level; a cycle visits
        // level l gamma^(L-l) times
        const int pl = H->o.profile_level > 0 && H->o.profile_level < H->L ? H->o.profile_level : H->L;
        long long visits = 1;
        for (int l = pl; l < H->L && visits < 4096; ++l) visits *= H->o.cycle;
        int pairs = (int)(2 * (H->fp32 ? H->o.inner_cycles : 1) * visits);
        H->pev.resize(2 * pairs);
        for (auto& e : H->pev) CK(cudaEventCreate(&e));
    }
    CK(cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal));
    H->rec_kernels = 0;
    H->recording = true;
    H->pev_used = 0;
    H->sweeps_per_iter = 0;
    int rc = record_iteration(H, H->cap);
    H->recording = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(H->cap, &g);
    if (rc != AAOMG_OK) return rc;
    if (e != cudaSuccess) return fail(AAOMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    H->graph = g;
    CK(cudaGraphInstantiate(&H->gexec, g, 0));
    H->graph_kernels = H->rec_kernels;
    return AAOMG_OK;
}

double* iter_x(mg_ctx* H) { return H->fp32 ? H->x64 : (double*)H->lev[H->L].x; }
double* iter_f(mg_ctx* H) { return H->fp32 ? H->f64 : (double*)H->lev[H->L].f; }

// fold the event timings of the last graph launch into the profile (the
// stream has been synchronised since that launch)
int collect_profile(mg_ctx* H) {
    if (!H->pending) return AAOMG_OK;
    H->pending = false;
    for (int p = 0; p + 1 < H->pev_used; p += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, H->pev[p], H->pev[p + 1]));
        H->prof_ms += ms;
    }
    H->prof_sweeps += H->sweeps_per_iter;
    return AAOMG_OK;
}

int run_iteration(mg_ctx* H, cudaStream_t s) {
    TraceRange tr("iteration (graph launch)");
    CK(cudaGraphLaunch(H->gexec, s));
    H->launches += H->graph_kernels;
    if (H->o.profile) H->pending = true;
    return AAOMG_OK;
}

int check_handle(mg_handle h) {
    if (!h) return fail(AAOMG_ERR_BAD_ARG, "null handle");
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return fail(AAOMG_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return AAOMG_OK;
}

int64_t vec_bytes(mg_ctx* H) { return (int64_t)2 * H->fine64.fs * (int64_t)sizeof(double); }

// The solve loop on the internal FP64 copies, as a state machine so that many
// handles can be driven at once: begin() queues the first residual and its
// norms; after that work has finished, step() reads the norms, decides, and
// queues the next iteration and residual.
struct SolveState {
    int it = 0;
    double r0 = 0.0, rr = 0.0;
    int status = AAOMG_OK;
};

int queue_norms(mg_ctx* H, cudaStream_t s) {
    Lev& v = H->lev[H->L];
    float* fin = H->fp32 ? (float*)v.f : nullptr;
    launch_resid64(H->fine64, iter_f(H), iter_x(H), nullptr, fin, v.ld, v.fs, H->part, kResidBlocks, H->red, s);
    H->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(H->h_red, H->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(H->norms_ready, s));
    return AAOMG_OK;
}

int solve_begin(mg_ctx* H, cudaStream_t s) {
    H->hist.clear();
    return queue_norms(H, s);
}

// after norms_ready: returns 1 when the solve is over (status in st), 0 if an
// iteration was queued, < 0 on a CUDA error
int solve_step(mg_ctx* H, double tol, SolveState& st, cudaStream_t s) {
    int rc = collect_profile(H);
    if (rc) return rc;
    double fn = H->h_red[1] > 0.0 ? H->h_red[1] : 1.0;
    st.rr = std::sqrt(H->h_red[0] / fn);
    H->hist.push_back(st.rr);
    if (st.it == 0) st.r0 = st.rr;
    if (!std::isfinite(st.rr) || st.rr > 1e6 * (st.r0 > 0 ? st.r0 : 1.0)) {
        st.status = fail(AAOMG_ERR_DIVERGED, "residual diverged");
        return 1;
    }
    if (st.rr <= tol) return 1;
    if (st.it >= H->o.max_iter) {
        st.status = fail(AAOMG_ERR_NOT_CONVERGED, "max_iter reached");
        return 1;
    }
    if ((rc = run_iteration(H, s))) return rc;
    ++st.it;
    if ((rc = queue_norms(H, s))) return rc;
    return 0;
}

int solve_internal(mg_ctx* H, double tol, int* iters, double* relres, cudaStream_t s) {
    TraceRange tr("solve L=%d alpha=%g %s", H->L, H->alpha, H->fp32 ? "fp32+refine" : "fp64");
    SolveState st;
    int rc = solve_begin(H, s);
    if (rc) return rc;
    for (;;) {
        CK(cudaEventSynchronize(H->norms_ready));
        rc = solve_step(H, tol, st, s);
        if (rc < 0) return rc;
        if (rc == 1) break;
    }
    if (iters) *iters = st.it;
    if (relres) *relres = st.rr;
    return st.status;
}

// The residual and its norms on the device only (no copy to the host): the
// FP64 defect of the iterate, its dual norm and that of f into H->red, and
// for FP32 cycles the scaled FP32 defect on the finest level.
int queue_norms_dev(mg_ctx* H, cudaStream_t s) {
    Lev& v = H->lev[H->L];
    float* fin = H->fp32 ? (float*)v.f : nullptr;
    launch_resid64(H->fine64, iter_f(H), iter_x(H), nullptr, fin, v.ld, v.fs, H->part, kResidBlocks, H->red, s);
    CK(cudaGetLastError());
    return AAOMG_OK;
}

// Record the batch graph: one branch per instance, each
//   residual norms of the initial iterate -> test -> while (test passed) {
//     one iteration (the handle's cycle or refinement step) -> norms -> test }
// so that a launch of the graph runs every instance to its own convergence
// with no host round trip.  The kernels of one iteration are those of the
// handle's own graph (record_iteration), recorded again into the while body.
int batch_record(mg_batch_ctx* B, bool pdl_off) {
    TraceRange tr("record batch graph (%d instances)", B->count);
    int rc = AAOMG_OK;
    g_pdl_off = pdl_off;
    std::vector<cudaStream_t> capturing;  // streams whose capture must be ended on failure
    auto bail = [&](int code, const std::string& msg) {
        for (cudaStream_t cs : capturing) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        g_pdl_off = false;
        return fail(code, msg);
    };
#define BCK(call)                                                                                           \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return bail(AAOMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    capturing.push_back(B->cap);
    BCK(cudaEventRecord(B->fork, B->cap));
    for (int k = 0; k < B->count && !rc; ++k) {
        mg_ctx* H = B->H[k];
        cudaStream_t s = H->own;
        BCK(cudaStreamWaitEvent(s, B->fork, 0));
        if ((rc = queue_norms_dev(H, s))) return bail(rc, g_err);
        cudaStreamCaptureStatus cst;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edata = nullptr;
        size_t nd = 0;
        BCK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edata, &nd));
        cudaGraphConditionalHandle ch;
        BCK(cudaGraphConditionalHandleCreate(&ch, g, 0, cudaGraphCondAssignDefault));
        k_batch_check<<<1, 32, 0, s>>>(H->red, B->d_state + k, B->d_hist + (size_t)k * B->hcap, B->hcap, B->d_tol,
                                        H->o.max_iter, ch, 1);
        BCK(cudaGetLastError());
        BCK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edata, &nd));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = ch;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode;
        BCK(cudaGraphAddNode(&wnode, g, deps, edata, nd, &np));
        BCK(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        BCK(cudaStreamBeginCaptureToGraph(H->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        capturing.push_back(H->cap);
        H->rec_kernels = 0;
        H->in_batch = B->count;
        rc = record_iteration(H, H->cap);
        H->in_batch = 0;
        if (rc || (rc = queue_norms_dev(H, H->cap))) return bail(rc, g_err);
        B->body_kernels[k] = H->rec_kernels + 3;
        k_batch_check<<<1, 32, 0, H->cap>>>(H->red, B->d_state + k, B->d_hist + (size_t)k * B->hcap, B->hcap,
                                             B->d_tol, H->o.max_iter, ch, 0);
        BCK(cudaGetLastError());
        cudaGraph_t done = nullptr;
        capturing.pop_back();
        BCK(cudaStreamEndCapture(H->cap, &done));
        BCK(cudaEventRecord(B->join[k], s));
        BCK(cudaStreamWaitEvent(B->cap, B->join[k], 0));
    }
    capturing.clear();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    g_pdl_off = false;
    if (e != cudaSuccess) return fail(AAOMG_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&B->gexec, g, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        B->gexec = nullptr;
        return fail(AAOMG_ERR_CUDA, std::string("batch graph instantiation: ") + cudaGetErrorString(e));
    }
    B->graph = g;
#undef BCK
    return AAOMG_OK;
}

// copy the caller's (FP64, paper's scaling) vector into the FP32 finest level
void to_inner(mg_ctx* H, const double* v, void* out, double s_l, cudaStream_t s) {
    Lev& w = H->lev[H->L];
    launch_to_f32(w.n, v, H->fine64.ld, H->fine64.fs, (float*)out, w.ld, w.fs, s_l, s);
}

}  // namespace

// ------------------------------------------------------------------ C ABI --
extern "C" {

const char* mg_strerror(int code) {
    switch (code) {
    case AAOMG_OK: return "ok";
    case AAOMG_ERR_BAD_ARG: return "bad argument";
    case AAOMG_ERR_OOM: return "out of memory";
    case AAOMG_ERR_CUDA: return "CUDA error";
    case AAOMG_ERR_NOT_CONVERGED: return "not converged";
    case AAOMG_ERR_DIVERGED: return "diverged";
    case AAOMG_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    default: return "unknown error";
    }
}

const char* mg_last_error(void) { return g_err.c_str(); }

void mg_destroy(mg_handle h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    cudaDeviceSynchronize();
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->own) cudaStreamDestroy(h->own);
    if (h->norms_ready) cudaEventDestroy(h->norms_ready);
    for (void* p : h->allocs) cudaFree(p);
    if (h->h_red) cudaFreeHost(h->h_red);
    delete h;
}

int mg_setup(int levels, double alpha, const mg_options* opt, mg_handle* out) {
    TraceRange tr("mg_setup L=%d alpha=%g", levels, alpha);
    if (!out) return fail(AAOMG_ERR_BAD_ARG, "out is null");
    *out = nullptr;
    if (levels < 1 || levels > AAOMG_MAX_LEVELS) return fail(AAOMG_ERR_BAD_ARG, "levels must be in [1, 13]");
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(AAOMG_ERR_BAD_ARG, "alpha must be positive and finite");
    mg_options o{};
    if (opt) o = *opt;
    if (o.smoother < 0 || o.smoother > MG_SMOOTHER_CGS) return fail(AAOMG_ERR_BAD_ARG, "unknown smoother");
    if (o.precision < 0 || o.precision > MG_PREC_FP32_REFINE) return fail(AAOMG_ERR_BAD_ARG, "unknown precision");
    if (o.cycle < 0 || o.cycle > 2) return fail(AAOMG_ERR_BAD_ARG, "cycle must be 1 (V) or 2 (W)");
    if (o.k_variant < 0 || o.k_variant > 1) return fail(AAOMG_ERR_BAD_ARG, "k_variant must be 0 or 1");
    const int dflt_nu = o.smoother == MG_SMOOTHER_SLSGS ? 1 : 2;
    if (o.nu_pre <= 0) o.nu_pre = dflt_nu;
    if (o.nu_post <= 0) o.nu_post = dflt_nu;
    if (o.cycle == 0) o.cycle = 2;
    if (!(o.tau > 0.0)) o.tau = 0.4;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.inner_cycles <= 0) o.inner_cycles = 3;

    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(AAOMG_ERR_NO_DEVICE, "no CUDA device");
    CK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return fail(AAOMG_ERR_NO_DEVICE, std::string("device is not sm_103: ") + prop.name);

    mg_ctx* H = new (std::nothrow) mg_ctx();
    if (!H) return fail(AAOMG_ERR_OOM, "host allocation");
    H->L = levels;
    H->alpha = alpha;
    H->beta = std::sqrt(alpha);
    H->o = o;
    H->dev = dev;
    H->fp32 = o.precision == MG_PREC_FP32_REFINE;
    H->nsm = prop.multiProcessorCount;
    if (o.small_max != 0) H->small_max = o.small_max;
    if (o.tile_w > 0 || o.tile_h > 0) {  // explicit tiling: the one-launch LSGS step on every level
        H->band_min = 0;
        H->small_max = -1;
    } else if (H->fp32) {
        // measured per LSGS step against the per-phase launches: 84 vs 144 us
        // at 1025^2, 156 vs 402 us at 2049^2; at 513^2 the autotuner's
        // smoothing calls and the five-solve bench favour the per-phase
        // launches (the band step holds every SM while its blocks run)
        H->band_min = H->small_max + 1 > 1025 ? H->small_max + 1 : 1025;
    } else {
        // FP64: the one-launch step's per-node arithmetic is bound by GB300's
        // FP64 rate (about 1/64 of FP32); the per-phase launches, which spread
        // it over the whole GPU, are 4.5x faster per step at 2049^2 nodes
        H->band_min = 1 << 30;
    }
    {
        cudaError_t e = H->fp32 ? strips_prepare<float>() : strips_prepare<double>();
        if (e != cudaSuccess) {
            delete H;
            return fail(AAOMG_ERR_CUDA, std::string("smoothing kernel attributes: ") + cudaGetErrorString(e));
        }
    }
    const double km = o.k_variant == 0 ? 1.0 : 0.0;
    {
        cudaError_t e = H->fp32 ? band_prepare<float>() : band_prepare<double>();
        if (e != cudaSuccess) {
            delete H;
            return fail(AAOMG_ERR_CUDA, std::string("band kernel attributes: ") + cudaGetErrorString(e));
        }
    }
    int rc = AAOMG_OK;
    {
        int n = 1 << levels;
        H->fine64 = make_params<double>(n, n + 1, (int64_t)(n + 1) * (n + 1), alpha, false, km, o.tau);
    }
    for (int l = 1; l <= levels; ++l) {
        Lev& v = H->lev[l];
        v.n = 1 << l;
        v.ld = v.n + 1;
        v.fs = (int64_t)v.ld * (v.n + 1);
        size_t es = H->fp32 ? sizeof(float) : sizeof(double);
        size_t bytes = es * 2 * (size_t)v.fs;
        if ((rc = dalloc(H, &v.x, bytes)) || (rc = dalloc(H, &v.x2, bytes)) || (rc = dalloc(H, &v.f, bytes)) ||
            (rc = dalloc(H, &v.rh, bytes)))
            break;
        CK(cudaMemset(v.x, 0, bytes));
        CK(cudaMemset(v.x2, 0, bytes));
        v.bg = H->fp32 ? band_grid<float>(v.n, o.tile_w, o.tile_h, H->nsm * band_blocks_per_sm<float>())
                       : band_grid<double>(v.n, o.tile_w, o.tile_h, H->nsm * band_blocks_per_sm<double>());
        v.band = v.n + 1 >= H->band_min;
        CK(cudaMemset(v.f, 0, bytes));
        CK(cudaMemset(v.rh, 0, bytes));
        v.pd = make_params<double>(v.n, v.ld, v.fs, alpha, false, km, o.tau);
        v.pf = make_params<float>(v.n, v.ld, v.fs, alpha, true, km, o.tau);
    }
    if (rc) {
        mg_destroy(H);
        return rc;
    }
    // One-launch smoothing calls on the levels with at most small_max nodes per
    // side: a cluster of cluster_size blocks on the mid-size levels if asked,
    // else the measured choice by level size and precision; a single block
    // where that is chosen or no cluster can run.
    for (int l = 2; l <= levels && !rc; ++l) {
        Lev& v = H->lev[l];
        if (v.n + 1 > H->small_max) continue;
        auto runs = [&](int cs) {
            return (H->fp32 ? strips_max_active<float>(v.n, cs) : strips_max_active<double>(v.n, cs)) > 0;
        };
        if (o.cluster_size > 1 && cluster_level(v.n)) {
            if (runs(o.cluster_size)) v.cs = o.cluster_size;
            else
                rc = fail(AAOMG_ERR_BAD_ARG, "cluster_size " + std::to_string(o.cluster_size) +
                                                 " cannot run on a level with " + std::to_string(v.n + 1) +
                                                 " nodes per side");
        } else if (o.cluster_size == 1) {
            v.cs = runs(1) ? 1 : 0;
        } else {
            for (int cs = default_cluster(v.n, H->fp32); cs >= 2 && !v.cs; cs /= 2)
                if (runs(cs)) v.cs = cs;
            if (!v.cs && runs(1)) v.cs = 1;
        }
        if (!rc && v.cs > 0)
            rc = H->fp32 ? build_class_table<float>(H, v, km) : build_class_table<double>(H, v, km);
        // 513 x 513 nodes (FP32 LSGS or sLSGS): the cluster kernel that keeps
        // only the residual on chip
        if (!rc && v.cs == 0 && H->fp32 && o.cluster_size == 0 &&
            (o.smoother == MG_SMOOTHER_LSGS || o.smoother == MG_SMOOTHER_SLSGS) && rg_max_active<float>(v.n) > 0) {
            v.rg = true;
            rc = build_class_table<float>(H, v, km);
        }
    }
    if (!rc && o.autotune) rc = H->fp32 ? autotune_levels<float>(H, km) : autotune_levels<double>(H, km);
    if (rc) {
        mg_destroy(H);
        return rc;
    }
    // Coarse end of the cycle: with coarse_level d (default 5), a problem with
    // levels <= d runs whole cycles in the single-block kernel; a larger one
    // replaces the gamma coarse-grid steps on level d by a dense map computed
    // here.  coarse_level 0 keeps grid-wide kernels on every level.
    int dcoarse = 0;
    if (o.coarse_level != 0) {
        int cap = max_cta_level<double>();
        dcoarse = o.coarse_level < 0 ? 5 : (o.coarse_level < cap ? o.coarse_level : cap);
        if (levels <= dcoarse) {
            H->lc = levels;
            cudaError_t e = H->fp32 ? coarse_prepare<float>() : coarse_prepare<double>();
            if (e != cudaSuccess) {
                mg_destroy(H);
                return fail(AAOMG_ERR_CUDA, std::string("coarse kernel attributes: ") + cudaGetErrorString(e));
            }
            if (H->fp32) H->cf = make_cta<float>(H, H->lc, true, km);
            else H->cd = make_cta<double>(H, H->lc, false, km);
        } else if (dcoarse >= 2) {
            H->ld = dcoarse;
        }
    }
    double inv[18 * 18];
    if (!coarse_inverse(alpha, H->fp32, km, inv)) {
        mg_destroy(H);
        return fail(AAOMG_ERR_BAD_ARG, "coarsest operator is singular");
    }
    int64_t n64 = H->fine64.fs;
    if ((rc = dalloc(H, (void**)&H->ainv, sizeof(inv))) || (rc = dalloc(H, (void**)&H->part, 2 * kResidBlocks * sizeof(double))) ||
        (rc = dalloc(H, (void**)&H->red, 2 * sizeof(double)))) {
        mg_destroy(H);
        return rc;
    }
    if (H->fp32 && ((rc = dalloc(H, (void**)&H->x64, 2 * n64 * sizeof(double))) ||
                    (rc = dalloc(H, (void**)&H->f64, 2 * n64 * sizeof(double))))) {
        mg_destroy(H);
        return rc;
    }
    if (cudaMallocHost((void**)&H->h_red, 2 * sizeof(double)) != cudaSuccess) {
        mg_destroy(H);
        return fail(AAOMG_ERR_OOM, "pinned host allocation");
    }
    cudaError_t e = cudaMemcpy(H->ainv, inv, sizeof(inv), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mg_destroy(H);
        return fail(AAOMG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (H->ld > 0 && (rc = build_dense_coarse(H, km))) {
        mg_destroy(H);
        return rc;
    }
    if ((rc = build_graph(H))) {
        mg_destroy(H);
        return rc;
    }
    if (cudaStreamCreateWithFlags(&H->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&H->norms_ready, cudaEventDisableTiming) != cudaSuccess) {
        mg_destroy(H);
        return fail(AAOMG_ERR_CUDA, "stream or event creation");
    }
    *out = H;
    return AAOMG_OK;
}

long long mg_num_nodes(mg_handle h) { return h ? (long long)h->fine64.fs : 0; }

long long mg_kernel_launches(mg_handle h) { return h ? h->launches : 0; }

int mg_rhs_from_yd(mg_handle h, const double* yD, double* f, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!yD || !f) return fail(AAOMG_ERR_BAD_ARG, "null vector");
    launch_rhs(h->fine64, yD, f, (cudaStream_t)stream);
    h->launches += 1;
    CK(cudaGetLastError());
    return AAOMG_OK;
}

int mg_residual(mg_handle h, const double* f, const double* x, double* r, double* relres, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x) return fail(AAOMG_ERR_BAD_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    launch_resid64(h->fine64, f, x, r, nullptr, 0, 0, h->part, kResidBlocks, h->red, s);
    h->launches += 2;
    CK(cudaGetLastError());
    if (relres) {
        CK(cudaMemcpyAsync(h->h_red, h->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double fn = h->h_red[1] > 0.0 ? h->h_red[1] : 1.0;
        *relres = std::sqrt(h->h_red[0] / fn);
    }
    return AAOMG_OK;
}

int mg_level_kernel(mg_handle h, int level, int* kind, int* blocks) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (level < 1 || level > h->L || !kind) return fail(AAOMG_ERR_BAD_ARG, "level out of range or null output");
    const Lev& v = h->lev[level];
    int k = MG_KERNEL_PHASES, b = 0;
    if (level == 1 || level <= h->lc || (h->ld > 0 && level <= h->ld)) {
        k = MG_KERNEL_COARSE;
    } else if (v.rg) {
        k = MG_KERNEL_STRIPS;
        b = 16;
    } else if (v.cs > 0) {
        k = MG_KERNEL_STRIPS;
        b = v.cs;
    } else if (v.band && h->o.smoother == MG_SMOOTHER_LSGS) {
        k = MG_KERNEL_BAND;
        b = v.bg.nb * v.bg.ns;
    }
    *kind = k;
    if (blocks) *blocks = b;
    return AAOMG_OK;
}

int mg_norms(mg_handle h, const double* x, double* norm_L, double* norm_Linv, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x || (!norm_L && !norm_Linv)) return fail(AAOMG_ERR_BAD_ARG, "null vector or no output");
    cudaStream_t s = (cudaStream_t)stream;
    launch_norms64(h->fine64, x, h->part, kResidBlocks, h->red, s);
    h->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_red, h->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (norm_L) *norm_L = std::sqrt(h->h_red[0]);
    if (norm_Linv) *norm_Linv = std::sqrt(h->h_red[1]);
    return AAOMG_OK;
}

int mg_smooth(mg_handle h, const double* f, double* x, int steps, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x || steps < 0) return fail(AAOMG_ERR_BAD_ARG, "null vector or negative steps");
    if (h->L < 2) return fail(AAOMG_ERR_BAD_ARG, "no smoothing on the coarsest grid (levels = 1)");
    cudaStream_t s = (cudaStream_t)stream;
    Lev& v = h->lev[h->L];
    size_t bytes = (size_t)vec_bytes(h);
    h->rec_kernels = 0;
    if (!h->fp32) {
        CK(cudaMemcpyAsync(v.f, f, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(v.x, x, bytes, cudaMemcpyDeviceToDevice, s));
        smooth<double>(h, h->L, steps, s);
        CK(cudaMemcpyAsync(x, v.x, bytes, cudaMemcpyDeviceToDevice, s));
    } else {
        to_inner(h, f, v.f, h->beta, s);
        to_inner(h, x, v.x, 1.0 / h->beta, s);
        smooth<float>(h, h->L, steps, s);
        launch_to_f64(v.n, (const float*)v.x, v.ld, v.fs, x, h->fine64.ld, h->fine64.fs, h->beta, s);
        h->rec_kernels += 3;
    }
    h->launches += h->rec_kernels;
    CK(cudaGetLastError());
    return AAOMG_OK;
}

int mg_restrict(mg_handle h, const double* f, const double* x, double* fc, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x || !fc) return fail(AAOMG_ERR_BAD_ARG, "null vector");
    if (h->L < 2) return fail(AAOMG_ERR_BAD_ARG, "restriction needs levels >= 2");
    cudaStream_t s = (cudaStream_t)stream;
    Lev& v = h->lev[h->L];
    Lev& c = h->lev[h->L - 1];
    size_t bytes = (size_t)vec_bytes(h);
    if (!h->fp32) {
        CK(cudaMemcpyAsync(v.f, f, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(v.x, x, bytes, cudaMemcpyDeviceToDevice, s));
        launch_restrict<double>(v.pd, c.pd, (const double*)v.f, (const double*)v.x, (double*)c.f, (double*)c.x, s);
        CK(cudaMemcpyAsync(fc, c.f, sizeof(double) * 2 * c.fs, cudaMemcpyDeviceToDevice, s));
        h->launches += 1;
    } else {
        to_inner(h, f, v.f, h->beta, s);
        to_inner(h, x, v.x, 1.0 / h->beta, s);
        launch_restrict<float>(v.pf, c.pf, (const float*)v.f, (const float*)v.x, (float*)c.f, (float*)c.x, s);
        launch_to_f64(c.n, (const float*)c.f, c.ld, c.fs, fc, c.n + 1, (int64_t)(c.n + 1) * (c.n + 1), 1.0 / h->beta,
                      s);
        h->launches += 4;
    }
    CK(cudaGetLastError());
    return AAOMG_OK;
}

int mg_prolong_add(mg_handle h, const double* xc, double* x, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!xc || !x) return fail(AAOMG_ERR_BAD_ARG, "null vector");
    if (h->L < 2) return fail(AAOMG_ERR_BAD_ARG, "prolongation needs levels >= 2");
    cudaStream_t s = (cudaStream_t)stream;
    Lev& v = h->lev[h->L];
    Lev& c = h->lev[h->L - 1];
    size_t bytes = (size_t)vec_bytes(h);
    if (!h->fp32) {
        CK(cudaMemcpyAsync(c.x, xc, sizeof(double) * 2 * c.fs, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(v.x, x, bytes, cudaMemcpyDeviceToDevice, s));
        launch_prolong<double>(v.pd, c.pd, (const double*)c.x, (double*)v.x, s);
        CK(cudaMemcpyAsync(x, v.x, bytes, cudaMemcpyDeviceToDevice, s));
        h->launches += 1;
    } else {
        launch_to_f32(c.n, xc, c.n + 1, (int64_t)(c.n + 1) * (c.n + 1), (float*)c.x, c.ld, c.fs, 1.0 / h->beta, s);
        to_inner(h, x, v.x, 1.0 / h->beta, s);
        launch_prolong<float>(v.pf, c.pf, (const float*)c.x, (float*)v.x, s);
        launch_to_f64(v.n, (const float*)v.x, v.ld, v.fs, x, h->fine64.ld, h->fine64.fs, h->beta, s);
        h->launches += 4;
    }
    CK(cudaGetLastError());
    return AAOMG_OK;
}

int mg_cycle(mg_handle h, const double* f, double* x, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x) return fail(AAOMG_ERR_BAD_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)vec_bytes(h);
    CK(cudaMemcpyAsync(iter_f(h), f, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(iter_x(h), x, bytes, cudaMemcpyDeviceToDevice, s));
    if (h->fp32) {
        Lev& v = h->lev[h->L];
        launch_resid64(h->fine64, iter_f(h), iter_x(h), nullptr, (float*)v.f, v.ld, v.fs, h->part, kResidBlocks, h->red, s);
        h->launches += 2;
    }
    if ((rc = run_iteration(h, s))) return rc;
    CK(cudaMemcpyAsync(x, iter_x(h), bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    return AAOMG_OK;
}

int mg_solve(mg_handle h, const double* f, double* x, double tol, int* iters, double* relres, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !x || !(tol >= 0.0)) return fail(AAOMG_ERR_BAD_ARG, "null vector or bad tol");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)vec_bytes(h);
    CK(cudaMemcpyAsync(iter_f(h), f, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(iter_x(h), x, bytes, cudaMemcpyDeviceToDevice, s));
    int status = solve_internal(h, tol, iters, relres, s);
    if (status == AAOMG_ERR_CUDA) return status;
    CK(cudaMemcpyAsync(x, iter_x(h), bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return status;
}

int mg_protocol_iterations(mg_handle h, const double* x0, double reduction, int max_iter, int* iters, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x0 || !iters || !(reduction > 0.0) || max_iter < 0)
        return fail(AAOMG_ERR_BAD_ARG, "null vector or output, reduction <= 0 or max_iter < 0");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)vec_bytes(h);
    // zero right-hand side, the random start as the iterate
    CK(cudaMemsetAsync(iter_f(h), 0, bytes, s));
    CK(cudaMemcpyAsync(iter_x(h), x0, bytes, cudaMemcpyDeviceToDevice, s));
    auto norm_L = [&](double& out) -> int {
        launch_norms64(h->fine64, iter_x(h), h->part, kResidBlocks, h->red, s);
        h->launches += 2;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h->h_red, h->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        out = std::sqrt(h->h_red[0]);
        return AAOMG_OK;
    };
    double e0 = 0.0, e = 0.0;
    if ((rc = norm_L(e0))) return rc;
    e = e0;
    int it = 0;
    h->hist.assign(1, 1.0);
    while (e > reduction * e0) {
        if (it >= max_iter) {
            *iters = -1;
            return fail(AAOMG_ERR_NOT_CONVERGED, "protocol: max_iter reached");
        }
        if (h->fp32) {
            // the refinement step's FP64 defect (f = 0) as the FP32 cycles' right-hand side
            Lev& v = h->lev[h->L];
            launch_resid64(h->fine64, iter_f(h), iter_x(h), nullptr, (float*)v.f, v.ld, v.fs, h->part, kResidBlocks,
                           h->red, s);
            h->launches += 2;
        }
        if ((rc = run_iteration(h, s))) return rc;
        ++it;
        if ((rc = norm_L(e))) return rc;
        h->hist.push_back(e0 > 0.0 ? e / e0 : 0.0);
        if (!std::isfinite(e)) {
            *iters = -1;
            return fail(AAOMG_ERR_DIVERGED, "protocol: the error norm is not finite");
        }
    }
    *iters = it;
    return AAOMG_OK;
}

int mg_solve_host(mg_handle h, const double* f_host, double* x_host, double tol, int* iters, double* relres,
                  void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f_host || !x_host || !(tol >= 0.0)) return fail(AAOMG_ERR_BAD_ARG, "null vector or bad tol");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)vec_bytes(h);
    CK(cudaMemcpyAsync(iter_f(h), f_host, bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(iter_x(h), x_host, bytes, cudaMemcpyHostToDevice, s));
    int status = solve_internal(h, tol, iters, relres, s);
    if (status == AAOMG_ERR_CUDA) return status;
    CK(cudaMemcpyAsync(x_host, iter_x(h), bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return status;
}

void mg_batch_destroy(mg_batch b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->d_state) cudaFree(b->d_state);
    if (b->d_hist) cudaFree(b->d_hist);
    if (b->d_tol) cudaFree(b->d_tol);
    if (b->h_state) cudaFreeHost(b->h_state);
    if (b->h_hist) cudaFreeHost(b->h_hist);
    if (b->h_tol) cudaFreeHost(b->h_tol);
    delete b;
}

int mg_batch_create(int count, const mg_handle* handles, mg_batch* out) {
    if (!out) return fail(AAOMG_ERR_BAD_ARG, "out is null");
    *out = nullptr;
    if (count < 1 || !handles) return fail(AAOMG_ERR_BAD_ARG, "a batch needs at least one handle");
    for (int k = 0; k < count; ++k) {
        if (!handles[k]) return fail(AAOMG_ERR_BAD_ARG, "null handle in batch");
        if (handles[k]->dev != handles[0]->dev) return fail(AAOMG_ERR_BAD_ARG, "the handles of a batch are on different devices");
        if (handles[k]->o.profile) return fail(AAOMG_ERR_BAD_ARG, "a profiled handle (profile = 1) cannot be batched");
        for (int q = 0; q < k; ++q)
            if (handles[q] == handles[k]) return fail(AAOMG_ERR_BAD_ARG, "a handle appears twice in the batch");
    }
    int rc = check_handle(handles[0]);
    if (rc) return rc;
    mg_batch_ctx* B = new (std::nothrow) mg_batch_ctx();
    if (!B) return fail(AAOMG_ERR_OOM, "host allocation");
    B->count = count;
    B->dev = handles[0]->dev;
    B->H.assign(handles, handles + count);
    B->body_kernels.assign(count, 0);
    B->join.assign(count, nullptr);
    for (int k = 0; k < count; ++k) B->hcap = std::max(B->hcap, handles[k]->o.max_iter + 1);
    auto cleanup = [&](int code) {
        mg_batch_destroy(B);
        return code;
    };
    cudaError_t e = cudaMalloc((void**)&B->d_state, sizeof(BatchState) * count);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_hist, sizeof(double) * (size_t)count * B->hcap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_tol, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_state, sizeof(BatchState) * count);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_hist, sizeof(double) * (size_t)count * B->hcap);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_tol, sizeof(double));
    if (e != cudaSuccess)
        return cleanup(fail(e == cudaErrorMemoryAllocation ? AAOMG_ERR_OOM : AAOMG_ERR_CUDA,
                            std::string("batch buffers: ") + cudaGetErrorString(e)));
    e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    for (int k = 0; k < count && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return cleanup(fail(AAOMG_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e)));
    // programmatic edges inside the while bodies where the driver accepts
    // them, else plain serialisation
    rc = batch_record(B, false);
    if (rc == AAOMG_ERR_CUDA) rc = batch_record(B, true);
    if (rc) return cleanup(rc);
    *out = B;
    return AAOMG_OK;
}

}  // extern "C"

namespace {

// Launch the batch graph on s with the tolerance tol (the instances' f and x
// already set).
int batch_launch(mg_batch b, double tol, cudaStream_t s) {
    TraceRange tr("batch graph launch (%d instances)", b->count);
    *b->h_tol = tol;
    CK(cudaMemcpyAsync(b->d_tol, b->h_tol, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaGraphLaunch(b->gexec, s));
    return AAOMG_OK;
}

// Read the instances' states and residual histories after the work queued on
// s, fill the outputs (each may be NULL) and return the first nonzero status.
int batch_finish(mg_batch b, cudaStream_t s, int* iters, double* relres, int* status) {
    CK(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(BatchState) * b->count, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(b->h_hist, b->d_hist, sizeof(double) * (size_t)b->count * b->hcap, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int first = AAOMG_OK;
    for (int k = 0; k < b->count; ++k) {
        mg_ctx* H = b->H[k];
        const BatchState& st = b->h_state[k];
        const int nh = std::min(st.it + 1, b->hcap);
        H->hist.assign(b->h_hist + (size_t)k * b->hcap, b->h_hist + (size_t)k * b->hcap + nh);
        H->launches += 3 + (long long)st.it * b->body_kernels[k];
        if (iters) iters[k] = st.it;
        if (relres) relres[k] = st.rr;
        if (status) status[k] = st.status;
        if (st.status != AAOMG_OK && first == AAOMG_OK) first = st.status;
    }
    if (first == AAOMG_ERR_NOT_CONVERGED) g_err = "max_iter reached";
    else if (first == AAOMG_ERR_DIVERGED) g_err = "residual diverged";
    return first;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// mg_batch_solve with the vectors in device memory (D2D copies) or in host
// memory (H2D in, D2H out); the copies are ordered on s around the launch.
int batch_solve_copy(mg_batch b, const double* const* f, double* const* x, double tol, int* iters, double* relres,
                     int* status, cudaStream_t s, bool host) {
    if (!b || !f || !x || !(tol >= 0.0)) return fail(AAOMG_ERR_BAD_ARG, "bad batch arguments");
    for (int k = 0; k < b->count; ++k)
        if (!f[k] || !x[k]) return fail(AAOMG_ERR_BAD_ARG, "null vector in batch");
    int rc = check_handle(b->H[0]);
    if (rc) return rc;
    const cudaMemcpyKind in = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int k = 0; k < b->count; ++k) {
        mg_ctx* H = b->H[k];
        size_t bytes = (size_t)vec_bytes(H);
        CK(cudaMemcpyAsync(iter_f(H), f[k], bytes, in, s));
        CK(cudaMemcpyAsync(iter_x(H), x[k], bytes, in, s));
    }
    if ((rc = batch_launch(b, tol, s))) return rc;
    for (int k = 0; k < b->count; ++k)
        CK(cudaMemcpyAsync(x[k], iter_x(b->H[k]), (size_t)vec_bytes(b->H[k]), out, s));
    return batch_finish(b, s, iters, relres, status);
}

}  // namespace

extern "C" {

int mg_batch_solve(mg_batch b, const double* const* f, double* const* x, double tol, int* iters, double* relres,
                   int* status, void* stream) {
    return batch_solve_copy(b, f, x, tol, iters, relres, status, (cudaStream_t)stream, false);
}

int mg_batch_solve_host(mg_batch b, const double* const* f_host, double* const* x_host, double tol, int* iters,
                        double* relres, int* status, void* stream) {
    return batch_solve_copy(b, f_host, x_host, tol, iters, relres, status, (cudaStream_t)stream, true);
}

int mg_batch_adjoint(mg_batch b, const double* const* x, const double* const* ubar, double* const* z,
                     double* const* gyD, double* dalpha, double tol, int* iters, void* stream) {
    if (!b || !x || !ubar || !z || !gyD || !dalpha || !(tol >= 0.0)) return fail(AAOMG_ERR_BAD_ARG, "bad batch arguments");
    for (int k = 0; k < b->count; ++k)
        if (!x[k] || !ubar[k] || !z[k] || !gyD[k]) return fail(AAOMG_ERR_BAD_ARG, "null vector in batch");
    int rc = check_handle(b->H[0]);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // adjoint right-hand sides (0, ubar / alpha) into the handles, z from zero
    for (int k = 0; k < b->count; ++k) {
        mg_ctx* H = b->H[k];
        launch_adjoint_rhs(H->fine64.fs, ubar[k], H->alpha, iter_f(H), s);
        CK(cudaMemsetAsync(iter_x(H), 0, (size_t)vec_bytes(H), s));
        H->launches += 1;
    }
    if ((rc = batch_launch(b, tol, s))) return rc;
    for (int k = 0; k < b->count; ++k) {
        mg_ctx* H = b->H[k];
        CK(cudaMemcpyAsync(z[k], iter_x(H), (size_t)vec_bytes(H), cudaMemcpyDeviceToDevice, s));
        launch_adjoint_terms(H->fine64, x[k], ubar[k], z[k], gyD[k], H->part, kResidBlocks, H->red, s);
        H->launches += 2;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(H->h_red, H->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    rc = batch_finish(b, s, iters, nullptr, nullptr);
    for (int k = 0; k < b->count; ++k) {
        const mg_ctx* H = b->H[k];
        dalpha[k] = -(H->h_red[0] + H->h_red[1]) / (H->alpha * H->alpha);
    }
    return rc;
}

int mg_solve_batch(int count, const mg_handle* handles, const double* const* f, double* const* x, double tol,
                   int* iters, double* relres, void* stream) {
    if (count < 0 || (count > 0 && (!handles || !f || !x)) || !(tol >= 0.0))
        return fail(AAOMG_ERR_BAD_ARG, "bad batch arguments");
    if (count == 0) return AAOMG_OK;
    mg_batch b = nullptr;
    int rc = mg_batch_create(count, handles, &b);
    if (rc) return rc;
    rc = mg_batch_solve(b, f, x, tol, iters, relres, nullptr, stream);
    std::string msg = g_err;
    mg_batch_destroy(b);
    g_err = msg;
    return rc;
}

int mg_control(mg_handle h, const double* x, double* u, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x || !u) return fail(AAOMG_ERR_BAD_ARG, "null vector");
    launch_control(h->fine64.fs, x, h->alpha, u, (cudaStream_t)stream);
    h->launches += 1;
    CK(cudaGetLastError());
    return AAOMG_OK;
}

int mg_adjoint(mg_handle h, const double* x, const double* ubar, double* z, double* gyD, double* dalpha, double tol,
               void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x || !ubar || !z || !gyD || !dalpha || !(tol >= 0.0)) return fail(AAOMG_ERR_BAD_ARG, "null vector or bad tol");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nn = h->fine64.fs;
    // adjoint right-hand side into the internal right-hand side, z from zero
    launch_adjoint_rhs(nn, ubar, h->alpha, iter_f(h), s);
    CK(cudaMemsetAsync(iter_x(h), 0, (size_t)vec_bytes(h), s));
    h->launches += 1;
    int it = 0;
    double rr = 0.0;
    int status = solve_internal(h, tol, &it, &rr, s);
    if (status == AAOMG_ERR_CUDA) return status;
    CK(cudaMemcpyAsync(z, iter_x(h), (size_t)vec_bytes(h), cudaMemcpyDeviceToDevice, s));
    launch_adjoint_terms(h->fine64, x, ubar, z, gyD, h->part, kResidBlocks, h->red, s);
    h->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_red, h->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *dalpha = -(h->h_red[0] + h->h_red[1]) / (h->alpha * h->alpha);
    return status;
}

int mg_get_profile(mg_handle h, double* smooth_ms, long long* sweeps) {
    int rc = check_handle(h);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    if ((rc = collect_profile(h))) return rc;
    if (smooth_ms) *smooth_ms = h->prof_ms;
    if (sweeps) *sweeps = h->prof_sweeps;
    return AAOMG_OK;
}

int mg_reset_profile(mg_handle h) {
    int rc = check_handle(h);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    h->pending = false;
    h->prof_ms = 0.0;
    h->prof_sweeps = 0;
    return AAOMG_OK;
}

int mg_get_history(mg_handle h, double* buf, int cap, int* n) {
    if (!h || (!buf && cap > 0)) return fail(AAOMG_ERR_BAD_ARG, "null handle or buffer");
    int k = (int)h->hist.size() < cap ? (int)h->hist.size() : cap;
    for (int i = 0; i < k; ++i) buf[i] = h->hist[i];
    if (n) *n = k;
    return AAOMG_OK;
}

}  // extern "C"
