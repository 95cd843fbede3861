/*
 * aaomg_stokes.h -- C ABI of the GB300 (sm_103a) all-at-once multigrid solver
 * for the discretised Stokes control problem.
 *
 * The method (Takacs, "Efficient smoothers for all-at-once multigrid methods
 * for Poisson and Stokes control problems", section 1, second model problem):
 *
 *   minimise 1/2 ||v - v_D||^2 + alpha/2 ||u||^2  subject to
 *   -Lap v + grad p = u,  div v = 0 in the unit square,  v = 0 on its boundary,
 *
 * discretised with Taylor-Hood elements (continuous P2 velocity and adjoint
 * velocity, zero on the boundary; continuous P1 pressure and adjoint pressure)
 * on the uniform triangulation with h = 2^-levels whose cells are split by
 * their SW-NE diagonal, gives the saddle-point system of eq. (mp3)
 *
 *   A x = f,  x = (v, p, lambda, mu),  f = (M v_D, 0, 0, 0),
 *   A = [[M, 0, K, D^T], [0, 0, D, 0], [K, D^T, -alpha^{-1} M, 0], [D, 0, 0, 0]],
 *
 * with M, K the vector P2 mass and stiffness matrices and D the discrete
 * divergence, (D v)_q = -int psi_q div v; the control is u = lambda / alpha.
 * p and mu are determined up to constants (the paper fixes int p = 0).  The
 * library solves it with the multigrid iteration of section 2 (V or W cycle,
 * smoothing by Algorithm 1 (NE, damped by tau; the paper's tau = 0.35), by
 * Algorithm 2 (LSGS) or by sLSGS, the transposes of the canonical embeddings
 * of the nested P2 and P1 spaces as restrictions, the solution with
 * int p = int mu = 0 on the coarsest grid h = 1/2) and the smoothing norm L of
 * section 2: blockdiag(W, P, alpha^{-1} W, alpha^{-1} P), W = diag(M +
 * alpha^{1/2} K), P = alpha diag(D W^{-1} D^T).  LSGS visits the unknowns
 * block by block (v_1, v_2, p, lambda_1, lambda_2, mu) and, within a block,
 * colour by colour ((a + 7b) mod 19 on the P2 half-step grid, (i + 2j) mod 7 on
 * the vertices); the unknowns of one colour touch disjoint rows of A, so each
 * colour is updated in parallel.  Arithmetic is FP64 throughout.
 *
 * Vectors.  Level L has n = 2^L cells per side.  A velocity component has one
 * unknown per interior node of the P2 half-step grid: node (a h/2, b h/2),
 * 1 <= a, b <= 2n-1, index (b-1)(2n-1) + (a-1), nv = (2n-1)^2 unknowns; a
 * pressure has one per vertex (i h, j h), 0 <= i, j <= n, index j(n+1) + i,
 * np = (n+1)^2 unknowns.  Every vector x, f or r is a contiguous array of
 * m = 4 nv + 2 np doubles in the block order (v_1, v_2, p, lambda_1,
 * lambda_2, mu).  A desired velocity v_D is given at all (2n+1)^2 nodes of the
 * half-step grid, first component then second (2 (2n+1)^2 doubles).
 *
 * Memory, streams and errors follow aaomg.h: vector arguments are device
 * pointers owned by the caller; `stream` is a cudaStream_t passed as void*
 * (NULL = legacy default stream); calls returning scalars synchronise with it.
 * Functions return AAOMG_OK or a negative AAOMG_ERR_* code; mg_last_error()
 * gives the message.  A handle is used by one host thread at a time.
 */
#ifndef AAOMG_STOKES_H
#define AAOMG_STOKES_H

#include "aaomg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_ctx* ms_handle;

#define MS_SMOOTHER_NE 0
#define MS_SMOOTHER_LSGS 1
#define MS_SMOOTHER_SLSGS 2

typedef struct {
    int smoother;  /* MS_SMOOTHER_*; default LSGS */
    int nu_pre;    /* pre-smoothing steps; <= 0: 2 (sLSGS: 1) */
    int nu_post;   /* post-smoothing steps; <= 0: 2 (sLSGS: 1) */
    int cycle;     /* 1: V, 2: W (default) */
    double tau;    /* NE damping; <= 0: 0.35 */
    int max_iter;  /* ms_solve iteration cap; <= 0: 100 */
    int block_max; /* levels up to this one smooth in one single-block launch per smoothing call
                      (iterate and residual in shared memory; at most 4); < 0: none; 0: 4 */
    int dense_level; /* the coarse-grid correction of this level (the gamma iterations of the levels
                        up to it, from zero) is applied as one dense linear map, built at set-up by
                        running those iterations on every unit vector: the same iterate up to
                        rounding, without the latency of the coarse levels' colour phases.  1..5
                        (below levels); 0: 5 when levels >= 7, 4 when levels is 5 or 6, else
                        none; < 0: none */
} ms_options;

/* Build the hierarchy for h = 2^-levels (1 <= levels <= 9; level 1, h = 1/2,
 * has 54 unknowns) and alpha > 0 (finite): assembles M, K and D of every level,
 * A, L and N_ii = sum_j A_ji^2 / L_jj (Algorithm 2), the embeddings, the
 * coarsest solution operator and the dense coarse-level map; allocates the
 * device workspaces on the current device (the level-5 map holds 2.6 GB).  opt
 * may be NULL (defaults).  Errors: BAD_ARG, NO_DEVICE, OOM, CUDA. */
AAOMG_API int ms_setup(int levels, double alpha, const ms_options* opt, ms_handle* out);

/* Free a handle (NULL is ignored).  Synchronises the device. */
AAOMG_API void ms_destroy(ms_handle h);

/* Sizes of level `level` (1..levels): out[0] = n, out[1] = nv, out[2] = np,
 * out[3] = m.  Errors: BAD_ARG. */
AAOMG_API int ms_sizes(ms_handle h, int level, int* out);

/* f = (M v_D, 0, 0, 0) on the finest level (M: the P2 mass matrix over all
 * half-step nodes, interior rows).  vD, f: device.  Errors: BAD_ARG, CUDA. */
AAOMG_API int ms_rhs_from_vd(ms_handle h, const double* vD, double* f, void* stream);

/* r = f - A x on the finest level; r may be NULL.  If relres is not NULL it
 * receives ||f - A x||_{L^-1} / ||f||_{L^-1} (synchronises).  Errors: BAD_ARG,
 * CUDA. */
AAOMG_API int ms_residual(ms_handle h, const double* f, const double* x, double* r, double* relres, void* stream);

/* `steps` smoothing steps of the configured smoother on the finest level, in
 * place on x (Algorithm 1 or 2 from the residual f - A x).  Errors: BAD_ARG,
 * CUDA. */
AAOMG_API int ms_smooth(ms_handle h, const double* f, double* x, int steps, void* stream);

/* One multigrid iteration (section 2) on the finest level, in place on x.
 * Errors: BAD_ARG, CUDA. */
AAOMG_API int ms_cycle(ms_handle h, const double* f, double* x, void* stream);

/* Iterate cycles from x until ||f - A x||_{L^-1} <= tol ||f||_{L^-1} (or
 * max_iter cycles); x in/out.  iters, relres may be NULL.  Synchronises.
 * Errors: BAD_ARG, CUDA, NOT_CONVERGED, DIVERGED. */
AAOMG_API int ms_solve(ms_handle h, const double* f, double* x, double tol, int* iters, double* relres, void* stream);

/* Subtract from p and from mu their means (int p = int mu = 0), in place.
 * Errors: BAD_ARG, CUDA. */
AAOMG_API int ms_normalize(ms_handle h, double* x, void* stream);

/* The control u = lambda / alpha (section 1: it is recovered from the Lagrange
 * multiplier) from a solution x: u has 2 nv doubles, first component then
 * second, on the interior P2 nodes.  x, u: device.  Errors: BAD_ARG, CUDA. */
AAOMG_API int ms_control(ms_handle h, const double* x, double* u, void* stream);

/* ||x||_L and ||x||_{L^-1} on the finest level (either pointer may be NULL;
 * synchronises).  Errors: BAD_ARG, CUDA. */
AAOMG_API int ms_norms(ms_handle h, const double* x, double* norm_L, double* norm_Linv, void* stream);

/* The protocol of section 3: zero right-hand side, initial guess x0 (device,
 * not modified), cycles until the error (the iterate with the means of p and
 * mu removed; the solution is 0) has dropped by `reduction` in ||.||_L; *iters
 * receives the count, -1 beyond max_iter.  Synchronises.  Errors: BAD_ARG,
 * CUDA. */
AAOMG_API int ms_protocol_iterations(ms_handle h, const double* x0, double reduction, int max_iter, int* iters,
                                     void* stream);

/* Number of kernels the library launched for this handle since ms_setup. */
AAOMG_API long long ms_kernel_launches(ms_handle h);

/* Entries of A on level `level`: *nnz the nonzeros of eq. (mp3)'s matrix as
 * assembled, *stored the entries the library holds (each row padded to a
 * multiple of 8).  For the algorithmic bytes of a smoothing step.  Errors:
 * BAD_ARG. */
AAOMG_API int ms_operator_entries(ms_handle h, int level, long long* nnz, long long* stored);

#ifdef __cplusplus
}
#endif

#endif /* AAOMG_STOKES_H */
