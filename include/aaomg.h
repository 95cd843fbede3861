/*
 * aaomg.h -- C ABI of the GB300 (sm_103a) all-at-once multigrid library for
 * the discretised Poisson control problem.
 *
 * The method (Takacs, "Efficient smoothers for all-at-once multigrid methods
 * for Poisson and Stokes control problems"):
 *
 *   minimise 1/2 ||y - y_D||^2 + alpha/2 ||u||^2  subject to  -Lap y + y = u,
 *   dy/dn = 0 on the boundary of the unit square            (section 1)
 *
 * discretised with Courant (P1) elements on the uniform triangulation with
 * h = 2^-levels whose cells are split by their SW-NE diagonal, gives the
 * saddle-point system of eq. (mp2)
 *
 *   A x = f,  A = [[M, K], [K, -alpha^{-1} M]],  x = (y, lambda),  f = (M y_D, 0),
 *
 * with M the mass matrix and K the matrix of (grad y, grad v) + (y, v); the
 * control is u = lambda / alpha.  The library solves it with the multigrid
 * iteration of section 2 (smoothing, defect restriction by the transpose of
 * the canonical embedding, recursive coarse correction, prolongation,
 * post-smoothing; exact solve on the coarsest grid h = 1/2), with the
 * normal-equation smoother (Algorithm 1), the least-squares Gauss-Seidel
 * smoother LSGS (Algorithm 2), its symmetric form sLSGS, or the collective
 * Gauss-Seidel smoother CGS.
 *
 * Vectors.  A grid level with n = 2^k cells per side has N = (n+1)^2 nodes;
 * node (i h, j h), 0 <= i, j <= n, has index j*(n+1) + i.  Every vector passed
 * to this library is a contiguous array of 2N doubles: the y (or first) field
 * in elements [0, N), the lambda (or second) field in [N, 2N).
 *
 * Memory.  Functions whose vector arguments are documented as device pointers
 * take CUDA device (or managed) memory on the current device, owned by the
 * caller; the library never frees them and keeps no reference after the call
 * returns.  The library owns its handle and the workspaces it allocates in
 * mg_setup; mg_destroy frees them.  A `stream` argument is a cudaStream_t
 * passed as void* (NULL = the legacy default stream); all device work of a call
 * is ordered on that stream, and calls that return scalars (iteration counts,
 * residual norms) synchronise with it before returning.
 *
 * Errors.  Every int-returning function returns AAOMG_OK (0) or a negative
 * AAOMG_ERR_* code; mg_strerror() names it and mg_last_error() gives the
 * message of the calling thread's last failure.  No C++ exception crosses this
 * interface.  A handle is not thread-safe: one host thread at a time.
 */
#ifndef AAOMG_H
#define AAOMG_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define AAOMG_API __attribute__((visibility("default")))
#else
#define AAOMG_API
#endif

#define AAOMG_OK 0
#define AAOMG_ERR_BAD_ARG (-1)       /* invalid argument: null pointer, level or alpha out of range */
#define AAOMG_ERR_OOM (-2)           /* device or host allocation failed */
#define AAOMG_ERR_CUDA (-3)          /* a CUDA runtime call failed (message in mg_last_error) */
#define AAOMG_ERR_NOT_CONVERGED (-4) /* max_iter reached above tol; x holds the last iterate */
#define AAOMG_ERR_DIVERGED (-5)      /* residual became NaN/Inf or grew by more than 1e6 */
#define AAOMG_ERR_NO_DEVICE (-7)     /* no CUDA device, or it is not sm_103 */

#define AAOMG_MAX_LEVELS 13

/* smoother (section 2) */
#define MG_SMOOTHER_NE 0    /* normal equation smoother, Algorithm 1, damped by tau */
#define MG_SMOOTHER_LSGS 1  /* least-squares Gauss-Seidel, Algorithm 2, undamped */
#define MG_SMOOTHER_SLSGS 2 /* symmetric LSGS: LSGS step then LSGS step in reversed order */
#define MG_SMOOTHER_CGS 3   /* collective Gauss-Seidel: the 2x2 block (y_i, lambda_i) of each node
                               solved in turn, nodes in the colour order (i + j) mod 3 */

/* precision */
#define MG_PREC_FP64 0        /* every operation in FP64 */
#define MG_PREC_FP32_REFINE 1 /* FP32 multigrid cycles inside FP64 iterative refinement */

typedef struct mg_ctx* mg_handle;

/* Options; an all-zero struct selects every default. */
typedef struct mg_options {
    int smoother;     /* MG_SMOOTHER_*; default NE (0) */
    int nu_pre;       /* pre-smoothing steps;  <= 0: 2 (sLSGS: 1) */
    int nu_post;      /* post-smoothing steps; <= 0: 2 (sLSGS: 1) */
    int cycle;        /* coarse-grid steps per level: 1 V-cycle, 2 W-cycle; 0: W */
    int precision;    /* MG_PREC_*; default FP64 */
    double tau;       /* NE damping; <= 0: 0.4 (the paper's value for Poisson control) */
    int k_variant;    /* 0: K = stiffness + mass (default); 1: K = bare stiffness matrix */
    int max_iter;     /* mg_solve iteration cap; <= 0: 100 */
    int inner_cycles; /* FP32_REFINE: FP32 cycles per refinement step; <= 0: 3 */
    int coarse_level; /* levels <= this run inside one single-block kernel; < 0: default, 0: none */
    int profile;      /* 1: time the smoothing calls of one level (profile_level) inside every
                         iteration (CUDA events) */
    int tile_w;       /* LSGS step kernel: owned columns per block; <= 0: widest the block allows */
    int tile_h;       /* LSGS step kernel: owned rows per block; <= 0: chosen to fill the GPU */
    int small_max;    /* levels with at most this many nodes per side smooth in one launch per
                         smoothing call (one block or one cluster: x and the residual in shared
                         memory up to 257 nodes per side; at 513, FP32 LSGS and sLSGS only, a
                         16-block cluster with the residual in shared memory and x in global
                         memory); 0: 513; < 0: never */
    int cluster_size; /* blocks per cluster of that launch on levels with 65, 129 or 257 nodes per
                         side (2..16); 0: by level size and precision (FP32: one block, 16, 16;
                         FP64: 8, 16, 16); 1: one block where it fits, else a launch per colour
                         phase.  A size that cannot run: BAD_ARG */
    int profile_level; /* with profile = 1: the level whose smoothing calls are timed; <= 0 or
                          > levels: the finest */
    int autotune;     /* 1: at set-up, time the candidate smoothing kernels of every level and keep
                         the fastest (one block or each cluster size that can run on levels up to
                         small_max nodes per side, unless cluster_size forces one; for LSGS above,
                         the one-launch step against a launch per colour phase); 0: the defaults */
} mg_options;

/* Build the hierarchy for h = 2^-levels (1 <= levels <= 13; level 1 is the
 * coarsest grid h = 1/2 with 18 unknowns) and regularisation alpha > 0
 * (finite).  Allocates all device workspaces on the current device.  On
 * success *out is a new handle.  Errors: BAD_ARG, NO_DEVICE, OOM, CUDA. */
AAOMG_API int mg_setup(int levels, double alpha, const mg_options* opt, mg_handle* out);

/* Free a handle and its workspaces (NULL is ignored).  Synchronises the device. */
AAOMG_API void mg_destroy(mg_handle h);

/* Number of nodes N per field on the finest level ((2^levels+1)^2). */
AAOMG_API long long mg_num_nodes(mg_handle h);

/* f = (M y_D, 0), eq. (mp2): yD (N doubles) and f (2N doubles) are device
 * pointers. */
AAOMG_API int mg_rhs_from_yd(mg_handle h, const double* yD, double* f, void* stream);

/* r = f - A x on the finest level (device pointers, 2N doubles each; r may be
 * NULL).  If relres is non-NULL it receives ||r||_{L^-1} / ||f||_{L^-1}, with
 * ||v||_{L^-1}^2 = v^T L^{-1} v and L = diag(Q) of section 2 (synchronises). */
AAOMG_API int mg_residual(mg_handle h, const double* f, const double* x, double* r, double* relres, void* stream);

/* `steps` smoothing steps of the configured smoother on the finest level:
 * x <- x + Ahat^{-1}(f - A x) (section 2; Algorithm 1, Algorithm 2, sLSGS or
 * the CGS block step), in place
 * on x.  In FP32_REFINE mode the steps run in FP32 on x and f rounded to
 * single precision.  Device pointers, 2N doubles each. */
AAOMG_API int mg_smooth(mg_handle h, const double* f, double* x, int steps, void* stream);

/* Defect restriction of section 2 on the finest level:
 * fc = I_k^{k-1} (f - A x), with I_k^{k-1} the transpose of the canonical
 * embedding.  f, x: 2N doubles; fc: 2Nc doubles for the next coarser level.
 * Requires levels >= 2.  Device pointers. */
AAOMG_API int mg_restrict(mg_handle h, const double* f, const double* x, double* fc, void* stream);

/* Prolongation and correction of section 2: x += I_{k-1}^k xc (canonical
 * embedding of the coarse P1 space).  xc: 2Nc doubles, x: 2N doubles.
 * Requires levels >= 2.  Device pointers. */
AAOMG_API int mg_prolong_add(mg_handle h, const double* xc, double* x, void* stream);

/* One multigrid iteration (section 2) on the finest level, in place on x.
 * FP64 mode: one cycle.  FP32_REFINE mode: one refinement step (FP64 defect,
 * `inner_cycles` FP32 cycles on it from zero, FP64 update).  Device pointers. */
AAOMG_API int mg_cycle(mg_handle h, const double* f, double* x, void* stream);

/* Iterate from the initial guess in x until ||f - A x||_{L^-1} <= tol *
 * ||f||_{L^-1} or max_iter iterations.  *iters (may be NULL) gets the number
 * of iterations, *relres (may be NULL) the final relative residual.  Returns
 * NOT_CONVERGED if the cap was hit (x holds the last iterate), DIVERGED on
 * NaN or blow-up.  Device pointers. */
AAOMG_API int mg_solve(mg_handle h, const double* f, double* x, double tol, int* iters, double* relres, void* stream);

/* The iteration count of section 3's protocol on the finest level: zero
 * right-hand side, initial iterate x0 (2N doubles, device, not modified), one
 * iteration (mg_cycle) at a time until the error ||x||_L (the exact solution
 * is 0) has dropped below reduction * ||x0||_L, with L = diag(Q) of section 2.
 * *iters receives the count, or -1 (status NOT_CONVERGED) if max_iter
 * iterations do not reach it, or -1 (DIVERGED) on a non-finite norm.
 * mg_get_history then gives ||x_k||_L / ||x0||_L.  Synchronises `stream` once
 * per iteration (the test is on the host). */
AAOMG_API int mg_protocol_iterations(mg_handle h, const double* x0, double reduction, int max_iter, int* iters,
                                     void* stream);

/* mg_solve with f and x in HOST memory (pinned or pageable): copies f and x to
 * the device, solves, and copies x back, all on `stream`. */
AAOMG_API int mg_solve_host(mg_handle h, const double* f_host, double* x_host, double tol, int* iters, double* relres,
                  void* stream);

/* Batched solves of independent problems (many right-hand sides, values of
 * alpha and grid sizes; the paper solves one problem at a time).
 *
 * mg_batch_create records ONE CUDA graph over `count` distinct handles (all on
 * the current device, none with opt.profile = 1): one branch per instance,
 * made of the residual norms of the initial iterate, a convergence test, and a
 * conditional while node whose body is one iteration of that handle (its
 * cycle, or its FP32 cycles and FP64 refinement update), the new residual norms
 * and the test again.  The tests run on the device (the same decisions as
 * mg_solve: diverged, converged to tol, max_iter reached), so one launch of the
 * graph takes every instance to its own convergence with no host round trip;
 * the branches are independent, so the GPU runs the instances' kernels
 * concurrently.  The batch keeps pointers to the handles: they must outlive it,
 * and a handle must not be used by another call while a batch solve runs.
 * Errors: BAD_ARG (null, repeated, profiled or multi-device handles), OOM, CUDA.
 */
typedef struct mg_batch_ctx* mg_batch;
AAOMG_API int mg_batch_create(int count, const mg_handle* handles, mg_batch* out);

/* Solve handles[k] A_k x_k = f_k from the initial guesses x_k to `tol` for
 * every k (f, x: arrays of `count` device pointers, 2N_k doubles each; x is
 * in/out): copies f_k and x_k into the handles, launches the batch graph on
 * `stream`, copies the solutions back and synchronises.  iters, relres and
 * status (NULL or arrays of count) receive each instance's iteration count,
 * final relative residual and status; mg_get_history of each handle gives its
 * residual history.  Returns the first nonzero instance status, else AAOMG_OK. */
AAOMG_API int mg_batch_solve(mg_batch b, const double* const* f, double* const* x, double tol, int* iters,
                             double* relres, int* status, void* stream);

/* mg_batch_solve with f_host and x_host arrays of HOST pointers (pinned or
 * pageable): the vectors are copied to the device, solved by one launch of the
 * batch graph and copied back, all on `stream`. */
AAOMG_API int mg_batch_solve_host(mg_batch b, const double* const* f_host, double* const* x_host, double tol,
                                  int* iters, double* relres, int* status, void* stream);

/* Batched adjoint of the solves (mg_adjoint for every instance at once): given
 * each instance's solution x_k of A_k x_k = (M y_D,k, 0) and ubar_k = dL/du_k
 * (N_k doubles), solves A_k z_k = (0, ubar_k / alpha_k) from zero to `tol` in
 * one launch of the batch graph and returns gyD_k = dL/dy_D,k = M z_k,y
 * (N_k doubles) and dalpha[k] = -alpha_k^{-2} (ubar_k . lambda_k +
 * z_k,lambda^T M lambda_k) (host array of count; eq. (mp2), dA/dalpha =
 * [[0,0],[0,alpha^{-2} M]]).  x, ubar, z (2N_k doubles, receives the adjoint
 * state), gyD: arrays of count device pointers.  iters (NULL or count ints)
 * receives the adjoint iteration counts.  Returns the first nonzero instance
 * status, else AAOMG_OK. */
AAOMG_API int mg_batch_adjoint(mg_batch b, const double* const* x, const double* const* ubar, double* const* z,
                               double* const* gyD, double* dalpha, double tol, int* iters, void* stream);

/* Free a batch (NULL is ignored); the handles stay valid.  Synchronises the device. */
AAOMG_API void mg_batch_destroy(mg_batch b);

/* One-shot batch: mg_batch_create, mg_batch_solve and mg_batch_destroy in one
 * call (the graph is recorded and instantiated each time; keep an mg_batch for
 * repeated solves).  Returns the first nonzero status of an instance, else
 * AAOMG_OK. */
AAOMG_API int mg_solve_batch(int count, const mg_handle* handles, const double* const* f, double* const* x, double tol,
                             int* iters, double* relres, void* stream);

/* The control u = alpha^{-1} lambda (eq. (mp2) and the relation below it) of
 * x = (y, lambda): x 2N doubles, u N doubles, device pointers. */
AAOMG_API int mg_control(mg_handle h, const double* x, double* u, void* stream);

/* Adjoint of the solve for a loss L(u) of the control u = lambda / alpha.
 * Given the solution x = (y, lambda) of A x = (M y_D, 0) and ubar = dL/du
 * (N doubles), solves A z = (0, ubar / alpha) to `tol` (A is symmetric, so the
 * adjoint operator is A itself) and returns
 *   gyD     = dL/dy_D  = M z_y                                   (N doubles),
 *   *dalpha = dL/dalpha = -alpha^{-2} (ubar . lambda + z_lambda^T M lambda),
 * the second term from dA/dalpha = [[0,0],[0,alpha^{-2} M]].  z (2N doubles)
 * receives the adjoint state.  Device pointers except dalpha (host). */
AAOMG_API int mg_adjoint(mg_handle h, const double* x, const double* ubar, double* z, double* gyD, double* dalpha,
                         double tol, void* stream);

/* The kernel that smooths level `level` (1..levels) inside the handle's cycle,
 * as chosen at set-up (defaults, options or autotuning): *kind is MG_KERNEL_*, *blocks
 * (may be NULL) the blocks per launch for STRIPS (1: one block, else the
 * cluster size) and BAND (the tiles), else 0. */
#define MG_KERNEL_PHASES 0 /* one launch per colour phase (per residual and update for NE) */
#define MG_KERNEL_STRIPS 1 /* whole smoothing call in one launch of one block or one cluster */
#define MG_KERNEL_BAND 2   /* one launch per LSGS step, wavefront over bands and segments */
#define MG_KERNEL_COARSE 3 /* no smoothing kernel: coarsest solve, dense coarse map or single-block cycle */
AAOMG_API int mg_level_kernel(mg_handle h, int level, int* kind, int* blocks);

/* ||x||_L and ||x||_{L^-1} of a vector x (2N doubles, device) on the finest
 * level, with L = diag(Q) of the paper's block preconditioner (section 2):
 * L_y = diag(M + alpha^{1/2} K), L_lambda = alpha^{-1} L_y.  ||.||_L is the norm
 * in which section 3 measures the error.  Either output may be NULL (not
 * both); results are written on the host after the stream has finished. */
AAOMG_API int mg_norms(mg_handle h, const double* x, double* norm_L, double* norm_Linv, void* stream);

/* Relative residual after each iteration of the last mg_solve: buf[0] is the
 * initial one; *n receives the count written (<= cap). */
AAOMG_API int mg_get_history(mg_handle h, double* buf, int cap, int* n);

/* With opt.profile = 1: total device time (ms) of the smoothing calls on the
 * profiled level (opt.profile_level, default the finest) inside the iterations
 * run since the last mg_reset_profile, and the number of smoothing steps
 * (sweeps) they cover; measured with CUDA events on the stream the kernels run
 * on. */
AAOMG_API int mg_get_profile(mg_handle h, double* smooth_ms, long long* sweeps);
AAOMG_API int mg_reset_profile(mg_handle h);

/* Kernel launches issued by this handle since it was created (for reports). */
AAOMG_API long long mg_kernel_launches(mg_handle h);

/* r = f - A x and ||r||_{L^-1} / ||f||_{L^-1} (as mg_residual) WITHOUT a handle
 * and without allocating any device memory.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate -- a program
 * with a device memory budget fixed at start-up, a framework whose caching
 * allocator owns all device memory, or a real-time loop that cannot afford the
 * device synchronisation cudaMalloc/cudaFree may cause.  Its scratch (row
 * partial sums) lives in a static device array of 4097 pairs of doubles
 * (about 64 KB) that every device using the library keeps until exit.
 *   levels:   1..12 (the finest grid, h = 2^-levels); 13 is rejected (BAD_ARG)
 *             because its 8193 grid rows exceed the static scratch;
 *   alpha > 0 and finite; k_variant 0 or 1 as in mg_options;
 *   f, x: device pointers, 2N doubles each; r: device pointer or NULL;
 *   relres: host pointer or NULL (if set, the call synchronises `stream`).
 * The first call on a device looks up the scratch address on that device
 * (cudaGetSymbolAddress), so make it before any stream capture.  All calls
 * share the scratch: calls that overlap on the GPU race and must be ordered by
 * the caller.  Errors: BAD_ARG, NO_DEVICE, CUDA (no message is recorded). */
AAOMG_API int mg_residual_noalloc(int levels, double alpha, int k_variant, const double* f, const double* x, double* r,
                                  double* relres, void* stream);

/* Name of an AAOMG_* code; message of the calling thread's last failure. */
/* The roofs of the library's kernels on the current device, measured with the
 * library's own microbenchmarks (the paper has no counterpart: measurement
 * only): the FP32 fused multiply-add rate (packed pairs, as the FP32 kernels
 * compute), the FP64 fused multiply-add rate, the read bandwidth of data
 * resident in L2 (a buffer of a quarter of the L2 size read repeatedly) and the
 * HBM copy bandwidth (2 GB read and 2 GB written).  Allocates about 4 GB for
 * the call and synchronises the device.  Errors: BAD_ARG, NO_DEVICE, OOM, CUDA. */
AAOMG_API int mg_device_peaks(double* fp32_tflops, double* fp64_tflops, double* l2_gbs, double* hbm_gbs);

AAOMG_API const char* mg_strerror(int code);
AAOMG_API const char* mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AAOMG_H */
