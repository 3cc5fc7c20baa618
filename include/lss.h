/*
 * lss.h - C ABI of the GB300 sparsify-and-sweep Lippmann-Schwinger solver.
 *
 * Liu & Ying, "Sparsify and sweep: an efficient preconditioner for the
 * Lippmann-Schwinger equation", arXiv:1705.09443.
 *
 * The library solves the discrete Lippmann-Schwinger equation (Sec. 2.1,
 * Eq. LS_d_c)
 *        (I + omega^2 K M) u = g   on I = {1..n}^d,  h = 1/(n+1),
 * with right-preconditioned restarted (flexible) GMRES whose preconditioner is
 * the sparsify-and-sweep operator P = E * Sweep * Q of Sec. 2.2-2.4
 * (Algorithms 1 and 2).  Every computation runs in the library's own CUDA
 * kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Vectors on I are complex128 (interleaved re, im doubles), row-major with
 *    x1 slowest: element (i1, i2) at offset (i1-1)*n + (i2-1) in 2D, element
 *    (i1, i2, i3) at ((i1-1)*n + (i2-1))*n + (i3-1) in 3D.  A batch of R
 *    vectors is R such arrays back to back (stride n^d complex numbers).
 *  - 3D grids (Sec. 3.1) use the same construction with the 27-point
 *    neighbourhood and the 26 PML directions; their slab subproblems are block
 *    tridiagonal along x2 with dense blocks of (slab layers) x n_tot unknowns,
 *    factored by block Gaussian elimination whose pivot blocks are inverted
 *    explicitly (Gauss-Jordan with partial pivoting inside each block).
 *  - Pointers named *_dev are device pointers owned by the caller; *_host are
 *    host pointers owned by the caller.  The library never frees them and keeps
 *    no reference after the call returns.
 *  - The library owns the context, the slab factors and all workspace.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *    work on it; entry points that return host-visible results (stats) block
 *    until those results are ready.
 *  - Return value: LSS_OK (0) or a negative LSS_ERR_* code; lss_last_error()
 *    then describes the failure.  A failed call leaves the context usable
 *    unless the code is LSS_ERR_CUDA.
 *
 * Environment switches (read at each call; each selects between two exact
 * implementations of the same operation, for comparison and testing):
 *  - LSS_SLAB_SOLVE=cr: 2D slab solves always by the block cyclic reduction
 *    (default: the 16-wide slabs of solves with R >= 16 by the block LU).
 *  - LSS_BATCH_THREADS=1: a batch context solves each instance on its own
 *    host thread (default: one lockstep Krylov driver for all instances).
 *  - LSS_SOLVE_NR=2: two right-hand sides per cyclic-reduction CTA on 16-wide
 *    slabs from the start (default: the autotuner decides).
 *  - LSS_TC_UPDATE=0: the 3D mixed factorization's rank updates on CUDA
 *    cores (default: 3xTF32 tcgen05 tensor cores).
 */
#ifndef LSS_H
#define LSS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lss_ctx lss_ctx;

/* Grid (Sec. 2.1, Sec. 3.1): dimension d (2 or 3), n points per unit length,
 * h = 1/(n+1), p_i = i h. */
typedef struct { int dim; int n; } lss_grid;

/* PML (Sec. 2.2.2): b_pml layers (eta = b_pml h) and the strength C of
 * sigma(x) = +-(C/omega)((x -+ ...)/eta)^2. */
typedef struct { int b_pml; double C; } lss_pml;

/* Sweep (Sec. 2.3-2.4): b_slab normal layers per slab along x1 (the first
 * slab adds the left PML, the last takes the remainder plus the right PML),
 * b_aux auxiliary moving-PML layers (0 = b_pml), n_samples squared-frequency
 * samples for the auxiliary stencils (0 = n).  fronts: 0 or 1 = one front
 * sweeping left to right (Algorithm 2); 2 = two fronts sweeping toward the
 * middle slab (n_slabs - 1) / 2 (Sec. 2.4 remark 1, the setting of Sec. 2.5):
 * the slabs right of it take their auxiliary PML on the right, the middle slab
 * on both sides (with b_slab + 2 b_aux <= 32 in 2D).  The transposed sweep,
 * the adjoint solve and the medium gradient are built for one front and return
 * LSS_ERR_UNSUPPORTED with two.  recursive (3D only; 0 in 2D, else
 * LSS_ERR_UNSUPPORTED): 1 = the recursive approach of Sec. 3.1, every slab
 * subproblem swept along x2 over quasi-1D sub-slab problems (the same
 * partition of x2, each padded before its first x2 layer with b_aux auxiliary
 * PML layers) instead of factored whole. */
typedef struct { int b_slab; int b_aux; int n_samples; int fronts; int recursive; } lss_slab;

/* GMRES (Sec. 2.5): restart length, relative tolerance on ||g - A u||/||g||,
 * cap on the total number of Arnoldi steps. */
typedef struct { int restart; double tol; int max_iter; } lss_gmres;

/* Per right-hand side results. */
typedef struct {
    int iters;            /* Arnoldi steps taken                              */
    int converged;        /* 1 if the Givens residual reached tol             */
    double relres_est;    /* Givens estimate |rho|/||g|| at exit              */
    double relres_true;   /* ||g - A u|| / ||g|| recomputed at exit           */
} lss_stats;

enum { LSS_FP64 = 0, LSS_MIXED = 1 };

enum {
    LSS_OK = 0,
    LSS_ERR_ARG = -1,          /* invalid argument (null pointer, size)         */
    LSS_ERR_OOM = -2,          /* device allocation failed                      */
    LSS_ERR_STATE = -3,        /* call out of order (e.g. solve before factor)  */
    LSS_ERR_SINGULAR = -4,     /* zero or non-finite pivot in a slab factor     */
    LSS_ERR_NOCONVERGE = -5,   /* GMRES hit max_iter; best iterate is written   */
    LSS_ERR_TIMEOUT = -6,      /* a bounded device wait expired                 */
    LSS_ERR_CUDA = -7,         /* CUDA runtime error                            */
    LSS_ERR_UNSUPPORTED = -8   /* configuration outside the supported range     */
};

/*
 * lss_setup - Algorithm 1 steps 1-3 and the operator data (Sec. 2.1-2.3).
 * Builds the Nystrom weights k (Sec. 2.1; k_0 = integral of G over the grid
 * cell), their FFT for the zero-padded convolution, the interior stencils
 * alpha, beta (Eq. alpha, Eq. beta), the PML stencils gamma (Eq. gamma) for the
 * physical PML and, per squared-frequency sample, for the moving PML
 * (Sec. 2.3), the slab partition, and assembles every slab subproblem
 * (Eq. Hwv_approx).
 *   out        receives the new context (NULL on failure)
 *   g          grid; 2D: n in [4, 2048]; 3D: n in [3, 128]
 *   omega      angular frequency > 0
 *   m_dev      device, n^d float64, m = 1 - 1/c^2 on I (row-major, x1 slowest)
 *   pml, slab  parameters above; 2D: every slab subproblem must be at most 32
 *              layers wide: b_aux + b_slab + b_pml <= 32 (the last slab);
 *              3D: (layers of the widest subproblem) x (n + 2 + 2 b_pml) must
 *              not exceed 1600 (LSS_ERR_UNSUPPORTED otherwise)
 *   precision  LSS_FP64 (all FP64) or LSS_MIXED (slab factors, sweep and the
 *              interface matrices in FP32; LS matvec, Arnoldi, Givens and the
 *              true residual in FP64; solves use flexible GMRES either way)
 * Copies m; the caller may free m_dev after the call.
 */
int lss_setup(lss_ctx **out, const lss_grid *g, double omega, const double *m_dev,
              const lss_pml *pml, const lss_slab *slab, int precision, void *stream);

/*
 * lss_set_medium - replace m on an existing context (same grid, omega and
 * parameters).  The Nystrom weights, their FFT, alpha, beta and the physical
 * PML stencils depend only on (n, omega) and are kept (Sec. 2.4, remark 3);
 * the squared-frequency samples, the moving-PML stencils and the slab
 * subproblems are rebuilt.  The context returns to the unfactored state.
 *   m_dev      device, n^d float64 (copied)
 */
int lss_set_medium(lss_ctx *c, const double *m_dev, void *stream);

/*
 * lss_factor - Algorithm 1 steps 4-8: block-tridiagonal LU (along x2, pivoting
 * inside each block) of every slab subproblem, all slabs in one launch, then
 * (2D) the interface maps that let the sweep of Algorithm 2 run slab-parallel.
 * In 3D every slab's pivot blocks D_k = A_k - C_k D_{k-1}^{-1} B_{k-1} are
 * inverted explicitly and stored; all slabs advance together.
 * Returns LSS_ERR_SINGULAR if a block pivot vanished.  Blocks the host.
 */
int lss_factor(lss_ctx *c, void *stream);

/*
 * lss_plane_wave_rhs - right-hand sides g = -omega^2 K (m .* u_I) (Sec. 2.1)
 * for R incident plane waves u_I = exp(i omega d . p).
 *   dirs_host  host, R x dim float64 unit directions
 *   g_dev      device, R x n^d complex128 (output)
 *   uI_dev     device, R x n^d complex128 (output) or NULL
 */
int lss_plane_wave_rhs(lss_ctx *c, const double *dirs_host, int R, void *g_dev,
                       void *uI_dev, void *stream);

/*
 * lss_apply_A - y = (I + omega^2 K M) x (transpose = 0) or
 * y = (I + omega^2 M K) x = A^T x (transpose = 1), Eq. LS_d_c, for R vectors;
 * zero-padded FFT convolution.  x_dev and y_dev may not alias.
 */
int lss_apply_A(lss_ctx *c, const void *x_dev, void *y_dev, int R, int transpose,
                void *stream);

/*
 * lss_apply_P - y = P x, the preconditioner of Sec. 2.2-2.4 (Algorithm 2):
 * f = Q x (alpha rows on I^h, Eq. Huf), the forward/backward moving-PML sweep
 * with the slab factors, restriction to I.  transpose = 1 applies the bilinear
 * transpose P^T = Q^T Sweep^T E^T: embedding of x on the grid, the sweep with
 * the transposed slab solves in reverse order (forward pass
 * w_i = v_i - H_{[i-1,i]}^T last(T~_{i-1}^T w_{i-1}), backward pass
 * x_i = T~_i^T (w_i - H_{[i+1,i]}^T first(x_{i+1}))), then Q^T (conj(alpha)
 * rows transposed).  The first transposed call after lss_factor also builds
 * the transposed sweep's interface maps.  Requires lss_factor.
 * x_dev, y_dev: R x n^d c128.  3D: transpose = 1 returns LSS_ERR_UNSUPPORTED;
 * the sweep of Algorithm 2 runs as one grid-synchronised launch (slab after
 * slab, block row after block row).
 */
int lss_apply_P(lss_ctx *c, const void *x_dev, void *y_dev, int R, int transpose,
                void *stream);

/*
 * lss_solve - solve (I + omega^2 K M) u = g for R right-hand sides with
 * flexible GMRES(restart), right preconditioned by P, x0 = 0, CGS2 Arnoldi in
 * FP64, per-RHS convergence masks (Sec. 2.5 uses standard restarted GMRES).
 *   g_dev      device, R x n^d complex128
 *   u_dev      device, R x n^d complex128 (output; best iterate on failure)
 *   stats      host, R entries (output), may be NULL
 * Returns LSS_ERR_NOCONVERGE if some RHS missed tol within max_iter.
 */
int lss_solve(lss_ctx *c, const void *g_dev, void *u_dev, int R, const lss_gmres *o,
              lss_stats *stats, void *stream);

/*
 * lss_adjoint_solve - solve A^T mu = rhs, A^T = I + omega^2 M K (the bilinear
 * transpose of Eq. LS_d_c; K is symmetric), for R right-hand sides with
 * flexible GMRES right-preconditioned by P^T (lss_apply_P, transpose = 1),
 * same options, statistics and errors as lss_solve.  For a real misfit L(u) of
 * a solution u of lss_solve, rhs = conj(dL/du) (dL/du = dL/dRe u + i dL/dIm u)
 * gives mu with dL/dm = Re((-omega^2 K mu) . (u + u_I)) (lss_medium_gradient).
 *   rhs_dev, mu_dev  device, R x n^d complex128
 * 2D grids only (LSS_ERR_UNSUPPORTED on a 3D context).
 */
int lss_adjoint_solve(lss_ctx *c, const void *rhs_dev, void *mu_dev, int R, const lss_gmres *o,
                      lss_stats *stats, void *stream);

/*
 * lss_medium_gradient - grad = sum_r Re((-omega^2 K mu_r) . (u_r + u_I,r)) on
 * I: the derivative of a real misfit with respect to m, from the adjoint
 * states mu (lss_adjoint_solve) and the scattered fields u of the plane waves
 * with directions dirs (u_I = exp(i omega d.p), Eq. LS_d).
 *   mu_dev, u_dev  device, R x n^d complex128
 *   dirs_host      host, R x 2 unit directions
 *   grad_dev       device, n^d float64 (output)
 * 2D grids only (LSS_ERR_UNSUPPORTED on a 3D context).
 */
int lss_medium_gradient(lss_ctx *c, const void *mu_dev, const void *u_dev, const double *dirs_host,
                        int R, double *grad_dev, void *stream);

/*
 * lss_helmholtz_solve - the sparsifying scheme as a direct discretization of
 * the Helmholtz equation (Sec. 4): solve the sparsified system
 *        H u~ = beta^* f   on the n_tot^2 grid,
 * i.e. alpha^* u_{mu_i} + omega^2 beta^* (m u)_{mu_i} = beta^* f_{mu_i} on I^h with
 * the PML rows of H, for R sources f (a discrete delta f = 1/h^2 at one point
 * gives about the Green's function, Sec. 4; with a medium m the equation is
 * (-Laplace - omega^2 (1 - m)) u = f).  Flexible GMRES on H (FP64, the
 * context's subproblem rows) right-preconditioned by the moving-PML sweep on
 * grid vectors; same options and statistics as lss_solve (relres is measured
 * with H on the grid).  2D grids only; requires lss_factor.
 *   f_dev      device, R x n^2 complex128 source values on I
 *   u_dev      device, R x n^2 complex128 (output): u~ restricted to I
 */
int lss_helmholtz_solve(lss_ctx *c, const void *f_dev, void *u_dev, int R, const lss_gmres *o,
                        lss_stats *stats, void *stream);

/*
 * lss_solve_host - the same solve with host buffers: copies g_host to the
 * device, solves, copies u back.  g_host, u_host: R x n^d complex128 (pinned
 * memory gives asynchronous copies).  Blocks the host.
 */
int lss_solve_host(lss_ctx *c, const void *g_host, void *u_host, int R,
                   const lss_gmres *o, lss_stats *stats, void *stream);

/*
 * lss_apply_slab - test hook: w = T~_i v, the moving-PML slab operator of
 * Eq. Hwv_approx (pad v with zeros on the auxiliary layers, solve the slab
 * subproblem with the stored factors, restrict to D_i).
 *   slab       0-based slab index
 *   v_dev, w_dev  device, R x (layers of D_i) x n_tot complex128 with
 *              n_tot = n + 2 + 2 b_pml, x1 layer slowest; in 3D
 *              R x (layers of D_i) x n_tot x n_tot (x1, then x2, then x3)
 */
int lss_apply_slab(lss_ctx *c, int slab, const void *v_dev, void *w_dev, int R,
                   void *stream);

/*
 * lss_apply_slab_noalloc - the same slab operator as lss_apply_slab, for
 * callers that must not reach the device allocator during the call: code
 * whose device memory is fully handed out up front (another framework's
 * caching allocator owns the rest of HBM), or latency-critical loops where a
 * workspace that grows through cudaMalloc/cudaFree would stall (cudaFree
 * synchronises the device).  The paper has no counterpart; this is a property
 * of the library, not of the method.
 * The call allocates nothing.  Its scratch is one fixed array of 8 MiB in
 * device memory that every GPU loading the library holds until the process
 * exits.  The first call on each device looks up that array's device address
 * (with the device current) and caches it; make that first call before any
 * stream capture on the device.  All calls share the array and it keeps the
 * last call's contents (nothing in it needs to start at zero): calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  A call that would need more than 8 MiB of scratch
 * (R x n_tot x P complex entries of the working precision, P = 16 when the
 * widest slab subproblem has at most 16 layers, else 32) returns
 * LSS_ERR_UNSUPPORTED without launching.
 * Arguments, layouts and ownership as for lss_apply_slab.  2D contexts only
 * (LSS_ERR_UNSUPPORTED on a 3D context); LSS_ERR_ARG on a batch context.
 * The cached address is valid while the device's primary context lives: do
 * not call this entry point again after cudaDeviceReset.
 */
int lss_apply_slab_noalloc(lss_ctx *c, int slab, const void *v_dev, void *w_dev, int R,
                           void *stream);

/* Sizes of the context: n_tot, number of slabs, first x1 index and number of
 * layers of slab i (x1 runs over -b_pml .. n+1+b_pml), FFT length. */
int lss_info(const lss_ctx *c, int *n_tot, int *n_slabs, int *fft_len);
int lss_slab_info(const lss_ctx *c, int slab, int *first_x1, int *n_layers, int *n_aux);

/* Interior stencils alpha, beta (Eq. alpha, Eq. beta) as 3^d complex128 each
 * (9 in 2D, 27 in 3D), copied to host arrays; lexicographic offsets, x1
 * slowest. */
int lss_get_stencils(const lss_ctx *c, double *alpha_host, double *beta_host);

/* Profiling.  lss_profile(c, 1) starts recording CUDA events (on the
 * caller's stream) around every kernel group of the library; lss_profile(c, 0)
 * stops.  lss_profile_read() waits for the recorded work, returns the summed
 * device milliseconds and launch counts per category since the previous read,
 * and clears them.  Categories (LSS_PROF_*): */
enum {
    LSS_PROF_MATVEC = 0,   /* LS operator: row FFT, column FFT x kernel, row IFFT  */
    LSS_PROF_SPARSIFY = 1, /* f = Q r                                             */
    LSS_PROF_SLAB_A = 2,   /* slab solves a_i = T~_i f_i (all slabs)              */
    LSS_PROF_RECUR = 3,    /* interface recurrences                               */
    LSS_PROF_SLAB_E = 4,   /* slab solves with the interface couplings            */
    LSS_PROF_FACTOR = 5,   /* block-tridiagonal LU of all slabs                   */
    LSS_PROF_IFACE = 6,    /* interface maps (multi-RHS slab solves)              */
    LSS_PROF_KRYLOV = 7,   /* Gram-Schmidt, norms, updates                        */
    LSS_PROF_SETUP = 8,    /* kernel table, stencils, assembly                    */
    LSS_PROF_NCAT = 9
};
int lss_profile(lss_ctx *c, int enable);

/*
 * lss_set_graphs - replay the kernels of each GMRES iteration (preconditioner,
 * operator, both Gram-Schmidt passes) from a CUDA graph (enable = 1, the
 * default) or launch them one by one (0).  Graphs are captured per basis
 * index, number of right-hand sides and transpose flag after a first solve
 * with the same R has sized every workspace; they are dropped when a
 * workspace is reallocated and are not used while profiling is on.  The
 * results are the same either way.  On a batch context: every instance.
 * The paper has no counterpart: this is how the library launches Sec. 2.5's
 * GMRES iterations, not part of the method.
 */
int lss_set_graphs(lss_ctx *c, int enable);
/*
 * lss_autotune - pick launch parameters for R right-hand sides by timing this
 * context's own operations (CUDA events, a few runs per candidate): the FFT
 * column group of the LS operator, the slab-solve shared-memory plan (ring
 * stages; right-hand sides in shared or global memory) and the recurrence's
 * ring depth.  2D grids only (LSS_ERR_UNSUPPORTED on a 3D context).  None of them changes any result (same arithmetic, same order),
 * so later solves agree bit for bit with untuned ones; only their speed
 * changes.  Requires a factored context; allocates and frees two vectors;
 * blocks the host.  On a batch: every instance.  The paper has no
 * counterpart (launch configuration only).
 *   chosen  host, 7 ints (may be NULL): column group, right-hand sides in
 *           global memory (0) or automatic (-1), ring stages (0 = automatic),
 *           recurrence stages, ring stages of the 32-wide slabs' launches
 *           (0 = as the others), slab solves within half the shared memory
 *           so that two CTAs share an SM (1) or not (0), right-hand sides
 *           per slab-solve CTA on 16-wide slabs (1 or 2)
 */
int lss_autotune(lss_ctx *c, int R, int *chosen, void *stream);

/* Iteration graphs held by the context (all instances of a batch): captured,
 * and refused (bodies that cannot be captured, e.g. with the grid-synchronised
 * recurrence of very many right-hand sides; those iterations run uncaptured). */
int lss_graph_count(const lss_ctx *c, int *captured, int *refused);
/* ms, launches: arrays of ncat entries (either may be NULL). */
int lss_profile_read(lss_ctx *c, double *ms, long long *launches, int ncat);

/*
 * Ragged instances: several independent problems of different grid size,
 * frequency and medium behind one context (the paper treats one problem at a
 * time; batching independent problems is this library's own form).  Each
 * instance is a full context with its own stream; a call on the batch forks
 * the caller's stream, drives every instance concurrently (one host thread
 * per instance, up to 32) and joins back, so small instances share the GPU.
 *
 * lss_setup_batch - lss_setup for n_inst instances (2D grids only).
 *   g, omega, m_dev  arrays of n_inst entries (grid, angular frequency, device
 *                    pointer to that instance's n_q^2 float64 medium)
 *   pml, slab, precision  shared by all instances
 * On a batch context lss_factor, lss_plane_wave_rhs, lss_apply_A,
 * lss_apply_P, lss_solve, lss_adjoint_solve, lss_medium_gradient,
 * lss_profile, lss_profile_read and lss_destroy act on every instance:
 *   vectors    instance q's R x n_q^2 complex128 values start at element
 *              R * (n_0^2 + ... + n_{q-1}^2) of the one device array passed
 *   stats      R x n_inst entries, instance-major (stats[q * R + r])
 *   gradient   instance q's n_q^2 values start at n_0^2 + ... + n_{q-1}^2
 *   directions R per instance, instance-major: n_inst x R x 2 float64 on the
 *              host (lss_plane_wave_rhs, lss_medium_gradient)
 * Errors: the first failing instance's code (LSS_ERR_NOCONVERGE only if no
 * instance failed otherwise), its message prefixed with "instance q: ".
 * lss_set_medium, lss_solve_host, lss_apply_slab(_noalloc), lss_info,
 * lss_slab_info and lss_get_stencils return LSS_ERR_ARG on a batch context:
 * call them on an instance.
 */
int lss_setup_batch(lss_ctx **out, int n_inst, const lss_grid *g, const double *omega,
                    const double *const *m_dev, const lss_pml *pml, const lss_slab *slab,
                    int precision, void *stream);
/* Number of instances and sum of n_q^2 over them; LSS_ERR_ARG if c is not a batch. */
int lss_batch_info(const lss_ctx *c, int *n_inst, long long *elems_per_rhs);
/* Instance q of a batch (owned by the batch: do not destroy it). */
int lss_batch_instance(lss_ctx *c, int q, lss_ctx **inst);

/*
 * lss_test_inject - fault injection for tests; the paper has no counterpart.
 * Nothing here touches memory outside the context's own arrays.
 *   what = 1  zero the coefficients of block row b (the x2 index + b_pml) of
 *             slab a's subproblem (its diagonal block in 3D); the context
 *             returns to the unfactored state, and the next lss_factor meets
 *             a zero pivot and returns LSS_ERR_SINGULAR
 *   what = 2  run the library's bounded device waits on conditions nothing
 *             satisfies (a grid barrier one arrival short, an mbarrier nobody
 *             arrives at); each gives up after the wait limit (about 2 s) and
 *             the call returns LSS_ERR_TIMEOUT; the context stays usable
 * Returns LSS_ERR_ARG for other values or on a batch context.
 */
int lss_test_inject(lss_ctx *c, int what, int a, long long b, void *stream);

/* Message of the last failure on this context ("" if none). */
const char *lss_last_error(const lss_ctx *c);

/* Frees the context and all device memory it owns.  NULL is ignored. */
void lss_destroy(lss_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* LSS_H */
