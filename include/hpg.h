/*
 * hpg.h -- C ABI of libhpg: hierarchical proximal Galerkin (hpG) on one GB300.
 *
 * The library solves the latent-variable proximal point (LVPP) subproblems of
 * Papadopoulos, "Hierarchical proximal Galerkin" (arXiv:2412.13733):
 *
 *   obstacle type, eq. (pG), Section 2.1 and 4.1:
 *     alpha_k (grad u, grad v) + (psi_k, v) = alpha_k (f, v) + (psi_{k-1}, v)
 *     (u, zeta) + (exp(-psi_k), zeta)       = (phi, zeta)
 *   gradient type, eq. (pG:gradient), Section 2.2 and 4.2:
 *     alpha_k (grad u, grad v) + (psi_k, grad v) = alpha_k (f, v) + (psi_{k-1}, grad v)
 *     (grad u, zeta) = (phi psi_k / sqrt(1 + |psi_k|^2), zeta)
 *
 * discretised with the hierarchical p-FEM basis of Section 3 (u: hats +
 * bubbles W_n, eq. (Wn); psi: cellwise Legendre, degree p-2 for obstacles and
 * p-1 (d components) for gradient constraints) on uniform tensor-product
 * quad/hex meshes.  Each subproblem is solved by Newton (Newton matrix G of
 * eq. (pG-matrix)); each Newton system by the Schur sequence of eq. (schur2),
 * with GMRES on the Schur complement S of eq. (schur4), right-preconditioned
 * by the cell-block-diagonal S-hat of eq. (schur-preconditioner) or
 * eq. (schur-preconditioner:gradient), whose blocks are factorised as
 * batched dense Cholesky on the device.
 *
 * Conventions
 * -----------
 *  - Every call returns an hpg_status; nothing aborts or throws across the ABI.
 *  - The caller owns every host buffer passed in; the library copies what it
 *    keeps.  The context owns all device memory it allocates.  A pointer
 *    argument documented as "device" must point to memory of the context's
 *    device; all others are host pointers.
 *  - Sizes: every output buffer comes with its length in elements; a length
 *    smaller than required returns HPG_ERR_ARG and writes nothing.
 *  - Threading: a context may be used by one host thread at a time.
 *
 * Coefficient orderings (shared with the CPU oracle by specification)
 * ------------------------------------------------------------------
 *  u (full):  tensor product of the 1D global numbering, x index fastest.
 *             1D numbering on m cells: hats 0..m first, then bubbles
 *             cell-major (bubble b of cell c at m + 1 + c (p - 1) + b).
 *             Length prod_j (m_j p + 1).
 *  u (interior): the entries of u (full) whose every 1D index is neither
 *             hat 0 nor hat m, in the same relative order.  Length
 *             prod_j (m_j p - 1).
 *  psi:       cell-major; cell c = c_x + m_x c_y (+ m_x m_y c_z); inside a
 *             cell [component][n^d coefficients, x degree fastest];
 *             n = p - 1 (obstacle) or p (gradient, d components).
 *  Newton vectors x = [u (interior); psi].
 */
#ifndef HPG_H
#define HPG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpg_ctx hpg_ctx;

typedef enum {
    HPG_OK = 0,
    HPG_ERR_ARG = 1,            /* bad argument, size or id                                  */
    HPG_ERR_OOM = 2,            /* device or host allocation failed                          */
    HPG_ERR_CUDA = 3,           /* a CUDA runtime call failed (see hpg_last_error)           */
    HPG_ERR_NEWTON_CAP = 4,     /* a subproblem hit the Newton iteration cap                 */
    HPG_ERR_KRYLOV_CAP = 5,     /* GMRES hit its cap before its tolerance (reported only)    */
    HPG_ERR_NONFINITE = 6,      /* NaN/Inf, or psi < -700 at a Gauss point (exp overflow)    */
    HPG_ERR_NOT_SPD = 7,        /* a cell block of -S-hat had a non-positive pivot in FP64
                                   (HPG_MIXED takes a failed step again in FP64 first)          */
    HPG_ERR_TIMEOUT = 8,        /* a bounded host wait expired                               */
    HPG_ERR_INFEASIBLE_BC = 9,  /* Dirichlet data violates the constraint on the boundary    */
    HPG_ERR_STATE = 10,         /* call out of order (e.g. solve before data were set)       */
    HPG_ERR_BUSY = 11           /* the problem is part of an unfinished batch or request     */
} hpg_status;

typedef enum {
    HPG_OBSTACLE_UPPER = 0,     /* u <= phi (the paper's form, eq. ad:obstacle)              */
    HPG_OBSTACLE_LOWER = 1,     /* u >= phi, solved as -u <= -phi with f, g negated          */
    HPG_GRADIENT = 2            /* |grad u| <= phi (eq. ad:gradient)                         */
} hpg_kind;

typedef enum {
    HPG_FP64 = 0,               /* every step in FP64                                        */
    HPG_MIXED = 1               /* FP64 residuals, exp and orthogonalisation; inner Schur
                                   operator and preconditioner in FP32 inside FP64 iterative
                                   refinement of each Newton system                           */
} hpg_precision;

/* How each Newton system G delta = F of eq. (pG-matrix) is solved (Section 4.3).
 * HPG_SCHUR: the Schur-complement sequence of eq. (schur2) with S-hat-preconditioned
 *   GMRES on S (the strategy the paper uses in 2D).
 * HPG_FGMRES_PD / _PLPD / _PF: flexible GMRES on G, right-preconditioned by the block
 *   preconditioner P_D = diag(A_alpha, S), P_L P_D, or P_F = P_L P_D P_R of eq. (schur4);
 *   S^{-1} is S-hat^{-1} for P_D and P_L P_D, and at most hpg_params.inner_max iterations of
 *   S-hat-preconditioned GMRES on S (relative tolerance 1e-5) for P_F ("P_F-(n)").
 *   A_alpha^{-1} is the exact fast diagonalisation in every strategy.  FP64 only. */
typedef enum {
    HPG_SCHUR = 0,
    HPG_FGMRES_PD = 1,
    HPG_FGMRES_PLPD = 2,
    HPG_FGMRES_PF = 3
} hpg_strategy;

/* Field callback: out[i] = field(x[i*dim], ..., x[i*dim+dim-1]) for i < npts. */
typedef void (*hpg_field_fn)(int npts, int dim, const double* x, double* out, void* user);

typedef struct {
    double beta;          /* E_beta = beta M_Psi (obstacle) or beta (grad_h zeta, grad_h zeta)
                             (gradient); Jacobian only, Section 4.1                           */
    double newton_tol;    /* absolute l2 norm of [F_u; F_psi]; default 1e-10                 */
    int    newton_max;    /* Newton cap per proximal step; default 50                         */
    int    krylov_max;    /* GMRES cap (no restart); default 150                              */
    double krylov_rtol;   /* GMRES relative tolerance ceiling; the forcing term is
                             min(krylov_rtol, ||F||) relative; default 1e-5                   */
    int    precision;     /* hpg_precision; default HPG_FP64                                  */
    int    ls_max;        /* line-search halvings; default 10                                 */
    int    refine_max;    /* HPG_MIXED: FP64 refinement sweeps per Newton system; default 8   */
    int    timing;        /* 1: record CUDA-event time per kernel class (hpg_get_kernel_times) */
    int    graphs;        /* 1 (default): GMRES runs as a device-side loop in one CUDA graph;
                             0: host-driven launches (for profilers that cannot trace
                             conditional graph nodes)                                          */
    int    fdm_tile_f32;  /* -1 (default): the FP32 fast-diagonalisation pass variant is picked
                             by timing all of them at set-up; 0 .. hpg_fdm_tile_count(HPG_MIXED)-1
                             forces one (the last six are tcgen05 3xTF32 tensor-core
                             kernels: two staging operands element by element, then four fed
                             by TMA with N tiles of 64, 128, 256 and 32 columns); changing it
                             releases the problem's device state                              */
    int    fdm_tile_f64;  /* the same for the FP64 passes                                     */
    int    strategy;      /* hpg_strategy; default HPG_SCHUR; the FGMRES strategies need
                             precision HPG_FP64 (HPG_ERR_ARG otherwise)                       */
    int    inner_max;     /* HPG_FGMRES_PF: inner GMRES iterations per application; default 10 */
    int    krylov_f32;    /* 0 (default): the GMRES basis and its Gram-Schmidt are FP64 in both
                             precisions (the mixed form keeps Krylov orthogonalisation in FP64);
                             1: with HPG_MIXED the FP32 inner solves store and orthogonalise
                             their basis in FP32 (per-lane products and updates in FP32, lane and
                             chunk sums, Hessenberg and Givens in FP64) -- faster, outside that
                             rule; the FP64 refinement still sets the accuracy.  Ignored for
                             HPG_FP64.                                                          */
    int    ainv_pcg;      /* 0 (default): A_alpha^{-1} is the exact fast diagonalisation;
                             1, 2, 3: in the FGMRES strategies HPG_FGMRES_PD and _PLPD,
                             A_alpha^{-1} is preconditioned CG (the inexact inverse of Section
                             6.5) with that preconditioner of hpg_stiffness_solve_pcg, to relative
                             tolerance ainv_rtol.  Ignored by HPG_SCHUR and HPG_FGMRES_PF, whose
                             A_alpha^{-1} runs inside the device-side GMRES loop               */
    double ainv_rtol;     /* relative tolerance of that CG; default 1e-10                       */
    int    fdm_tune_batch;/* 1 (default): the set-up autotuner picks the fast-diagonalisation
                             variant that is fastest for this problem alone; B in 2..64: the
                             variant with the least time per problem when B same-shape problems
                             run in one lockstep launch (hpg_solve_batch).  A group runs its
                             members' variant, so solving alone and in a batch give the same
                             bits either way; changing it releases the device state            */
} hpg_params;

#define HPG_MAX_ALPHA 128

typedef struct {
    int    status;                         /* hpg_status of the last solve                 */
    int    alpha_steps;                    /* proximal subproblems solved                  */
    int    newton_total;                   /* Newton iterations (linear solves)            */
    int    newton_per_step[HPG_MAX_ALPHA]; /* Newton iterations per proximal step          */
    long long krylov_total;                /* inner GMRES iterations over the solve        */
    int    refine_total;                   /* HPG_MIXED refinement sweeps over the solve   */
    int    ls_fail;                        /* line searches that ran out of halvings       */
    int    krylov_cap_hits;                /* GMRES solves that stopped at the cap         */
    double final_residual;                 /* ||F|| at the end of the last subproblem      */
    double solve_ms;                       /* wall time of the last hpg_solve (host clock) */
    long long n_u;                         /* interior u unknowns                          */
    long long n_psi;                       /* psi unknowns                                 */
    long long kernel_launches;             /* libhpg kernels launched by the last solve    */
    long long h2d_bytes;                   /* problem data copied host->device by it       */
    int    fdm_tile_f32;                   /* FDM GEMM tile variant picked by the autotuner */
    int    fdm_tile_f64;                   /*   (FP32 and FP64 passes)                      */
    long long fgmres_total;                /* outer FGMRES iterations (FGMRES strategies)  */
    long long ainv_total;                  /* applications of A_alpha^{-1} over the solve  */
    long long ainv_iters;                  /* CG iterations of those applications (ainv_pcg) */
    /* HPG_MIXED fallback: a proximal step whose mixed Newton iteration fails (a
       non-positive pivot of the FP32 S-hat elimination, a line search that ends on a
       non-finite trial point, the Newton cap) is solved again from its starting point in
       FP64, and so is the rest of the solve.  newton_total counts the discarded steps too,
       newton_per_step the FP64 ones.  A lockstep-group member that falls back is solved
       again on its own after the group, which gives the result of solving it alone. */
    int    fp64_from_step;                 /* proximal step (1-based) of the fallback, or 0 */
    int    fp64_newton_steps;              /* Newton steps taken in FP64 after it          */
} hpg_stats;

/* Kernel classes timed when hpg_params.timing = 1. */
typedef enum {
    HPG_K_EVAL = 0,       /* Gauss evaluation of the latent nonlinearity                   */
    HPG_K_RESIDUAL = 1,   /* Newton residual F_u, F_psi and its norm                       */
    HPG_K_FACTOR = 2,     /* S-hat cell-block assembly + batched Cholesky + inverse        */
    HPG_K_PRECOND = 3,    /* S-hat^{-1} apply                                              */
    HPG_K_BAPPLY = 4,     /* B apply                                                       */
    HPG_K_FDM = 5,        /* A_alpha^{-1} apply (fast diagonalisation, all passes)         */
    HPG_K_SCHUR = 6,      /* -(D + E) z - B^T t  (rest of the S apply)                     */
    HPG_K_ORTHO = 7,      /* GMRES orthogonalisation, norms, Givens                        */
    HPG_K_NEWTON_APPLY = 8,/* FP64 matrix-free G apply (mixed-precision refinement)        */
    HPG_K_UPDATE = 9,     /* vector updates                                                */
    HPG_K_COUNT = 10
} hpg_kernel_class;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` (a cudaStream_t,
 * may be NULL) is the stream every launch of this context goes to; NULL makes
 * the context create its own non-blocking stream. */
hpg_status hpg_create(hpg_ctx** out, int device, void* cuda_stream);
/* Free every device buffer and the context.  NULL is accepted. */
hpg_status hpg_destroy(hpg_ctx* ctx);
/* Human-readable name of a status code (static string). */
const char* hpg_status_str(hpg_status s);
/* Last detailed error message of this context (static per context; never NULL). */
const char* hpg_last_error(hpg_ctx* ctx);
/* Fill `p` with the defaults listed in hpg_params. */
void hpg_default_params(hpg_params* p);

/* ---------------------------------------------------------------- problem */

/* Uniform tensor-product mesh of (lo[j], hi[j]) with cells[j] cells in
 * direction j < dim (dim 2 or 3), partial degree p for u, constraint kind.
 * Obstacle kinds need 2 <= p <= 33; gradient needs 1 <= p <= 32, and one cell's
 * latent coefficients and Gauss values must fit the per-cell kernels' shared memory
 * (200 KB: 2 n^d + n^2 doubles, and 6 nb + 2 n^2 for the cell operators), which caps
 * p near 15 for 3D obstacles and 10 for 3D gradient constraints.  The psi
 * pairing is the paper's (Section 4.1: degree p-2; Section 4.2: degree p-1).
 * Returns a problem id in *pid (valid until hpg_problem_free/hpg_destroy). */
hpg_status hpg_problem_create(hpg_ctx* ctx, int dim, const double* lo, const double* hi,
                              const int* cells, int p, hpg_kind kind, int* pid);
hpg_status hpg_problem_free(hpg_ctx* ctx, int pid);

/* Sizes of the problem's vectors (any pointer may be NULL). n_quad = Gauss
 * points of the latent-variable rule (q = n per direction per cell). */
hpg_status hpg_problem_sizes(hpg_ctx* ctx, int pid, size_t* n_u_full, size_t* n_u_interior,
                             size_t* n_psi, size_t* n_quad);

/* Right-hand side f: callback evaluated at setup on (p+2)^d Gauss points per
 * cell, or a constant.  Default f = 0. */
hpg_status hpg_set_rhs(hpg_ctx* ctx, int pid, hpg_field_fn f, void* user);
hpg_status hpg_set_rhs_const(hpg_ctx* ctx, int pid, double f);

/* Constraint phi (eq. ad:obstacle / ad:gradient), evaluated at the latent
 * Gauss points.  Required before solving.  hpg_quad_points returns those
 * points (n_quad x dim, cell-major, point index x fastest inside a cell);
 * hpg_set_constraint_values takes phi at them directly (length n_quad). */
hpg_status hpg_set_constraint(hpg_ctx* ctx, int pid, hpg_field_fn phi, void* user);
hpg_status hpg_quad_points(hpg_ctx* ctx, int pid, double* pts, size_t len);
hpg_status hpg_set_constraint_values(hpg_ctx* ctx, int pid, const double* phi_q, size_t len);

/* Dirichlet datum g (NULL: u = 0 on the boundary).  Realised by the lifting
 * rule: vertex hats take g at the vertex, each boundary edge's bubbles the
 * H^1_0-seminorm projection of g minus its linear interpolant, faces by the
 * tensor product of that 1D rule. */
hpg_status hpg_set_dirichlet(hpg_ctx* ctx, int pid, hpg_field_fn g, void* user);

/* alpha_k schedule: alpha_k = min(a1 * 2^{(k-1)/2}, cap) until it repeats
 * (Sections 6.1-6.5), or an explicit list (count <= HPG_MAX_ALPHA). */
hpg_status hpg_set_alpha_schedule(hpg_ctx* ctx, int pid, double a1, double cap);
hpg_status hpg_set_alpha_list(hpg_ctx* ctx, int pid, const double* alphas, int count);
/* alpha_k = min(a1 growth^{k-1}, cap) for k = 1 .. max_steps (growth >= 1, max_steps <=
 * HPG_MAX_ALPHA); the schedule ends at the first step that reaches cap (cap_twice = 0:
 * "terminate once alpha_k = cap", as for the QVI of Section 6.4: a1 = 2^-6, growth 4, cap 1
 * gives 2^-6, 2^-4, 2^-2, 1) or after cap has been repeated once (cap_twice = 1, the rule of
 * hpg_set_alpha_schedule with growth sqrt(2)). */
hpg_status hpg_set_alpha_growth(hpg_ctx* ctx, int pid, double a1, double growth, double cap, int max_steps,
                                int cap_twice);

hpg_status hpg_set_params(hpg_ctx* ctx, int pid, const hpg_params* params);

/* ------------------------------------------------------------------ solve */

/* Run the full proximal loop (psi_0 = 0, u_0 = lifting; each subproblem warm
 * started from the previous one).  Blocking.  Returns HPG_OK or the first
 * failure (also in hpg_stats.status). */
hpg_status hpg_solve(hpg_ctx* ctx, int pid);

/* Solve several independent problems with their work overlapping on the
 * device: up to hpg_set_concurrency() host workers, each on its own CUDA
 * stream forked from (and joined back to) the context's stream, take the
 * problems in order.  Each problem's arithmetic is exactly that of hpg_solve,
 * so a result does not depend on what else is in the batch.  Ids must be
 * distinct.  Blocking.  Returns HPG_OK if every problem converged, else the
 * first failure in id order; per-problem status in hpg_stats. */
hpg_status hpg_solve_batch(hpg_ctx* ctx, const int* pids, int count);
/* Number of concurrent workers/streams of hpg_solve_batch (1..64, default 8).
 * With more than 8 streams, set the environment variable
 * CUDA_DEVICE_MAX_CONNECTIONS (e.g. to 32) before the process creates its CUDA
 * context: with the driver's default of 8 hardware work queues, streams share
 * queues and their kernels wait on each other. */
hpg_status hpg_set_concurrency(hpg_ctx* ctx, int streams);

/* Results of the last solve (u in the caller's sign convention). */
hpg_status hpg_get_u(hpg_ctx* ctx, int pid, double* u_full, size_t len);
hpg_status hpg_get_psi(hpg_ctx* ctx, int pid, double* psi, size_t len);
hpg_status hpg_get_stats(hpg_ctx* ctx, int pid, hpg_stats* stats);
/* u_h at npts points (npts x dim).  Also the feasible reconstruction
 * phi - exp(-psi_h) for obstacles (eq. pG) when `feasible` != NULL; it is
 * defined only at the latent Gauss points (length n_quad). */
hpg_status hpg_eval_u(hpg_ctx* ctx, int pid, const double* pts, int npts, double* out);
hpg_status hpg_feasible_u(hpg_ctx* ctx, int pid, double* out_q, size_t len);
/* Accuracy of the last solve against a reference u (full coefficients, caller's sign,
 * length n_u_full): *err = ||u_h - u_ref||_{L2(Omega)} and, when ref_norm is not NULL,
 * *ref_norm = ||u_ref||_{L2(Omega)}, both exact through the 1D mass matrices of
 * Section 3 (M = M_1 (x) ... (x) M_d over the full tensor-product basis).  Host
 * arithmetic; the reference stays the caller's. */
hpg_status hpg_l2_error(hpg_ctx* ctx, int pid, const double* u_ref, size_t len, double* err, double* ref_norm);
/* Accumulated per-kernel-class device time (ms) and launch counts since the
 * last reset, recorded only when params.timing = 1. */
hpg_status hpg_get_kernel_times(hpg_ctx* ctx, int pid, double* ms, long long* launches, int count);
hpg_status hpg_reset_kernel_times(hpg_ctx* ctx, int pid);
/* Enqueue `reps` back-to-back applications of one kernel class (hpg_kernel_class:
 * HPG_K_EVAL, _FACTOR, _PRECOND, _BAPPLY, _FDM, _SCHUR, _NEWTON_APPLY or _ORTHO) on
 * the state left by the last solve, in arithmetic `precision`, on the context's
 * stream, without synchronising: bracket it with CUDA events on that stream
 * to time the kernels in their solver launch configuration.  The launches are
 * captured into a CUDA graph on the first call for a given (class, precision,
 * reps) and replayed on later calls, so time the second call.  Needs a prior
 * hpg_solve or hpg_set_state (+ hpg_factor_precond for _PRECOND/_SCHUR);
 * the kernels write only scratch buffers.  _ORTHO is one Arnoldi step (FP64
 * basis for HPG_FP64, float basis for HPG_MIXED) with both Gram-Schmidt passes
 * (two dot passes, two update passes, Givens) at j = krylov_max / 2 on the
 * Krylov basis buffer, whose contents it overwrites; the HPG_MIXED _PRECOND and
 * _SCHUR launches also read and write that buffer, as in the solver. */
hpg_status hpg_launch_kernel(hpg_ctx* ctx, int pid, int kernel_class, int precision, int reps);
/* Measured SIMT FMA throughput of the context's device (TFLOP/s, 2 flops per FMA):
 * FP32 for HPG_MIXED, FP64 for HPG_FP64; eight independent FMA chains per thread,
 * 8 blocks of 256 threads per SM, best of three timed launches on the context's
 * stream (synchronises it).  *sm_count (may be NULL) receives the SM count.  The
 * roofline denominators of the FP32/FP64-bound kernels; not part of the method. */
hpg_status hpg_measure_fma_peak(hpg_ctx* ctx, int precision, double* tflops, int* sm_count);
/* The same for a batch: `reps` back-to-back launches of one kernel class, each serving
 * every problem of pids[0..count-1] in the lockstep configuration hpg_solve_batch uses
 * for them (one launch per step for the whole group).  The problems must have been
 * solved and share shape and parameters (HPG_ERR_STATE otherwise).  Classes HPG_K_FDM,
 * _PRECOND, _BAPPLY, _SCHUR, _FACTOR, _NEWTON_APPLY, _EVAL; captured once per (class,
 * precision, reps) and replayed; writes only scratch buffers. */
hpg_status hpg_launch_kernel_batch(hpg_ctx* ctx, const int* pids, int count, int kernel_class, int precision,
                                   int reps);
/* Number of fast-diagonalisation pass variants for `precision` (HPG_MIXED: FP32
 * passes, HPG_FP64: FP64 passes); valid values of hpg_params.fdm_tile_f32/_f64
 * are 0 .. count-1.  Returns 0 for an unknown precision. */
int hpg_fdm_tile_count(int precision);

/* ------------------------------------------------------------ request loop
 * Continuous batching of independent solves.  The client creates and fills
 * problems as usual and submits them; `workers` host threads, each with its
 * own CUDA stream, take queued requests in arrival order as soon as they are
 * free and the request's device footprint fits in `device_budget_bytes`
 * (0: 80% of the device memory free at start), first fit.  Running requests
 * overlap on the GPU; each one's arithmetic is exactly that of hpg_solve.
 * A request's device bytes count against the budget from admission until its
 * solve ends; the result (u_h, psi_h, stats) is then kept in host memory and
 * the problem's device buffers are released (a later hpg_solve or
 * component call re-creates them).  While queued or running, every call on
 * that problem except hpg_poll/hpg_wait returns HPG_ERR_BUSY. */
hpg_status hpg_server_start(hpg_ctx* ctx, int workers, size_t device_budget_bytes);
/* Finish running and queued requests that fit, join the workers. */
hpg_status hpg_server_stop(hpg_ctx* ctx);
/* Queue problem `pid`; returns a ticket.  HPG_ERR_OOM if it can never fit. */
hpg_status hpg_submit(hpg_ctx* ctx, int pid, long long* ticket);
/* Non-blocking: *done = 1 once finished, *result its hpg_status. */
hpg_status hpg_poll(hpg_ctx* ctx, long long ticket, int* done, hpg_status* result);
/* Bounded wait: HPG_ERR_TIMEOUT if not finished within timeout_ms. */
hpg_status hpg_wait(hpg_ctx* ctx, long long ticket, double timeout_ms, hpg_status* result);
/* times3 = {queued ms, running ms, submit-to-done ms} (0 while unfinished). */
hpg_status hpg_ticket_times(hpg_ctx* ctx, long long ticket, double* times3);
/* Admission order among queued requests that fit the budget: 0 (default) arrival order;
 * 1 largest work first (unknowns x degree), so that long solves start early and short
 * ones fill the gaps.  HPG_ERR_STATE without a running loop. */
hpg_status hpg_server_policy(hpg_ctx* ctx, int policy);
/* Message of a finished request that failed: which step failed and why (the text
 * hpg_last_error gives after a failing hpg_solve), truncated to len-1 bytes and
 * NUL-terminated; an empty string while unfinished or after success. */
hpg_status hpg_ticket_error(hpg_ctx* ctx, long long ticket, char* buf, size_t len);
/* Bytes currently charged to the budget (running requests), and the
 * footprint estimate for problem pid (pid ignored when estimate is NULL). */
hpg_status hpg_server_memory(hpg_ctx* ctx, int pid, size_t* in_use, size_t* estimate);

/* ------------------------------------------- component operators (testing)
 * These act on an explicit state (u, psi, psi_prev, alpha) uploaded by
 * hpg_set_state, on host vectors in the orderings above.  precision is an
 * hpg_precision: which arithmetic the operator runs in (results are FP64). */

/* Upload (u full, psi, psi_prev, alpha) and evaluate the latent nonlinearity
 * at the Gauss points.  u is in the solver's internal sign (for
 * HPG_OBSTACLE_LOWER the negated field). */
hpg_status hpg_set_state(hpg_ctx* ctx, int pid, const double* u_full, const double* psi,
                         const double* psi_prev, double alpha);
/* Newton residual [F_u (interior); F_psi] of eq. (pG) / (pG:gradient) and its l2 norm. */
hpg_status hpg_residual(hpg_ctx* ctx, int pid, double* F, size_t len, double* norm);
/* y = G x with G of eq. (pG-matrix) (including -E_beta), matrix-free, FP64. */
hpg_status hpg_apply_newton(hpg_ctx* ctx, int pid, const double* x, double* y, size_t len);
/* y = A_alpha^{-1} x on interior u vectors (exact fast diagonalisation). */
hpg_status hpg_apply_stiffness_inv(hpg_ctx* ctx, int pid, int precision, const double* x,
                                   double* y, size_t len);
/* Assemble and factorise the S-hat cell blocks for the current state; the
 * blocks of -S-hat before factorisation are copied to `blocks` when not NULL
 * (Nc x nb x nb, nb = n^d (obstacle) or d n^d (gradient)). */
hpg_status hpg_factor_precond(hpg_ctx* ctx, int pid, int precision, double* blocks, size_t len);
/* y = S-hat^{-1} x (needs hpg_factor_precond). */
hpg_status hpg_apply_precond_inv(hpg_ctx* ctx, int pid, int precision, const double* x,
                                 double* y, size_t len);
/* y = S x, S = -(D_psi + E_beta + B^T A_alpha^{-1} B) of eq. (schur4). */
hpg_status hpg_apply_schur(hpg_ctx* ctx, int pid, int precision, const double* x, double* y,
                           size_t len);
/* y_dev = A_alpha^{-1} x_dev, the same FP64 fast-diagonalisation apply as
 * hpg_apply_stiffness_inv, for callers that cannot allocate device memory at
 * call time: real-time loops that forbid allocation after start-up (cudaMalloc
 * may synchronise the device and takes unbounded time), and applications that
 * hand all device memory to their own pool or budget up front, so that an
 * extra cudaMalloc would fail or fragment it.  The paper has no counterpart;
 * this is a library service.
 * x_dev, y_dev: device pointers of length n_u_interior (len >= that); they may
 * alias.  Its intermediate tensors live in one fixed device array of the
 * library (4 MiB, held by every GPU that loads libhpg until exit), so it
 * accepts at most 262144 interior unknowns (HPG_ERR_ARG beyond, with a message
 * in hpg_last_error) and calls no allocator.  The problem's operators must
 * already be on the device (after hpg_solve or hpg_set_state), else
 * HPG_ERR_STATE.  The first call on a device looks up the array's device
 * address once; make that first call before any stream capture.  Work is
 * enqueued on the context's stream; y_dev is ready when that stream is.
 * Every call shares the array, so calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller. */
hpg_status hpg_apply_stiffness_inv_noalloc(hpg_ctx* ctx, int pid, double alpha, const double* x_dev, double* y_dev,
                                           size_t len);
/* x = A_alpha^{-1} b by preconditioned CG (host vectors of n_u interior entries), to
 * ||b - A_alpha x|| <= max(atol, rtol ||b||) or maxit iterations; *its = iterations.
 * Both preconditioners are additive Schwarz methods of the p-version whose coarse space
 * is the vertex (all-hat) functions -- the Q1 stiffness of the mesh, solved exactly by
 * fast diagonalisation (Section 6.5 uses algebraic multigrid instead):
 *   precond 1: block Jacobi over the entities of the hierarchical basis, the bubble
 *              functions of every edge, face and cell interior forming dense blocks;
 *   precond 2: overlapping, one block per cell holding all its interior dofs (the
 *              principal submatrix of A), the cells' corrections summed per dof;
 *   precond 3: overlapping, one patch per interior vertex -- the interior of its star
 *              of cells, a tensor-product box -- solved exactly by fast diagonalisation
 *              of the 1D restrictions of the pencil; the patches' corrections summed
 *              per dof (the p-robust vertex-based method).  Its boxes (2p-1)^d must fit
 *              in shared memory (HPG_ERR_ARG beyond).
 * Needs the problem's operators on the device (after hpg_solve or hpg_set_state). */
hpg_status hpg_stiffness_solve_pcg(hpg_ctx* ctx, int pid, int precond, double alpha, const double* b, double* x,
                                   size_t len, double rtol, double atol, int maxit, int* its);
/* ---------------------------------------------------------------- thermoforming QVI */
/* The quasi-variational inequality of Section 6.4 (thermoforming): the membrane u of
 * an upper-obstacle problem (this problem: HPG_OBSTACLE_UPPER, its rhs, Dirichlet data
 * and alpha schedule as set) under the obstacle Phi_0 + xi T, where the mould
 * temperature T in U_{h,p} (all dofs, no boundary condition) solves
 *     (grad T, grad q) + gamma (T, q) = (g(Phi_0 + xi T - u), q)   for all q,
 *     g(s) = g0 for s <= 0, g0 (1 - s) for 0 < s < 1, 0 for s >= 1.
 * Fixed point from T_0 = 0: (I) the obstacle problem with phi = Phi_0 + xi T_i at the
 * latent Gauss points (a full hpG solve, psi_0 = 0); (II) T_{i+1} by Newton on the T
 * equation from T_i, each Newton system by GMRES right-preconditioned with
 * (A + gamma M)^{-1} (fast diagonalisation of the full-space 1D pencils), until
 * ||R(T)||_2 <= t_tol; stop once ||u_{i+1} - u_i||_{H^1} <= tol (i >= 1).  The nonsmooth
 * integral (g(.), q) uses nq Gauss points per direction per cell. */
typedef struct {
    double gamma;         /* > 0; default 1                                            */
    double g0;            /* >= 0; default 0.2                                         */
    double tol;           /* H^1 stopping tolerance of the fixed point; default 3e-3   */
    double t_tol;         /* absolute ||R(T)||_2 of the T Newton; default 1e-11        */
    int    max_fp;        /* fixed-point cap (<= HPG_QVI_MAX_FP); default 30           */
    int    nq;            /* Gauss points per direction per cell of the T equation;
                             p + 2 by default (0)                                       */
    int    t_newton_max;  /* Newton cap of one T solve; default 50                     */
    int    t_krylov_max;  /* GMRES cap of one T Newton system; default 200             */
    double t_krylov_rtol; /* GMRES relative tolerance; default 1.5e-8 (Section 6.4)    */
} hpg_qvi_params;

#define HPG_QVI_MAX_FP 64

typedef struct {
    int    status;                      /* hpg_status of the QVI solve                  */
    int    iterations;                  /* fixed-point iterations taken                 */
    int    converged;                   /* 1 when the H^1 test was met                  */
    int    newton_total;                /* Newton steps of the obstacle solves          */
    int    t_newton_total;              /* Newton steps of the T solves                 */
    long long t_krylov_total;           /* GMRES iterations of the T Newton systems     */
    double du_h1[HPG_QVI_MAX_FP];       /* ||u_i - u_{i-1}||_{H^1} per iteration (entry 0: 0) */
    int    newton_per_fp[HPG_QVI_MAX_FP];   /* obstacle Newton steps per iteration       */
    int    t_newton_per_fp[HPG_QVI_MAX_FP]; /* T Newton steps per iteration              */
    double t_residual;                  /* ||R(T)||_2 at the end                        */
    double solve_ms;                    /* wall time (host clock)                       */
    long long kernel_launches;          /* libhpg kernels launched by the QVI solve     */
    long long krylov_total;             /* GMRES iterations of the obstacle Newton systems */
} hpg_qvi_stats;

/* Defaults of hpg_qvi_params. */
hpg_status hpg_qvi_default_params(hpg_qvi_params* out);
/* The T-equation Gauss points of problem pid (nq per direction per cell; 0: p + 2):
 * Nc nq^d points, cell-major (cells as psi), x index fastest inside a cell; pts holds
 * len >= Nc nq^d dim doubles. */
hpg_status hpg_qvi_points(hpg_ctx* ctx, int pid, int nq, double* pts, size_t len);
/* Solve the QVI.  phi0_lat, xi_lat: Phi_0 and xi at the latent Gauss points
 * (hpg_quad_points order, n_lat = Nq values each); phi0_q, xi_q: at the T-equation
 * points of hpg_qvi_points for params->nq (n_q values each).  Afterwards hpg_get_u and
 * hpg_get_psi give the last obstacle solve, hpg_qvi_get_T the temperature, and the
 * problem's constraint is the last obstacle Phi_0 + xi T_i.  Errors: HPG_ERR_ARG for a
 * kind other than HPG_OBSTACLE_UPPER, wrong lengths or parameters, or cells too large
 * for shared memory ((max(p+1, nq))^d doubles twice); the obstacle solve's status when
 * it fails (hpg_last_error names the iteration); HPG_ERR_NEWTON_CAP when a T Newton
 * or the fixed point runs out. */
hpg_status hpg_qvi_solve(hpg_ctx* ctx, int pid, const hpg_qvi_params* params, const double* phi0_lat,
                         const double* xi_lat, size_t n_lat, const double* phi0_q, const double* xi_q, size_t n_q,
                         hpg_qvi_stats* stats);
/* The temperature T of the last hpg_qvi_solve (full U_{h,p} coefficients, len >= the
 * full u length). */
hpg_status hpg_qvi_get_T(hpg_ctx* ctx, int pid, double* T_full, size_t len);
/* Solve G delta = F(state) by eq. (schur2) + GMRES (relative tolerance rtol);
 * returns delta and the GMRES iteration count. */
hpg_status hpg_newton_direction(hpg_ctx* ctx, int pid, int precision, double rtol, double* delta,
                                size_t len, int* krylov_its);

#ifdef __cplusplus
}
#endif
#endif /* HPG_H */
