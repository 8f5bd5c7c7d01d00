/*
 * ph.h -- C ABI of libph: one Newton predictor-corrector step of polynomial
 * homotopy continuation in complex double-double (DD) and quad-double (QD)
 * arithmetic on one GPU (sm_103a), after Verschelde & Yu, "Accelerating
 * Polynomial Homotopy Continuation on a Graphics Processing Unit with Double
 * Double and Quad Double Arithmetic" (2015).
 *
 * Conventions (all entry points):
 *  - Every call returns a ph_status; nothing throws or aborts across the ABI.
 *    On an error the context keeps a message for ph_last_error().
 *  - Multi-limb numbers: a real in L limbs (L = 2 for DD, 4 for QD) is L
 *    doubles, leading limb first, whose exact sum is the value.  A vector of m
 *    complex numbers is m*2*L doubles laid out [limb][re|im][index]; an N x n
 *    complex matrix is column-major [limb][re|im][column][row].
 *  - Array arguments may be host or device pointers; the library asks the CUDA
 *    runtime which, copies host data in and out itself, and works on device
 *    data in place.  Inputs are only read; the caller keeps ownership of every
 *    buffer it passes.  Outputs go to caller-provided buffers.
 *  - Work runs on the stream given to ph_init (NULL = the legacy default
 *    stream); calls return once their results are in the caller's buffers.
 *  - A context is not thread-safe: one host thread per context at a time.
 *  - Waits inside the library's own kernels are bounded; a wait that runs out
 *    makes the call return PH_TIMEOUT with the context still usable.
 */
#ifndef PH_H
#define PH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { PH_D = 1, PH_DD = 2, PH_QD = 4 } ph_prec;     /* value = limbs per real */

typedef enum {
  PH_OK = 0,
  PH_EINVAL = 1,     /* invalid argument (sizes, indices, layout, parameters)   */
  PH_ENOMEM = 2,     /* device or host allocation failed                         */
  PH_ECUDA = 3,      /* a CUDA runtime call failed (message in ph_last_error)    */
  PH_DIVERGED = 4,   /* ||x||_inf exceeded ph_track_params.max_x                 */
  PH_MAXSTEPS = 5,   /* more than max_steps predictor-corrector steps            */
  PH_STEPMIN = 6,    /* the step size fell below min_dt                          */
  PH_NONFINITE = 7,  /* a non-finite start point, or a zero column in the QR     */
  PH_TIMEOUT = 8     /* a bounded device-side wait ran out                        */
} ph_status;

typedef struct ph_ctx ph_ctx;
typedef struct ph_system ph_system;

/* Creates a context on CUDA device `device`, working on `cuda_stream`
 * (a cudaStream_t, may be NULL).  *ctx receives the handle. */
ph_status ph_init(ph_ctx **ctx, int device, void *cuda_stream);

/* Destroys a context (systems loaded into it must be freed first). */
ph_status ph_destroy(ph_ctx *ctx);

/* The message of the last failed call on this context ("" if none). */
const char *ph_last_error(ph_ctx *ctx);

/* Loads a polynomial system of N polynomials in n variables, N >= n (Section
 * 2, input specification), given fully expanded (Section 3.1: every polynomial
 * as the list of its monomials and their coefficients):
 *   polynomial i owns terms term_ptr[i] .. term_ptr[i+1]-1   (term_ptr: N+1);
 *   term k owns the pairs var_ptr[k] .. var_ptr[k+1]-1        (var_ptr: M+1);
 *   pair p is variable var_idx[p] in [0, n) with exponent var_exp[p] >= 1;
 *   the variables of one term are distinct; a term with no pair is a constant;
 *   coeff holds the M complex coefficients, [L][2][M] doubles.
 * The arrays are copied to the device once (Section 3.1: the structures and
 * coefficients cross to the device only at the start); the system keeps the
 * instruction layout the evaluation kernels read.  PH_EINVAL for any
 * malformed index, pointer array or exponent. */
ph_status ph_system_load(ph_ctx *ctx, ph_prec prec, int N, int n,
                         const int32_t *term_ptr, const int32_t *var_ptr,
                         const int32_t *var_idx, const int32_t *var_exp,
                         const double *coeff, ph_system **out);

/* Frees a system and its device memory. */
ph_status ph_system_free(ph_system *sys);

/* Values h [L][2][N] and Jacobian J [L][2][n][N] (column-major) of the
 * homotopy h(x,t) = gamma (1-t)^k g(x) + t^k f(x) (Section 2, Eq. (1)) at the
 * point x [L][2][n]:
 *   g      start system, or NULL for the total-degree system
 *          g_i = x_i^{d_i} - 1 with d_i the degree of f_i (needs N == n);
 *   gamma  [L][2] complex constant; NULL evaluates f alone (h = f, J = Jf);
 *   k      relaxation exponent >= 1 (the paper uses k >= 2; k = 1 is the
 *          plain linear homotopy);
 *   t      the real parameter, L limbs (only read when gamma != NULL).
 * Monomials are differentiated in the reverse mode (Speelpenning products
 * with a common factor for exponents > 1, Section 3.2) and summed into h and J
 * (Section 3.3). */
ph_status ph_eval_jac(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                      const double *gamma, int k, const double *t, const double *x,
                      double *h, double *J);

/* Least-squares solution dx [L][2][n] of J dx = rhs for an N x n matrix J
 * [L][2][n][N] (N >= n) and rhs [L][2][N], by modified Gram-Schmidt on the
 * augmented matrix [J | rhs] and back substitution (Introduction: MGS instead
 * of LU with pivoting; Section 3.1, GPU_Modified_Gram_Schmidt).  resid_norm,
 * if not NULL, receives ||J dx - rhs||_2 in double (a host pointer).
 * PH_NONFINITE if a column becomes zero (rank deficiency). */
ph_status ph_mgs_solve(ph_ctx *ctx, ph_prec prec, int N, int n, const double *J,
                       const double *rhs, double *dx, double *resid_norm);

/* Path-tracking parameters (Section 2 and Fig. 3; the paper leaves the values open). */
typedef struct {
  double max_dt;      /* largest step size h_max, also the first step size      */
  double min_dt;      /* smallest step size h_min: halving below it ends the
                         path with PH_STEPMIN                                     */
  double tol_res;     /* Newton succeeds when ||h(x,t)||_inf < tol_res           */
  double tol_dx;      /* ... or when ||dx||_inf < tol_dx (after the update)       */
  double max_res;     /* residual bound for the first Newton iteration           */
  double max_x;       /* ||x||_inf above this after an accepted step: PH_DIVERGED */
  int32_t max_steps;  /* more than this many steps: PH_MAXSTEPS                  */
  int32_t max_newton; /* Newton iterations per step (P.max_iteration)            */
  int32_t pred_order; /* largest degree of the extrapolation predictor (0..8)    */
  int32_t relax_k;    /* k in gamma (1-t)^k g + t^k f, >= 1                      */
  int32_t fixed_steps;/* > 0: fixed schedule t_j = j / fixed_steps with exactly
                         max_newton updates per step, no test, no rejection      */
  int32_t control;    /* 0: the whole path is one graph launch, steps decided on
                         the device; 1: the host launches one step at a time and
                         reads the controller state back after each (the paper's
                         host-side step control, Section 3.1)                    */
  /* The precision form (no counterpart in the paper, whose corrector runs in
   * DD/QD throughout).  lin_prec selects the precision of the Newton system:
   *   0  working precision (DD/QD), the paper's corrector;
   *   1  IEEE double: the residual h(x,t) is evaluated and the update x += dx
   *      accumulated in working precision, while the Jacobian is evaluated at
   *      the rounded x and factored (MGS) in double; the residual is scaled by
   *      a power of two before it is rounded.  Each iteration contracts the
   *      error by about kappa(J) u_double instead of squaring it;
   *   2  the same in IEEE single;
   *   3  automatic: single where it costs no convergence, else double.  A
   *      solve is single when the previous factorization's condition
   *      estimate kappa (max r_kk / min r_kk) is at most cond_f32 and, after
   *      the step's first iteration, the current error, estimated as the
   *      square of the last update norm, is at least kappa 2^-24 (the single
   *      solve's relative error), so Newton's quadratic convergence holds.
   * In 2 and 3 a single-precision factorization that is not finite is redone
   * in double.  On adaptive steps a low-precision corrector gets one
   * iteration beyond max_newton when its previous update was below
   * sqrt(tol_dx) (the working-precision corrector would have squared that
   * update below tol_dx and succeeded).  A step whose low-precision corrector
   * fails is
   * corrected once more from its predicted point one precision up before it
   * counts as a failure (step size halved): in double if it solved in single
   * under lin_prec 2; in working precision if a double solve had
   * kappa u_double above 1e-6 or the corrector failed although an update
   * below sqrt(tol_dx) was followed by another.
   * A corrector that fails while its updates are still large follows the
   * working-precision iterates to kappa u_low, and so does their failure.
   * A failed corrector whose last three updates contracted, but more slowly
   * than quadratically (ratios r1, r0 below 1 with r0 > r1^1.5: its solves
   * limit it, whatever kappa shows), is corrected again in working precision,
   * and the rest of the path runs in working precision (stats wp_rest).
   * Steps to t >= endgame_t run in working precision throughout (the end
   * game).
   * ph_track_paths and the serving loop take 0..3; ph_track_path takes 0 and
   * 1 (its step graph holds both kernel sets, one of them gated off per
   * iteration). */
  int32_t lin_prec;
  /* 1 (with an explicit start system g): every row i where g_i is the zero
   * polynomial (no terms) is held fixed, h_i = f_i instead of t^k f_i.  This
   * is the monodromy homotopy of Section 4.2, {f = 0, alpha (1-t) L + t K = 0}:
   * target [f; K], start [0; L], gamma = alpha; f is evaluated once.  0: every
   * row moves.  PH_EINVAL with the total-degree start system. */
  int32_t fixed_rows;
  double endgame_t;   /* <= 0: 1.0 (only the step that lands on t = 1)           */
  double cond_f32;    /* threshold of lin_prec 3; <= 0: 1e3                       */
  /* > 0: the corrector's tolerance, for both of its tests, on the steps to
   * t < 1; the step that lands on t = 1 keeps tol_res and tol_dx, so the end
   * point has their accuracy.  0: tol_res and tol_dx on every step.  (The
   * paper's corrector tests, Section 2, Eq. (3), and Fig. 2, name tolerances
   * without values; how tight they must be on the way is left open.) */
  double tol_path;
} ph_track_params;

/* Outcome of one tracked path. */
typedef struct {
  int32_t status;       /* ph_status of the path                                 */
  int32_t steps;        /* predictor-corrector steps taken                       */
  int32_t accepted;     /* steps whose corrector succeeded                        */
  int32_t rejected;     /* steps whose corrector failed (step size halved)       */
  int32_t newton_iters; /* evaluations of h and J (corrector iterations)         */
  int32_t updates;      /* applied Newton updates x += dx                         */
  double t_final;       /* t of the last accepted point                           */
  double res;           /* last residual norm seen by the corrector              */
  double dx;            /* last update norm seen by the corrector                */
  int64_t launches;     /* kernels the library launched for this path            */
  int32_t solves_f64;   /* Newton systems solved in double (lin_prec != 0)        */
  int32_t solves_f32;   /* ... and in single                                       */
  int32_t escalated;    /* steps whose low-precision corrector failed and that
                           were corrected again one precision up                 */
  int32_t wp_rest;      /* 1 if the precision form left the rest of the path to
                           working precision (a failed low-precision corrector
                           whose updates contracted only linearly)              */
  double cond;          /* condition estimate of the last low-precision solve    */
} ph_path_stats;

/* One step of the schedule actually taken, for replay. */
typedef struct {
  double t;             /* the t the step tried                                   */
  double res;           /* last residual norm of its corrector                    */
  double dx;            /* last update norm of its corrector                      */
  int32_t accepted;     /* 1 if the corrector succeeded                           */
  int32_t updates;      /* Newton updates applied during the step                */
} ph_step_record;

/* Tracks one solution path of h(x,t) = gamma (1-t)^k g(x) + t^k f(x) from the
 * start solution x0 of g at t = 0 to t = 1 (Section 2, input-output
 * specification; Fig. 2 and Fig. 3):
 *   t := min(1, t + dt); predict x by extrapolation through the last accepted
 *   points (degree min(pred_order, #accepted - 1), Section 3.1); run Newton's
 *   method (fail if the residual grows, succeed if ||h|| < tol_res or
 *   ||dx|| < tol_dx); on success keep the point and, after more than two
 *   successes in a row, double dt up to max_dt; on failure go back to the last
 *   accepted point and halve dt.
 * With params->control = 0 the whole loop runs on the device (one CUDA graph
 * launch per path) and the host reads the result once at the end; with 1 the
 * host launches one step (one graph) at a time, as in the paper.
 * params->lin_prec is 0 or 1 here (PH_EINVAL otherwise): with 1 each step's
 * Newton systems below endgame_t are evaluated and solved in IEEE double
 * (see ph_track_params), the rest as with 0.
 *   f, g, gamma  as in ph_eval_jac (gamma is required here);
 *   x0           start solution [L][2][n];
 *   x_out        end point [L][2][n] (the last accepted point);
 *   stats        may be NULL;
 *   log, log_cap optional schedule log (host memory, NULL/0 for none); the
 *                first min(steps, log_cap) steps are recorded.
 * Returns the path status (PH_OK when t = 1 was reached). */
ph_status ph_track_path(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                        const double *gamma, const double *x0,
                        const ph_track_params *params, double *x_out,
                        ph_path_stats *stats, ph_step_record *log, int log_cap);

/* Tracks npaths solution paths of the same homotopy, each from its own start
 * point, to t = 1: the many-path form.  The paper accelerates one path at a
 * time (Section 3; many paths are its companion work); this entry point keeps
 * the GPU busy with many.  One persistent kernel: each thread block takes the
 * next unstarted path, tracks it to its end with the same predictor, corrector,
 * MGS and step control as ph_track_path (params->control is ignored), stores
 * the end point and takes the next path, so paths of uneven length balance.
 *   x0     [npaths][L][2][n] start points; x_out [npaths][L][2][n] end points;
 *   stats  [npaths] (may be NULL); log [npaths][log_cap] (may be NULL/0): the
 *          first log_cap steps of each path.
 * Returns PH_OK when the launch completed; each path's status is in stats. */
ph_status ph_track_paths(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                         const double *gamma, int npaths, const double *x0,
                         const ph_track_params *params, double *x_out, ph_path_stats *stats,
                         ph_step_record *log, int log_cap);

/* A continuous-batching request loop for path-tracking jobs of different sizes
 * and precisions (the paper tracks one path at a time; a service receives jobs
 * while others run).  Each job gets its own workspace (point, history, step
 * size, Jacobian) carved from one device pool of pool_bytes: a job is admitted
 * only when its footprint fits in the free pool, otherwise it waits on the host
 * in arrival order; a finished job's region returns to the pool.  Admitted jobs
 * go to a queue in host-mapped memory that one persistent kernel works: each
 * block claims the next job, tracks it whole (same algorithm as
 * ph_track_paths), publishes the result and claims the next, so jobs submitted
 * while others run start as soon as a block is free and overlap them.  A job's
 * result does not depend on what runs beside it.  A host thread reaps results,
 * admits waiting jobs and relaunches the kernel when it has gone idle. */
typedef struct ph_server ph_server;
typedef struct {
  int32_t max_n;        /* largest number of variables of a job run by one block */
  int32_t max_blocks;   /* resident blocks, 0 = two per SM                      */
  int64_t pool_bytes;   /* device pool for the jobs' workspaces                 */
  int32_t queue_cap;    /* jobs on the device at once (table slots)             */
  /* > 0: the large-job route.  A job with more than big_n variables (any
   * number, not bounded by max_n) is not given to one block, whose O(n^3)
   * solve would take one SM minutes: it runs alone on the whole GPU through
   * the single-path tracker (ph_track_path) on a context of the server's own,
   * in arrival order.  When such a job is next, no further small job is
   * admitted, the small jobs on the device finish, the large one runs, then
   * admission resumes.  Its systems must stay loaded until it is done.
   * 0: every job runs on one block (and n <= max_n). */
  int32_t big_n;
} ph_server_config;

ph_status ph_server_create(ph_ctx *ctx, const ph_server_config *cfg, ph_server **out);
/* Submits one job (f, g, gamma, x0 and params as in ph_track_path, host or
 * device arrays, copied); returns at once with its id.  PH_EINVAL if f has more
 * than max_n variables, PH_ENOMEM if its workspace exceeds the whole pool. */
ph_status ph_server_submit(ph_server *srv, const ph_system *f, const ph_system *g,
                           const double *gamma, const double *x0,
                           const ph_track_params *params, int64_t *job_id);
/* *done = 1 and the results (end point [L][2][n], statistics, submit-to-finish
 * latency in ms, each optional) once the job has finished; the job is then
 * forgotten.  *done = 0 while it runs. */
ph_status ph_server_poll(ph_server *srv, int64_t job_id, int *done, double *x_out,
                         ph_path_stats *stats, double *latency_ms);
/* ph_server_poll that waits up to timeout_ms (PH_TIMEOUT if not done by then). */
ph_status ph_server_wait(ph_server *srv, int64_t job_id, int timeout_ms, double *x_out,
                         ph_path_stats *stats, double *latency_ms);
/* Jobs waiting for admission and on the device, kernel launches so far, free
 * pool bytes (each optional). */
ph_status ph_server_info(ph_server *srv, int64_t *waiting, int64_t *on_device,
                         int64_t *kernel_launches, int64_t *pool_free_bytes);
/* Device workspace a job of this homotopy takes from the pool, in bytes. */
ph_status ph_server_job_bytes(ph_server *srv, const ph_system *f, const ph_system *g,
                              int64_t *bytes);
/* Stops the loop (running jobs finish first) and frees the server. */
ph_status ph_server_destroy(ph_server *srv);

/* The least-squares solve has three variants (the paper has one MGS kernel;
 * the choice is this library's, per GPU and shape):
 *   PH_MGS_GRID     one block per column, each pivot handed to the blocks
 *                   that need it through a flag in L2 (size 0);
 *   PH_MGS_CLUSTER  the whole matrix in the shared memory of one thread-block
 *                   cluster, pivots passed by cluster barrier and distributed
 *                   shared memory (size: the cluster's CTAs, 8 or 16; only
 *                   where the matrix fits);
 *   PH_MGS_TILED    the trailing matrix cut into tiles of R row blocks by
 *                   column groups over every SM, one grid barrier per pivot,
 *                   the next pivot's dot products fused into the update
 *                   (size: R; after the paper's tiled MGS, Introduction).
 * ph_mgs_variant reports the variant this context uses for an N x n system
 * of precision prec: the first use of a shape times every variant that
 * applies (the tiled one for each row-block count worth trying) on a scratch
 * matrix and keeps the fastest.  ms (optional, 3 doubles) receives the
 * measured milliseconds of the grid, cluster and best tiled variant, -1 where
 * a variant does not apply or was not measured (a pinned shape). */
typedef enum { PH_MGS_GRID = 0, PH_MGS_CLUSTER = 1, PH_MGS_TILED = 2 } ph_mgs_kind;
ph_status ph_mgs_variant(ph_ctx *ctx, ph_prec prec, int N, int n, int *kind, int *size,
                         double *ms);

/* Pins the variant this context uses for an N x n system of precision prec,
 * in place of the timing: kind PH_MGS_GRID (size ignored), PH_MGS_CLUSTER
 * with the cluster size the shape takes (PH_EINVAL otherwise, or if the shape
 * does not fit a cluster), PH_MGS_TILED with R row blocks (PH_EINVAL if R
 * exceeds the SMs or the rows, or its tiles do not fit shared memory); kind
 * -1 returns the shape to the timed choice.  The variants round differently
 * (their dot products are summed in different orders), so pinning one makes
 * a context's results the same from run to run; tests pin each to check it.
 * A path graph captured with the previous choice is rebuilt on next use. */
ph_status ph_mgs_set_variant(ph_ctx *ctx, ph_prec prec, int N, int n, int kind, int size);

/* The number of lanes (threads) per output of the summation kernel used for f
 * (with g): *lanes = 1, 2, 4, 8, 16 or 32, chosen by timing each on the
 * system's first evaluation (Section 3.3 of the paper times its summation with
 * 1 to 32 threads per sum; here the choice is made per system and GPU).
 * ms (optional, 6 doubles) receives the measured times for 1 .. 32 lanes, -1
 * where not measured. */
ph_status ph_sum_lanes(ph_ctx *ctx, const ph_system *f, const ph_system *g, int *lanes,
                       double *ms);

/* The summation's lanes per output inside the many-path and serving kernels
 * (one thread block per path), the paper's threads per sum (Section 3.3):
 * ph_track_paths times 1, 2, 4, 8, 16 and 32 lanes on its first batch of a
 * system that fills the GPU (as many paths as SMs or more) -- one corrector
 * iteration of a full GPU of blocks per choice -- and keeps the fastest on f;
 * until then, and for the serving loop's jobs of a system never batched, 4.
 * ph_block_lanes reports the lanes in use and (ms, optional, 6 doubles) the
 * measured milliseconds per launch of each choice, -1 where not measured;
 * ph_set_block_lanes pins a choice (0: back to untimed, timed again by the
 * next batch that fills the GPU). */
ph_status ph_block_lanes(ph_ctx *ctx, const ph_system *f, int *lanes, double *ms);
ph_status ph_set_block_lanes(ph_ctx *ctx, const ph_system *f, int lanes);

/* Host-side step-size controller of the path tracker, exported so it can be
 * checked without a GPU: the same code runs inside the device controller.
 * Fig. 3. */
typedef struct {
  double t, dt;
  int32_t nsucc, nsteps, done, status;
} ph_ctrl_state;

void ph_ctrl_init(ph_ctrl_state *c, const ph_track_params *p);
/* The next t to try, or -1 once the controller has stopped. */
double ph_ctrl_next_t(ph_ctrl_state *c, const ph_track_params *p);
/* Reports the corrector's outcome at t_new. */
void ph_ctrl_report(ph_ctrl_state *c, const ph_track_params *p, double t_new, int success);
/* The precision form's test on three successive update norms d2, d1, d0 of a
 * low-precision corrector (see ph_track_params.lin_prec): 1 if they contract
 * (d1/d2 < 1, d0/d1 < 1) more slowly than quadratically (d0/d1 > (d1/d2)^1.5),
 * else 0; 0 for non-positive or non-finite input. */
int ph_ctrl_linear_contraction(double d2, double d1, double d0);

/* Measurement support (Section 5 reports per-kernel times; the roofline of
 * this FP64-bound path needs the FP64 rate of the device it runs on).
 *
 * ph_profile_newton runs `reps` corrector iterations at (x, t) outside any graph
 * and times each of its kernels with CUDA events on the context's stream;
 * ms_out[0..3] receive the average milliseconds per launch of: the power table
 * and homotopy factors, the monomial AD, the summation/assembly, and the MGS
 * solve with back substitution.  Arguments as in ph_eval_jac (gamma required).
 *
 * ph_fp64_peak times a kernel of independent FP64 fused multiply-adds on every
 * SM for about `ms_target` milliseconds and returns the rate in G lane-ops/s
 * (one DFMA of one thread = one op; 2 flops). */
ph_status ph_profile_newton(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                            const double *gamma, int k, const double *t, const double *x,
                            int reps, double *ms_out);
ph_status ph_fp64_peak(ph_ctx *ctx, double ms_target, double *gops);

/* The execution-unit rates the kernels' design rests on, measured on the
 * context's device in G operations per second: rates[0] FP64 fused
 * multiply-adds on the FP64 pipe (as ph_fp64_peak), rates[1] FP64 fused
 * multiply-adds on the tensor cores (mma.sync m8n8k4 .f64: 256 per warp
 * instruction), rates[2] 32-bit integer multiply-adds.  The tensor-core rate
 * below the FP64 pipe's is why no MGS update runs on the tensor cores; the
 * integer rate is what the exact integer reductions of the solvers use. */
ph_status ph_unit_rates(ph_ctx *ctx, double *rates);

/* A least-squares solve like ph_mgs_solve for callers that must not allocate
 * device memory: processes whose device memory belongs to another allocator
 * (a framework's caching allocator or a fixed arena, where one more
 * cudaMalloc fails or takes the owner's memory), and real-time loops that
 * cannot afford an allocation's implicit device synchronisation.  The paper
 * has no counterpart; this is a convenience of this library.
 *   No context is needed and nothing is allocated: the scratch is one static
 *   4 MiB device array that each GPU loading the library keeps until exit.
 *   Sizes whose scratch (augmented matrix, projections, norms, solution) does
 *   not fit return PH_EINVAL (n = N up to 353 in D, 254 in DD, 175 in QD).
 *   device, cuda_stream  the GPU (made current for the call) and the stream
 *                        (a cudaStream_t, may be NULL) the work runs on;
 *   J, rhs, dx, resid_norm  as in ph_mgs_solve (host or device arrays).
 *   It always runs the grid MGS kernel (one block per column), whereas a
 *   context may pick the cluster variant by timing (ph_mgs_variant): the
 *   results agree with ph_mgs_solve to the solver's rounding tolerance, not
 *   bit for bit.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and may load the module.  Every call shares the
 *   array, so calls that overlap on the GPU race: serialise them.  The call
 *   reads its status back and returns after synchronising its stream; a
 *   stream that is being captured is refused (PH_EINVAL, nothing enqueued). */
ph_status ph_mgs_solve_static(int device, void *cuda_stream, ph_prec prec, int N, int n,
                              const double *J, const double *rhs, double *dx,
                              double *resid_norm);

/* Failure handling (the paper has no counterpart).
 *
 * ph_set_wait_limit: the limit, in milliseconds, of every bounded device-side
 * wait in this context's kernels (the pivot hand-offs and grid barriers of the
 * least-squares solves); 2000 by default.  A wait that runs out makes the
 * call (or the path) end with PH_TIMEOUT and leaves the context usable.
 *
 * ph_set_memory_limit: a cap, in bytes, on the device memory that all of this
 * process's libph objects hold together (0, the default: none); *in_use
 * (optional) receives what they hold now.  An allocation beyond the cap fails
 * as on a full device (PH_ENOMEM), so a caller can keep the library within a
 * share of the GPU; it also lets tests reach every allocation-failure path
 * without exhausting a device.
 *
 * ph_debug_withhold_pivot: test support.  From now on, the least-squares
 * solves of this context withhold the hand-off of pivot k (the grid kernel
 * never publishes its flag; the tiled kernel's block 0 never arrives at its
 * barrier), so the other blocks' bounded waits run out and the call returns
 * PH_TIMEOUT; k < 0 restores normal operation.  Nothing faults and nothing
 * waits beyond the wait limit. */
ph_status ph_set_wait_limit(ph_ctx *ctx, double ms);

/* Test support for the solvers' reductions: the exact sum over one warp of 32
 * double-double (limbs 2) or quad-double (limbs 4) values in[32][limbs] (host
 * array), rounded back to limbs doubles in out[limbs] (host array): the
 * fixed-point integer reduction the MGS kernels use for their dot products
 * and norms (each input truncated below 2^-116 (DD) / 2^-244 (QD) of the
 * largest; the total correctly rounded limb by limb). */
ph_status ph_debug_warp_sum(int device, int limbs, const double *in, double *out);

/* Test support for the fixed-point updates of the MGS kernels: for each of
 * count cases, in[case][6][limbs] (host array) holds a, ar, b, ai, c and the
 * sign sg (its leading limb, +1 or -1), and out[case][limbs] (host array)
 * receives a - ar b + sg ai c as the MGS kernels form it in fixed point:
 * limbs 2 (double-double) the exact products of the leading limbs and the
 * cross products summed as 128-bit integers and rounded to two limbs; limbs 4
 * (quad-double) 256-bit fixed-point values, products of their top words,
 * exact sums and the four-limb round-back.  count <= 65536.  PH_EINVAL on a
 * bad argument, PH_ENOMEM / PH_ECUDA on a failed device allocation or copy. */
ph_status ph_debug_update(int device, int limbs, int count, const double *in, double *out);
ph_status ph_set_memory_limit(int64_t bytes, int64_t *in_use);
ph_status ph_debug_withhold_pivot(ph_ctx *ctx, int k);

/* Library version string. */
const char *ph_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PH_H */
