/*
 * glasso.h - C ABI of the GB300 multilevel proximal-Newton solver for sparse
 * inverse covariance estimation (Treister, Turek, Yavneh, arXiv 1607.00315).
 *
 * The problem (Section 5, eq. MLE_l1_prior):
 *     A* = argmin_{A > 0}  -log det A + tr(S A) + lambda * sum_ij |A_ij|,
 * with S the empirical covariance of the samples (eq. cov_estimate) and the
 * diagonal penalised.  A* is unique for lambda > 0.
 *
 * Conventions for every entry point:
 *  - Matrices are dense, row-major, n x n, leading dimension n, FP64 unless
 *    stated.  Symmetric inputs are read in full; outputs are written in full.
 *  - Pair lists are upper-triangle index pairs (i <= j) as two int32 arrays,
 *    in row-major order (i ascending, then j ascending); a pair (i, j)
 *    stands for both A_ij and A_ji.
 *  - The caller owns every buffer it passes.  Inputs are borrowed for the
 *    duration of the call only, except for glasso_submit (see there).
 *  - No call aborts, traps or throws: every failure is a status code.
 *    GLASSO_ECUDA means a CUDA runtime call failed; the message is kept in
 *    the context (glasso_last_error).
 *  - Step-level entry points (glasso_potrf ... glasso_line_search) take
 *    DEVICE pointers, run on the context's stream and return when their
 *    results are complete.  They expose the individual steps of one
 *    relaxation for testing and measurement; glasso_solve runs them all.
 */
#ifndef GLASSO_H
#define GLASSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glasso_ctx glasso_ctx; /* opaque; bound to one device */

typedef enum {
    GLASSO_OK = 0,
    GLASSO_EINVAL = 1,       /* bad argument (n < 1, lambda <= 0, NaN, asymmetric S, ...) */
    GLASSO_ENOMEM = 2,       /* device allocation failed or footprint above the budget */
    GLASSO_ENOTPD = 3,       /* initial iterate not positive definite (S_ii + lambda <= 0) */
    GLASSO_ELINESEARCH = 4,  /* no step length passed the line search */
    GLASSO_EMAXITER = 5,     /* tolerance not reached within max_cycles */
    GLASSO_EAGAIN = 6,       /* glasso_poll: not finished yet */
    GLASSO_ETIMEOUT = 7,     /* a bounded device wait ran out (a grid barrier of the CD sweep, or
                                a tensor-core pipeline wait); the kernel returned early, the
                                context stays usable, A_out is not written */
    GLASSO_ECUDA = 8         /* a CUDA runtime call failed */
} glasso_status;

enum { GLASSO_FP64 = 0, GLASSO_MIXED = 1 };          /* precision modes */
enum { GLASSO_INPUT_S = 0, GLASSO_INPUT_X = 1 };     /* what `data` holds */
enum { GLASSO_F64 = 0, GLASSO_F32 = 1 };             /* element type of `data` */
enum { GLASSO_HOST = 0, GLASSO_DEVICE = 1 };         /* where `data`, A0 and outputs live */

typedef struct {
    int device;              /* CUDA device ordinal */
    size_t mem_budget_bytes; /* 0 = no limit; solves whose footprint exceeds it get ENOMEM */
    int precision;           /* GLASSO_FP64 or GLASSO_MIXED */
} glasso_config;

typedef struct {
    int input;        /* GLASSO_INPUT_S: data is S (n x n); GLASSO_INPUT_X: data is X (m x n, one sample per row) */
    int dtype;        /* GLASSO_F64 or GLASSO_F32 (X only; S is always FP64) */
    int location;     /* GLASSO_HOST or GLASSO_DEVICE for data, A0, A_out and W_out */
    const void *data;
    int64_t n, m;     /* m: number of samples (INPUT_X only) */
    int center;       /* INPUT_X: subtract the sample mean before forming S */
    double lambda;    /* > 0 */
    double tol;       /* stop when the relative KKT residual is <= tol */
    int max_cycles;   /* ML-cycles (Algorithm 1) before GLASSO_EMAXITER; <= 0 means 200 */
    const double *A0; /* optional warm start (n x n, positive definite); NULL: diag(1/(S_ii + lambda)) */
    int one_level;    /* 0: the ML-cycle of Algorithm 1; nonzero: the one-level method of the paper's
                         comparison (Section 8) -- every cycle a single relaxation on the full free set */
    int continuation; /* nonzero: the continuation strategy (end of Section 2, schedule of Section 8):
                         before the cycles, one full-free-set relaxation at each of lambda_4 > lambda_3 >
                         lambda_2, lambda_s = lambda + (s-1)(lambda_4 - lambda)/3, lambda_4 =
                         (max_{i!=j} |S_ij| + lambda)/2 (no stages when that maximum is <= lambda).
                         These relaxations count in `relaxations` and `max_nnz`, not in `cycles`;
                         max_cycles bounds the cycles at lambda.  Combines with either method. */
    int screen;       /* nonzero: exact screening.  The minimiser is block diagonal over the connected
                         components of {(i,j): i != j, |S_ij| > lambda}; isolated vertices get the closed
                         form A_ii = 1/(S_ii + lambda), and the remaining vertices are solved as one
                         sub-problem (the method never couples two components: their pairs never enter
                         the free set).  Same minimiser; the statistics are the sub-problem's plus the
                         isolated vertices' (objective, log det, nnz). */
    int inner;        /* Newton-direction solver of each relaxation: GLASSO_INNER_CD (0, the default):
                         CD sweeps, min(1 + floor(k/3), 10) in cycle k; GLASSO_INNER_PCD_CG (1): PCD-CG
                         (glasso_pcd) to relative precision 1e-4 (Section 8), at most 500 iterations;
                         GLASSO_INNER_AUTO (2): per relaxation, PCD-CG when the CD sweeps would update
                         at least GLASSO_AUTO_PCD_WORK coordinates in their serial chain (pairs x
                         sweeps; the environment variable of that name overrides it), else CD sweeps */
} glasso_problem;

enum { GLASSO_INNER_CD = 0, GLASSO_INNER_PCD_CG = 1, GLASSO_INNER_AUTO = 2 };
#define GLASSO_AUTO_PCD_WORK 20000

typedef struct {
    int status;          /* glasso_status of this solve */
    int cycles;          /* ML-cycles run */
    int relaxations;     /* proximal-Newton relaxations (all levels) */
    int ls_trials;       /* Cholesky trials in the line searches */
    double objective;    /* F(A) at return */
    double rel_kkt;      /* sum |min-norm subgradient| / ||A||_1 at return */
    double max_kkt;      /* max |min-norm subgradient| at return */
    double logdet;       /* log det A at return */
    double seconds;      /* wall time of the solve */
    int64_t nnz;         /* nonzeros of A (both triangles) */
    int64_t max_nnz;     /* largest nnz(A) at the fine-level free-set scans and at return (the
                            paper's max-supp, sampled where the full free set is formed) */
    int64_t components;  /* screen: connected components of {|S_ij| > lambda}; 0 without screening */
    int64_t max_block;   /* screen: vertices in the largest component; 0 without screening */
    int64_t inner_iters; /* CD sweeps or PCD-CG iterations, summed over the relaxations */
    double flops;        /* glasso_solve_batch_fused: the solve's algorithmic FP64 operations
                            (n^3/3 per factorisation, 2n^3/3 per inverse, 2n per coordinate
                            of a sweep + 2n per row it updates); 0 elsewhere */
} glasso_info;

/* ---- context -------------------------------------------------------- */

/* Create a context on cfg->device.  Allocates nothing on the device until the
 * first call that needs memory.  *out is NULL on failure. */
glasso_status glasso_create(const glasso_config *cfg, glasso_ctx **out);

/* Release every device buffer and stream of the context.  NULL is ignored. */
void glasso_destroy(glasso_ctx *ctx);

/* Run all later work of this context on `stream` (a cudaStream_t; NULL puts
 * the context back on its own stream).  The stream stays owned by the caller. */
glasso_status glasso_set_stream(glasso_ctx *ctx, void *stream);

/* Human-readable name of a status code (static storage). */
const char *glasso_strerror(glasso_status s);

/* Text of the last CUDA error seen by this context ("" if none). */
const char *glasso_last_error(glasso_ctx *ctx);

/* ---- solver --------------------------------------------------------- */

/* Solve one problem by the ML-cycle (Algorithm 1, nu = nu_c = 1, hierarchy of
 * Section 7) with the dense proximal-Newton relaxation of Sections 5.1-5.2.
 * A_out (required) and W_out (optional, = A^{-1}) are n x n in the location
 * given by p->location.  info (optional) receives the statistics; the return
 * value equals info->status. */
glasso_status glasso_solve(glasso_ctx *ctx, const glasso_problem *p, double *A_out,
                           double *W_out, glasso_info *info);

/* Solve `count` problems (e.g. several subjects, or lambda paths) on the
 * device.  A_out[k] receives the solution of p[k]; infos[k] (if infos is not
 * NULL) its statistics.  When p[k].A0 is NULL and k > 0 and warm_from_prev is
 * set, problem k starts from the solution of problem k-1 if both have the
 * same n, input kind and data pointer (continuation along decreasing lambda,
 * Section 2).  Problems that do not continue one another (and, with
 * warm_from_prev, each maximal run of continuing problems) are solved
 * concurrently through the context's serving slots; a run is solved in order
 * on one slot.  Inputs are copied to host memory before solving, so they may
 * be in either location.  Returns the first non-OK status, or GLASSO_OK. */
glasso_status glasso_solve_batch(glasso_ctx *ctx, const glasso_problem *p, int count,
                                 int warm_from_prev, double **A_out, glasso_info *infos);

/* The batched solver in ONE persistent launch (many small problems, e.g.
 * lambda paths of several subjects).  Same arguments and warm-start rule as
 * glasso_solve_batch: A_out[k] (in p[k].location) receives the solution of
 * p[k], infos[k] its statistics; with warm_from_prev a maximal run of
 * problems on the same data (same n, input kind and data pointer, A0 NULL
 * after the first) is one lambda path, each problem warm started from the
 * previous solution (continuation, end of Section 2).
 * Each CTA of the launch takes a path from a device-side queue (longest
 * first) and runs every step of the ML-cycle of Algorithm 1 (hierarchy of
 * Section 7, CD sweeps on the Newton LASSO of eq. Quad_MLE_l1_prior, the
 * Armijo line search of Section 6.1.2, the Section 8 KKT stop) itself, in
 * FP64, whatever the context's precision; no host round trip between steps,
 * relaxations or problems.  infos[k].seconds is the solve's own device time;
 * with profiling on (glasso_set_profiling), the kernel classes of
 * glasso_get_profile receive the CTAs' summed device time per step: 0 the
 * factorisations of the iterate, 1 the inverses, 2 the free-set scans and the
 * hierarchy, 3 the CD sweeps, 4 the line searches.
 * Requires 1 <= n <= GLASSO_FUSED_MAX_N, screen = 0, continuation = 0 and
 * inner CD or AUTO (AUTO takes the CD sweeps here); otherwise GLASSO_EINVAL
 * before any work.  GLASSO_ENOMEM when the launch's memory (inputs, outputs
 * and one workspace of about 6 n_max^2 doubles per CTA) exceeds the budget.
 * Returns the first non-OK status, or GLASSO_OK. */
#define GLASSO_FUSED_MAX_N 512
glasso_status glasso_solve_batch_fused(glasso_ctx *ctx, const glasso_problem *p, int count,
                                       int warm_from_prev, double **A_out, glasso_info *infos);

/* Asynchronous serving interface.  glasso_submit copies the problem's inputs
 * before returning (the caller may free them at once), queues the solve and
 * returns a ticket.  A_out must stay valid until glasso_poll reports the
 * ticket finished.  glasso_poll waits up to timeout_us microseconds (0: do
 * not wait) and returns GLASSO_EAGAIN while the solve is running, or the
 * solve's status once it has finished (info filled, ticket retired).  Solves
 * from several tickets run concurrently on the device. */
glasso_status glasso_submit(glasso_ctx *ctx, const glasso_problem *p, double *A_out,
                            uint64_t *ticket);
glasso_status glasso_poll(glasso_ctx *ctx, uint64_t ticket, int64_t timeout_us,
                          glasso_info *info);

/* ---- timing of the solver's kernel classes ---------------------------- */

/* Kernel classes timed with CUDA events on the context's stream when
 * profiling is on: 0 Cholesky of the iterate, 1 inverse (W = A^{-1}),
 * 2 level-0 free-set scan, 3 CD sweeps, 4 line-search Cholesky trials,
 * 5 Newton-Schulz refinement GEMMs of W (mixed precision). */
#define GLASSO_PROF_CLASSES 6

/* Code-path counters (all contexts, counted always, since the last reset):
 * which variant of a step the solves took. */
#define GLASSO_PATHS 11
enum {
    GLASSO_PATH_CD_LAG2 = 0,       /* FP32 sweeps by the pipelined chain-CTA kernel */
    GLASSO_PATH_CD_PERSIST32 = 1,  /* FP32 sweeps by the one-copy kernel (its matrices did not fit) */
    GLASSO_PATH_CD_CHAIN64 = 2,    /* sweeps with an FP64 resolution chain */
    GLASSO_PATH_LS_SERIES2 = 3,    /* mixed line-search trials decided by the two-term log-det series */
    GLASSO_PATH_LS_SERIES6 = 4,    /* ... by the six-term series */
    GLASSO_PATH_TC_FACTOR = 5,     /* tensor-core factorisations (line-search trials and fresh W) */
    GLASSO_PATH_TC_LEAVES = 6,     /* diagonal leaves factored inside them */
    GLASSO_PATH_NS_STEPS = 7,      /* Newton-Schulz refinement GEMMs of W */
    GLASSO_PATH_TC_DAG = 8,        /* diagonal blocks (up to 32 x 128) factored and inverted by one
                                      persistent task-graph launch inside them */
    GLASSO_PATH_TC_TUNED = 9       /* task-graph launches timed by the grid autotuner (the first
                                      call per block size; GLASSO_AUTOTUNE=0 turns it off) */,
    GLASSO_PATH_FUSED = 10         /* problems solved inside a fused batched launch
                                      (glasso_solve_batch_fused) */
};

typedef struct {
    double ms[GLASSO_PROF_CLASSES];        /* summed device time */
    long long launches[GLASSO_PROF_CLASSES];
    double work[GLASSO_PROF_CLASSES];      /* algorithmic flops (0, 1, 4, 5) or bytes (2, 3) */
    long long kernels;                     /* kernels launched by the library (all contexts,
                                              counted always) since the last reset */
    long long paths[GLASSO_PATHS];         /* GLASSO_PATH_* counters since the last reset */
} glasso_profile;

/* Turn event timing of the kernel classes on (on != 0) or off.  Off by
 * default; costs two events per timed call. */
glasso_status glasso_set_profiling(glasso_ctx *ctx, int on);

/* Copy the accumulated timings (and zero them when reset != 0).  The kernel
 * count is kept whether or not profiling is on. */
glasso_status glasso_get_profile(glasso_ctx *ctx, glasso_profile *out, int reset);

/* ---- fault injection (tests of the error paths) ---------------------- */

/* The paper has no counterpart: these knobs let tests drive the solver's
 * failure paths without a GPU fault.  They act on the context's own solves
 * and step-level calls (glasso_solve, glasso_cd_sweeps, glasso_line_search,
 * ...), not on solves run through the serving slots (glasso_submit,
 * glasso_solve_batch).  All are off (0) when the context is created. */
enum {
    GLASSO_DEBUG_WAIT_CYCLES = 1,      /* limit of each grid-barrier wait of the CD sweep in SM cycles
                                          (0: the default, about 2 s); value >= 0 */
    GLASSO_DEBUG_WAIT_UNREACHABLE = 2, /* nonzero: the CD sweep's grid barrier waits for one arrival more
                                          than the grid holds, so every wait runs to its limit; the sweep
                                          returns early and the call reports GLASSO_ETIMEOUT */
    GLASSO_DEBUG_LS_REJECT = 3,        /* nonzero: every line-search trial is rejected (Section 6.1.2's
                                          backtracking runs out of trials: GLASSO_ELINESEARCH) */
    GLASSO_DEBUG_TC_DAG_TILES = 4      /* not a fault: the largest diagonal block, in 128-row tiles,
                                          that the mixed factorisation hands to one persistent
                                          task-graph launch (larger ones recurse): 0 the default (32),
                                          1 none (recursion down to one-tile leaves), 2 .. 32 that
                                          many; so every variant stays testable and comparable */
};

/* Set one knob.  GLASSO_EINVAL for an unknown knob or a value out of its range. */
glasso_status glasso_set_debug(glasso_ctx *ctx, int knob, int64_t value);

/* ---- step-level entry points (device pointers) ----------------------- */

/* a1. S = (1/m) X^T X (eq. cov_estimate), X m x n row-major of `dtype`
 * (GLASSO_F64 or GLASSO_F32), S n x n FP64.  With center != 0 the sample mean
 * is subtracted first.  FP64 X is accumulated in FP64; FP32 X on the tensor
 * cores (TF32 inputs, FP32 accumulation) in GLASSO_MIXED contexts and in FP64
 * otherwise. */
glasso_status glasso_form_S(glasso_ctx *ctx, const void *X, int dtype, int64_t m, int64_t n,
                            int center, double *S);

/* a2. Cholesky factorisation in place: on return the lower triangle of A
 * holds L with A = L L^T (upper triangle untouched).  *info = 0, or k+1 when
 * the k-th pivot is not positive (A not positive definite: the line-search
 * feasibility test of Section 6.1.2); *logdet = 2 sum_i log L_ii when
 * *info = 0.  Blocked right-looking; FP64. */
glasso_status glasso_potrf(glasso_ctx *ctx, double *A, int64_t n, int *info, double *logdet);

/* a3. W = A^{-1} = L^{-T} L^{-1} from the Cholesky factor L (lower triangle
 * read), eq. gradHes.  W is written in full.  FP64. */
glasso_status glasso_inverse(glasso_ctx *ctx, const double *L, int64_t n, double *W);

/* a2 + a3 in the arithmetic of the mixed-precision solve: A (lower triangle
 * read, FP64) is rounded to FP32 and factored, A = L L^T, with the inverse
 * factor X = L^{-1} formed alongside (recursive blocking; every O(n^3)
 * contraction on the tensor cores as a split-TF32 product, about 2^-21
 * relative error per product, FP32 accumulation); then W = X^T X = A^{-1}
 * (eq. gradHes; not refined) is written in full as FP64.  *info and *logdet
 * as glasso_potrf (log det accumulated in FP64 from the FP32 pivots); W is
 * left unwritten when *info != 0.  A is not modified.  Needs a
 * GLASSO_MIXED context (else GLASSO_EINVAL). */
glasso_status glasso_cholinv_mixed(glasso_ctx *ctx, const double *A, int64_t n, double *W, int *info,
                                   double *logdet);

/* a4. Free set of eq. active_set, {(i,j): A_ij != 0 or |(S - W)_ij| > lambda},
 * restricted to a candidate set C_l (eq. MLE_l1_prior_C).  When cand_i is
 * NULL all upper-triangle pairs are candidates and the scan also returns the
 * relative KKT residual (min-norm subgradient, eq. subgradient1, over all
 * (i, j), divided by ||A||_1) in *rel_kkt and its max norm in *max_kkt
 * (either may be NULL); otherwise cand_i/cand_j (ncand pairs, device) are
 * filtered in their order.  out_i/out_j (device, capacity n(n+1)/2 for the
 * full scan, ncand otherwise) receive the free pairs in candidate order,
 * absg (device, optional) |S - W| on them; *count their number. */
glasso_status glasso_free_set(glasso_ctx *ctx, const double *S, const double *W,
                              const double *A, int64_t n, double lambda,
                              const int32_t *cand_i, const int32_t *cand_j, int64_t ncand,
                              int32_t *out_i, int32_t *out_j, double *absg, int64_t *count,
                              double *rel_kkt, double *max_kkt);

/* a5. Multilevel hierarchy (Section 3.2, Section 7): given the previous fine
 * free set (nf pairs) with |G| on each (absg, device) and a support flag
 * (insupp, device uint8), tag[p] (device uint8) receives the coarsest level
 * whose set C_l holds pair p and *levels the number L of levels:
 * |C_1| = max(ceil(nf/2), |supp|), |C_{l+1}| = max(ceil(|C_l|/2), |supp|)
 * until |C_L| = |supp|; C_l = support + the non-support pairs of largest |G|
 * (ties: earlier pair first).  nf <= 2^31 - 1. */
glasso_status glasso_hierarchy(glasso_ctx *ctx, const double *absg, const uint8_t *insupp,
                               int64_t nf, uint8_t *tag, int *levels);

/* a6. nsweeps coordinate-descent sweeps over the pair list on the Newton
 * LASSO of eq. Quad_MLE_l1_prior,
 *   min_Delta tr(Delta (S - W)) + 1/2 tr(Delta W Delta W) + lambda ||A + Delta||_1,
 * in list order.  Each coordinate takes the exact 1-D minimiser
 * mu = -c + S_{lambda/a}(c - b/a) (eq. 1d_l1 and eq. shrinkage) with
 * a = W_ij^2 + W_ii W_jj (W_ii^2 on the diagonal), b = (S - W)_ij + (W Delta W)_ij,
 * c = A_ij + Delta_ij.  D (np, device) holds Delta on the pairs and U (n x n,
 * device) = Delta W; both are read and updated.  The result equals the
 * sequential sweep up to floating-point reassociation.  In a GLASSO_MIXED
 * context the sweep is the mixed solve's: W and U rounded to FP32, the
 * resolution chain in FP32, the increments of Delta in FP64 (exact zeros of
 * the shrinkage kept); U is returned converted to FP64. */
glasso_status glasso_cd_sweeps(glasso_ctx *ctx, const double *S, const double *W,
                               const double *A, int64_t n, double lambda, const int32_t *pi,
                               const int32_t *pj, int64_t np, int nsweeps, double *D, double *U);

/* a6 (alternative inner solver).  PCD-CG on the same Newton LASSO as
 * glasso_cd_sweeps: the generalised parallel coordinate descent direction
 * (Section 2, eq. IST_direction with D = the diagonal of the Hessian) -- every
 * coordinate's own 1-D minimiser d_p = S_{lambda/a}(c - b/a) - c at once --
 * with the exact minimising step along the search direction (the model is a
 * convex quadratic plus a piecewise-linear term: its kinks are walked in
 * increasing order, and a coordinate that lands on its kink becomes an
 * exact zero), accelerated by non-linear conjugate gradients (Section 6.3;
 * Polak-Ribiere-plus coefficient in the pair inner product with weight 2 off
 * the diagonal, reset to the PCD direction when not a descent direction).
 * A coordinate whose own minimiser is zero and that the step no longer moves
 * is set to its exact zero.  cg == 0 gives plain PCD.  Stops after `iters`
 * iterations, when the direction is zero, when the step is zero, or for
 * rtol > 0 once max|d| <= rtol * max|d| of the first iteration.  D (np,
 * device) holds Delta on the pairs (in/out; b starts from (W Delta W) of the
 * given Delta); U (n x n, device) receives Delta W (its input is not read).
 * *iters_done (host, may be NULL) receives the iterations taken.  In a
 * GLASSO_MIXED context the products with W run in FP32 (the mixed solve's
 * arithmetic) and U is returned converted to FP64. */
glasso_status glasso_pcd(glasso_ctx *ctx, const double *S, const double *W, const double *A, int64_t n,
                         double lambda, const int32_t *pi, const int32_t *pj, int64_t np, int iters,
                         int cg, double rtol, double *D, double *U, int *iters_done);

/* a7. Armijo backtracking line search (eq. Line-search; Section 6.1.2 with
 * alpha_0 = 1, beta = 1/2): the first alpha = 2^-t, t < max_trials, for which
 * A + alpha Delta is positive definite and
 *   F(A + alpha Delta) <= F_A + sigma alpha delta + 1e-12 max(|F_A|, n),
 *   delta = tr((S - W) Delta) + lambda (||A + Delta||_1 - ||A||_1),
 * where F_A = F(A) is passed in (the last term absorbs objective rounding).
 * On success A (device, n x n) becomes A + alpha Delta and the outputs are
 * set; otherwise GLASSO_ELINESEARCH and A is unchanged. */
glasso_status glasso_line_search(glasso_ctx *ctx, const double *S, const double *W, double *A,
                                 int64_t n, double lambda, const int32_t *pi, const int32_t *pj,
                                 int64_t np, const double *D, double F_A, double sigma,
                                 int max_trials, double *F_new, double *alpha, int *trials);

/* Screening: connected components of the graph {(i, j): i != j, |S_ij| > lambda}
 * on S (n x n, device, symmetric; only the upper triangle is read).
 * comp (device, n int32) receives for each vertex the smallest vertex of its
 * component (so labels are independent of the order of discovery); *ncomp
 * (host, may be NULL) the number of components.  Lock-free union-find; a
 * retry bound that the algorithm cannot reach is checked and reported as
 * GLASSO_ECUDA. */
glasso_status glasso_components(glasso_ctx *ctx, const double *S, int64_t n, double lambda,
                                int32_t *comp, int64_t *ncomp);

/* F(A) = -log det A + tr(S A) + lambda ||A||_1 (eq. MLE_l1_prior); *info as
 * glasso_potrf (F undefined when *info != 0). */
glasso_status glasso_objective(glasso_ctx *ctx, const double *S, const double *A, int64_t n,
                               double lambda, double *F, int *info);

/* BCD-IC's line-search log det (Section 6, the update of Algorithm 2;
 * eq. Schurs_lemma, eq. logdet_blocks, eq. Schurs_PDness): for a block I and
 * a direction Delta that vanishes outside the rows and columns of I,
 *   log det(A + alpha Delta) = log det A_22 + log det(B_0 + alpha B_1 + alpha^2 B_2)
 * with B_0 = A_11 - A_12 A_22^{-1} A_21, B_1 = Delta_11 - Delta_12 A_22^{-1} A_21
 * - A_12 A_22^{-1} Delta_21, B_2 = -Delta_12 A_22^{-1} Delta_21 ("1" = I, "2"
 * the other indices); A + alpha Delta is positive definite iff A_22 and the
 * |I| x |I| matrix are.  FP64 on the device in any context.
 * A: n x n FP64, device, symmetric (A_22 is read from it); pi, pj, D: the np
 * pairs of Delta (i <= j, device); inI: n bytes on the device, nonzero for
 * the indices of I.  *code (host): 0 with *logdet set; 1 when A_22, 2 when
 * the small matrix is not positive definite; -1 when Delta has a nonzero
 * pair outside the rows and columns of I.  GLASSO_EINVAL for bad arguments
 * or a pair index outside [0, n).  Allocates its scratch on the context's
 * stream and synchronises it. */
glasso_status glasso_bcd_logdet(glasso_ctx *ctx, const double *A, int64_t n, const int32_t *pi,
                                const int32_t *pj, int64_t np, const double *D, const uint8_t *inI,
                                double alpha, double *logdet, int *code);

/* One BCD-IC iteration (Section 6, Algorithm 2) on the device, A updated in
 * place.  The columns are split into consecutive blocks of `block` columns
 * (0: one block), treated in order; for each, at the current iterate: W from
 * the FP64 factorisation, the block's free set (eq. active_set_j: free pairs
 * with a row or column in the block), the Newton direction on it
 * (eq. sub_Quad_MLE_l1_prior) by nsweeps CD sweeps (inner = GLASSO_INNER_CD)
 * or PCD-CG to relative precision 1e-4 (GLASSO_INNER_PCD_CG), and the line
 * search over alpha = 2^-t (t < 30) with log det(A + alpha Delta) from the
 * Schur complement (glasso_bcd_logdet).  rule 1: the sample minimising F
 * subject to positive definiteness (Section 6.1.2: the first sample not
 * improved on by the next); rule 0: Armijo (sigma = 1e-4).  Both accept only
 * F(A + alpha Delta) <= F(A) + 1e-12 max(|F(A)|, n).  S, A: n x n FP64 on the
 * device.  *F (optional): F of the result; *moved: blocks with a nonzero
 * direction; *trials: samples evaluated.  GLASSO_ENOTPD when A is not
 * positive definite, GLASSO_ELINESEARCH when no sample passes (A keeps the
 * blocks done so far). */
glasso_status glasso_bcd_iteration(glasso_ctx *ctx, const double *S, double *A, int64_t n, double lambda,
                                   int64_t block, int inner, int nsweeps, int rule, double *F,
                                   int *moved, int *trials);

/* ML-BCD (Sections 6-7): the ML-cycle of Algorithm 1 (hierarchy of Section 7,
 * the Section 8 KKT stop at tol) with one BCD-IC iteration (as
 * glasso_bcd_iteration, blocks of `block` columns) as the relaxation on each
 * level, the block free sets taken within C_l; from A0 = diag(1/(S_ii +
 * lambda)); nsweeps = min(1 + floor(k/3), 10) CD sweeps in cycle k (inner =
 * GLASSO_INNER_CD) or PCD-CG; one_level != 0: BCD-IC alone.  The control runs
 * on the host, every step on the device.  S (input) and A (output): n x n
 * FP64 on the device.  info (optional): status, cycles, relaxations, samples
 * (ls_trials), objective, KKT residuals, log det, nnz.  Returns the status. */
glasso_status glasso_solve_bcd(glasso_ctx *ctx, const double *S, int64_t n, double lambda, double tol,
                               int max_cycles, int64_t block, int inner, int rule, int one_level, double *A,
                               glasso_info *info);

/* ---- allocation-free entry point ------------------------------------- */

/* Largest n accepted by glasso_free_set_noalloc. */
#define GLASSO_NOALLOC_MAX_N 4096

/* The level-0 free-set scan of glasso_free_set (all candidate pairs, with the
 * relative KKT residual), for callers that must not allocate device memory:
 * code running under another framework's memory manager, which owns the
 * device heap, or latency-critical loops that cannot take cudaMalloc's
 * implicit device-wide synchronisation.  The paper has no counterpart; this
 * is a deployment variant of the same kernels.
 *
 * It needs no context and allocates nothing.  Its scratch (about 2.3 MB: the
 * row bit masks, row counts, partial sums and result scalars for n up to
 * GLASSO_NOALLOC_MAX_N) is one fixed array in device memory that every GPU
 * loading the library holds until the process exits.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.
 *
 * Arguments and outputs are those of glasso_free_set with cand_i = NULL:
 * S, W, A are device n x n; out_i/out_j (capacity n(n+1)/2) and absg
 * (optional) are device; count, rel_kkt, max_kkt are host.  Work runs on
 * `stream` (a cudaStream_t, NULL for the legacy default stream) and the call
 * returns when the outputs are complete.  n > GLASSO_NOALLOC_MAX_N returns
 * GLASSO_EINVAL; CUDA failures return GLASSO_ECUDA.
 *
 * All calls in the process share the one scratch array, which keeps the last
 * call's contents: calls that overlap on the GPU (from several host threads
 * or streams) race on it and must be serialised by the caller. */
glasso_status glasso_free_set_noalloc(const double *S, const double *W, const double *A,
                                      int64_t n, double lambda, int32_t *out_i,
                                      int32_t *out_j, double *absg, int64_t *count,
                                      double *rel_kkt, double *max_kkt, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GLASSO_H */
