/*
 * clr.h -- C ABI of the GB300 interior-point conic solver.
 *
 * Problem (Eq. P of arXiv:2412.19027, "CuClarabel", Sec. 1):
 *
 *     minimize    1/2 x'Px + q'x
 *     subject to  Ax + s = b,  s in K = K_1 x ... x K_p
 *
 * with dual (Eq. D)  maximize -1/2 x'Px - b'z  s.t.  Px + A'z = -q, z in K*.
 * K is a product of zero, nonnegative, second-order, exponential, power and
 * positive-semidefinite cones (Sec. 2.1).  The solver runs the homogeneous-
 * embedding predictor-corrector interior-point method of Algorithm 1 (Sec.
 * 3.2): setup (equilibration, initialisation, symbolic KKT analysis) on the
 * host, then every iteration on one GPU.
 *
 * Conventions shared by every entry point
 *  - Return value: int status code, CLR_OK (0) on success, a negative CLR_E_*
 *    on failure.  No entry point exits, aborts or traps.  The solver's own
 *    outcome (solved, infeasible, ...) is a separate clr_status in clr_info;
 *    a solve that ends in MAX_ITER is still a successful call.
 *  - Ownership: every input array is caller-owned HOST memory, read during
 *    the call and deep-copied; the library keeps no caller pointer.  Outputs
 *    go into caller-owned host buffers of the stated length.  Device memory
 *    is owned by the solver object and freed by clr_free.
 *  - Threads: a clr_solver may be used by one host thread at a time.
 *  - Index types: column pointers int64, row indices int32, values double.
 */
#ifndef CLR_H
#define CLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum clr_error {
  CLR_OK = 0,
  CLR_E_INVALID = -1,     /* malformed input: NaN/Inf, bad pattern, bad cone list */
  CLR_E_DIM = -2,         /* dimensions disagree (cone dims vs m, vector lengths) */
  CLR_E_UNSUPPORTED = -3, /* e.g. PSD cones of different orders or order > 32 */
  CLR_E_OOM = -4,         /* device or host allocation failed */
  CLR_E_CUDA = -5,        /* a CUDA call failed; clr_last_cuda_error() has details */
  CLR_E_TIMEOUT = -6,     /* a bounded device wait ran out */
  CLR_E_AGAIN = -7,       /* result not ready yet */
  CLR_E_STATE = -8        /* call out of order (e.g. solution before solve) */
};

/* Solver outcome (Sec. 2.2 termination and infeasibility tests). */
enum clr_status {
  CLR_UNSOLVED = 0,
  CLR_SOLVED = 1,
  CLR_PRIMAL_INFEASIBLE = 2,
  CLR_DUAL_INFEASIBLE = 3,
  CLR_MAX_ITER = 4,
  CLR_INSUFFICIENT_PROGRESS = 5,
  CLR_NUMERICAL_ERROR = 6
};

/* Cone types (Sec. 2.1).  CLR_PSD_TRI: dim = k(k+1)/2 rows holding the svec
 * of a k x k symmetric matrix -- upper triangle, column by column, entries
 * above the diagonal multiplied by sqrt(2).  Every PSD cone has order
 * k <= 32 (the paper's bound, Sec. 2.1 footnote and Sec. 3.4); cones of
 * different orders may be mixed (the paper requires one order and names mixed
 * orders as future work, Sec. 6).  CLR_EXP and CLR_POW have dim 3; alpha is
 * the power cone exponent in (0, 1). */
enum clr_cone_type { CLR_ZERO = 0, CLR_NONNEG = 1, CLR_SOC = 2, CLR_EXP = 3, CLR_POW = 4, CLR_PSD_TRI = 5 };

typedef struct {
  int32_t type;  /* clr_cone_type */
  int32_t dim;   /* number of rows of s (and of A, b) the cone covers */
  double alpha;  /* power-cone exponent; ignored otherwise */
} clr_cone;

/* Compressed sparse column matrix: colptr[ncols+1], rowind[nnz], val[nnz].
 * Row indices within a column must be strictly increasing. */
typedef struct {
  int64_t nrows, ncols, nnz;
  const int64_t* colptr;
  const int32_t* rowind;
  const double* val;
} clr_csc;

/* Settings.  clr_default_settings fills the values below; each one is
 * printed in the paper where noted, otherwise it is this library's reading. */
typedef struct {
  double eps_feas;        /* termination tolerance (Eq. termination-check); default 1e-8 */
  double eps_inf;         /* infeasibility tolerance (Eq. infeasibility-check); 1e-8 */
  int32_t max_iter;       /* 200 */
  int32_t factor_bits;    /* LDL^T precision (Sec. 3.6): 64 (FP64), 32 (FP32), or 16: FP32 factor whose
                             large-front updates multiply BF16-rounded operands on the tensor cores with
                             FP32 accumulation (the 16-bit-products variant; defaults as for 32) */
  double static_reg;      /* delta_s: 1e-8 (FP64), sqrt(eps_32) ~ 3.45e-4 (FP32) (Sec. 3.6) */
  double static_reg_dyn;  /* delta_d in delta = delta_s + delta_d max|K_ii|: eps_64^2 */
  double dyn_reg_eps;     /* pivot threshold of dynamic regularisation: 1e-13 (FP64), 1e-6 (FP32) */
  double dyn_reg_delta;   /* replacement pivot magnitude: 2e-7 (FP64), 1e-4 (FP32) */
  int32_t ir_max_steps;   /* T_max = 10 (Sec. 3.6) */
  double ir_abstol;       /* t_abs = 1e-12 (Sec. 3.6) */
  double ir_reltol;       /* t_rel = 1e-12 (Sec. 3.6) */
  double ir_stop_ratio;   /* 0 (off): else stop refining once a step reduces ||r|| by less than this factor */
  int32_t equilibrate;    /* 1: modified Ruiz scaling at setup (Alg. 1 step 1) */
  int32_t ruiz_passes;    /* 10 */
  double scale_min;       /* 1e-4: clamp of every equilibration factor */
  double scale_max;       /* 1e4 */
  double step_fraction;   /* 0.99 (Alg. 1 step 11) */
  double backtrack;       /* 0.8 (Sec. 2.2, exp/pow step length) */
  double nbhd_beta;       /* 1e-6 (Sec. 2.2, neighbourhood N(beta)) */
  double min_step;        /* 1e-10: smaller combined steps end the solve */
  int32_t use_graph;      /* 1: replay each iteration as a captured CUDA graph */
  int32_t verbose;        /* 0 */
  int32_t fp64_escalation; /* factor_bits 32/16 only, 1 (default): when the refinement of a KKT solve ends with
                              ||r||_inf > 1e-4 max(1, ||rhs||_inf) (or NaN) the iteration is not taken and the solve
                              goes on with the FP64 factor and the FP64 regularisation defaults (for every problem
                              of a cohort); 0: never */
  int32_t big_front_schedule; /* large fronts: 1 (default) one dataflow launch per level, tile tasks started as
                                 their inputs are ready; with the FP32 factor, on the levels where a schedule
                                 simulated at setup from measured task times is shorter that way, its
                                 trailing and E updates run on the tensor cores (tcgen05 kind::tf32, each
                                 operand split into high and low TF32 parts, FP32 accumulation; operand tiles
                                 staged by TMA); 3 the tensor-core launch on every level; 2 CUDA-core
                                 products only; 0 three launches per 64-column panel.  The 16-bit-products
                                 variant always uses the per-panel launches. */
  int32_t small_front_max;    /* fronts of at most this order are factored by one CTA each in shared memory,
                                 larger ones by the big-front kernels; 0 (default): 128 (FP32 / 16-bit
                                 products), 96 (FP64); at most 224 (FP32) / 160 (FP64) */
  int32_t amalgamation;       /* relaxed supernode amalgamation: 0 off, 1 (default) column thresholds
                                 4 / 16 / 48, 2 thresholds 8 / 32 / 96 (same zero ratios) */
  double escalate_ratio;      /* factor_bits 32/16 with fp64_escalation: also escalate when a KKT solve of an
                                 iteration ends its refinement above t_abs + t_rel ||rhs|| with ||r||_inf larger
                                 than escalate_ratio times the largest entry of the iterate's scaled residual G
                                 while the primal or dual residual is still more than 100 times its termination
                                 tolerance (the direction is then too inexact to reduce it); default 0.1, 0 = off */
  int32_t soc_expand_dim;     /* second-order cones of at least this many rows (Sec. 3.3 names cones of
                                 thousands of rows, multistage portfolios) enter the KKT matrix in sparse
                                 form -- H = eta^2 (I + u u' - v v') as its diagonal plus two extra rows and
                                 columns per cone, [-eta^2 I, eta u, eta v; eta u', 1, 0; eta v', 0, -1] --
                                 instead of a dense d x d block (not in the paper, which factors with
                                 cuDSS); default 33, 0 = never */
  int32_t pull_lists_direct;  /* 1 (default): the factorization's extend-add source lists of a front whose
                                 children contribute densely are placed directly by counting each target's
                                 sources; 0: always by sorting (target, source) pairs.  Both give the same
                                 lists (clr_symbolic_stats.maps_digest); 0 is slower and exists to check that */
} clr_settings;

typedef struct {
  int32_t status;          /* clr_status */
  int32_t iterations;
  int32_t ir_steps_total;  /* refinement steps summed over all KKT solves */
  int32_t dyn_reg_hits;    /* pivots replaced by dynamic regularisation (last factor) */
  double obj_primal;       /* g_p (Eq. residuals-objectives), unscaled */
  double obj_dual;         /* g_d */
  double res_primal;       /* ||r_p||_inf */
  double res_dual;         /* ||r_d||_inf */
  double gap_abs;          /* |g_p - g_d| */
  double gap_rel;          /* |g_p - g_d| / max(1, min(|g_p|, |g_d|)) */
  double mu, tau, kappa;   /* complementarity measure (scaled space) and the embedding scalars */
  double setup_s;          /* host wall time of clr_setup */
  double solve_s;          /* host wall time of the last clr_solve */
  int32_t fp64_from_iter;  /* iteration from which the FP64 factor was used after an escalation, -1 if none */
  int32_t pad;
} clr_info;

/* Statistics of the symbolic KKT analysis done at setup. */
typedef struct {
  int64_t n, m, kkt_dim;   /* N = n + m; m counts the two auxiliary rows of each expanded SOC (the last
                              rows of the reordered constraint block; clr_get_symbolic's row_perm and
                              clr_get_scaling's E cover the caller's rows only) */
  int64_t kkt_nnz_lower;   /* structural nonzeros of the lower triangle of K */
  int64_t l_nnz;           /* nonzeros of L (supernodal, including the diagonal) */
  double factor_flops;     /* flops of the exact factor (multiply-adds x 2; explicit zeros excluded) */
  int64_t n_supernodes;
  int64_t n_levels;        /* depth of the supernodal elimination tree */
  int64_t max_front;       /* largest frontal matrix order */
  int64_t front_pool_entries; /* entries of the frontal-matrix pool */
  int64_t n_dense_rows;    /* rows treated as dense by the ordering */
  int64_t ordering;        /* 0: AMD on the KKT pattern; 1: cone rows first, then x by AMD (fewer flops) */
  int64_t l_nnz_exact;     /* nnz of the exact factor pattern (l_nnz adds the explicit zeros of merged supernodes) */
  int64_t l_nnz_counted;   /* the same from column counts of the order, without forming the factor */
  double factor_flops_stored; /* flops the supernodal factorization performs (explicit zeros included) */
  uint64_t maps_digest;    /* hash (FNV-1a's step over whole entries) of the elimination order and of
                              every index map of the numeric phase (value scatter, extend-add and solve
                              pull lists, push rounds): equal digests mean the same device arithmetic,
                              e.g. across hosts or settings */
} clr_symbolic_stats;

/* Device-side timing of the last clr_solve, from CUDA events recorded inside
 * the captured graphs on the solver's stream. */
typedef struct {
  int64_t kernel_launches;  /* kernels launched by the last solve (graph nodes x replays) */
  int32_t iterations;
  int32_t factorizations;   /* numeric factorizations (initialisation included) */
  double init_ms;           /* initial point (incl. its factorization and solves) */
  double resid_cones_ms;    /* residuals, termination tests, scaling H (all iterations) */
  double factor_ms;         /* numeric LDL^T (all iterations) */
  double solve_step_ms;     /* KKT solves with refinement, directions, step lengths, update */
  double factor_flops;      /* flops of one numeric factorization (symbolic count) */
  double factor64_ms;       /* the part of factor_ms spent in iterations with the FP64 factor */
  int32_t factorizations64; /* iterations factored with the FP64 factor (factor_bits 64, or after escalation) */
  int32_t pad;
} clr_perf;

typedef struct clr_solver clr_solver;

/* Fill *out with the defaults for a factorization precision (64, 32 or 16).
 * CLR_E_INVALID for any other factor_bits or a NULL out. */
int clr_default_settings(clr_settings* out, int32_t factor_bits);

/* Setup phase of Algorithm 1 (steps 1-2): validate, reorder the cones into
 * zero, nonneg, SOC, exp, pow, PSD with all zero and all nonneg cones merged
 * (Sec. 3.3, 3.5), equilibrate, assemble the KKT pattern of Eq. linsys_2x2,
 * compute the AMD ordering, elimination tree and supernodes, and upload the
 * data to the current CUDA device.
 *   P_upper  n x n, upper triangle of P only (entries below the diagonal give
 *            CLR_E_INVALID); P must be positive semidefinite (not checked).
 *   q        length n.   A  m x n.   b  length m.
 *   cones    ncones entries whose dims add up to m, in row order of A and b.
 *   st       settings, or NULL for clr_default_settings(.., 64).
 * On success *out owns device memory; free it with clr_free.  On failure
 * *out is NULL.  Errors: CLR_E_INVALID (NaN/Inf, pattern), CLR_E_DIM,
 * CLR_E_UNSUPPORTED, CLR_E_OOM, CLR_E_CUDA. */
int clr_setup(clr_solver** out, const clr_csc* P_upper, const double* q, const clr_csc* A, const double* b,
              const clr_cone* cones, int32_t ncones, const clr_settings* st);

/* Host-only part of clr_setup (validation, reordering, equilibration, KKT
 * pattern, ordering, symbolic factorization); touches no GPU.  The object can
 * be queried with clr_get_symbolic_stats / clr_get_symbolic and freed with
 * clr_free, but not solved. */
int clr_analyze(clr_solver** out, const clr_csc* P_upper, const double* q, const clr_csc* A, const double* b,
                const clr_cone* cones, int32_t ncones, const clr_settings* st);

/* Solve phase of Algorithm 1: initial point, then iterations until the
 * termination or infeasibility tests pass, max_iter is reached, or the step
 * length falls below min_step.  Blocking.  Each call starts from scratch
 * (data as set up, or as replaced by clr_update_qb / clr_update_PA). */
int clr_solve(clr_solver* s);

/* clr_solve in parts, for callers that interleave iterations with other work or
 * time them (the same kernels and graphs as clr_solve):
 *   clr_solve_begin    starts a solve from scratch: the initial point (Alg. 1
 *                      step 2), queued on the solver's stream;
 *   clr_solve_iterate  runs up to k (>= 0) passes of the iteration (Alg. 1 steps
 *                      3-11; blocking), stopping early once every problem has
 *                      stopped (then *done = 1, else 0); *iters_run = the
 *                      iterations completed (a pass that only finds the
 *                      termination test satisfied completes none);
 *   clr_solve_end      finishes the solve (results readable with
 *                      clr_get_solution).
 * done and iters_run may be NULL.  CLR_E_STATE if the solver holds no device
 * data (clr_analyze), CLR_E_INVALID on k < 0. */
int clr_solve_begin(clr_solver* s);
int clr_solve_iterate(clr_solver* s, int32_t k, int32_t* done, int32_t* iters_run);
int clr_solve_end(clr_solver* s);

/* Copy the result to host buffers (any may be NULL): x (n), s (m), z (m) in
 * the caller's original row order, un-scaled.  SOLVED: x/tau, s/tau, z/tau.
 * PRIMAL_INFEASIBLE: z = certificate normalised to b'z = -1, x and s NaN.
 * DUAL_INFEASIBLE: x, s normalised to q'x = -1, z NaN.
 * CLR_E_STATE before the first clr_solve. */
int clr_get_solution(const clr_solver* s, double* x, double* sl, double* z, clr_info* info);

/* Replace q and b (host, lengths n and m, caller's row order) keeping P, A,
 * the cones and the symbolic analysis (parametric re-solve, Sec. 4.6).  The
 * equilibration computed at setup is kept.  CLR_E_INVALID on NaN/Inf. */
int clr_update_qb(clr_solver* s, const double* q, const double* b);

/* Replace the values of P and/or A, same sparsity patterns as at setup
 * (parametric programming, Sec. 4.6: the coefficients change, the solver and
 * its symbolic factorization are reused).  Px (host): nnz(P_upper) values in
 * the CSC order of the P_upper given to setup; Ax (host): nnz(A) values in the
 * CSC order of A.  Either may be NULL (kept).  An entry set to 0 stays in the
 * pattern.  The equilibration computed at setup is kept and applied to the new
 * values; the fill-reducing order, the supernodes and every device buffer are
 * reused.  The next clr_solve starts from scratch on the new data.
 * CLR_E_INVALID on NaN/Inf (nothing is changed then). */
int clr_update_PA(clr_solver* s, const double* Px, const double* Ax);

int clr_get_symbolic_stats(const clr_solver* s, clr_symbolic_stats* out);

/* ------------------------------------------------------------------------
 * Cohorts ("batches"): many independent problems in one solver.  The paper
 * solves one problem at a time; for many small problems of uneven size the
 * per-iteration device step runs over all of them at once: the problems are
 * merged block-diagonally (x stacked; constraint rows family-major, each
 * family holding its rows of every problem in turn) and one launch of each
 * kernel -- one replay of the iteration's CUDA graph -- advances every
 * problem.  Every scalar of Algorithm 1 (tau, kappa, mu, step lengths,
 * sigma, regularisation, refinement counters, status) is kept per problem,
 * reductions are summed per problem in a fixed order, and each problem keeps
 * its own equilibration and fill-reducing order, so a problem's iterates are
 * the ones it has when solved alone (up to the row grouping of the K
 * products).  A problem that stops (solved, infeasible, ...) is frozen while
 * the others go on; the solve returns when every problem has stopped.
 * ------------------------------------------------------------------------ */

/* One problem of a cohort: the arguments of clr_setup, all host, read during
 * the call only. */
typedef struct {
  const clr_csc* P_upper;
  const double* q;
  const clr_csc* A;
  const double* b;
  const clr_cone* cones;
  int32_t ncones;
} clr_problem;

/* Setup of nprob >= 1 problems as one solver (the host analysis of each
 * problem runs on worker threads).  Errors as clr_setup, for the first failing
 * problem.  clr_solve solves every problem; clr_get_solution and
 * clr_update_qb act on problem 0; clr_get_perf covers the cohort. */
int clr_batch_setup(clr_solver** out, int32_t nprob, const clr_problem* probs, const clr_settings* st);

/* Host-only part of clr_batch_setup (as clr_analyze for one problem): the
 * merged cohort can be inspected with clr_get_symbolic_stats but not solved. */
int clr_batch_analyze(clr_solver** out, int32_t nprob, const clr_problem* probs, const clr_settings* st);

/* Number of problems held by a solver (1 after clr_setup). */
int32_t clr_batch_size(const clr_solver* s);

/* clr_get_solution for problem i of the cohort (CLR_E_INVALID if i is out of range). */
int clr_batch_get(const clr_solver* s, int32_t i, double* x, double* sl, double* z, clr_info* info);

/* clr_update_qb for problem i of the cohort. */
int clr_batch_update_qb(clr_solver* s, int32_t i, const double* q, const double* b);

/* clr_update_PA for problem i of the cohort (its own P and A patterns). */
int clr_batch_update_PA(clr_solver* s, int32_t i, const double* Px, const double* Ax);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  The paper has no
 * serving layer; this is the production pattern for streams of small solves
 * (e.g. one model-predictive-control QP per controller and period).
 * Submitted problems are copied, analysed on host worker threads, and
 * admitted as cohorts (see clr_batch_setup) whenever one of max_active slots
 * is free and the device memory in use is below device_bytes: every analysed
 * request waiting at that moment joins the new cohort (at most max_cohort).
 * Up to max_active cohorts run at once on their own CUDA streams with their
 * IPM iterations interleaved, so requests that arrive while others are on the
 * GPU start as soon as a slot and memory free up.  A result is handed out as
 * soon as its problem stops, not when its cohort does; it equals the result
 * of clr_setup + clr_solve on the same problem up to the rounding of the K
 * products.  All host threads are owned by the server.
 * ------------------------------------------------------------------------ */
/* Autotuner of the factorization's blocking parameters (small_front_max,
 * amalgamation, big_front_schedule) for a cohort of problems: every candidate
 * (small_front_max in {64, 96, 128, 160} plus 192 for FP32 factors, amalgamation
 * 0..2, schedules 0 and 1, and 2 for FP32 factors) is set up as a cohort of `probs` with the other fields
 * of *base and solved for `iters` (>= 1) IPM iterations; the device time per
 * iteration (CUDA events: residuals, scaling, factorization, solves, steps)
 * picks the winner.  With cache_path non-NULL the result is looked up first
 * in that text file under a key made of the factor precision, the cohort size,
 * total n, m, nnz(P), nnz(A) and cone counts per family, and appended to it
 * after a run (one line per key).  out: the chosen fields, its ms per
 * iteration and that of *base's own fields.  Host-side analysis is repeated
 * per candidate, so the call takes seconds for large problems.  Errors: as
 * clr_batch_setup; CLR_E_INVALID for iters < 1. */
typedef struct {
  int32_t small_front_max, amalgamation, big_front_schedule;
  int32_t candidates;        /* candidates timed (0 when read from the cache) */
  double ms_per_iter;        /* chosen fields */
  double base_ms_per_iter;   /* *base's fields (-1 when read from the cache) */
  int32_t from_cache, pad;
} clr_tune_result;
int clr_autotune(int32_t nprob, const clr_problem* probs, const clr_settings* base, int32_t iters,
                 const char* cache_path, clr_tune_result* out);

typedef struct clr_server clr_server;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int64_t cohorts;          /* cohorts formed so far */
  int64_t max_cohort_seen;  /* largest cohort formed */
  int64_t peak_bytes;       /* device memory held by live cohorts, peak */
  int64_t bytes_in_use;     /* ... now */
} clr_server_stats;

/* Start a server on the current CUDA device.  st: settings of every solve
 * (NULL: clr_default_settings(.., 64); use_graph is forced on).  device_bytes
 * is the admission budget: a new cohort is formed while the live cohorts hold
 * less than it (or none is live).  One builder forms and uploads cohorts one
 * at a time and a cohort's size is known once it is on the device, so the
 * peak (clr_server_stats.peak_bytes) can exceed the budget by at most the
 * last cohort admitted.  A cohort whose upload fails (the device has no room:
 * CLR_E_OOM or CLR_E_CUDA) hands that error to each of its tickets.  Errors:
 * CLR_E_INVALID (zero budget, max_cohort < 1, max_active < 1), CLR_E_CUDA. */
int clr_server_create(clr_server** out, size_t device_bytes, int32_t max_cohort, int32_t max_active,
                      const clr_settings* st);

/* Queue one problem (deep-copied; never waits for the GPU).  *ticket
 * identifies it in clr_server_poll / clr_server_wait.  Input errors found by
 * the analysis are returned by poll/wait for that ticket. */
int clr_server_submit(clr_server* sv, const clr_problem* p, uint64_t* ticket);

/* CLR_E_AGAIN while the ticket is not done.  Once done: its result as
 * clr_get_solution gives it (any output may be NULL), or its error code; the
 * ticket is then released (CLR_E_INVALID afterwards).  In info, setup_s is the
 * time from submit to the end of the host analysis and solve_s the latency
 * from submit to the result being readable. */
int clr_server_poll(clr_server* sv, uint64_t ticket, double* x, double* sl, double* z, clr_info* info);

/* As clr_server_poll, waiting up to timeout_s seconds (CLR_E_TIMEOUT). */
int clr_server_wait(clr_server* sv, uint64_t ticket, double timeout_s, double* x, double* sl, double* z,
                    clr_info* info);

int clr_server_get_stats(clr_server* sv, clr_server_stats* out);

/* Stop the threads, wait for work on the device, free everything.  Tickets
 * not yet done are dropped. */
int clr_server_destroy(clr_server* sv);

/* Device timing and launch count of the last clr_solve (CLR_E_STATE before it). */
int clr_get_perf(const clr_solver* s, clr_perf* out);

/* Export the symbolic factorization for inspection.  perm (length N): the
 * fill-reducing order, perm[k] = KKT index eliminated k-th (KKT index i < n is
 * x_i, n + j is row j of the reordered constraint block).  sn_ptr (n_supernodes
 * + 1): columns of supernode J are perm-positions sn_ptr[J] .. sn_ptr[J+1]-1.
 * sn_parent (n_supernodes): parent supernode or -1.  row_ptr (n_supernodes+1)
 * and rows (row_ptr[n_supernodes]): perm-positions of the rows of each front,
 * its own columns first.  row_perm (the caller's m): reordered constraint row i is caller
 * row row_perm[i].  Any output may be NULL; sizes from clr_get_symbolic_stats
 * (rows total: query with rows == NULL and read *rows_len). */
int clr_get_symbolic(const clr_solver* s, int64_t* perm, int64_t* sn_ptr, int64_t* sn_parent, int64_t* row_ptr,
                     int64_t* rows, int64_t* rows_len, int64_t* row_perm);

/* Equilibration scalings: D (n), E (the caller's m, reordered rows), c (1 value). */
int clr_get_scaling(const clr_solver* s, double* D, double* E, double* c);

/* Per-iteration log of the last solve, up to cap rows of 12 doubles:
 * iter, mu, pcost, dcost, res_primal, res_dual, gap, alpha_a, sigma,
 * alpha_c, ir_steps, tau.  Returns the number of rows written in *rows. */
int clr_get_history(const clr_solver* s, double* out, int32_t cap, int32_t* rows);

/* Bind the solver's work to a CUDA stream (cudaStream_t passed as void*;
 * NULL = the solver's own stream).  The stream must outlive the solver. */
int clr_set_stream(clr_solver* s, void* cuda_stream);

/* Device-memory allocator used by every later clr_setup (process-wide).
 * alloc returns NULL on failure; both are called on the setup thread.
 * Passing NULL functions restores cudaMalloc/cudaFree. */
typedef void* (*clr_alloc_fn)(size_t bytes, void* ctx);
typedef void (*clr_free_fn)(void* ptr, size_t bytes, void* ctx);
int clr_set_allocator(clr_alloc_fn alloc_fn, clr_free_fn free_fn, void* ctx);

void clr_free(clr_solver* s);
const char* clr_error_string(int code);
const char* clr_status_string(int status);
/* Text of the last CUDA error seen by this thread ("" if none). */
const char* clr_last_cuda_error(void);

/* ------------------------------------------------------------------------
 * Step-level entry points.  Each runs one step of the per-iteration device
 * path on its own, on host arrays, so that it can be checked against a
 * reference.  They allocate and free their own device memory per call.
 * ------------------------------------------------------------------------ */

/* Scaling matrices H of one cone list (Alg. 1 step 4, Appendix A): for each
 * cone, its dense dim x dim block H (row-major) is written to H_out at the
 * cone's packed offset sum(dim_i^2).  s, z: length sum(dim).  mu: global
 * complementarity measure used by the exp/pow BFGS scaling.  Zero cones give
 * H = 0.  The cones are not reordered. */
int clr_cones_scaling(const clr_cone* cones, int32_t ncones, const double* s, const double* z, double mu,
                      double* H_out);

/* Largest step alpha <= alpha_max with s + alpha ds in K and z + alpha dz in
 * K* (Sec. 2.2), over the given cones, as the affine step computes it
 * (symmetric cones exact, exp/pow by backtracking with ratio 0.8 from the
 * symmetric-cone value). */
int clr_cones_step_length(const clr_cone* cones, int32_t ncones, const double* s, const double* z,
                          const double* ds, const double* dz, double alpha_max, double* alpha_out);

/* Combined-step d_s of Eq. ds-correction-step for every cone, with the
 * Mehrotra (symmetric) or third-order (exp/pow) correction built from the
 * affine directions ds_a, dz_a.  Zero cones give 0. */
int clr_cones_combined_ds(const clr_cone* cones, int32_t ncones, const double* s, const double* z,
                          const double* ds_a, const double* dz_a, double sigma_mu, double* ds_out);

/* Device time of the cone steps on one cone list, for roofline measurement
 * (the scaling of Alg. 1 step 4 with the KKT block write, the step-length
 * ratio tests of Sec. 2.2, the combined-step d_s of Eq. ds-correction-step).
 * s, z, ds, dz (length sum(dim), caller-owned host arrays) are uploaded once;
 * each step then runs `reps` (>= 1) times back to back after one untimed
 * call, bracketed by CUDA events on the default stream, and out receives the
 * mean device milliseconds per call.  The exp/pow line search is not timed
 * (step_ms covers the symmetric families).  Inputs larger than the L2 cache
 * (~129 MB) give DRAM-bound figures.  out->rows = sum(dim), out->kkt_values =
 * number of packed H entries written per scaling call.  Errors:
 * CLR_E_INVALID (null pointers, reps < 1), CLR_E_UNSUPPORTED (cone list as
 * for clr_cones_scaling), CLR_E_OOM, CLR_E_CUDA. */
typedef struct {
  double scaling_ms, step_ms, combined_ds_ms;
  int64_t rows, kkt_values;
} clr_cone_times;
int clr_cones_time(const clr_cone* cones, int32_t ncones, const double* s, const double* z, const double* ds,
                   const double* dz, double mu, int32_t reps, clr_cone_times* out);

/* Sparse LDL^T of a symmetric quasi-definite matrix (Sec. 3.6) with the same
 * supernodal factorization the solver uses.  K_lower: lower triangle (CSC,
 * diagonal present in every column).  signs[N]: +1 or -1, the expected sign
 * of each pivot (dynamic regularisation replaces a pivot d with
 * sign*dyn_reg_delta when sign*d <= dyn_reg_eps).  No static regularisation
 * is added here.  order: NULL for the library's AMD ordering, else a
 * caller permutation (order[k] = index eliminated k-th).  factor_bits 64/32/16.
 * x_out = K^{-1} rhs (no refinement); D_out (optional, N): pivots in the
 * caller's numbering.  big_front_schedule: the large fronts' schedule, as the
 * setting of the same name (0 per-panel launches; dataflow: 1 tensor-core
 * updates for factor_bits 32 on the levels chosen at setup, 2 CUDA-core
 * products, 3 tensor-core updates on every level). */
int clr_ldl_solve(const clr_csc* K_lower, const double* signs, const int64_t* order, int32_t factor_bits,
                  double dyn_reg_eps, double dyn_reg_delta, const double* rhs, double* x_out, double* D_out,
                  int32_t* dyn_hits_out, int32_t big_front_schedule);

/* Arithmetic peaks of the current GPU measured by the library's own kernels,
 * the denominators of the benchmark's roofline fractions (the paper reports
 * none): FP64 and FP32 FMA throughput of the CUDA cores, and tcgen05 tensor
 * throughput for kind::tf32 and kind::f16 with BF16 operands (FP32
 * accumulation; M = 128, N = 256 MMAs issued back to back from shared-memory
 * operands, one CTA per SM).  Each figure is the best of `reps` (>= 1)
 * launches timed with CUDA events on `stream` (cudaStream_t as void*, NULL:
 * legacy default stream); *_ms are those launches' durations.  Allocates and
 * frees a few MB of scratch.  tc_timeouts != 0 means a tensor-core wait ran out
 * (the tensor figures are then invalid).  Errors: CLR_E_INVALID (out NULL,
 * reps < 1), CLR_E_CUDA.  Changes no clock or other GPU setting. */
typedef struct {
  double fp64_fma_tflops, fp32_fma_tflops, tf32_tc_tflops, bf16_tc_tflops;
  double fp64_ms, fp32_ms, tf32_ms, bf16_ms;
  int32_t sms, tc_timeouts;
} clr_peaks;
int clr_probe_peaks(int32_t reps, void* stream, clr_peaks* out);

/* ------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory where they need a
 * solve -- code running while a CUDA graph is being captured (cudaMalloc is
 * not allowed there), real-time control loops that must not allocate after
 * start-up (e.g. one small KKT solve per period of a predictive controller),
 * and plug-ins whose device memory belongs to a host framework.
 * ------------------------------------------------------------------------ */

/* Largest system order accepted by clr_dense_ldl_solve_noalloc. */
#define CLR_NOALLOC_MAX_N 128

/* Dense LDL^T (natural order, no pivoting, dynamic regularisation as in
 * clr_ldl_solve) and solve of one quasi-definite system, on DEVICE pointers:
 *   K      N x N column-major, lower triangle read (upper ignored)
 *   signs  N expected pivot signs (> 0: +1, else -1)
 *   rhs    N;  x (output) N, may be the same buffer as rhs (in-place solve);
 *          D (output, may be NULL) N pivots; K must not overlap x or D
 *   dyn_hits (output, device int, may be NULL): pivots replaced
 *   stream cudaStream_t as void* (NULL: legacy default stream)
 * No device memory is allocated or freed: the working matrix lives in one
 * static device array of CLR_NOALLOC_MAX_N^2 doubles (128 KiB) that every GPU
 * loading the library keeps until the process exits.  N > CLR_NOALLOC_MAX_N
 * gives CLR_E_UNSUPPORTED; N < 0 or a NULL required pointer CLR_E_INVALID.
 * The first call on a device resolves that array's address with
 * cudaGetSymbolAddress (with the device current); make the first call on each
 * device before any stream capture.  All calls on a device share the array:
 * calls whose kernels overlap on the GPU (different streams without ordering)
 * race on it.  Asynchronous: the results are ready when the stream is. */
int clr_dense_ldl_solve_noalloc(const double* K, const double* signs, int32_t N, const double* rhs, double* x,
                                double* D, double dyn_reg_eps, double dyn_reg_delta, int32_t* dyn_hits,
                                void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CLR_H */
