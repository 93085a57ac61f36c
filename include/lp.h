/*
 * lp.h -- C ABI of the GB300 restarted-PDHG linear-programming library
 * (liblp.so, built for sm_103a).
 *
 * Method: Applegate, Hinder, Lu, Lubin, "Faster first-order primal-dual
 * methods for linear programming using restarts and sharpness".
 *
 * Problem (Eq. LP-Lag, widened to box bounds and signed rows):
 *     min_{x in X} max_{y in Y}  L(x, y) = c^T x - y^T A x + b^T y,
 *     X = prod_j [lb_j, ub_j],  Y = prod_i Y_i with
 *     Y_i = R          for LP_ROW_EQ  ((A x)_i =  b_i),
 *     Y_i = [0, inf)   for LP_ROW_GE  ((A x)_i >= b_i),
 *     Y_i = (-inf, 0]  for LP_ROW_LE  ((A x)_i <= b_i).
 *
 * Conventions for every entry point:
 *   - A is m x n, given in CSR form with int32 indices; nnz < 2^31.
 *   - Array arguments of lp_create may be host or device memory (detected
 *     per pointer); all other array arguments are DEVICE pointers unless
 *     the name starts with host_.  Device arrays are read/written in stream
 *     order on the given stream.
 *   - cuda_stream is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.
 *   - The library copies every input at lp_create; the caller may free or
 *     reuse its buffers once lp_create returns.  Outputs go to caller
 *     buffers.  The handle owns all device memory it allocates.
 *   - Errors are reported as lp_status codes, never as exceptions; the
 *     message of the last error on the calling thread is lp_last_error().
 *   - A handle may be used by one host thread at a time.
 */
#ifndef LP_GB300_LP_H
#define LP_GB300_LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_problem *lp_handle;

typedef enum {
  LP_OK = 0,
  LP_ERR_INVALID_ARG = 1, /* bad size, pointer, CSR structure, NaN, bound */
  LP_ERR_CUDA = 2,        /* a CUDA runtime call failed                  */
  LP_ERR_OOM = 3,         /* device or host allocation failed            */
  LP_ITER_LIMIT = 4,      /* max_iter reached before the tolerance       */
  LP_ERR_NUMERICAL = 5,   /* NaN or Inf met in an iterate or residual    */
  LP_ERR_TIMEOUT = 6,     /* reserved: a bounded device wait expired     */
  LP_ERR_NOT_SOLVED = 7   /* no solve has run on this handle yet         */
} lp_status;

enum { LP_ROW_EQ = 0, LP_ROW_GE = 1, LP_ROW_LE = 2 };

/* Arithmetic of the iterations.  FP64: everything in double.  MIXED: the
 * PDHG iterations run in FP32 (FP32 matrix values, iterates, FP32
 * accumulation) on a scaled correction dz = s (z - z^{n,0}) around the
 * restart point of Algorithm 1; the running average, the KKT and
 * normalized-gap checks, the restart point and the correction data
 * (residuals formed at every restart) stay in FP64.  Re-forming the
 * correction at each restart is a residual-correction refinement, so the
 * solution reaches FP64 accuracy. */
enum { LP_PRECISION_FP64 = 0, LP_PRECISION_MIXED = 1 };

/* Restart schemes of Section 4 (fixed frequency, Eq. define:t-star;
 * adaptive, Eq. adaptive-restart-scheme) and Section 7 (no restarts; the
 * flexible scheme of Remark "Flexible restarts"). */
enum {
  LP_RESTART_NONE = 0,
  LP_RESTART_FIXED = 1,
  LP_RESTART_ADAPTIVE = 2,
  LP_RESTART_FLEXIBLE = 3
};

/* Estimators of sigma_max(A) for eta = 0.9 / sigma_max(A) (Section 7).
 * Both work on A^T A from the same start vector: the power iteration's
 * Rayleigh quotient, or the largest Ritz value of the Lanczos process
 * (the same quantity from the same products, converging in far fewer
 * steps; both approach sigma_max^2 from below). */
enum { LP_SIGMA_POWER = 0, LP_SIGMA_LANCZOS = 1 };

typedef struct {
  double beta;            /* restart contraction factor (Remark on the choice of beta: e^-1) */
  int32_t check_every;    /* K: restart/termination checks every K iterations (Section 7 uses 30) */
  int32_t restart_scheme; /* LP_RESTART_* */
  int64_t tau0;           /* first restart length for n = 0 (iterations; 0 = K) */
  int64_t fixed_len;      /* restart length of LP_RESTART_FIXED (iterations) */
  double omega;           /* primal weight: tau = eta/omega, sigma = eta*omega (Section 7) */
  double eta;             /* base step; 0 = 0.9 / sigma_max(A) (estimator: sigma_method) */
  int32_t power_iters;    /* step cap of the sigma_max estimator (default 5000) */
  double power_tol;       /* relative change of the sigma_max^2 estimate to stop (1e-10) */
  int64_t max_iter;       /* iteration limit of one lp_solve call */
  int32_t long_row_threshold; /* rows at least this long get a whole warp (32 lanes) (512) */
  int32_t trace_capacity; /* per-check trace rows kept on device (65536) */
  int32_t spmv_unroll;    /* gathers in flight per lane, column pass (A^T y): 2, 4, 8; negative
                             values -2, -4 add a software pipeline over the matrix stream;
                             adding 100 (or -100 for negative values) caps the registers for
                             higher occupancy (-2) */
  int32_t spmv_unroll_rows; /* the same for the row pass (A xhat) (-4) */
  int32_t lane_steps;     /* rows longer than single_lane_max get the fewest lanes G (power of
                             two <= 32) with ceil(len / G) <= lane_steps (16) */
  int32_t single_lane_max; /* rows of at most this many elements get one lane each (64) */
  int32_t spmv_mode;      /* reserved, must be 0 */
  int32_t precision;      /* LP_PRECISION_FP64 (default) or LP_PRECISION_MIXED */
  int32_t lane_auto;      /* > 0: per matrix, halve single_lane_max and lane_steps until the
                             layout has at least lane_auto x (SM count) slices (warps); 0: use
                             the given lane policy as is (32) */
  int32_t autotune;       /* 1: at lp_create, time every unroll variant of the column and row
                             passes on this problem and keep the fastest (overrides spmv_unroll
                             and spmv_unroll_rows; results do not depend on the variant: every
                             variant sums each row in the same order); 0: use them as given (1) */
  int32_t sigma_method;   /* estimator of sigma_max(A) when eta = 0: LP_SIGMA_LANCZOS (default;
                             at most min(power_iters, 1024) steps) or LP_SIGMA_POWER (Section 7's
                             power iteration); both stop when the estimate of sigma_max^2 changes
                             by at most power_tol (relative) */
  int32_t device_layout;  /* 1: build the library's layout (CSC copy, length orders, slices) on the
                             GPU (default); 0: on the host cores.  Both give the same arrays.
                             lp_batch_create always builds on the host */
  int32_t split_row_len;  /* a row of A or A^T with a whole warp (long_row_threshold or more
                             elements) longer than this is cut into chunks of at most this many
                             elements, one warp each, whose partial sums the last chunk to finish
                             adds in chunk order: no warp walks a very long row alone.  A positive
                             multiple of 32, or 0 for never (512 = 32 x lane_steps: a chunk takes no
                             more steps than an ordinary slice) */
} lp_options;

typedef struct {
  int64_t iters;        /* iterations since the last lp_create / lp_set_state */
  int64_t restarts;     /* outer-loop count n of Algorithm 1 */
  int64_t checks;       /* restart/termination checks run */
  int32_t status;       /* lp_status of the last lp_solve / lp_iterate */
  int32_t returned;     /* solution candidate: 0 = running average, 1 = current iterate */
  double kkt_avg[5];    /* at the last check, average:  r_p, r_d, p, d, relative KKT */
  double kkt_cur[5];    /* at the last check, current iterate: same layout */
  double eta, sigma_max, omega, tau, sigma;
  double rho_stored;    /* gap stored at the last restart, Eq. (adaptive-restart-scheme) */
  double last_rho;      /* normalized duality gap at the last check */
  double last_radius;   /* its radius ||zbar - z^{n,0}|| */
  int64_t nnz_padded;   /* stored nonzeros of one copy of A including padding */
  int32_t n_long_rows, n_long_cols; /* rows of A / of A^T handled by a whole warp */
  double setup_ms[4];   /* lp_create phases: input copy + validation, host layout (CSC,
                           permutations, slices), device upload, sigma_max estimate */
  int32_t spmv_unroll, spmv_unroll_rows; /* kernel variants in use (tuned or given) */
  int32_t sigma_steps;  /* steps of the sigma_max estimator (0 when eta was given) */
  int32_t graph_kernels; /* kernel launches per replay of the graph of K iterations + check
                            (0 until the first lp_solve / lp_iterate builds it) */
  int32_t n_split_slices; /* chunk slices of split rows in A and A^T together (split_row_len) */
} lp_info;

/* Defaults: beta = e^-1, K = 64, ADAPTIVE, tau0 = K, omega = 1, eta = 0
 * (auto), power_iters = 5000, power_tol = 1e-10, max_iter = 1e7, autotune = 1,
 * sigma_method = LP_SIGMA_LANCZOS, device_layout = 1, split_row_len = 512. */
void lp_default_options(lp_options *opt);

/*
 * Creates a problem handle (the LP data of Eq. LP-Lag and the setup of
 * Section 7: eta = 0.9 / sigma_max(A), sigma_max estimated on A^T A as
 * opt->sigma_method says, unless opt->eta > 0).
 *   row_ptr[m+1], col_idx[nnz], val[nnz]: CSR of A; row_ptr[0] = 0,
 *     nondecreasing, row_ptr[m] = nnz; col_idx in [0, n); a column may
 *     appear at most once per row (duplicates are rejected).
 *   c[n], lb[n], ub[n]: objective and bounds; lb = -INFINITY / ub = INFINITY
 *     mean no bound; lb <= ub, lb < INFINITY, ub > -INFINITY.
 *   b[m], row_type[m] (LP_ROW_*): right-hand side and row sense.
 *   opt: may be NULL for defaults.
 * Every value must be finite except the infinite bounds.  The starting
 * point z^{0,0} is zero projected onto X x Y.  Returns LP_ERR_INVALID_ARG
 * on any violation (message in lp_last_error), LP_ERR_OOM, LP_ERR_CUDA.
 */
lp_status lp_create(int32_t m, int32_t n, int64_t nnz, const int32_t *row_ptr,
                    const int32_t *col_idx, const double *val, const double *c,
                    const double *b, const double *lb, const double *ub,
                    const int8_t *row_type, const lp_options *opt,
                    void *cuda_stream, lp_handle *out);

/*
 * Runs Algorithm 1 (restarted PDHG) from the handle's current state until
 * the relative KKT error of the running average or of the current iterate
 * is <= tol at a check (every K iterations; the average wins ties), or
 * until opt.max_iter further iterations.  Returns LP_OK, LP_ITER_LIMIT,
 * LP_ERR_NUMERICAL, LP_ERR_INVALID_ARG (tol <= 0) or LP_ERR_CUDA.  Blocks
 * the host until the solve ends (one 4-byte read per check).
 */
lp_status lp_solve(lp_handle h, double tol, void *cuda_stream);

/*
 * Enqueues n_checks blocks of K PDHG iterations, each followed by a check
 * (KKT, normalized gap, restart decision), without any host
 * synchronization.  Blocks after convergence (relative KKT <= tol) do no
 * work.  The iteration count is not capped by max_iter.  Returns LP_OK or
 * an error of the enqueue.
 */
lp_status lp_iterate(lp_handle h, int32_t n_checks, double tol, void *cuda_stream);

/* Copies the solution candidate (see lp_info.returned) into x[n], y[m]
 * (device or host pointers); LP_ERR_NOT_SOLVED before any solve. */
lp_status lp_get_solution(lp_handle h, double *x, double *y, void *cuda_stream);

/* Copies the full iteration state of Algorithm 1 -- current iterate (x, y),
 * running average (xbar, ybar), restart point (x0, y0) -- in the caller's
 * (unpermuted) order; any pointer may be NULL to skip it.  Host or device
 * pointers.  Synchronizes the stream. */
lp_status lp_get_state(lp_handle h, double *x, double *y, double *xbar,
                       double *ybar, double *x0, double *y0, void *cuda_stream);

/* Warm start: sets z^{0,0} = proj_{X x Y}(x, y) (host or device pointers,
 * NULL = zero) and resets the restart state and counters. */
lp_status lp_set_state(lp_handle h, const double *x, const double *y, void *cuda_stream);

/* Counters, step sizes and the residuals of the last check (host struct). */
lp_status lp_get_info(lp_handle h, lp_info *host_info);

/* Per-check log (Figure 2's series): 6 doubles per check
 * {iteration, rho, restarted, relKKT(avg), relKKT(cur), radius}, oldest
 * first, at most capacity rows; *host_count receives the number written. */
lp_status lp_get_trace(lp_handle h, double *host_rows, int64_t capacity,
                       int64_t *host_count);

/*
 * Normalized duality gap, Eq. (rhorz), of the LP at (x, y) for radius r
 * under the weighted norm ||(x, y)||^2 = omega ||x||^2 + ||y||^2 / omega:
 * the linear trust region of Section 6.3 solved by a parallel search over
 * the multiplier (Algorithm 2's answer).  x[n], y[m] (host or device) in the
 * caller's order, inside X x Y.  *host_rho receives rho_r; r = 0 gives 0.
 * Allocates and frees its own scratch (split-row counters included), so it
 * may overlap a solve on the same handle.  Synchronizes the stream.
 */
lp_status lp_normalized_gap(lp_handle h, const double *x, const double *y,
                            double r, double *host_rho, void *cuda_stream);

/*
 * lp_normalized_gap without any device allocation.  The paper has no
 * counterpart; this entry point exists for callers that cannot let a
 * library allocate device memory (a latency-bound host loop, since cudaFree
 * synchronizes the device; a process whose framework already reserved
 * nearly all device memory; code that must leave the allocation state
 * untouched while other work is queued).
 * Same arguments as lp_normalized_gap and the same result, bit for bit (the
 * same kernels and reduction order).  Scratch is a fixed 16 MiB device array
 * inside the library (held on every GPU that loads it until exit), so
 * n + m must be <= 262,144; larger problems, or split rows whose partial
 * sums do not fit beside the rest, return LP_ERR_INVALID_ARG.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  All
 * calls of this entry point share the array: two of them that overlap on
 * the GPU race and must be serialized by the caller.  Neither gap entry
 * point writes anything the handle's other calls use (the split-row
 * counters and partial sums are the call's own), so a gap call may overlap
 * a solve on the same handle.  Synchronizes the stream.
 */
lp_status lp_normalized_gap_static(lp_handle h, const double *x, const double *y,
                                   double r, double *host_rho, void *cuda_stream);

/*
 * Profiling hook: enqueues reps launches of one hot-path kernel alone --
 * which = 0: the primal step (column pass, Eq. PDHG-update first line),
 * which = 1: the dual step (row pass, second line) -- on the stream, with
 * the averaging weight of the block's first iteration.  It advances the
 * iterate like real steps do (without checks), so use it on a handle whose
 * solve state no longer matters.  Bracket it with events to time a kernel.
 */
lp_status lp_profile_kernel(lp_handle h, int32_t which, int32_t reps, void *cuda_stream);

/*
 * Primal-weight selection of Section 7: for each omega in host_omegas[count]
 * (each > 0), restart from the projection of zero onto X x Y and run
 * `iters` iterations of PDHG without restarts (iters >= K; checks every K),
 * with tau = eta/omega, sigma = eta*omega; host_kkt[k] receives the smaller
 * relative KKT error of the average and the current iterate at the last
 * check.  Then the handle takes the omega with the smallest value (first on
 * ties; *host_best receives it), its restart scheme is restored, and its
 * state is reset to the projection of zero.  Synchronizes the stream.
 */
lp_status lp_select_omega(lp_handle h, const double *host_omegas, int32_t count,
                          int64_t iters, double *host_kkt, double *host_best,
                          void *cuda_stream);

/*
 * Unrolled forward for differentiation (an extension: the paper has no
 * gradients): runs exactly `iters` iterations of Algorithm 1 from the
 * current state (iters a multiple of K; FP64; adaptive, fixed or no
 * restarts; no termination test), keeping a checkpoint of (x, y, xbar, ybar)
 * and the inner iteration count at the start of every block of K
 * iterations and the restart decision of every check.  The unrolled map's
 * output is the running average (xbar, ybar) after the last check.
 */
lp_status lp_solve_recorded(lp_handle h, int64_t iters, void *cuda_stream);

/*
 * Adjoint of the recorded unrolled map (c, b) -> (xbar, ybar): given
 * dl_dx[n] = dL/dxbar and dl_dy[m] = dL/dybar (NULL = 0), writes
 * dl_dc[n] = dL/dc and dl_db[m] = dL/db (host or device pointers, caller's
 * order).  Restart decisions and the clamp / projection masks of every step
 * are those of the recorded solve (the map is differentiated where they do
 * not change); blocks are recomputed from their checkpoints in reverse
 * order, each adjoint step running the transposed products of the forward
 * step.  Leaves the state of the recorded solve.  LP_ERR_NOT_SOLVED without
 * a recording.  Synchronizes the stream.
 */
lp_status lp_backward(lp_handle h, const double *dl_dx, const double *dl_dy,
                      double *dl_dc, double *dl_db, void *cuda_stream);

/* Releases every resource of the handle (NULL is a no-op).  Waits for the
 * stream of the handle's latest call that enqueued work (and for the
 * handle's own capture stream), not for the whole device; work on other
 * streams that still reads the handle must be finished by the caller. */
void lp_destroy(lp_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char *lp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LP_GB300_LP_H */
