/*
 * lp_batch.h -- C ABI of the batched restarted-PDHG solver in liblp.so:
 * many independent LPs of uneven sizes solved together on one GPU, each
 * with its own restart state (Algorithm 1 per problem: inner count t, outer
 * count n, stored normalized gap, restart point z^{n,0}, status).
 *
 * The paper solves one LP at a time; batching is an extension.  Every
 * problem of a batch follows exactly the iteration of the single-problem
 * solver (include/lp.h) with its own step sizes (eta_k = 0.9 / sigma_max(A_k)
 * unless opt->eta > 0; tau = eta/omega, sigma = eta*omega, Section 7), its
 * own restart checks (every K_k iterations, adaptive restarts of Eq.
 * adaptive-restart-scheme on the normalized duality gap of Section 6.3)
 * and its own termination test (relative KKT error <= tol).
 *
 * Input: the block-diagonal LP of the batch, in the conventions of
 * lp_create (CSR with int32 indices, host or device arrays), plus the
 * problem boundaries host_row_start[count + 1] and host_col_start[count + 1]
 * (host arrays, nondecreasing, starting at 0): problem k owns rows
 * [host_row_start[k], host_row_start[k+1]) and columns
 * [host_col_start[k], host_col_start[k+1]); each of its rows may reference
 * only its own columns.  Vectors (c, lb, ub, b, row_type, solutions) are
 * the concatenation of the problems' vectors in that order.  Every problem
 * needs at least one column; it may have no rows.
 *
 * Launch shape: every PDHG step of the batch is two kernel launches (a
 * column pass and a row pass over the slices of all running problems, from
 * a work list rebuilt at each check), and the checks of all problems due at
 * a block boundary run together (one block of threads per problem for
 * reductions and for the multiplier search).  Problems that have stopped
 * cost nothing.  Errors, streams and ownership as in lp.h.
 */
#ifndef LP_GB300_LP_BATCH_H
#define LP_GB300_LP_BATCH_H

#include "lp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_batch *lp_batch_handle;

/* Choices of the batch's own tuner (lp_batch_create with autotune != 0).
 * Kernel variants are timed on the batch itself; the check period of each
 * size class (problems binned by nonzeros, powers of 4) is the smallest
 * K_base * 2^s (s <= max_k_shift) whose measured check cost is at most
 * check_budget times the cost of the class's K iterations. */
typedef struct {
  int32_t autotune;       /* 0: use opt as given (every problem K = opt->check_every) */
  int32_t max_k_shift;    /* largest s in K = K_base * 2^s (default 2) */
  double check_budget;    /* check cost / iteration cost per class (default 0.05) */
} lp_batch_tuning;

typedef struct {
  int64_t iters;        /* iterations of this problem since create */
  int64_t restarts;     /* outer-loop count n of Algorithm 1 */
  int64_t checks;       /* restart/termination checks run */
  int32_t status;       /* LP_OK (converged), LP_ITER_LIMIT, LP_ERR_NUMERICAL, LP_ERR_NOT_SOLVED */
  int32_t returned;     /* solution candidate: 0 = running average, 1 = current iterate */
  int32_t check_every;  /* K of this problem */
  int32_t size_class;   /* tuner's class (floor(log4(nnz / 64)), clamped to [0, 7]) */
  double kkt_avg[5];    /* at the last check: r_p, r_d, p, d, relative KKT (average) */
  double kkt_cur[5];    /* same for the current iterate */
  double eta, sigma_max, tau, sigma;
  double rho_stored;    /* gap stored at the last restart */
  double last_rho;      /* normalized duality gap at the last check */
  double omega;         /* primal weight in use (tau = eta/omega, sigma = eta*omega) */
  int32_t sigma_steps;  /* steps of the sigma_max estimator (0 when eta was given) */
} lp_batch_problem_info;

typedef struct {
  int32_t count;        /* problems in the batch */
  int32_t running;      /* problems still iterating after the last check */
  int32_t m, n;         /* rows and columns of the whole batch */
  int64_t nnz;          /* nonzeros of the whole batch */
  int64_t blocks;       /* blocks of K_base iterations run by the batch */
  int32_t k_base;       /* K_base = opt->check_every */
  int32_t spmv_unroll, spmv_unroll_rows; /* kernel variants in use (lp_options codes) */
  int32_t grid_cols, grid_rows;          /* blocks of the column / row pass launches */
  int32_t n_classes;    /* size classes present */
  int32_t class_k[8];   /* check period chosen per size class (0 = class empty) */
  double class_iter_ms[8];  /* tuner: one iteration of the class running alone (ms) */
  double class_check_ms[8]; /* tuner: one check of the class running alone (ms) */
  double tune_ms;       /* time spent by the tuner at create */
  double setup_ms;      /* total time of lp_batch_create */
} lp_batch_info;

/* Defaults: autotune = 1, max_k_shift = 2, check_budget = 0.05. */
void lp_batch_default_tuning(lp_batch_tuning *t);

/*
 * Creates a batch.  count >= 1; the arrays are described in the header
 * comment (nnz < 2^31, m + n + 2048 count < 2^31 for the whole batch).
 * opt applies to every problem (NULL = lp_default_options), including
 * opt->precision (LP_PRECISION_MIXED: the mixed-precision iteration of
 * lp.h with a correction scale per problem); spmv_mode must be 0.  tuning
 * may be NULL (no tuning).  The
 * starting point of every problem is zero projected onto X x Y.  Returns
 * LP_ERR_INVALID_ARG on any violation (message in lp_last_error),
 * LP_ERR_OOM, LP_ERR_CUDA, LP_ERR_NUMERICAL (sigma_max of a problem is 0
 * and opt->eta = 0).
 */
lp_status lp_batch_create(int32_t count, const int32_t *host_row_start,
                          const int32_t *host_col_start, int64_t nnz,
                          const int32_t *row_ptr, const int32_t *col_idx,
                          const double *val, const double *c, const double *b,
                          const double *lb, const double *ub, const int8_t *row_type,
                          const lp_options *opt, const lp_batch_tuning *tuning,
                          void *cuda_stream, lp_batch_handle *out);

/* Overrides the check period of every problem (host_k[count], each a
 * positive multiple of K_base = opt->check_every) and resets the iteration
 * state to the projection of zero.  Used to reproduce a schedule. */
lp_status lp_batch_set_check_every(lp_batch_handle h, const int32_t *host_k, void *cuda_stream);

/*
 * Primal-weight selection of Section 7 for every problem at once: for each
 * omega in host_omegas[n_omegas] (each > 0), every problem restarts from the
 * projection of zero and runs `iters` iterations (a multiple of K_base) of
 * PDHG without restarts, with tau = eta_k/omega, sigma = eta_k*omega;
 * host_kkt[k * n_omegas + j] (may be NULL) receives problem k's smaller
 * relative KKT error of the average and the current iterate at its last
 * check for omega j.  Each problem then keeps the omega with its smallest
 * value (first on ties; host_best[count], may be NULL, receives it), the
 * restart scheme is restored, and every problem is reset to the projection
 * of zero.  Synchronizes the stream.
 */
lp_status lp_batch_select_omega(lp_batch_handle h, const double *host_omegas, int32_t n_omegas,
                                int64_t iters, double *host_kkt, double *host_best,
                                void *cuda_stream);

/* Warm start: every problem restarts Algorithm 1 from z^{0,0} = proj(x, y)
 * (concatenated in the caller's order, host or device; NULL = zero), with its
 * counters and restart state reset.  Synchronizes the stream. */
lp_status lp_batch_set_state(lp_batch_handle h, const double *x, const double *y, void *cuda_stream);

/*
 * Runs every problem that has not met the tolerance (and has not failed)
 * until its relative KKT error is <= tol at one of its checks, or until it
 * has run opt.max_iter further iterations.  Returns LP_OK if every problem
 * converged, else LP_ERR_NUMERICAL if one failed, else LP_ITER_LIMIT;
 * per-problem results via lp_batch_get_info.  Blocks the host until the
 * solve ends (one 4-byte read per block of K_base iterations).
 */
lp_status lp_batch_solve(lp_batch_handle h, double tol, void *cuda_stream);

/* Enqueues n_blocks blocks of K_base iterations plus checks, without host
 * synchronization (iteration limits are still applied per problem). */
lp_status lp_batch_iterate(lp_batch_handle h, int32_t n_blocks, double tol, void *cuda_stream);

/* Each problem's solution candidate, concatenated in the caller's order:
 * x[n], y[m] (host or device).  LP_ERR_NOT_SOLVED before any solve. */
lp_status lp_batch_get_solution(lp_batch_handle h, double *x, double *y, void *cuda_stream);

/* Full iteration state (x, y, xbar, ybar, x0, y0), concatenated in the
 * caller's order; NULL pointers are skipped.  Synchronizes the stream. */
lp_status lp_batch_get_state(lp_batch_handle h, double *x, double *y, double *xbar,
                             double *ybar, double *x0, double *y0, void *cuda_stream);

/* Batch summary (host struct) and, if host_problems is not NULL, the
 * first min(capacity, count) problems' results. */
lp_status lp_batch_get_info(lp_batch_handle h, lp_batch_info *host_info,
                            lp_batch_problem_info *host_problems, int32_t capacity);

/*
 * Unrolled forward for differentiation (the paper has no gradients): runs
 * exactly `iters` iterations of every problem from the current state (iters
 * a multiple of K_base = opt->check_every; FP64; adaptive, fixed or no
 * restarts; no termination test), keeping a checkpoint of (x, y, xbar, ybar)
 * of the whole batch and every problem's inner iteration count at the start
 * of every block of K_base iterations, and whether each block's check
 * restarted each problem.  The unrolled map of problem k is its running
 * average (xbar_k, ybar_k) after the last block.  LP_ERR_NUMERICAL if a
 * problem fails during the recording.
 */
lp_status lp_batch_solve_recorded(lp_batch_handle h, int64_t iters, void *cuda_stream);

/*
 * Adjoint of the recorded unrolled maps (c, b) -> (xbar, ybar), all problems
 * at once: given dl_dx[n] = dL/dxbar and dl_dy[m] = dL/dybar (concatenated,
 * caller's order; NULL = 0), writes dl_dc[n] and dl_db[m] (host or device).
 * Per problem this is lp_backward of lp.h: restart decisions and clamp /
 * projection masks held at the recorded ones, blocks recomputed from their
 * checkpoints in reverse order, each adjoint step running the transposed
 * products of the forward step with that problem's tau, sigma and averaging
 * weights.  Leaves the state of the recorded solve.  LP_ERR_NOT_SOLVED
 * without a recording.  Synchronizes the stream.
 */
lp_status lp_batch_backward(lp_batch_handle h, const double *dl_dx, const double *dl_dy,
                            double *dl_dc, double *dl_db, void *cuda_stream);

/* Releases every resource of the batch (NULL is a no-op). */
void lp_batch_destroy(lp_batch_handle h);

#ifdef __cplusplus
}
#endif
#endif /* LP_GB300_LP_BATCH_H */
