/*
 * Plain FP64 CPU oracle for restarted PDHG on linear programs.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Method (Applegate, Hinder, Lu, Lubin, "Faster first-order primal-dual
 * methods for linear programming using restarts and sharpness"):
 *
 *   LP saddle point, Eq. (LP-Lag), widened to box bounds and row signs:
 *       L(x, y) = c^T x - y^T A x + b^T y,   x in X = prod [l_j, u_j],
 *       y in Y = prod Y_i,  Y_i = R (equality row), [0, inf) (>= row),
 *       (-inf, 0] (<= row).
 *   PDHG step, Eq. (PDHG-update) with separate primal/dual steps
 *   (footnote of Section 2, primal weight of Section 7):
 *       x+ = proj_X(x - tau (c - A^T y)),
 *       y+ = proj_Y(y + sigma (b - A (2 x+ - x))),
 *       tau = eta / omega, sigma = eta * omega.
 *   Restarted loop with running average, Algorithm 1; adaptive restart
 *   rule, Eq. (adaptive-restart-scheme); normalized duality gap, Eq. (rhorz),
 *   evaluated with the linear trust-region algorithm of Section 6.3 and
 *   Algorithm 2 (Appendix F); KKT error from the system K z >= h of
 *   Eq. (define:K-and-h-for-lp), made relative (see orc_kkt).
 *
 * Conventions: A is m x n in CSR form (row_ptr int64 [m+1], col_idx int32,
 * val double).  Infinite bounds are +-INFINITY.  Everything is double.
 * Compiled with -ffp-contract=off so that a*b+c is two roundings, as
 * written.
 *
 * The loops whose iterations are independent (the row products of A x,
 * the elementwise parts of the PDHG step, the averages) carry OpenMP
 * pragmas.  The tests use the default build, without -fopenmp: the
 * pragmas are ignored and the code runs on one thread exactly as written.
 * A second build with -fopenmp (liboracle_omp.so) is used only to time the
 * oracle on all host cores; the loops it splits have no dependence between
 * iterations (no sum is split), so it computes the same values bit for bit,
 * and A^T y stays a serial scatter over the rows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_ROW_EQ = 0, ORC_ROW_GE = 1, ORC_ROW_LE = 2 };
enum { ORC_RESTART_NONE = 0, ORC_RESTART_FIXED = 1, ORC_RESTART_ADAPTIVE = 2,
       ORC_RESTART_FLEXIBLE = 3, ORC_RESTART_SCHEDULE = 4 };
enum { ORC_OK = 0, ORC_ITER_LIMIT = 4, ORC_NUMERICAL = 5 };

typedef struct {
  int32_t m, n;
  const int64_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
  const double *c, *b, *lb, *ub;
  const int8_t *row_type;
} orc_lp;

/* ---------------------------------------------------------------- basics */

/* out = A x (definition of the matrix-vector product). */
void orc_matvec(const orc_lp *lp, const double *x, double *out) {
  #pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < lp->m; ++i) {
    double s = 0.0;
    for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
      s += lp->val[p] * x[lp->col_idx[p]];
    out[i] = s;
  }
}

/* out = A^T y, accumulated row by row from the CSR form. */
void orc_matvec_t(const orc_lp *lp, const double *y, double *out) {
  for (int32_t j = 0; j < lp->n; ++j) out[j] = 0.0;
  for (int32_t i = 0; i < lp->m; ++i)
    for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
      out[lp->col_idx[p]] += lp->val[p] * y[i];
}

static double clamp(double v, double lo, double hi) {
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

/* Bounds of Y_i: the dual variable of an equality row is free, of a >= row
 * nonnegative, of a <= row nonpositive (sign of y in -y^T(Ax - b)). */
static void dual_bounds(int8_t t, double *lo, double *hi) {
  *lo = (t == ORC_ROW_GE) ? 0.0 : -INFINITY;
  *hi = (t == ORC_ROW_LE) ? 0.0 : INFINITY;
}

static double sq(double v) { return v * v; }

/* ------------------------------------------------------------ PDHG step */

/*
 * One PDHG step, Eq. (PDHG-update) with primal step tau and dual step sigma:
 *   x+ = proj_X(x - tau (c - A^T y))
 *   y+ = proj_Y(y + sigma (b - A (2 x+ - x)))
 * work must hold n + m doubles.
 */
void orc_pdhg_step(const orc_lp *lp, double tau, double sigma, const double *x,
                   const double *y, double *x_new, double *y_new,
                   double *work) {
  double *aty = work;          /* [n] */
  double *ax = work + lp->n;   /* [m] */
  orc_matvec_t(lp, y, aty);
  #pragma omp parallel for schedule(static)
  for (int32_t j = 0; j < lp->n; ++j)
    x_new[j] = clamp(x[j] - tau * (lp->c[j] - aty[j]), lp->lb[j], lp->ub[j]);
  /* extrapolated point 2 x+ - x, stored temporarily in aty */
  #pragma omp parallel for schedule(static)
  for (int32_t j = 0; j < lp->n; ++j) aty[j] = 2.0 * x_new[j] - x[j];
  orc_matvec(lp, aty, ax);
  #pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < lp->m; ++i) {
    double lo, hi;
    dual_bounds(lp->row_type[i], &lo, &hi);
    y_new[i] = clamp(y[i] + sigma * (lp->b[i] - ax[i]), lo, hi);
  }
}

/* ------------------------------------------------ power iteration (Sec. 7) */

/* SplitMix64 output function (Steele, Lea, Flood 2014; the form in Vigna's
 * public-domain splitmix64.c), used as a counter-based generator: the j-th
 * value is the mix of (j + 1) * golden gamma. */
static uint64_t splitmix64_at(uint64_t j) {
  uint64_t z = (j + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/*
 * Largest singular value of A by power iteration on A^T A (Section 7 names
 * power iteration without details).  Start at v_j = 0.5 + u_j, u_j uniform
 * in [0, 1) from SplitMix64 at counter j (a start orthogonal to the top
 * singular vector, as the all-ones vector is for symmetric network
 * matrices, would converge to a smaller value), normalized;
 * v <- A^T A v / ||A^T A v||; stop when the Rayleigh estimate
 * ||A v||^2 changes by less than tol relative, or after max_iter steps.
 */
double orc_sigma_max(const orc_lp *lp, int32_t max_iter, double tol) {
  int32_t n = lp->n, m = lp->m;
  double *v = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
  double *av = malloc(sizeof(double) * (m > 0 ? m : 1));
  double nv = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    v[j] = 0.5 + (double)(splitmix64_at((uint64_t)j) >> 11) * 0x1.0p-53;
    nv += v[j] * v[j];
  }
  nv = sqrt(nv);
  for (int32_t j = 0; j < n; ++j) v[j] /= nv;
  double est = 0.0;
  for (int32_t it = 0; it < max_iter; ++it) {
    orc_matvec(lp, v, av);
    double ray = 0.0; /* v^T A^T A v with ||v|| = 1 */
    for (int32_t i = 0; i < m; ++i) ray += av[i] * av[i];
    orc_matvec_t(lp, av, w);
    double nw = 0.0;
    for (int32_t j = 0; j < n; ++j) nw += w[j] * w[j];
    nw = sqrt(nw);
    int done = (it > 0 && fabs(ray - est) <= tol * ray);
    est = ray;
    if (nw == 0.0 || done) break;
    for (int32_t j = 0; j < n; ++j) v[j] = w[j] / nw;
  }
  free(v); free(w); free(av);
  return sqrt(est);
}

/* ----------------------------------------- linear trust region (Alg. 2) */

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/*
 * Algorithm 2 (Appendix F): minimize g^T zt over { zt >= l, ||zt - z|| <= r }
 * for g > 0, l <= z, Euclidean norm.  The optimum is
 * zt(lambda) = max(z - lambda g, l) for the largest lambda with
 * ||zt(lambda) - z|| <= r (Section 6.3).  Breakpoints
 * lambda_hat_i = (z_i - l_i) / g_i; median elimination as in Algorithm 2,
 * with the median taken as the lower median of a sorted copy.
 *
 * Writes the multiplier to *lambda_out (INFINITY when the full clamp zt = l
 * is inside the ball) and the minimizer to zt.  N may be 0.
 */
void orc_trust_region_lower(int64_t N, const double *z, const double *l,
                            const double *g, double r, double *zt,
                            double *lambda_out) {
  double *lam = malloc(sizeof(double) * (N > 0 ? N : 1));
  double *buf = malloc(sizeof(double) * (N > 0 ? N : 1));
  int64_t *I = malloc(sizeof(int64_t) * (N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i)
    lam[i] = isinf(l[i]) ? INFINITY : (z[i] - l[i]) / g[i];

  /* if ||l - z|| <= r return zt(inf) = l */
  double full = 0.0;
  for (int64_t i = 0; i < N; ++i) full += sq(l[i] - z[i]);
  double lambda;
  if (full <= r * r) {
    lambda = INFINITY;
  } else {
    double lam_lo = 0.0, lam_hi = INFINITY;
    double f_lo = 0.0, f_hi = 0.0;
    int64_t nI = 0;
    for (int64_t i = 0; i < N; ++i) {
      if (lam[i] <= lam_lo) f_lo += sq(l[i] - z[i]);
      if (lam[i] >= lam_hi) f_hi += sq(g[i]);
      if (lam_lo < lam[i] && lam[i] < lam_hi) I[nI++] = i;
    }
    while (nI > 0) {
      for (int64_t k = 0; k < nI; ++k) buf[k] = lam[I[k]];
      qsort(buf, (size_t)nI, sizeof(double), cmp_double);
      double lam_mid = buf[(nI - 1) / 2];
      /* f_mid = ||zt(lam_mid) - z||^2 */
      double f_mid = f_lo + f_hi * lam_mid * lam_mid;
      for (int64_t k = 0; k < nI; ++k) {
        int64_t i = I[k];
        double d = fmax(z[i] - lam_mid * g[i], l[i]) - z[i];
        f_mid += d * d;
      }
      int64_t keep = 0;
      if (f_mid < r * r) {
        lam_lo = lam_mid;
        for (int64_t k = 0; k < nI; ++k) {
          int64_t i = I[k];
          if (lam[i] <= lam_mid) f_lo += sq(l[i] - z[i]);
          else I[keep++] = i;
        }
      } else {
        lam_hi = lam_mid;
        for (int64_t k = 0; k < nI; ++k) {
          int64_t i = I[k];
          if (lam[i] >= lam_mid) f_hi += sq(g[i]);
          else I[keep++] = i;
        }
      }
      nI = keep;
    }
    lambda = sqrt((r * r - f_lo) / f_hi);
  }
  for (int64_t i = 0; i < N; ++i)
    zt[i] = isinf(lambda) ? l[i] : fmax(z[i] - lambda * g[i], l[i]);
  *lambda_out = lambda;
  free(lam); free(buf); free(I);
}

/*
 * Two-sided linear trust region: minimize g^T zt over
 * { lo <= zt <= hi, ||zt - z|| <= r }.  Reduced to Algorithm 2's form as in
 * Section 6.3: a coordinate with g_i > 0 only moves down (its lower bound
 * is the binding one); a coordinate with g_i < 0 is mirrored
 * (z_i -> -z_i, g_i -> -g_i, l_i -> -hi_i); a coordinate with g_i = 0
 * does not change the objective and stays at z_i.
 * Returns the multiplier; writes the minimizer to zt.
 */
double orc_trust_region(int64_t N, const double *z, const double *lo,
                        const double *hi, const double *g, double r,
                        double *zt) {
  double *zz = malloc(sizeof(double) * (N > 0 ? N : 1));
  double *ll = malloc(sizeof(double) * (N > 0 ? N : 1));
  double *gg = malloc(sizeof(double) * (N > 0 ? N : 1));
  double *out = malloc(sizeof(double) * (N > 0 ? N : 1));
  int64_t *map = malloc(sizeof(int64_t) * (N > 0 ? N : 1));
  int64_t K = 0;
  for (int64_t i = 0; i < N; ++i) {
    zt[i] = z[i];
    if (g[i] > 0.0) {
      zz[K] = z[i]; ll[K] = lo[i]; gg[K] = g[i]; map[K++] = i;
    } else if (g[i] < 0.0) {
      zz[K] = -z[i]; ll[K] = -hi[i]; gg[K] = -g[i]; map[K++] = i;
    }
  }
  double lambda;
  orc_trust_region_lower(K, zz, ll, gg, r, out, &lambda);
  for (int64_t k = 0; k < K; ++k) {
    int64_t i = map[k];
    zt[i] = (g[i] > 0.0) ? out[k] : -out[k];
  }
  free(zz); free(ll); free(gg); free(out); free(map);
  return lambda;
}

/* ------------------------------------- normalized duality gap, Eq. (rhorz) */

/*
 * rho_r(z) for the LP Lagrangian with the weighted Euclidean norm
 * ||(x, y)||_w^2 = omega ||x||^2 + ||y||^2 / omega (the Euclidean norm of
 * the rescaled space of the Section 2 footnote; plain Euclidean at
 * omega = 1, the norm Section 6.2 and Section 7 use for PDHG).
 *
 * By Eq. (bilinear-0), L(x, yt) - L(xt, y) = F(z)^T (z - zt) with
 * F(z) = (c - A^T y, A x - b), so the maximizer of Eq. (rhorz-pos) is the
 * minimizer of the linear trust region (Section 6.3) with objective F(z)
 * over W_r(z) = Z intersected with the ball.  The problem is solved in the
 * rescaled coordinates x' = sqrt(omega) x, y' = y / sqrt(omega), where the
 * objective becomes F_x / sqrt(omega), F_y sqrt(omega).
 *
 * r == 0 returns 0 (Proposition "avoid trivial setting": a zero radius
 * means z is optimal and rho_0 is never needed, Section 6.1).
 */
double orc_normalized_gap(const orc_lp *lp, double omega, const double *x,
                          const double *y, double r) {
  int32_t n = lp->n, m = lp->m;
  if (r == 0.0) return 0.0;
  int64_t N = (int64_t)n + m;
  double *aty = malloc(sizeof(double) * (n > 0 ? n : 1));
  double *ax = malloc(sizeof(double) * (m > 0 ? m : 1));
  double *z = malloc(sizeof(double) * N), *lo = malloc(sizeof(double) * N);
  double *hi = malloc(sizeof(double) * N), *g = malloc(sizeof(double) * N);
  double *zt = malloc(sizeof(double) * N);
  orc_matvec_t(lp, y, aty);
  orc_matvec(lp, x, ax);
  double sw = sqrt(omega);
  for (int32_t j = 0; j < n; ++j) {
    double F = lp->c[j] - aty[j];
    z[j] = sw * x[j];
    lo[j] = sw * lp->lb[j];
    hi[j] = sw * lp->ub[j];
    g[j] = F / sw;
  }
  for (int32_t i = 0; i < m; ++i) {
    double F = ax[i] - lp->b[i];
    double dlo, dhi;
    dual_bounds(lp->row_type[i], &dlo, &dhi);
    z[n + i] = y[i] / sw;
    lo[n + i] = dlo / sw;
    hi[n + i] = dhi / sw;
    g[n + i] = F * sw;
  }
  orc_trust_region(N, z, lo, hi, g, r, zt);
  double gap = 0.0; /* F(z)^T (z - zt) in rescaled coordinates */
  for (int64_t k = 0; k < N; ++k) gap += g[k] * (z[k] - zt[k]);
  free(aty); free(ax); free(z); free(lo); free(hi); free(g); free(zt);
  return gap / r;
}

/* Weighted distance ||(x - x0, y - y0)||_w. */
double orc_weighted_dist(int32_t n, int32_t m, double omega, const double *x,
                         const double *y, const double *x0, const double *y0) {
  double sx = 0.0, sy = 0.0;
  for (int32_t j = 0; j < n; ++j) sx += sq(x[j] - x0[j]);
  for (int32_t i = 0; i < m; ++i) sy += sq(y[i] - y0[i]);
  return sqrt(omega * sx + sy / omega);
}

/* ----------------------------------------------------------- KKT error */

/*
 * KKT residuals of (x, y).  For standard form (Ax = b, x >= 0) these are
 * the three blocks of (h - K z)^+ of Eq. (define:K-and-h-for-lp) that are
 * not identically zero on X x Y; for general bounds and row signs:
 *   primal residual r_p = ||v||, v_i = (Ax - b)_i on EQ rows,
 *       min(0, (Ax - b)_i) on GE rows, max(0, (Ax - b)_i) on LE rows;
 *   reduced costs lam = c - A^T y; Lambda_j = {0} for a free column,
 *       [0, inf) with only l_j finite, (-inf, 0] with only u_j finite,
 *       R with both finite; dual residual r_d = ||lam - proj_Lambda(lam)||;
 *   primal objective p = c^T x; dual objective
 *       d = b^T y + sum_j (l_j [lt_j]^+ - u_j [lt_j]^-), lt = proj_Lambda(lam),
 *       finite bounds only;
 *   relative KKT = max(r_p / (1 + ||b||), r_d / (1 + ||c||),
 *                      |p - d| / (1 + |p| + |d|)).
 * out = {r_p, r_d, p, d, relative KKT}.
 */
void orc_kkt(const orc_lp *lp, const double *x, const double *y,
             double *out) {
  int32_t n = lp->n, m = lp->m;
  double *aty = malloc(sizeof(double) * (n > 0 ? n : 1));
  double *ax = malloc(sizeof(double) * (m > 0 ? m : 1));
  orc_matvec_t(lp, y, aty);
  orc_matvec(lp, x, ax);
  double rp = 0.0, rd = 0.0, p = 0.0, d = 0.0, nb = 0.0, nc = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    double v = ax[i] - lp->b[i];
    if (lp->row_type[i] == ORC_ROW_GE) v = fmin(v, 0.0);
    if (lp->row_type[i] == ORC_ROW_LE) v = fmax(v, 0.0);
    rp += v * v;
    d += lp->b[i] * y[i];
    nb += lp->b[i] * lp->b[i];
  }
  for (int32_t j = 0; j < n; ++j) {
    double lam = lp->c[j] - aty[j];
    int lf = isfinite(lp->lb[j]), uf = isfinite(lp->ub[j]);
    double lo = lf ? 0.0 : (uf ? -INFINITY : 0.0);
    double hi = uf ? 0.0 : (lf ? INFINITY : 0.0);
    if (lf && uf) { lo = -INFINITY; hi = INFINITY; }
    double lt = clamp(lam, lo, hi);
    rd += sq(lam - lt);
    p += lp->c[j] * x[j];
    nc += lp->c[j] * lp->c[j];
    if (lf && lt > 0.0) d += lp->lb[j] * lt;
    if (uf && lt < 0.0) d += lp->ub[j] * lt;
  }
  rp = sqrt(rp);
  rd = sqrt(rd);
  double rel = fmax(rp / (1.0 + sqrt(nb)), rd / (1.0 + sqrt(nc)));
  rel = fmax(rel, fabs(p - d) / (1.0 + fabs(p) + fabs(d)));
  out[0] = rp; out[1] = rd; out[2] = p; out[3] = d; out[4] = rel;
  free(aty); free(ax);
}

/* ------------------------------------------- restarted PDHG, Algorithm 1 */

typedef struct {
  double eta, omega, beta, tol;
  int64_t max_iter;
  int32_t check_every;    /* K: restart and termination checks at k % K == 0 */
  int32_t restart_scheme; /* ORC_RESTART_* */
  int64_t tau0;           /* first restart length (n = 0 branch) */
  int64_t fixed_len;      /* restart length of the fixed-frequency scheme */
  const int8_t *schedule; /* SCHEDULE: restart at check c iff schedule[c - 1] != 0 */
  int64_t nschedule;
} orc_options;

typedef struct {
  int64_t iters, restarts, inner_t;
  int32_t status;   /* ORC_OK / ORC_ITER_LIMIT / ORC_NUMERICAL */
  int32_t returned; /* 0: average, 1: current iterate */
  double rho_stored;
  double kkt_avg[5], kkt_cur[5];
  int64_t n_checks;
} orc_info;

/*
 * Algorithm 1 with PDHG as the primal-dual step.
 *
 * State arrays (all caller-owned; on entry x, y hold z^{0,0}):
 *   x[n], y[m]      current iterate z^{n,t}
 *   xbar, ybar      running average zbar^{n,t} (line "average" of Alg. 1)
 *   x0, y0          restart point z^{n,0}
 * On return every array holds the final state; info->returned names the
 * solution candidate (0: the average xbar/ybar, 1: the current x/y), the
 * one that met the tolerance at the deciding check, else the one with the
 * smaller relative KKT error at the last check.
 *
 * Every check_every iterations (Section 7: 30) the relative KKT error is
 * evaluated at the average and at the current iterate (Table 3 counts a
 * run as solved when either candidate meets the tolerance; here the
 * average wins ties), and the
 * restart rule runs:
 *   ADAPTIVE, Eq. (adaptive-restart-scheme): restart when
 *     rho_{||zbar - z^{n,0}||}(zbar) <= beta * rho_{||z^{n,0} - z^{n-1,0}||}(z^{n,0})
 *   for n >= 1, and when t >= tau0 for n = 0.  The right-hand gap is the gap
 *   computed at the restart that produced z^{n,0} (same point, same
 *   radius), so it is stored instead of recomputed.
 *   FLEXIBLE, Eq. (flexible-restart-scheme): before the test, the average is
 *   replaced by the current iterate when the latter has the smaller gap.
 *   FIXED, Eq. (define:t-star): restart when t >= fixed_len.
 *   NONE: never restart.
 *   SCHEDULE: restart at the checks the caller flags (decisions held
 *   fixed, so that the unrolled map is a fixed composition of steps).
 * On restart z^{n+1,0} <- zbar and the iteration continues from zbar.
 *
 * trace (optional, may be NULL): per check 6 doubles
 *   {iteration, rho, restarted, kkt_avg_rel, kkt_cur_rel, radius},
 *   up to trace_cap checks.
 */
int32_t orc_solve(const orc_lp *lp, const orc_options *opt, double *x,
                  double *y, double *xbar, double *ybar, double *x0,
                  double *y0, orc_info *info, double *trace,
                  int64_t trace_cap) {
  int32_t n = lp->n, m = lp->m;
  double tau = opt->eta / opt->omega, sigma = opt->eta * opt->omega;
  double *xn = malloc(sizeof(double) * (n > 0 ? n : 1));
  double *yn = malloc(sizeof(double) * (m > 0 ? m : 1));
  double *work = malloc(sizeof(double) * ((int64_t)n + m + 1));
  memcpy(x0, x, sizeof(double) * n);
  memcpy(y0, y, sizeof(double) * m);
  memcpy(xbar, x, sizeof(double) * n);
  memcpy(ybar, y, sizeof(double) * m);
  int64_t k = 0, t = 0, restarts = 0, checks = 0;
  double rho_stored = NAN;
  int32_t status = ORC_ITER_LIMIT, returned = 0;
  double ka[5] = {NAN, NAN, NAN, NAN, INFINITY};
  double kc[5] = {NAN, NAN, NAN, NAN, INFINITY};
  while (k < opt->max_iter) {
    orc_pdhg_step(lp, tau, sigma, x, y, xn, yn, work);
    memcpy(x, xn, sizeof(double) * n);
    memcpy(y, yn, sizeof(double) * m);
    /* zbar^{n,t+1} = t/(t+1) zbar^{n,t} + 1/(t+1) z^{n,t+1} */
    #pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < n; ++j)
      xbar[j] = ((double)t * xbar[j] + x[j]) / (double)(t + 1);
    #pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < m; ++i)
      ybar[i] = ((double)t * ybar[i] + y[i]) / (double)(t + 1);
    ++t;
    ++k;
    if (k % opt->check_every != 0) continue;
    ++checks;
    orc_kkt(lp, xbar, ybar, ka);
    orc_kkt(lp, x, y, kc);
    if (!isfinite(ka[4]) || !isfinite(kc[4])) { status = ORC_NUMERICAL; break; }
    if (ka[4] <= opt->tol || kc[4] <= opt->tol) {
      status = ORC_OK;
      returned = (ka[4] <= opt->tol) ? 0 : 1;
      break;
    }
    double r = orc_weighted_dist(n, m, opt->omega, xbar, ybar, x0, y0);
    double rho = NAN;
    int restart = 0;
    if (opt->restart_scheme == ORC_RESTART_ADAPTIVE ||
        opt->restart_scheme == ORC_RESTART_FLEXIBLE) {
      rho = orc_normalized_gap(lp, opt->omega, xbar, ybar, r);
      if (opt->restart_scheme == ORC_RESTART_FLEXIBLE) {
        double rc = orc_weighted_dist(n, m, opt->omega, x, y, x0, y0);
        double rho_c = orc_normalized_gap(lp, opt->omega, x, y, rc);
        if (rho_c < rho) {
          memcpy(xbar, x, sizeof(double) * n);
          memcpy(ybar, y, sizeof(double) * m);
          rho = rho_c;
          r = rc;
        }
      }
      restart = (restarts == 0) ? (t >= opt->tau0) : (rho <= opt->beta * rho_stored);
    } else if (opt->restart_scheme == ORC_RESTART_FIXED) {
      restart = (t >= opt->fixed_len);
    } else if (opt->restart_scheme == ORC_RESTART_SCHEDULE) {
      /* restart decisions given from outside (the unrolled map with its
         decisions held fixed, for finite differences of the adjoint) */
      restart = (checks <= opt->nschedule) && opt->schedule[checks - 1] != 0;
    }
    if (trace && checks <= trace_cap) {
      double *row = trace + 6 * (checks - 1);
      row[0] = (double)k; row[1] = rho; row[2] = restart;
      row[3] = ka[4]; row[4] = kc[4]; row[5] = r;
    }
    if (restart) {
      memcpy(x0, xbar, sizeof(double) * n);
      memcpy(y0, ybar, sizeof(double) * m);
      memcpy(x, xbar, sizeof(double) * n);
      memcpy(y, ybar, sizeof(double) * m);
      rho_stored = rho;
      ++restarts;
      t = 0;
    }
  }
  if (status == ORC_ITER_LIMIT && checks > 0) returned = (ka[4] <= kc[4]) ? 0 : 1;
  info->iters = k;
  info->restarts = restarts;
  info->inner_t = t;
  info->status = status;
  info->returned = returned;
  info->rho_stored = rho_stored;
  info->n_checks = checks;
  memcpy(info->kkt_avg, ka, sizeof ka);
  memcpy(info->kkt_cur, kc, sizeof kc);
  free(xn); free(yn); free(work);
  return status;
}
