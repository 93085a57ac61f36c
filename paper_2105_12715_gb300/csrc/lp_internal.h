// Internal declarations shared by the two translation units of liblp.so
// (lp_kernels.cu: device code and launchers; lp_api.cu: the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lpg {

constexpr int kWarp = 32;
constexpr int kBlock = 256;           // threads per block of the SpMV kernels
constexpr int kWarpsPerBlock = kBlock / kWarp;
constexpr int kBuckets = 256;         // buckets per pass of the multiplier search
constexpr int kSearchPasses = 8;      // 8 x 8 bits cover a 64-bit key
constexpr int kHistWarps = 4;         // warps per block of the histogram kernel
constexpr uint64_t kNoKey = ~0ull;    // element that takes no part in the search
constexpr int32_t kRunning = -1;      // DevState::status while iterating

// One copy of A (or A^T) in the library's device layout.  Rows are in the
// library's permuted order: rows [0, nlong) are "long" and stored CSR-style
// (one warp per row); rows [nlong, nrows) are grouped in slices of 32
// consecutive rows stored column-major inside the slice (SELL-32): element
// k of the slice's lane l sits at slice_ptr[s] + 32 k + l, padded with
// zero values up to the slice's longest row.
struct SellMat {
  int32_t nrows;
  int32_t ncols;
  int32_t nlong;
  int32_t nslices;
  const int64_t *long_ptr;   // [nlong + 1]
  const int32_t *long_idx;
  const double *long_val;
  const int64_t *slice_ptr;  // [nslices + 1], element offsets, multiples of 32
  const int32_t *idx;
  const double *val;
};

// Reduced quantities of one check.  _A: running average, _C: current
// iterate.  GAP*: data of the multiplier search (finite-breakpoint sums and
// the squared objective of coordinates that never reach a bound).
enum Quantity {
  Q_RP2_A, Q_RP2_C, Q_RD2_A, Q_RD2_C, Q_POBJ_A, Q_POBJ_C, Q_DOBJ_A, Q_DOBJ_C,
  Q_RRX_A, Q_RRY_A, Q_D2_A, Q_GD_A, Q_G2INF_A,
  Q_RRX_C, Q_RRY_C, Q_D2_C, Q_GD_C, Q_G2INF_C,
  Q_BAD, NQ
};

// State of one search for the trust-region multiplier lambda* of
// Section 6.3 (largest lambda with ||zt(lambda) - z||^2 <= r^2).
struct LSearch {
  double r2;        // r^2
  double f_lo;      // sum d^2 over breakpoints known to lie below lambda*
  double e_lo;      // sum |g| d over the same coordinates
  double f_hi;      // sum g^2 over breakpoints known to lie above lambda*
  unsigned long long prefix;  // fixed high bits of lambda*'s bracket
  int32_t done;
  int32_t pad;
  double lambda;    // result (INFINITY: full clamp)
  double rho_r;     // result: rho * r = sum_clamped |g| d + lambda f_hi
};

struct DevState {
  double tau, sigma, omega, beta, tol;
  double norm_b, norm_c;
  int64_t t0;          // inner iterations since the restart, at block start
  int64_t iters;       // iterations since create / set_state
  int64_t checks;
  int64_t restarts;    // n of Algorithm 1
  int64_t tau0, fixed_len;
  int32_t K;
  int32_t scheme;
  int32_t status;      // kRunning or a final lp_status
  int32_t returned;    // 0: average, 1: current iterate
  int32_t restart_now; // decision of the last check, read by the copy kernel
  int32_t use_cur;     // flexible scheme: current iterate replaced the average
  double rho_stored, last_rho, last_r;
  double kkt_a[5], kkt_c[5];
  LSearch ls[2];       // [0] average, [1] current iterate (flexible scheme)
  int64_t trace_count;
  int32_t trace_cap;
  int32_t given_radius; // standalone gap evaluation: radius taken from r_given
  double r_given;
  // power iteration
  double pw_est, pw_nw;
  int32_t pw_done;
  int32_t pw_iters;
  int32_t pw_max;
  int32_t pad2;
  double pw_tol;
};

// Device arrays of one problem, permuted order.
struct DevVecs {
  double *c, *lb, *ub, *b;
  int8_t *row_type;
  double *x, *xhat, *xbar, *x0;
  double *y, *ybar, *y0;
};

// Scratch of the check and of the multiplier search.
struct CheckScratch {
  double *partials;        // [NQ][pstride]
  int32_t pstride;
  int32_t cols_grid, rows_grid;
  uint64_t *keys[2];       // [n + m] per candidate
  double *d2[2], *g2[2], *gd[2];
  double *hpart;           // [2][hist_grid][4][kBuckets]
  int32_t hist_grid;
};

// ---- launchers (lp_kernels.cu) ----
void launch_primal_step(const SellMat &AT, const DevVecs &v, DevState *st,
                        const double *w, int k, cudaStream_t s);
void launch_dual_step(const SellMat &A, const DevVecs &v, DevState *st,
                      const double *w, int k, cudaStream_t s);
void launch_check(const SellMat &A, const SellMat &AT, const DevVecs &v,
                  DevState *st, double *w, const CheckScratch &cs, int n,
                  int m, int nsearch, double *trace, bool decide,
                  cudaStream_t s);
void launch_advance(DevState *st, double *w, int r, cudaStream_t s);
void launch_spmv(const SellMat &A, const double *v, double *out, cudaStream_t s,
                 DevState *st_guard);
void launch_power_iteration_step(const SellMat &A, const SellMat &AT,
                                 double *v, double *av, double *w,
                                 DevState *st, double *partials, int pstride,
                                 int grid, int n, int m, cudaStream_t s);
void launch_gather(double *out, const double *in, const int32_t *perm, int64_t n,
                   cudaStream_t s);
void launch_scatter(double *out, const double *in, const int32_t *perm, int64_t n,
                    cudaStream_t s);
void launch_project(const DevVecs &v, int n, int m, cudaStream_t s);
void launch_fill(double *p, double val, int64_t n, cudaStream_t s);
void launch_weights(DevState *st, double *w, cudaStream_t s);
void launch_norms(const DevVecs &v, DevState *st, double *partials, int pstride,
                  int grid, int n, int m, cudaStream_t s);
int check_grid_for(const SellMat &A, int num_sms);

}  // namespace lpg
