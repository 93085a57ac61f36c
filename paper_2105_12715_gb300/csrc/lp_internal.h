// Internal declarations shared by the translation units of liblp.so
// (lp_kernels.cu: device code and launchers; lp_api.cu: the C ABI;
// lp_batch.cu: the batched solver).
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

// Per-slice metadata of the sliced layout (see SellMat).
struct SliceInfo {
  int64_t off;    // element offset of the slice (multiple of 32)
  int32_t row0;   // first row of the slice (permuted order)
  int32_t len_g;  // (steps << 3) | log2(G): steps of 32 elements, G lanes per row
};

// One copy of A (or A^T) in the library's device layout.  Rows are in the
// library's permuted order (longest first).  Consecutive rows of similar
// length form a slice handled by one warp: each row gets G lanes
// (G = 1, 2, ..., 32, chosen from the row length so that a lane walks about
// 8-15 elements), so a slice holds 32 / G rows.  Element k of the slice's
// i-th row sits at off + 32 * (k / G) + i * G + (k % G): every warp-wide
// load of the matrix stream is 32 consecutive elements.  Rows are padded
// with zero values up to the slice's longest row (a multiple of G).
// info has nslices + 1 entries; the last one holds the end offset and nrows.
//
// Split rows: a row longer than the split length (a whole-warp row) is cut
// into chunks of at most that many elements, one warp slice each (G = 32),
// so that no warp walks a very long row alone.  These chunk slices come
// first (the split rows are the longest); split[s] says which chunk slice s
// is.  Each chunk writes its partial sums to split_part; the last chunk of
// a row to finish (arrival counter split_cnt[first], reset by it) adds the
// partials in chunk order and runs the row's epilogue.
struct SplitSlice {
  int32_t chunk;    // chunk index within its row
  int32_t nchunks;  // chunks of the row
  int32_t first;    // slice index of the row's chunk 0 (its counter index)
  int32_t begin;    // element offset of the chunk within the row
};
struct SellMat {
  int32_t nrows;
  int32_t ncols;
  int32_t nslices;
  int32_t n_warp_rows;      // rows with G = 32 (a whole warp per row)
  const SliceInfo *info;    // [nslices + 1]
  const int32_t *idx;
  const double *val;
  const float *valf;        // FP32 copy of val (mixed precision), or null
  int32_t nsplit = 0;                  // chunk slices (slices 0 .. nsplit - 1)
  const SplitSlice *split = nullptr;   // [nsplit]
  double *split_part = nullptr;        // [2 nsplit] partial sums of the chunks
  int32_t *split_cnt = nullptr;        // [nsplit] arrival counters (at index first), zero between passes
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
  // sigma_max estimator (power iteration or Lanczos): estimate of sigma_max^2,
  // steps taken, done flag
  double pw_est, pw_nw;
  int32_t pw_done;
  int32_t pw_iters;
  int32_t pw_max;
  int32_t pad2;
  double pw_tol;
  // cross-block reductions (last-block pattern; counters return to 0)
  double tot[NQ];
  unsigned int fin_counter;
  unsigned int sel_counter[2];
  int32_t mixed;        // 1: mixed-precision iterations (MixVecs)
  double mix_s;         // scale of the current correction
};

// Device arrays of one problem, permuted order.
struct DevVecs {
  double *c, *lb, *ub, *b;
  long long *lbk, *ubk;  // order keys of lb, ub (integer-pipe clamps)
  int8_t *row_type;
  double *x, *xhat, *xbar, *x0;
  double *y, *ybar, *y0;
};

// Mixed-precision state (FP32 iterations on scaled corrections).  Within an
// outer loop of Algorithm 1 the iterate is z = z^{n,0} + dz / s, where
// z^{n,0} (x0, y0, FP64) is the restart point and s the scale chosen at the
// restart; dz runs PDHG in FP32 on the correction data below, which is
// re-formed in FP64 at every restart (residual correction).
struct MixVecs {
  float *cf, *lf, *uf;     // [n] s (c - A^T y0), s (l - x0), s (u - x0)
  float *dx, *dxhat;       // [n]
  double *dxbar;           // [n] FP64 average of dx
  float *bf, *ylo, *yhi;   // [m] s (b - A x0), s (Y_lo - y0), s (Y_hi - y0)
  float *dy;               // [m]
  double *dybar;           // [m]
  double *lam[2];          // [n] c - A^T y of the average / current candidate (from the check)
  double *gy[2];           // [m] A x - b of the average / current candidate
};

// Adjoint state of the unrolled iteration (FP64).
struct AdjVecs {
  double *ax, *axb, *ac, *v;  // [n]
  double *ay, *ayb, *ab, *u;  // [m]
};

// Coefficients of the Lanczos tridiagonal matrix (sigma_max estimate):
// alpha[0..cap-1] on the diagonal, beta[0..cap-1] below it.
struct LanczosT {
  double *alpha, *beta;
  int32_t cap;
};
constexpr int kLanczosMax = 1024;  // longest Lanczos run (steps)

// Scratch of the check and of the multiplier search.
struct CheckScratch {
  double *partials;        // [NQ][pstride]
  int32_t pstride;
  int32_t cols_grid, rows_grid;
  uint64_t *keys[2];       // [n + m] per candidate
  double *d2[2], *g2[2], *gd[2];
  double *hpart;           // [2][hist_grid][4][kBuckets]
  double *btot;            // [2][4][kBuckets] bucket totals of the current pass
  int32_t hist_grid;
  double *pair_x, *pair_y; // [2n], [2m]: (xbar, x) and (ybar, y) interleaved for the check's
                           // gathers (16-byte aligned); null: gather the two vectors apart
  // multiplier search candidate lists: per histogram warp cand_cap slots (elements of
  // the bracket after the first pass) and a count; null: every pass scans all elements
  int32_t *cand[2], *ccnt[2];
  int64_t cand_cap;
};

// Launch with programmatic stream serialization: the kernel may be scheduled
// while its predecessor in the stream finishes (it must call pdl_enter()
// before reading the predecessor's results).  Works inside stream capture.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), int grid, int block, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---- device layout construction (lp_layout.cu) ----
// Input error bits of lay_validate (and lay_dup).
enum : int32_t {
  kLayBadRowPtr = 1, kLayBadColIdx = 2, kLayBadVal = 4, kLayBadC = 8, kLayBadBounds = 16,
  kLayBadB = 32, kLayBadRowType = 64, kLayDuplicate = 128
};
// Runs of equal lane count in the length-sorted order: run q holds rows
// [g0[q], g0[q] + ...) with 2^lg[q] lanes per row; its slices start at
// slice index s0[q] (runs in order, empty runs left out).
struct LayRuns {
  int32_t count;
  int32_t lg[6];
  int64_t g0[6];
  int64_t s0[6];
};
void lay_validate(const int32_t *rp, int32_t m, int64_t nnz, const int32_t *ci, int32_t n,
                  const double *v, const double *c, const double *lb, const double *ub,
                  const double *b, const int8_t *rt, int32_t *flags, int nsm, cudaStream_t s);
void lay_row_of(const int32_t *rp, int32_t m, int64_t nnz, int32_t *row_of, int nsm,
                cudaStream_t s);
void lay_iota(int32_t *a, int64_t count, int nsm, cudaStream_t s);
int64_t lay_scan_scratch(int64_t len);
void lay_exclusive_scan(const int64_t *in, int64_t len, int64_t *out, int64_t *sums,
                        cudaStream_t s);
int64_t lay_radix_tiles(int64_t count);
void lay_radix_sort(uint32_t *keys, int32_t *pay, uint32_t *keys_alt, int32_t *pay_alt,
                    int64_t count, int bits, int64_t *gh, int64_t *goff, int64_t *sums,
                    cudaStream_t s, bool *in_alt);
void lay_col_count(const int32_t *ci, int64_t nnz, int64_t *cnt, int nsm, cudaStream_t s);
void lay_csc_gather(const int32_t *pos, const int32_t *row_of, const double *v, int64_t nnz,
                    int32_t *ri, double *cv, int nsm, cudaStream_t s);
void lay_dup(const uint32_t *col, const int32_t *ri, int64_t nnz, int32_t *flags, int nsm,
             cudaStream_t s);
template <class P>
void lay_lengths(const P *ptr, int32_t count, int64_t *mx, uint32_t *key, int64_t mxv,
                 int64_t *hist, int nsm, cudaStream_t s);
void lay_inverse(const int32_t *perm, int32_t count, int32_t *inv, int nsm, cudaStream_t s);
// Slices of one operator: the chunk slices of the nsr split rows first
// (nsplit of them, SplitSlice records in split; nch and cstart are nsr-long
// scratch), then the runs of ordinary rows from slice nsplit on.
template <class P>
void lay_slices(const LayRuns &runs, const int32_t *perm, const P *ptr, int64_t nslices,
                int32_t nrows, SliceInfo *info, int64_t *width, int64_t *off, int64_t *sums,
                int nsm, cudaStream_t s, int64_t nsr, int64_t nsplit, int32_t split_len,
                SplitSlice *split, int64_t *nch, int64_t *cstart);
template <class P>
void lay_fill(const SliceInfo *info, int64_t nslices, const int32_t *perm, const P *ptr,
              const int32_t *ind, const double *val, const int32_t *relabel, int32_t *idx,
              double *vout, float *vf, int nsm, cudaStream_t s, const SplitSlice *split,
              int64_t nsplit, int32_t split_len);
void lay_vectors(const int32_t *perm_x, int32_t n, const double *c, const double *lb,
                 const double *ub, double *pc, double *pl, double *pu, long long *lk,
                 long long *uk, const int32_t *perm_y, int32_t m, const double *b,
                 const int8_t *rt, double *pb, int8_t *prt, int nsm, cudaStream_t s);

// ---- launchers (lp_kernels.cu) ----
void launch_primal_step(const SellMat &AT, const DevVecs &v, DevState *st,
                        const double *w, int k, int unroll, int grid_cap, cudaStream_t s);
void launch_dual_step(const SellMat &A, const DevVecs &v, DevState *st,
                      const double *w, int k, int unroll, int grid_cap, cudaStream_t s);
void launch_check(const SellMat &A, const SellMat &AT, const DevVecs &v,
                  DevState *st, double *w, const CheckScratch &cs, int n,
                  int m, int nsearch, double *trace, bool decide,
                  cudaStream_t s, const MixVecs *mv = nullptr);
void launch_advance(DevState *st, double *w, int r, cudaStream_t s);
void launch_spmv(const SellMat &A, const double *v, double *out, cudaStream_t s,
                 DevState *st_guard);
void launch_power_iteration_step(const SellMat &A, const SellMat &AT,
                                 double *v, double *av, double *w,
                                 DevState *st, double *partials, int pstride,
                                 int grid, int n, int m, cudaStream_t s);
void launch_lanczos_step(const SellMat &A, const SellMat &AT, const double *v, double *av,
                         double *w, const double *vprev, DevState *st, const LanczosT &T, int k,
                         bool evaluate, double *partials, int pstride, int grid, int n,
                         cudaStream_t s);
void launch_start_vector(const int32_t *perm, double *v, int n, double *partials, int pstride,
                         int grid, cudaStream_t s);
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
int split_grid(const SellMat &A);
void launch_primal_mix(const SellMat &AT, const MixVecs &mv, DevState *st, const double *w,
                       int k, int unroll, cudaStream_t s);
void launch_dual_mix(const SellMat &A, const MixVecs &mv, const DevVecs &v, DevState *st,
                     const double *w, int k, int unroll, cudaStream_t s);
void launch_combine(const DevVecs &v, const MixVecs &mv, DevState *st, int n, int m, int force,
                    cudaStream_t s);
void launch_recenter(const DevVecs &v, const MixVecs &mv, DevState *st, int n, int m, int force,
                     cudaStream_t s);
void launch_residuals(const SellMat &A, const SellMat &AT, const DevVecs &v, const MixVecs &mv,
                      int n, int m, cudaStream_t s);
void launch_forward_masked(const SellMat &A, const SellMat &AT, const DevVecs &v, double tau,
                           double sigma, double w, uint8_t *mx, uint8_t *my, cudaStream_t s);
void launch_adjoint_step(const SellMat &A, const SellMat &AT, const AdjVecs &a,
                         const uint8_t *mx, const uint8_t *my_prev, double tau, double sigma,
                         double w, double w_prev, int has_prev, cudaStream_t s);
void launch_adjoint_block_start(const AdjVecs &a, const uint8_t *my_last, int restarted,
                                double sigma, double w, int n, int m, cudaStream_t s);

}  // namespace lpg
