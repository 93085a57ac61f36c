// Device code of liblp.so: the restarted-PDHG hot path for sm_103a.
//
// Per iteration (Eq. PDHG-update, tau = eta/omega, sigma = eta*omega):
//   primal_kernel: column pass over A^T (SELL-32 layout, gathers y)
//       x+ = clamp(x - tau (c - A^T y), l, u), xhat = 2 x+ - x,
//       xbar += w_t (x+ - xbar)                     (Algorithm 1, average)
//   dual_kernel:   row pass over A (SELL-32 layout, gathers xhat)
//       y+ = proj_Y(y + sigma (b - A xhat)),  ybar += w_t (y+ - ybar)
// Every K iterations, the check (Section 7: restart and termination tests):
//   check_cols / check_rows: A^T [ybar, y] and A [xbar, x] with fused
//       epilogues for the KKT residuals, the radius ||zbar - z^{n,0}|| and
//       the breakpoints of the linear trust region (Section 6.3);
//   check_finalize: fixed-order reduction, relative KKT, termination;
//   hist / select (x8): search for the trust-region multiplier lambda* over
//       the bit patterns of the breakpoints, 8 bits per pass;
//   check_decide: normalized gap rho = (sum_clamped |g| d + lambda* f_hi)/r,
//       restart rule of Eq. (adaptive-restart-scheme), next averaging weights;
//   restart_copy: z^{n+1,0} <- zbar and z <- zbar on restart.
// All reductions run in a fixed order, so results are bitwise reproducible
// for a given problem and launch configuration.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "lp_internal.h"
#include "spmv_core.cuh"

namespace lpg {
namespace {

// ------------------------------------------------------------ iteration

// SPLIT: the chunk slices of split rows (a second, small launch; see SellMat).
template <int U, bool PIPE, int MINB, bool SPLIT = false>
__global__ void __launch_bounds__(kBlock, MINB) primal_kernel(SellMat AT, const double *__restrict__ y,
                                                        PrimalEpi epi, const DevState *st,
                                                        const double *__restrict__ w, int k) {
  pdl_enter();
  if (st->status != kRunning) return;
  epi.tau = st->tau;
  epi.w = w[k];
  process_all<1, U, PIPE, false, SPLIT>(AT, y, (const double *)nullptr, epi);
}

template <int U, bool PIPE, int MINB, bool SPLIT = false>
__global__ void __launch_bounds__(kBlock, MINB) dual_kernel(SellMat A, const double *__restrict__ xhat,
                                                      DualEpi epi, const DevState *st,
                                                      const double *__restrict__ w, int k) {
  pdl_enter();
  if (st->status != kRunning) return;
  epi.sigma = st->sigma;
  epi.w = w[k];
  process_all<1, U, PIPE, false, SPLIT>(A, xhat, (const double *)nullptr, epi);
}

template <bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) spmv_kernel(SellMat A, const double *__restrict__ v,
                                                      StoreEpi epi, const DevState *st) {
  if (st && (st->status != kRunning || st->pw_done)) return;
  process_all<1, kUnroll, false, false, SPLIT>(A, v, (const double *)nullptr, epi);
}

template <int U, bool PIPE, bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) primal_mix_kernel(SellMat AT, const float *__restrict__ dy,
                                                            PrimalMixEpi epi, const DevState *st,
                                                            const double *__restrict__ w, int k) {
  pdl_enter();
  if (st->status != kRunning) return;
  epi.tau = (float)st->tau;
  epi.w = w[k];
  process_all<1, U, PIPE, false, SPLIT>(AT, dy, (const float *)nullptr, epi);
}

template <int U, bool PIPE, bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) dual_mix_kernel(SellMat A, const float *__restrict__ dxhat,
                                                          DualMixEpi epi, const DevState *st,
                                                          const double *__restrict__ w, int k) {
  pdl_enter();
  if (st->status != kRunning) return;
  epi.sigma = (float)st->sigma;
  epi.w = w[k];
  process_all<1, U, PIPE, false, SPLIT>(A, dxhat, (const float *)nullptr, epi);
}

__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  return fmin(fmax(v, lo), hi);
}

// FP64 iterate and average in original coordinates, z = z^{n,0} + dz / s,
// projected onto X x Y (removes the FP32 rounding of the bounds).
__global__ void combine_kernel(DevVecs v, MixVecs mv, const DevState *st, int n, int m,
                               int force) {
  if (!force && st->status != kRunning) return;
  const double inv = 1.0 / st->mix_s;
  const int64_t total = (int64_t)n + m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const double x0 = v.x0[i], l = v.lb[i], u = v.ub[i];
      v.x[i] = clampd(fma((double)mv.dx[i], inv, x0), l, u);
      v.xbar[i] = clampd(fma(mv.dxbar[i], inv, x0), l, u);
    } else {
      const int64_t r = i - n;
      const int t = v.row_type[r];
      const double lo = (t == 1) ? 0.0 : -INFINITY, hi = (t == 2) ? 0.0 : INFINITY;
      const double y0 = v.y0[r];
      v.y[r] = clampd(fma((double)mv.dy[r], inv, y0), lo, hi);
      v.ybar[r] = clampd(fma(mv.dybar[r], inv, y0), lo, hi);
    }
  }
}

// Re-forms the correction at a restart (or when forced, at set-up): with the
// new restart point z^{n,0} and scale s (set by the restart decision), the
// correction data are s times the FP64 residuals of the chosen candidate,
// and dz starts at 0.  Without a restart, the flexible scheme's
// replacement of the average by the current iterate is applied to dz.
__global__ void recenter_kernel(DevVecs v, MixVecs mv, const DevState *st, int n, int m,
                                int force) {
  if (!force && st->status != kRunning) return;
  const int rs = force ? 1 : st->restart_now, uc = force ? 0 : st->use_cur;
  if (!rs && !uc) return;
  const double s = st->mix_s;
  const double *lam = mv.lam[uc], *gy = mv.gy[uc];
  const int64_t total = (int64_t)n + m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      if (rs) {
        const double x0 = v.x0[i];
        mv.cf[i] = (float)(s * lam[i]);
        mv.lf[i] = (float)(s * (v.lb[i] - x0));
        mv.uf[i] = (float)(s * (v.ub[i] - x0));
        mv.dx[i] = 0.0f;
        mv.dxhat[i] = 0.0f;
        mv.dxbar[i] = 0.0;
      } else {
        mv.dxbar[i] = (double)mv.dx[i];
      }
    } else {
      const int64_t r = i - n;
      if (rs) {
        const int t = v.row_type[r];
        const double lo = (t == 1) ? 0.0 : -INFINITY, hi = (t == 2) ? 0.0 : INFINITY;
        const double y0 = v.y0[r];
        mv.bf[r] = (float)(-s * gy[r]);
        mv.ylo[r] = (float)(s * (lo - y0));
        mv.yhi[r] = (float)(s * (hi - y0));
        mv.dy[r] = 0.0f;
        mv.dybar[r] = 0.0;
      } else {
        mv.dybar[r] = (double)mv.dy[r];
      }
    }
  }
}

// Residuals of the restart point at set-up: lam = c - A^T y0, gy = A x0 - b
// (aty and ax hold A^T y0 and A x0).
__global__ void residuals_kernel(DevVecs v, MixVecs mv, const double *aty, const double *ax,
                                 int n, int m) {
  const int64_t total = (int64_t)n + m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      mv.lam[0][i] = v.c[i] - aty[i];
    } else {
      const int64_t r = i - n;
      mv.gy[0][r] = ax[r] - v.b[r];
    }
  }
}

// ------------------------------------------------------------ adjoint
//
// Reverse mode of the unrolled iteration with the clamp/projection masks of
// a recomputed forward block and the restart decisions held fixed.  With
// adjoints (ax, ay, axb, ayb) of the outputs (x, y, xbar, ybar) of step k:
//   u   = D_y (ay + w ayb),  grad_b += sigma u,  ayb <- (1 - w) ayb
//   v   = D_x (ax + w axb - 2 sigma A^T u),       grad_c -= tau v
//   ax <- v + sigma A^T u,   axb <- (1 - w) axb,  ay <- u + tau A v
// (dual half of Eq. PDHG-update, then the extrapolation 2x+ - x, then the
// primal half; the running average of Algorithm 1 is linear).  A restart
// (x <- xbar) moves ax into axb.

// Forward step with masks, for the recomputation of one block.
template <bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) primal_mask_kernel(SellMat AT,
                                                             const double *__restrict__ y,
                                                             PrimalEpi epi, double tau, double w) {
  epi.tau = tau;
  epi.w = w;
  process_all<1, 2, true, false, SPLIT>(AT, y, (const double *)nullptr, epi);
}

template <bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) dual_mask_kernel(SellMat A,
                                                           const double *__restrict__ xhat,
                                                           DualEpi epi, double sigma, double w) {
  epi.sigma = sigma;
  epi.w = w;
  process_all<1, 4, true, false, SPLIT>(A, xhat, (const double *)nullptr, epi);
}

template <bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) adj_cols_kernel(SellMat AT, const double *__restrict__ u,
                                                          AdjColsEpi epi) {
  process_all<1, 2, true, false, SPLIT>(AT, u, (const double *)nullptr, epi);
}

template <bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) adj_rows_kernel(SellMat A, const double *__restrict__ v,
                                                          AdjRowsEpi epi) {
  process_all<1, 4, true, false, SPLIT>(A, v, (const double *)nullptr, epi);
}

// Start of a reverse block: the restart after the block (if any), then u of
// the block's last step.
__global__ void adj_block_start_kernel(double *ax, double *axb, double *ay, double *ayb, double *u,
                                       double *ab, const uint8_t *my_last, int restarted,
                                       double sigma, double w, int n, int m) {
  const int64_t total = (int64_t)n + m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      if (restarted) {
        axb[i] += ax[i];
        ax[i] = 0.0;
      }
    } else {
      const int64_t r = i - n;
      double a = ay[r], yb = ayb[r];
      if (restarted) {
        yb += a;
        a = 0.0;
        ay[r] = 0.0;
      }
      const double up = my_last[r] ? fma(w, yb, a) : 0.0;
      ab[r] = fma(sigma, up, ab[r]);
      ayb[r] = (1.0 - w) * yb;
      u[r] = up;
    }
  }
}

// ---------------------------------------------------------------- check

// PAIR: v0 holds the two gathered vectors interleaved (pack_pairs_kernel), v1 is unused.
template <class Epi, bool PAIR, bool SPLIT = false>
__global__ void __launch_bounds__(kBlock) check_kernel(SellMat A, const double *__restrict__ v0,
                                                       const double *__restrict__ v1, Epi epi,
                                                       const DevState *st, double *partials,
                                                       int pstride, int poff) {
  if (st->status != kRunning) return;
  if (!st->given_radius) {
    epi.gap_a = (st->scheme == kSchemeAdaptive || st->scheme == kSchemeFlexible);
    epi.gap_c = (st->scheme == kSchemeFlexible);
  }
  const double om = st->omega;
  epi.sw = sqrt(om);
  epi.isw = 1.0 / epi.sw;
#pragma unroll
  for (int i = 0; i < NQ; ++i) epi.q[i] = 0.0;
  process_all<2, kUnroll2, false, PAIR, SPLIT>(A, v0, v1, epi);
  block_reduce_store_mask<NQ>(epi.q, Epi::kUsed | (epi.gap_c ? Epi::kUsedGapC : 0u), partials,
                              pstride, poff + (int)blockIdx.x);
}

// out[2i] = a[i], out[2i+1] = b[i]: the two vectors a check pass gathers,
// interleaved so that one 16-byte gather serves both.
__global__ void __launch_bounds__(kBlock) pack_pairs_kernel(const double *__restrict__ a,
                                                            const double *__restrict__ b,
                                                            int64_t n, double2 *out,
                                                            const DevState *st) {
  if (st->status != kRunning) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2(a[i], b[i]);
}

// Reduction of the check's partial sums: block q sums quantity q over the
// partial blocks in a fixed order (strided per thread, then a fixed tree);
// the last block to finish (threadfence + counter; no waiting) applies the
// termination test and prepares the multiplier search.  Spreading the FP64
// additions over NQ blocks keeps them off a single SM's FP64 pipe.
__global__ void __launch_bounds__(kBlock) check_finalize_kernel(DevState *st,
                                                                const double *partials,
                                                                int pstride, int nparts) {
  if (st->status != kRunning) return;
  __shared__ double red[kBlock];
  __shared__ bool last;
  const int q = blockIdx.x;
  double acc = 0.0;
  for (int p = threadIdx.x; p < nparts; p += kBlock) acc += partials[(size_t)q * pstride + p];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->tot[q] = red[0];
    __threadfence();
    last = (atomicAdd(&st->fin_counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x != 0) return;
  __threadfence();
  st->fin_counter = 0u;
  double tot[NQ];
  const volatile double *vt = st->tot;
  for (int i = 0; i < NQ; ++i) tot[i] = vt[i];
  const double om = st->omega;
  if (st->given_radius) {  // standalone gap evaluation
    init_search(st->ls[0], st->r_given, tot[Q_D2_A], tot[Q_GD_A], tot[Q_G2INF_A]);
    return;
  }
  st->iters += st->K;
  st->checks += 1;
  kkt_from(tot, Q_RP2_A, Q_RD2_A, Q_POBJ_A, Q_DOBJ_A, st->norm_b, st->norm_c, st->kkt_a);
  kkt_from(tot, Q_RP2_C, Q_RD2_C, Q_POBJ_C, Q_DOBJ_C, st->norm_b, st->norm_c, st->kkt_c);
  const double ra = st->kkt_a[4], rc = st->kkt_c[4];
  st->ls[0].done = 1;
  st->ls[1].done = 1;
  if (tot[Q_BAD] > 0.0 || !isfinite(ra) || !isfinite(rc)) {
    st->status = kStatusNumerical;
    return;
  }
  if (ra <= st->tol) {
    st->status = kStatusOK;
    st->returned = 0;
    return;
  }
  if (rc <= st->tol) {
    st->status = kStatusOK;
    st->returned = 1;
    return;
  }
  st->returned = (ra <= rc) ? 0 : 1;
  if (st->scheme == kSchemeAdaptive || st->scheme == kSchemeFlexible) {
    const double r = sqrt(om * tot[Q_RRX_A] + tot[Q_RRY_A] / om);
    init_search(st->ls[0], r, tot[Q_D2_A], tot[Q_GD_A], tot[Q_G2INF_A]);
    st->last_r = r;
  }
  if (st->scheme == kSchemeFlexible) {
    const double r = sqrt(om * tot[Q_RRX_C] + tot[Q_RRY_C] / om);
    init_search(st->ls[1], r, tot[Q_D2_C], tot[Q_GD_C], tot[Q_G2INF_C]);
  }
}

// ----------------------------------------------- multiplier search (Sec. 6.3)
//
// f(lambda) = ||zt(lambda) - z||^2 = sum_{lam_i <= lambda} d_i^2
//           + lambda^2 sum_{lam_i > lambda} g_i^2 is continuous and
// nondecreasing; lambda* is its largest point with f <= r^2.  Pass p splits
// the current bracket (keys sharing the fixed prefix) into 256 buckets by
// bits [56 - 8p, 64 - 8p) of the breakpoint's bit pattern (monotone in the
// value for nonnegative doubles) and accumulates, per bucket, the count,
// sum d^2, sum g^2 and sum d g.  Bucket edges e_k are evaluated exactly;
// the bracket shrinks to the last bucket with f(e_k) <= r^2.  The search
// ends when that bucket is empty or after the 8th pass, then
// lambda* = sqrt((r^2 - f_lo) / f_hi), the closed form of Algorithm 2.
//
// Within a warp, lanes that fall in the same bucket are summed by the
// group's lowest lane in lane order (match_any), so the per-bucket sums
// are deterministic.

__global__ void __launch_bounds__(kHistWarps *kWarp) ls_hist_kernel(
    const uint64_t *__restrict__ keys0, const double *__restrict__ d20,
    const double *__restrict__ g20, const double *__restrict__ gd0,
    const uint64_t *__restrict__ keys1, const double *__restrict__ d21,
    const double *__restrict__ g21, const double *__restrict__ gd1, int64_t N,
    const DevState *st, int pass, double *hpart, int32_t *cand0, int32_t *cand1, int32_t *ccnt0,
    int32_t *ccnt1, int64_t wcap) {
  const int sidx = blockIdx.y;
  const LSearch &L = st->ls[sidx];
  if (L.done) return;
  const uint64_t *keys = sidx ? keys1 : keys0;
  const double *d2 = sidx ? d21 : d20;
  const double *g2 = sidx ? g21 : g20;
  const double *gd = sidx ? gd1 : gd0;
  const int shift = 56 - 8 * pass;
  const uint64_t pre = L.prefix;
  __shared__ double hist[kHistWarps][kBuckets][3];
  __shared__ unsigned cnt[kHistWarps][kBuckets];
  __shared__ double stage[kHistWarps][kWarp][3];
  for (int i = threadIdx.x; i < kHistWarps * kBuckets; i += blockDim.x) {
    (&hist[0][0][0])[3 * i] = 0.0;
    (&hist[0][0][0])[3 * i + 1] = 0.0;
    (&hist[0][0][0])[3 * i + 2] = 0.0;
    (&cnt[0][0])[i] = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
  // Candidate lists: in pass 1 each warp keeps, in its scan order, the
  // elements inside the bracket of pass 0; later passes read only that list
  // (its elements are a superset of every later bracket's).  Without lists
  // (cand0 null) every pass scans all N elements.
  const int64_t gw = (int64_t)blockIdx.x * kHistWarps + warp;
  int32_t *cand = cand0 ? (sidx ? cand1 : cand0) + gw * wcap : nullptr;
  int32_t *ccnt = sidx ? ccnt1 : ccnt0;
  // element e (or -1): is it in the current bracket, and in which bucket
  auto classify = [&](int64_t e, bool &act, int &bk) {
    act = false;
    bk = -1;
    if (e >= 0) {
      const uint64_t k = keys[e];
      if (k != kNoKey && (pass == 0 || (k >> (shift + 8)) == (pre >> (shift + 8)))) {
        act = true;
        bk = (int)((k >> shift) & 255u);
      }
    }
  };
  auto add = [&](int64_t e, bool act, int bk) {
    if (__ballot_sync(kFull, act) == 0u) return;
    double vd = 0.0, vg = 0.0, ve = 0.0;
    if (act) {
      vd = d2[e];
      vg = g2[e];
      ve = gd[e];
    }
    const unsigned grp = __match_any_sync(kFull, bk);
    const bool leader = act && (grp & ((1u << lane) - 1u)) == 0u;
    const unsigned leaders = __ballot_sync(kFull, leader);
    const int ndist = __popc(leaders);
    const int maxg = (int)__reduce_max_sync(kFull, act ? (unsigned)__popc(grp) : 0u);
    if (15 * ndist < 3 * maxg) {
      // few distinct buckets: one warp-wide butterfly sum per bucket
      unsigned rem = leaders;
      while (rem) {
        const int l = __ffs(rem) - 1;
        rem &= rem - 1u;
        const int b = __shfl_sync(kFull, bk, l);
        const bool mine = act && bk == b;
        const unsigned mm = __ballot_sync(kFull, mine);
        double sd = mine ? vd : 0.0, sg = mine ? vg : 0.0, se = mine ? ve : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sd += __shfl_xor_sync(kFull, sd, o);
          sg += __shfl_xor_sync(kFull, sg, o);
          se += __shfl_xor_sync(kFull, se, o);
        }
        if (lane == 0) {
          hist[warp][b][0] += sd;
          hist[warp][b][1] += sg;
          hist[warp][b][2] += se;
          cnt[warp][b] += (unsigned)__popc(mm);
        }
        __syncwarp();
      }
    } else {
      // many distinct buckets: each group's lowest lane sums its group in lane order
      if (act) {
        stage[warp][lane][0] = vd;
        stage[warp][lane][1] = vg;
        stage[warp][lane][2] = ve;
      }
      __syncwarp();
      if (leader) {
        double sd = 0.0, sg = 0.0, se = 0.0;
        unsigned gm = grp;
        while (gm) {
          const int l = __ffs(gm) - 1;
          gm &= gm - 1u;
          sd += stage[warp][l][0];
          sg += stage[warp][l][1];
          se += stage[warp][l][2];
        }
        hist[warp][bk][0] += sd;
        hist[warp][bk][1] += sg;
        hist[warp][bk][2] += se;
        cnt[warp][bk] += (unsigned)__popc(grp);
      }
    }
    __syncwarp();
  };
  if (cand && pass >= 2) {
    const int32_t count = ccnt[gw];
    for (int32_t i0 = 0; i0 < count; i0 += kWarp) {
      const int64_t e = i0 + lane < count ? (int64_t)cand[i0 + lane] : -1;
      bool act;
      int bk;
      classify(e, act, bk);
      add(e, act, bk);
    }
  } else {
    const int64_t stride = (int64_t)gridDim.x * kHistWarps * kWarp;
    int32_t count = 0;
    for (int64_t base = gw * kWarp; base < N; base += stride) {
      const int64_t e = base + lane < N ? base + lane : -1;
      bool act;
      int bk;
      classify(e, act, bk);
      if (cand && pass == 1) {
        const unsigned bal = __ballot_sync(kFull, act);
        if (act) cand[count + __popc(bal & ((1u << lane) - 1u))] = (int32_t)e;
        count += __popc(bal);
      }
      add(e, act, bk);
    }
    if (cand && pass == 1 && lane == 0) ccnt[gw] = count;
  }
  __syncthreads();
  double *out = hpart + ((size_t)sidx * gridDim.x + blockIdx.x) * 4 * kBuckets;
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) {
    double c = 0.0, sd = 0.0, sg = 0.0, se = 0.0;
    for (int w = 0; w < kHistWarps; ++w) {
      c += (double)cnt[w][b];
      sd += hist[w][b][0];
      sg += hist[w][b][1];
      se += hist[w][b][2];
    }
    out[b] = c;
    out[kBuckets + b] = sd;
    out[2 * kBuckets + b] = sg;
    out[3 * kBuckets + b] = se;
  }
}

// Block (b, search) sums bucket b's four values over the histogram blocks
// in a fixed order; the last block to finish (threadfence + counter) picks
// the bracket.  The FP64 additions are spread over 256 blocks.
__global__ void __launch_bounds__(kBuckets) ls_select_kernel(DevState *st, int pass,
                                                             const double *hpart, double *btot,
                                                             int hist_grid) {
  const int sidx = blockIdx.y;
  LSearch &L = st->ls[sidx];
  if (L.done) return;
  const int tid = threadIdx.x, bucket = blockIdx.x;
  __shared__ double red[4][kBuckets];
  __shared__ bool last;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const double *base = hpart + (size_t)sidx * hist_grid * 4 * kBuckets;
  for (int blk = tid; blk < hist_grid; blk += kBuckets) {
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += base[((size_t)blk * 4 + q) * kBuckets + bucket];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][tid] = acc[q];
  __syncthreads();
  for (int o = kBuckets / 2; o > 0; o >>= 1) {
    if (tid < o) {
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][tid] += red[q][tid + o];
    }
    __syncthreads();
  }
  double *bt = btot + (size_t)sidx * 4 * kBuckets;
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) bt[q * kBuckets + bucket] = red[q][0];
    __threadfence();
    last = (atomicAdd(&st->sel_counter[sidx], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int b = tid;
  __shared__ double cnt[kBuckets], sd[kBuckets], sg[kBuckets], se[kBuckets];
  __shared__ double cum_d[kBuckets + 1], cum_e[kBuckets + 1], tail_g[kBuckets + 1];
  __shared__ double wt[3][8];
  __shared__ int kstar;
  const volatile double *vb = bt;
  cnt[b] = vb[b];
  sd[b] = vb[kBuckets + b];
  sg[b] = vb[2 * kBuckets + b];
  se[b] = vb[3 * kBuckets + b];
  if (tid == 0) {
    kstar = -1;
    st->sel_counter[sidx] = 0u;
  }
  __syncthreads();
  // exclusive prefix sums of d^2 and d g, suffix sums of g^2 (fixed order)
  double pd = 0.0, pe = 0.0, pg = 0.0;
  if (tid < kBuckets) {  // warps 0..7, whole warps
    pd = scan256(sd[b], wt[0]);
    pe = scan256(se[b], wt[1]);
    pg = scan256(sg[kBuckets - 1 - b], wt[2]);  // reversed order: suffix sums
  }
  __syncthreads();
  if (tid < kBuckets) {
    double od = 0.0, oe = 0.0, og = 0.0;
    for (int w = 0; w < (b >> 5); ++w) {
      od += wt[0][w];
      oe += wt[1][w];
      og += wt[2][w];
    }
    cum_d[b + 1] = od + pd;
    cum_e[b + 1] = oe + pe;
    tail_g[kBuckets - 1 - b] = og + pg;
    if (b == 0) {
      cum_d[0] = 0.0;
      cum_e[0] = 0.0;
      tail_g[kBuckets] = 0.0;
    }
  }
  __syncthreads();
  if (tid < kBuckets) {
    const int shift = 56 - 8 * pass;
    const uint64_t edge_bits = L.prefix | ((uint64_t)b << shift);
    const double edge = __longlong_as_double((long long)edge_bits);
    bool ok = false;
    if ((edge_bits >> 63) == 0ull && isfinite(edge)) {  // edges are nonnegative finite doubles
      const double f = L.f_lo + cum_d[b] + edge * edge * (L.f_hi + tail_g[b]);
      ok = f <= L.r2;
    }
    if (ok) atomicMax(&kstar, b);
  }
  __syncthreads();
  if (tid != 0) return;
  const int k = kstar < 0 ? 0 : kstar;
  const int shift = 56 - 8 * pass;
  L.f_lo += cum_d[k];
  L.e_lo += cum_e[k];
  L.f_hi += tail_g[k + 1];
  L.prefix = L.prefix | ((uint64_t)k << shift);
  if (cnt[k] == 0.0 || pass == kSearchPasses - 1) {
    if (cnt[k] != 0.0) {  // last pass: breakpoints equal to the edge are clamped
      L.f_lo += sd[k];
      L.e_lo += se[k];
    }
    if (L.f_hi > 0.0) {
      L.lambda = sqrt(fmax(L.r2 - L.f_lo, 0.0) / L.f_hi);
      L.rho_r = L.e_lo + L.lambda * L.f_hi;
    } else {
      L.lambda = INFINITY;
      L.rho_r = L.e_lo;
    }
    L.done = 1;
  }
}

// Restart decision (Eq. adaptive-restart-scheme / flexible / fixed), trace
// row, and the averaging weights w_k = 1 / (t0 + k + 1) of the next block.
__global__ void __launch_bounds__(kBlock) check_decide_kernel(DevState *st, double *w,
                                                              double *trace) {
  __shared__ int64_t t0s;
  __shared__ int active;
  if (threadIdx.x == 0) {
    active = (st->status == kRunning);
    if (active) {
      const int scheme = st->scheme;
      double rho = NAN, r = st->last_r;
      int use_cur = 0;
      if (scheme == kSchemeAdaptive || scheme == kSchemeFlexible) {
        const LSearch &La = st->ls[0];
        r = sqrt(La.r2);
        rho = (La.r2 > 0.0) ? La.rho_r / r : 0.0;
        if (scheme == kSchemeFlexible) {
          const LSearch &Lc = st->ls[1];
          const double rc = sqrt(Lc.r2);
          const double rho_c = (Lc.r2 > 0.0) ? Lc.rho_r / rc : 0.0;
          if (rho_c < rho) {
            use_cur = 1;
            rho = rho_c;
            r = rc;
          }
        }
      }
      const int64_t t = st->t0 + st->K;
      int restart = 0;
      if (scheme == kSchemeAdaptive || scheme == kSchemeFlexible)
        restart = (st->restarts == 0) ? (t >= st->tau0) : (rho <= st->beta * st->rho_stored);
      else if (scheme == kSchemeFixed)
        restart = (t >= st->fixed_len);
      if (trace && st->trace_count < st->trace_cap) {
        double *row = trace + 6 * st->trace_count;
        row[0] = (double)st->iters;
        row[1] = rho;
        row[2] = (double)restart;
        row[3] = st->kkt_a[4];
        row[4] = st->kkt_c[4];
        row[5] = r;
      }
      st->trace_count += 1;
      st->last_rho = rho;
      st->last_r = r;
      st->use_cur = use_cur;
      st->restart_now = restart;
      if (restart) {
        st->rho_stored = rho;
        st->restarts += 1;
        st->t0 = 0;
        // mixed precision: the next correction is scaled by the distance moved
        if (st->mixed && r > 0.0 && isfinite(r)) st->mix_s = fmin(1.0 / r, 1e12);
      } else {
        st->t0 = t;
      }
    }
    t0s = st->t0;
  }
  __syncthreads();
  if (!active) return;
  for (int k = threadIdx.x; k < st->K; k += blockDim.x) w[k] = 1.0 / (double)(t0s + k + 1);
}

__global__ void restart_copy_kernel(DevVecs v, const DevState *st, int n, int m) {
  if (st->status != kRunning) return;
  const int rs = st->restart_now, uc = st->use_cur;
  if (!rs && !uc) return;
  const int64_t total = (int64_t)n + m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const double s = uc ? v.x[i] : v.xbar[i];
      if (rs) {
        v.x0[i] = s;
        v.x[i] = s;
      }
      v.xbar[i] = s;
    } else {
      const int64_t k = i - n;
      const double s = uc ? v.y[k] : v.ybar[k];
      if (rs) {
        v.y0[k] = s;
        v.y[k] = s;
      }
      v.ybar[k] = s;
    }
  }
}

__global__ void advance_kernel(DevState *st, double *w, int r) {
  __shared__ int64_t t0s;
  __shared__ int active;
  if (threadIdx.x == 0) {
    active = (st->status == kRunning);
    if (active) {
      st->iters += r;
      st->t0 += r;
    }
    t0s = st->t0;
  }
  __syncthreads();
  if (!active) return;
  for (int k = threadIdx.x; k < st->K; k += blockDim.x) w[k] = 1.0 / (double)(t0s + k + 1);
}

__global__ void weights_kernel(const DevState *st, double *w) {
  const int64_t t0 = st->t0;
  for (int k = threadIdx.x; k < st->K; k += blockDim.x) w[k] = 1.0 / (double)(t0 + k + 1);
}

// ------------------------------------------------------ power iteration

__global__ void __launch_bounds__(kBlock) sumsq_kernel(const double *__restrict__ v, int64_t n,
                                                       double *partials, int pstride, int slot,
                                                       const DevState *st) {
  if (st && st->pw_done) return;
  double q[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[0] += v[i] * v[i];
  block_reduce_store<1>(q, partials + (size_t)slot * pstride, pstride, (int)blockIdx.x);
}

__device__ double sum_fixed(const double *p, int count, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += p[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Power iteration on A^T A (Section 7): ray = ||A v||^2 for ||v|| = 1,
// stop when |ray - est| <= tol * ray (after the first step) or A^T A v = 0.
__global__ void __launch_bounds__(kBlock) power_finalize_kernel(DevState *st,
                                                                const double *partials,
                                                                int pstride, int nparts) {
  if (st->pw_done) return;
  __shared__ double red[kBlock];
  const double ray = sum_fixed(partials, nparts, red);
  const double nw2 = sum_fixed(partials + pstride, nparts, red);
  if (threadIdx.x != 0) return;
  const double nw = sqrt(nw2);
  const int done = (st->pw_iters > 0 && fabs(ray - st->pw_est) <= st->pw_tol * ray);
  st->pw_est = ray;
  st->pw_iters += 1;
  st->pw_nw = nw;
  if (nw == 0.0 || done || st->pw_iters >= st->pw_max) st->pw_done = 1;
}

__global__ void power_scale_kernel(double *v, const double *w, int64_t n, const DevState *st) {
  if (st->pw_done) return;
  const double nw = st->pw_nw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] / nw;
}

// ------------------------------------------------------- Lanczos (sigma_max)
//
// sigma_max(A)^2 is the largest eigenvalue of A^T A; the Lanczos process on
// A^T A estimates it by the largest eigenvalue (Ritz value) of the
// tridiagonal matrix it builds, in far fewer products than the power
// iteration.  Step k, with w = A^T A v_k from two SpMVs:
//   alpha_k = v_k . w,  w <- w - alpha_k v_k - beta_{k-1} v_{k-1},
//   beta_k = ||w||,     v_{k+1} = w / beta_k.
// The Ritz value is evaluated every few steps; the run stops when it changes
// by at most pw_tol relative to the previous evaluation, at beta_k = 0 (an
// invariant subspace: the Ritz value is exact) or at the step cap.  Every
// block re-sums the block partials of a reduction in the same fixed order,
// so all blocks see the same alpha_k and beta_k.
__global__ void __launch_bounds__(kBlock) lz_dot_kernel(const double *__restrict__ v,
                                                        const double *__restrict__ w, int64_t n,
                                                        double *partials, int pstride,
                                                        const DevState *st) {
  if (st->pw_done) return;
  double q[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[0] += v[i] * w[i];
  block_reduce_store<1>(q, partials, pstride, (int)blockIdx.x);
}

__global__ void __launch_bounds__(kBlock) lz_update_kernel(double *w, const double *v,
                                                           const double *vprev, int64_t n,
                                                           double *partials, int pstride,
                                                           int nparts, const DevState *st,
                                                           LanczosT T, int k) {
  if (st->pw_done) return;
  __shared__ double red[kBlock];
  const double alpha = sum_fixed(partials, nparts, red);
  if (blockIdx.x == 0 && threadIdx.x == 0) T.alpha[k] = alpha;
  const double bprev = k > 0 ? T.beta[k - 1] : 0.0;
  double q[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double r = w[i] - alpha * v[i];
    if (k > 0) r -= bprev * vprev[i];
    w[i] = r;
    q[0] += r * r;
  }
  block_reduce_store<1>(q, partials + pstride, pstride, (int)blockIdx.x);
}

__global__ void __launch_bounds__(kBlock) lz_scale_kernel(double *w, int64_t n,
                                                          const double *partials, int pstride,
                                                          int nparts, const DevState *st,
                                                          LanczosT T, int k) {
  if (st->pw_done) return;
  __shared__ double red[kBlock];
  const double beta = sqrt(sum_fixed(partials + pstride, nparts, red));
  if (blockIdx.x == 0 && threadIdx.x == 0) T.beta[k] = beta;
  if (!(beta > 0.0)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = w[i] / beta;
}

// One warp.  After step k: the Ritz value of the (k+1) x (k+1) matrix.
__global__ void lz_ritz_kernel(DevState *st, LanczosT T, int k, int evaluate) {
  if (st->pw_done) return;
  const double beta = T.beta[k];
  const bool last = (k + 1 >= T.cap) || !(beta > 0.0);
  if (!evaluate && !last) return;
  const double theta = tridiag_top_eig(T.alpha, T.beta, k + 1);
  if (threadIdx.x == 0) {
    const int conv = (st->pw_iters > 0 && fabs(theta - st->pw_est) <= st->pw_tol * theta);
    st->pw_est = theta;
    st->pw_iters = k + 1;
    if (conv || last) st->pw_done = 1;
  }
}

// Start vector of the sigma_max estimators: v_r = 0.5 + u(perm[r]), u(j) the
// top 53 bits of SplitMix64 (Steele, Lea and Flood, 2014) at counter j (the
// original column index) as a fraction in [0, 1); then v /= ||v|| with the
// norm from fixed-order block partials.
__global__ void __launch_bounds__(kBlock) start_vector_kernel(const int32_t *__restrict__ perm,
                                                              double *v, int64_t n) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = ((uint64_t)perm[r] + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[r] = 0.5 + (double)(z >> 11) * 0x1.0p-53;
  }
}

__global__ void __launch_bounds__(kBlock) scale_inv_norm_kernel(double *v, int64_t n,
                                                                const double *partials,
                                                                int nparts) {
  __shared__ double red[kBlock];
  const double nv = sqrt(sum_fixed(partials, nparts, red));
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    v[r] = v[r] / nv;
}

__global__ void norms_finalize_kernel(DevState *st, const double *partials, int pstride,
                                      int nparts) {
  __shared__ double red[kBlock];
  const double b2 = sum_fixed(partials, nparts, red);
  const double c2 = sum_fixed(partials + pstride, nparts, red);
  if (threadIdx.x == 0) {
    st->norm_b = sqrt(b2);
    st->norm_c = sqrt(c2);
  }
}

// -------------------------------------------------------------- utilities

__global__ void gather_kernel(double *out, const double *in, const int32_t *perm, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}

__global__ void scatter_kernel(double *out, const double *in, const int32_t *perm, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = in[i];
}

__global__ void fill_kernel(double *p, double val, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = val;
}

// z <- proj_{X x Y}(z); average and restart point <- z.
__global__ void project_kernel(DevVecs v, int n, int m) {
  const int64_t total = (int64_t)n + m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const double xv = fmin(fmax(v.x[i], v.lb[i]), v.ub[i]);
      v.x[i] = xv;
      v.xbar[i] = xv;
      v.x0[i] = xv;
      v.xhat[i] = xv;
    } else {
      const int64_t k = i - n;
      double yv = v.y[k];
      if (v.row_type[k] == 1) yv = fmax(yv, 0.0);
      else if (v.row_type[k] == 2) yv = fmin(yv, 0.0);
      v.y[k] = yv;
      v.ybar[k] = yv;
      v.y0[k] = yv;
    }
  }
}

int grid_for(int64_t n, int num_sms) {
  int64_t g = (n + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int item_grid(const SellMat &A) {
  const int64_t items = A.nslices;
  int64_t g = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// Blocks of the second launch that handles the chunk slices of split rows
// (one warp per chunk slice); 0 when the matrix has none.
int split_grid(const SellMat &A) {
  return A.nsplit > 0 ? (A.nsplit + kWarpsPerBlock - 1) / kWarpsPerBlock : 0;
}

namespace {

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 132;
  }
  return g_num_sms;
}

}  // namespace

// One wave of resident blocks (the check kernels loop over the slices): the
// per-block reduction of the check's quantities is paid once per resident
// block.
int check_grid_for(const SellMat &A, int nsm) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, check_kernel<CheckColsEpi, true>, kBlock,
                                                      0) != cudaSuccess ||
        b < 1) {
      cudaGetLastError();
      b = 2;
    }
    return b;
  }();
  const int64_t items = A.nslices;
  int64_t g = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int64_t cap = (int64_t)nsm * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// unroll: 2, 4, 8 = register batches; -2, -4 = software-pipelined batches.
// |unroll| >= 100 (e.g. 102, -104): the same with registers capped for 5
// (column pass) or 4 (row pass) resident blocks of 256 threads.
template <int U, bool PIPE>
void primal_launch(int occ, int g, cudaStream_t s, const SellMat &AT, const double *y,
                   const PrimalEpi &epi, DevState *st, const double *w, int k) {
  if (AT.nsplit > 0)
    launch_pdl(primal_kernel<U, PIPE, 1, true>, split_grid(AT) + g, kBlock, s, AT, y, epi, st, w,
               k);
  else if (occ) launch_pdl(primal_kernel<U, PIPE, 5>, g, kBlock, s, AT, y, epi, st, w, k);
  else launch_pdl(primal_kernel<U, PIPE, 1>, g, kBlock, s, AT, y, epi, st, w, k);
}

template <int U, bool PIPE>
void dual_launch(int occ, int g, cudaStream_t s, const SellMat &A, const double *xhat,
                 const DualEpi &epi, DevState *st, const double *w, int k) {
  if (A.nsplit > 0)
    launch_pdl(dual_kernel<U, PIPE, 1, true>, split_grid(A) + g, kBlock, s, A, xhat, epi, st, w,
               k);
  else if (occ) launch_pdl(dual_kernel<U, PIPE, 4>, g, kBlock, s, A, xhat, epi, st, w, k);
  else launch_pdl(dual_kernel<U, PIPE, 1>, g, kBlock, s, A, xhat, epi, st, w, k);
}

void launch_primal_step(const SellMat &AT, const DevVecs &v, DevState *st, const double *w,
                        int k, int unroll, int grid_cap, cudaStream_t s) {
  PrimalEpi epi{v.c, v.lbk, v.ubk, v.x, v.xhat, v.xbar, 0.0, 0.0, nullptr};
  const int g = grid_cap > 0 ? std::min(item_grid(AT), grid_cap) : item_grid(AT);
  const int occ = (unroll >= 100 || unroll <= -100) ? 1 : 0;
  switch (unroll % 100) {
    case 2: primal_launch<2, false>(occ, g, s, AT, v.y, epi, st, w, k); break;
    case 8: primal_launch<8, false>(occ, g, s, AT, v.y, epi, st, w, k); break;
    case -2: primal_launch<2, true>(occ, g, s, AT, v.y, epi, st, w, k); break;
    case -4: primal_launch<4, true>(occ, g, s, AT, v.y, epi, st, w, k); break;
    default: primal_launch<4, false>(occ, g, s, AT, v.y, epi, st, w, k); break;
  }
}

void launch_dual_step(const SellMat &A, const DevVecs &v, DevState *st, const double *w, int k,
                      int unroll, int grid_cap, cudaStream_t s) {
  DualEpi epi{v.b, v.row_type, v.y, v.ybar, 0.0, 0.0, nullptr};
  const int g = grid_cap > 0 ? std::min(item_grid(A), grid_cap) : item_grid(A);
  const int occ = (unroll >= 100 || unroll <= -100) ? 1 : 0;
  switch (unroll % 100) {
    case 2: dual_launch<2, false>(occ, g, s, A, v.xhat, epi, st, w, k); break;
    case 8: dual_launch<8, false>(occ, g, s, A, v.xhat, epi, st, w, k); break;
    case -2: dual_launch<2, true>(occ, g, s, A, v.xhat, epi, st, w, k); break;
    case -4: dual_launch<4, true>(occ, g, s, A, v.xhat, epi, st, w, k); break;
    default: dual_launch<4, false>(occ, g, s, A, v.xhat, epi, st, w, k); break;
  }
}

void launch_check(const SellMat &A, const SellMat &AT, const DevVecs &v, DevState *st, double *w,
                  const CheckScratch &cs, int n, int m, int nsearch, double *trace,
                  bool decide, cudaStream_t s, const MixVecs *mv) {
  if (mv) launch_combine(v, *mv, st, n, m, 0, s);
  CheckColsEpi ce{};
  if (mv) {
    ce.lam_out0 = mv->lam[0];
    ce.lam_out1 = mv->lam[1];
  }
  ce.c = v.c; ce.lb = v.lb; ce.ub = v.ub; ce.xbar = v.xbar; ce.x = v.x; ce.x0 = v.x0;
  ce.ga = GapOut{cs.keys[0], cs.d2[0], cs.g2[0], cs.gd[0]};
  ce.gc = GapOut{cs.keys[1], cs.d2[1], cs.g2[1], cs.gd[1]};
  ce.gap_a = 1;  // overridden on device from the scheme unless a radius is given
  ce.gap_c = 0;
  CheckRowsEpi re{};
  re.b = v.b; re.rt = v.row_type; re.ybar = v.ybar; re.y = v.y; re.y0 = v.y0;
  re.ga = ce.ga;
  re.gc = ce.gc;
  re.off = n;
  re.gap_a = 1;
  re.gap_c = 0;
  if (mv) {
    re.gy_out0 = mv->gy[0];
    re.gy_out1 = mv->gy[1];
  }
  const bool pair = cs.pair_y && cs.pair_x;
  if (pair) {
    if (m > 0)
      pack_pairs_kernel<<<grid_for(m, num_sms()), kBlock, 0, s>>>(
          v.ybar, v.y, m, reinterpret_cast<double2 *>(cs.pair_y), st);
    if (n > 0)
      pack_pairs_kernel<<<grid_for(n, num_sms()), kBlock, 0, s>>>(
          v.xbar, v.x, n, reinterpret_cast<double2 *>(cs.pair_x), st);
  }
  // with split rows, the SPLIT instantiation with the chunk blocks in front;
  // every block writes one partial slot, columns' slots first
  const int sc = split_grid(AT), sr = split_grid(A);
  const int gc = sc + cs.cols_grid, gr = sr + cs.rows_grid;
  const double *c0 = pair ? cs.pair_y : v.ybar, *c1 = pair ? nullptr : v.y;
  const double *r0 = pair ? cs.pair_x : v.xbar, *r1 = pair ? nullptr : v.x;
  double *P = cs.partials;
  const int ps = cs.pstride;
  // after the blocks' slots, one reduction slot per chunk slice of each
  // matrix's split rows (every one written by every check pass)
  ce.split_slots = AT.nsplit > 0 ? P + gc + gr : nullptr;
  ce.slot_stride = ps;
  re.split_slots = A.nsplit > 0 ? P + gc + gr + AT.nsplit : nullptr;
  re.slot_stride = ps;
  const int nparts = gc + gr + AT.nsplit + A.nsplit;
  if (sc > 0 && pair)
    check_kernel<CheckColsEpi, true, true><<<gc, kBlock, 0, s>>>(AT, c0, c1, ce, st, P, ps, 0);
  else if (sc > 0)
    check_kernel<CheckColsEpi, false, true><<<gc, kBlock, 0, s>>>(AT, c0, c1, ce, st, P, ps, 0);
  else if (pair)
    check_kernel<CheckColsEpi, true><<<gc, kBlock, 0, s>>>(AT, c0, c1, ce, st, P, ps, 0);
  else
    check_kernel<CheckColsEpi, false><<<gc, kBlock, 0, s>>>(AT, c0, c1, ce, st, P, ps, 0);
  if (sr > 0 && pair)
    check_kernel<CheckRowsEpi, true, true><<<gr, kBlock, 0, s>>>(A, r0, r1, re, st, P, ps, gc);
  else if (sr > 0)
    check_kernel<CheckRowsEpi, false, true><<<gr, kBlock, 0, s>>>(A, r0, r1, re, st, P, ps, gc);
  else if (pair)
    check_kernel<CheckRowsEpi, true><<<gr, kBlock, 0, s>>>(A, r0, r1, re, st, P, ps, gc);
  else
    check_kernel<CheckRowsEpi, false><<<gr, kBlock, 0, s>>>(A, r0, r1, re, st, P, ps, gc);
  check_finalize_kernel<<<NQ, kBlock, 0, s>>>(st, cs.partials, cs.pstride, nparts);
  if (nsearch > 0) {
    const int64_t N = (int64_t)n + m;
    for (int p = 0; p < kSearchPasses; ++p) {
      ls_hist_kernel<<<dim3(cs.hist_grid, nsearch), kHistWarps * kWarp, 0, s>>>(
          cs.keys[0], cs.d2[0], cs.g2[0], cs.gd[0], cs.keys[1], cs.d2[1], cs.g2[1], cs.gd[1], N,
          st, p, cs.hpart, cs.cand[0], cs.cand[1], cs.ccnt[0], cs.ccnt[1], cs.cand_cap);
      ls_select_kernel<<<dim3(kBuckets, nsearch), kBuckets, 0, s>>>(st, p, cs.hpart, cs.btot,
                                                                 cs.hist_grid);
    }
  }
  if (decide) {
    check_decide_kernel<<<1, kBlock, 0, s>>>(st, w, trace);
    restart_copy_kernel<<<grid_for((int64_t)n + m, num_sms()), kBlock, 0, s>>>(v, st, n, m);
    if (mv) launch_recenter(v, *mv, st, n, m, 0, s);
  }
}

template <int U, bool PIPE>
void primal_mix_launch(int g, cudaStream_t s, const SellMat &AT, const float *dy,
                       const PrimalMixEpi &epi, DevState *st, const double *w, int k) {
  if (AT.nsplit > 0)
    launch_pdl(primal_mix_kernel<U, PIPE, true>, split_grid(AT) + g, kBlock, s, AT, dy, epi, st, w,
               k);
  else launch_pdl(primal_mix_kernel<U, PIPE>, g, kBlock, s, AT, dy, epi, st, w, k);
}

template <int U, bool PIPE>
void dual_mix_launch(int g, cudaStream_t s, const SellMat &A, const float *dxhat,
                     const DualMixEpi &epi, DevState *st, const double *w, int k) {
  if (A.nsplit > 0)
    launch_pdl(dual_mix_kernel<U, PIPE, true>, split_grid(A) + g, kBlock, s, A, dxhat, epi, st, w,
               k);
  else launch_pdl(dual_mix_kernel<U, PIPE>, g, kBlock, s, A, dxhat, epi, st, w, k);
}

void launch_primal_mix(const SellMat &AT, const MixVecs &mv, DevState *st, const double *w,
                       int k, int unroll, cudaStream_t s) {
  PrimalMixEpi epi{mv.cf, mv.lf, mv.uf, mv.dx, mv.dxhat, mv.dxbar, 0.0f, 0.0};
  const int g = item_grid(AT);
  switch (unroll % 100) {
    case 2: primal_mix_launch<2, false>(g, s, AT, mv.dy, epi, st, w, k); break;
    case 4: primal_mix_launch<4, false>(g, s, AT, mv.dy, epi, st, w, k); break;
    case -4: primal_mix_launch<4, true>(g, s, AT, mv.dy, epi, st, w, k); break;
    default: primal_mix_launch<2, true>(g, s, AT, mv.dy, epi, st, w, k); break;
  }
}

void launch_dual_mix(const SellMat &A, const MixVecs &mv, const DevVecs &, DevState *st,
                     const double *w, int k, int unroll, cudaStream_t s) {
  DualMixEpi epi{mv.bf, mv.ylo, mv.yhi, mv.dy, mv.dybar, 0.0f, 0.0};
  const int g = item_grid(A);
  switch (unroll % 100) {
    case 2: dual_mix_launch<2, false>(g, s, A, mv.dxhat, epi, st, w, k); break;
    case 4: dual_mix_launch<4, false>(g, s, A, mv.dxhat, epi, st, w, k); break;
    case -2: dual_mix_launch<2, true>(g, s, A, mv.dxhat, epi, st, w, k); break;
    default: dual_mix_launch<4, true>(g, s, A, mv.dxhat, epi, st, w, k); break;
  }
}

void launch_combine(const DevVecs &v, const MixVecs &mv, DevState *st, int n, int m, int force,
                    cudaStream_t s) {
  combine_kernel<<<grid_for((int64_t)n + m, num_sms()), kBlock, 0, s>>>(v, mv, st, n, m, force);
}

void launch_recenter(const DevVecs &v, const MixVecs &mv, DevState *st, int n, int m, int force,
                     cudaStream_t s) {
  recenter_kernel<<<grid_for((int64_t)n + m, num_sms()), kBlock, 0, s>>>(v, mv, st, n, m, force);
}

void launch_residuals(const SellMat &A, const SellMat &AT, const DevVecs &v, const MixVecs &mv,
                      int n, int m, cudaStream_t s) {
  // A^T y0 into lam[1], A x0 into gy[1] (scratch), then the residuals
  launch_spmv(AT, v.y0, mv.lam[1], s, nullptr);
  launch_spmv(A, v.x0, mv.gy[1], s, nullptr);
  residuals_kernel<<<grid_for((int64_t)n + m, num_sms()), kBlock, 0, s>>>(v, mv, mv.lam[1],
                                                                          mv.gy[1], n, m);
}

void launch_forward_masked(const SellMat &A, const SellMat &AT, const DevVecs &v, double tau,
                           double sigma, double w, uint8_t *mx, uint8_t *my, cudaStream_t s) {
  PrimalEpi pe{v.c, v.lbk, v.ubk, v.x, v.xhat, v.xbar, 0.0, 0.0, mx};
  if (AT.nsplit > 0)
    primal_mask_kernel<true><<<split_grid(AT) + item_grid(AT), kBlock, 0, s>>>(AT, v.y, pe, tau, w);
  else
    primal_mask_kernel<<<item_grid(AT), kBlock, 0, s>>>(AT, v.y, pe, tau, w);
  DualEpi de{v.b, v.row_type, v.y, v.ybar, 0.0, 0.0, my};
  if (A.nsplit > 0)
    dual_mask_kernel<true><<<split_grid(A) + item_grid(A), kBlock, 0, s>>>(A, v.xhat, de, sigma, w);
  else
    dual_mask_kernel<<<item_grid(A), kBlock, 0, s>>>(A, v.xhat, de, sigma, w);
}

void launch_adjoint_step(const SellMat &A, const SellMat &AT, const AdjVecs &a,
                         const uint8_t *mx, const uint8_t *my_prev, double tau, double sigma,
                         double w, double w_prev, int has_prev, cudaStream_t s) {
  AdjColsEpi ce{a.ax, a.axb, a.ac, a.v, mx, tau, sigma, w};
  if (AT.nsplit > 0)
    adj_cols_kernel<true><<<split_grid(AT) + item_grid(AT), kBlock, 0, s>>>(AT, a.u, ce);
  else
    adj_cols_kernel<<<item_grid(AT), kBlock, 0, s>>>(AT, a.u, ce);
  AdjRowsEpi re{a.ay, a.ayb, a.ab, a.u, my_prev, tau, sigma, w_prev, has_prev};
  if (A.nsplit > 0)
    adj_rows_kernel<true><<<split_grid(A) + item_grid(A), kBlock, 0, s>>>(A, a.v, re);
  else
    adj_rows_kernel<<<item_grid(A), kBlock, 0, s>>>(A, a.v, re);
}

void launch_adjoint_block_start(const AdjVecs &a, const uint8_t *my_last, int restarted,
                                double sigma, double w, int n, int m, cudaStream_t s) {
  adj_block_start_kernel<<<grid_for((int64_t)n + m, num_sms()), kBlock, 0, s>>>(
      a.ax, a.axb, a.ay, a.ayb, a.u, a.ab, my_last, restarted, sigma, w, n, m);
}

void launch_advance(DevState *st, double *w, int r, cudaStream_t s) {
  advance_kernel<<<1, kBlock, 0, s>>>(st, w, r);
}

void launch_weights(DevState *st, double *w, cudaStream_t s) {
  weights_kernel<<<1, kBlock, 0, s>>>(st, w);
}

void launch_spmv(const SellMat &A, const double *v, double *out, cudaStream_t s,
                 DevState *st_guard) {
  StoreEpi epi{out};
  if (A.nsplit > 0)
    spmv_kernel<true><<<split_grid(A) + item_grid(A), kBlock, 0, s>>>(A, v, epi, st_guard);
  else
    spmv_kernel<<<item_grid(A), kBlock, 0, s>>>(A, v, epi, st_guard);
}

void launch_power_iteration_step(const SellMat &A, const SellMat &AT, double *v, double *av,
                                 double *w, DevState *st, double *partials, int pstride,
                                 int grid, int n, int m, cudaStream_t s) {
  launch_spmv(A, v, av, s, st);
  sumsq_kernel<<<grid, kBlock, 0, s>>>(av, m, partials, pstride, 0, st);
  launch_spmv(AT, av, w, s, st);
  sumsq_kernel<<<grid, kBlock, 0, s>>>(w, n, partials, pstride, 1, st);
  power_finalize_kernel<<<1, kBlock, 0, s>>>(st, partials, pstride, grid);
  power_scale_kernel<<<grid_for(n, num_sms()), kBlock, 0, s>>>(v, w, n, st);
}

void launch_lanczos_step(const SellMat &A, const SellMat &AT, const double *v, double *av,
                         double *w, const double *vprev, DevState *st, const LanczosT &T, int k,
                         bool evaluate, double *partials, int pstride, int grid, int n,
                         cudaStream_t s) {
  launch_spmv(A, v, av, s, st);
  launch_spmv(AT, av, w, s, st);
  lz_dot_kernel<<<grid, kBlock, 0, s>>>(v, w, n, partials, pstride, st);
  lz_update_kernel<<<grid, kBlock, 0, s>>>(w, v, vprev, n, partials, pstride, grid, st, T, k);
  lz_scale_kernel<<<grid, kBlock, 0, s>>>(w, n, partials, pstride, grid, st, T, k);
  lz_ritz_kernel<<<1, kWarp, 0, s>>>(st, T, k, evaluate ? 1 : 0);
}

void launch_start_vector(const int32_t *perm, double *v, int n, double *partials, int pstride,
                         int grid, cudaStream_t s) {
  start_vector_kernel<<<grid, kBlock, 0, s>>>(perm, v, n);
  sumsq_kernel<<<grid, kBlock, 0, s>>>(v, n, partials, pstride, 0, nullptr);
  scale_inv_norm_kernel<<<grid, kBlock, 0, s>>>(v, n, partials, grid);
}

void launch_norms(const DevVecs &v, DevState *st, double *partials, int pstride, int grid, int n,
                  int m, cudaStream_t s) {
  sumsq_kernel<<<grid, kBlock, 0, s>>>(v.b, m, partials, pstride, 0, nullptr);
  sumsq_kernel<<<grid, kBlock, 0, s>>>(v.c, n, partials, pstride, 1, nullptr);
  norms_finalize_kernel<<<1, kBlock, 0, s>>>(st, partials, pstride, grid);
}

void launch_gather(double *out, const double *in, const int32_t *perm, int64_t n,
                   cudaStream_t s) {
  if (n > 0) gather_kernel<<<grid_for(n, num_sms()), kBlock, 0, s>>>(out, in, perm, n);
}

void launch_scatter(double *out, const double *in, const int32_t *perm, int64_t n,
                    cudaStream_t s) {
  if (n > 0) scatter_kernel<<<grid_for(n, num_sms()), kBlock, 0, s>>>(out, in, perm, n);
}

void launch_project(const DevVecs &v, int n, int m, cudaStream_t s) {
  const int64_t total = (int64_t)n + m;
  if (total > 0) project_kernel<<<grid_for(total, num_sms()), kBlock, 0, s>>>(v, n, m);
}

void launch_fill(double *p, double val, int64_t n, cudaStream_t s) {
  if (n > 0) fill_kernel<<<grid_for(n, num_sms()), kBlock, 0, s>>>(p, val, n);
}

}  // namespace lpg
