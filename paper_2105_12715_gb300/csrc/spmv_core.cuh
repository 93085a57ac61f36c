// SpMV core of the sliced layout and the fused epilogues of the PDHG step
// and of the check, shared by the single-problem kernels (lp_kernels.cu)
// and the batched kernels (lp_batch.cu).  Header-only device code.
#pragma once

#include <cmath>
#include <cstdint>

#include "lp_internal.h"

namespace lpg {
namespace {
constexpr unsigned kFull = 0xffffffffu;
constexpr int kUnroll = 8;   // gathers in flight per lane, one vector (plain SpMV)
constexpr int kUnroll2 = 4;  // gathers in flight per lane and vector, two vectors
constexpr int kStatusOK = 0;
constexpr int kStatusNumerical = 5;
constexpr int kSchemeFixed = 1, kSchemeAdaptive = 2, kSchemeFlexible = 3;

__device__ __forceinline__ double sq(double v) { return v * v; }

// Programmatic dependent launch (iteration kernels, launched with
// launch_pdl): let the next kernel in the stream be scheduled while this one
// drains, then wait until the previous kernel has completed and its writes
// are visible -- before any read of its results.  Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------ SpMV core
//
// Row sums of one slice (one warp).  Each lane walks its row's elements
// k = g, g + G, g + 2G, ... in stored order, U steps at a time: the U
// index and value loads of a batch are issued together, then the U
// gathers, then the FMAs, so a lane has U gathers in flight.  The G lanes of
// a row are then combined by a butterfly (the same sum in every lane of the
// group), and the group's first lane runs the epilogue.  The epilogue's
// operands are loaded before the row loop.  NV = 1 or 2 gathered vectors.
// T is the value type of the matrix copy, of the gathered vectors and of
// the accumulators (double for the FP64 path, float for the mixed path).
// PAIR (NV = 2, double): the two vectors are stored interleaved at v0
// (element i of both in one 16-byte pair), so one 16-byte gather, one
// sector, fetches both operands of an element; the sums are the same.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ const double *vals_of(const SellMat &A, double) { return A.val; }
__device__ __forceinline__ const float *vals_of(const SellMat &A, float) { return A.valf; }

template <int NV, int U, bool PIPE, bool PAIR = false, typename T, class Epi>
__device__ __forceinline__ void process_item(const SellMat &A, const T *__restrict__ v0,
                                             const T *__restrict__ v1, int item, int lane,
                                             Epi &epi) {
  const SliceInfo a = A.info[item];
  const int32_t row_end = A.info[item + 1].row0;
  const int lg = a.len_g & 7;
  const int steps = a.len_g >> 3;
  const int row = a.row0 + (lane >> lg);
  const bool owner = ((lane & ((1 << lg) - 1)) == 0) && row < row_end;
  typename Epi::Pre pre{};
  if (owner) pre = epi.load(row);
  const int32_t *ip = A.idx + a.off + lane;
  const T *vp = vals_of(A, T(0)) + a.off + lane;
  T a0 = owner ? epi.init(pre) : T(0), a1 = T(0);
  int32_t j[U];
  T c[U];
  if (PIPE) {  // software pipeline: the next batch's index/value loads overlap this batch's gathers
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < steps) {
        j[u] = __ldcs(ip + (size_t)kWarp * u);
        c[u] = __ldcs(vp + (size_t)kWarp * u);
      }
    }
  }
  for (int t = 0; t < steps; t += U) {
    T g[U], h[U];
    if (!PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (t + u < steps) {
          j[u] = __ldcs(ip + (size_t)kWarp * (t + u));
          c[u] = __ldcs(vp + (size_t)kWarp * (t + u));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u < steps) {
        if constexpr (PAIR) {
          const double2 p = __ldg(reinterpret_cast<const double2 *>(v0) + j[u]);
          g[u] = p.x;
          h[u] = p.y;
        } else {
          g[u] = __ldg(v0 + j[u]);
          if (NV == 2) h[u] = __ldg(v1 + j[u]);
        }
      }
    }
    int32_t jn[U];
    T cn[U];
    if (PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (t + U + u < steps) {
          jn[u] = __ldcs(ip + (size_t)kWarp * (t + U + u));
          cn[u] = __ldcs(vp + (size_t)kWarp * (t + U + u));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u < steps) {
        a0 = fma_t(c[u], g[u], a0);
        if (NV == 2) a1 = fma_t(c[u], h[u], a1);
      }
    }
    if (PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        j[u] = jn[u];
        c[u] = cn[u];
      }
    }
  }
  for (int o = (1 << lg) >> 1; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(kFull, a0, o);
    if (NV == 2) a1 += __shfl_xor_sync(kFull, a1, o);
  }
  if (owner) epi.store(row, a0, a1, pre);
}

// Epilogues that accumulate reductions (the check's) declare kSplitSlots:
// the reductions of a split row then go to a slot of their own instead of
// the block of whichever chunk arrived last (see process_split_item).
template <class E, class = void>
struct SplitSlotsOf {
  static constexpr bool value = false;
};
template <class E>
struct SplitSlotsOf<E, decltype((void)E::kSplitSlots, void())> {
  static constexpr bool value = E::kSplitSlots;
};

// One chunk slice of a split row (see SellMat): the warp sums its chunk in
// the order of process_item (U loads, U gathers, U FMAs per lane, then the
// 32-lane butterfly); chunk 0 starts from the epilogue's initial value.
// Lane 0 publishes the partial sums; the last chunk of the row to arrive
// adds all partials in chunk order and runs the epilogue, then resets the
// row's counter for the next pass.  Every chunk's sum, and their order, is
// fixed, so the result is deterministic.  For an accumulating epilogue,
// every chunk slice first clears its own reduction slot, and the last
// arrival moves the row's reductions into the slot of the row's first
// chunk: each split row's terms land in a fixed slot, which the finalize
// adds in slot order, whichever block arrived last.
template <int NV, int U, bool PIPE, bool PAIR, typename T, class Epi>
__device__ __forceinline__ void process_split_item(const SellMat &A, const T *__restrict__ v0,
                                                const T *__restrict__ v1, int item, int lane,
                                                Epi &epi) {
  const SliceInfo a = A.info[item];
  const SplitSlice sp = A.split[item];
  const int steps = a.len_g >> 3;  // G = 32: one row, lane l holds elements l, l + 32, ...
  const int row = a.row0;
  T a0 = T(0), a1 = T(0);
  if (sp.chunk == 0 && lane == 0) {
    const typename Epi::Pre pre = epi.load(row);
    a0 = epi.init(pre);
  }
  const int32_t *ip = A.idx + a.off + lane;
  const T *vp = vals_of(A, T(0)) + a.off + lane;
  for (int t = 0; t < steps; t += U) {
    int32_t j[U];
    T c[U], g[U], h[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u < steps) {
        j[u] = __ldcs(ip + (size_t)kWarp * (t + u));
        c[u] = __ldcs(vp + (size_t)kWarp * (t + u));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u < steps) {
        if constexpr (PAIR) {
          const double2 p = __ldg(reinterpret_cast<const double2 *>(v0) + j[u]);
          g[u] = p.x;
          h[u] = p.y;
        } else {
          g[u] = __ldg(v0 + j[u]);
          if (NV == 2) h[u] = __ldg(v1 + j[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u < steps) {
        a0 = fma_t(c[u], g[u], a0);
        if (NV == 2) a1 = fma_t(c[u], h[u], a1);
      }
    }
  }
  for (int o = kWarp >> 1; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(kFull, a0, o);
    if (NV == 2) a1 += __shfl_xor_sync(kFull, a1, o);
  }
  if (lane != 0) return;
  if constexpr (SplitSlotsOf<Epi>::value) {
    if (item != sp.first) epi.zero_split_slot(item);
  }
  A.split_part[2 * (size_t)item] = (double)a0;
  A.split_part[2 * (size_t)item + 1] = (double)a1;
  __threadfence();
  if (atomicAdd(&A.split_cnt[sp.first], 1) != sp.nchunks - 1) return;
  __threadfence();
  const volatile double *part = A.split_part;
  T s0 = T(0), s1 = T(0);
  for (int c = 0; c < sp.nchunks; ++c) {
    s0 += (T)part[2 * (size_t)(sp.first + c)];
    s1 += (T)part[2 * (size_t)(sp.first + c) + 1];
  }
  A.split_cnt[sp.first] = 0;
  const typename Epi::Pre pre = epi.load(row);
  epi.store(row, s0, s1, pre);
  if constexpr (SplitSlotsOf<Epi>::value) epi.flush_split_slot(sp.first);
}

// The slices of a pass, one warp per slice.  SPLIT = false: matrices
// without split rows (the kernels compiled as always).  SPLIT = true (a
// separate instantiation the launchers pick only for matrices with split
// rows, launched with split_grid(A) extra blocks in front): the first
// blocks take the chunk slices, one warp each, and the others the ordinary
// slices, so the chunks, started first, overlap the rest of the pass.
template <int NV, int U, bool PIPE = false, bool PAIR = false, bool SPLIT = false, typename T,
          class Epi>
__device__ __forceinline__ void process_all(const SellMat &A, const T *v0, const T *v1,
                                            Epi &epi) {
  const int lane = threadIdx.x & (kWarp - 1);
  int first_block = 0;
  if constexpr (SPLIT) {
    first_block = (A.nsplit + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if ((int)blockIdx.x < first_block) {
      const int it = (int)blockIdx.x * kWarpsPerBlock + (int)(threadIdx.x >> 5);
      if (it < A.nsplit) process_split_item<NV, U, PIPE, PAIR>(A, v0, v1, it, lane, epi);
      return;
    }
  }
  const int warp = (int)(((blockIdx.x - first_block) * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x - first_block) * blockDim.x) >> 5;
  for (int it = A.nsplit + warp; it < A.nslices; it += nwarps)
    process_item<NV, U, PIPE, PAIR>(A, v0, v1, it, lane, epi);
}

// Fixed-order block reduction of NV2 per-thread values; thread q < NV2 of
// the block writes the block's value q to partials[q * pstride + col].
template <int NV2>
__device__ __forceinline__ void block_reduce_store(const double (&q)[NV2], double *partials,
                                                   int pstride, int col) {
  __shared__ double sh[kBlock / kWarp][NV2];
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV2; ++i) {
    double v = q[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0) sh[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV2) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][threadIdx.x];
    partials[(size_t)threadIdx.x * pstride + col] = s;
  }
}

// The same for the quantities whose bit is set in mask (uniform across the
// block); the others are stored as 0 without a reduction.  The check
// kernels use it to skip the quantities their epilogue never touches: on
// GB300 each FP64 addition of the butterflies costs as much as a nonzero's
// FMA.
template <int NV2>
__device__ __forceinline__ void block_reduce_store_mask(const double (&q)[NV2], uint32_t mask,
                                                        double *partials, int pstride,
                                                        int col) {
  __shared__ double sh[kBlock / kWarp][NV2];
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV2; ++i) {
    if (!((mask >> i) & 1u)) continue;
    double v = q[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0) sh[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV2) {
    double s = 0.0;
    if ((mask >> threadIdx.x) & 1u)
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][threadIdx.x];
    partials[(size_t)threadIdx.x * pstride + col] = s;
  }
}

// -------------------------------------------------------------- epilogues

// Order-preserving map of a double's bit pattern to a signed integer
// (negative values: all bits but the sign flipped); it is its own inverse.
// Clamps and sign projections compare these keys on the integer pipe
// instead of issuing FP64 min/max (GB300 runs 2 FP64 operations per cycle
// per SM).
__device__ __forceinline__ long long ord_key(long long b) {
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

// Eq. (PDHG-update), primal half, and Algorithm 1's running average.  The
// row sum starts at -c_j, so it ends as (A^T y)_j - c_j = -g_j.  lbk/ubk are
// the bounds' order keys.
struct PrimalEpi {
  const double *__restrict__ c;
  const long long *__restrict__ lbk;
  const long long *__restrict__ ubk;
  double *x, *xhat, *xbar;
  double tau, w;
  uint8_t *mask;  // adjoint recording: 1 where the clamp is inactive, or null
  struct Pre { double c, x, xb; long long lk, uk; };
  __device__ __forceinline__ Pre load(int j) const { return {c[j], x[j], xbar[j], lbk[j], ubk[j]}; }
  __device__ __forceinline__ double init(const Pre &p) const { return -p.c; }
  __device__ __forceinline__ void store(int j, double neg_g, double, const Pre &p) const {
    const double v = fma(tau, neg_g, p.x);  // x - tau (c - A^T y)
    long long k = ord_key(__double_as_longlong(v));
    if (mask) mask[j] = (k > p.lk && k < p.uk) ? 1 : 0;
    k = k < p.lk ? p.lk : k;
    k = k > p.uk ? p.uk : k;
    const double xn = __longlong_as_double(ord_key(k));
    x[j] = xn;
    xhat[j] = fma(2.0, xn, -p.x);
    xbar[j] = fma(w, xn - p.xb, p.xb);
  }
};

// Eq. (PDHG-update), dual half: projection onto Y_i by row sense (on the
// integer pipe: a negative double has a negative bit pattern).  The row sum
// starts at -b_i, so it ends as (A xhat)_i - b_i.
struct DualEpi {
  const double *__restrict__ b;
  const int8_t *__restrict__ rt;
  double *y, *ybar;
  double sigma, w;
  uint8_t *mask;  // adjoint recording: 1 where the projection is inactive, or null
  struct Pre { double b, y, yb; int t; };
  __device__ __forceinline__ Pre load(int i) const { return {b[i], y[i], ybar[i], (int)rt[i]}; }
  __device__ __forceinline__ double init(const Pre &p) const { return -p.b; }
  __device__ __forceinline__ void store(int i, double r, double, const Pre &p) const {
    long long bits = __double_as_longlong(fma(-sigma, r, p.y));  // y + sigma (b - A xhat)
    if (mask) mask[i] = (p.t == 0 || (p.t == 1 && bits > 0) || (p.t == 2 && bits < 0)) ? 1 : 0;
    if (p.t == 1 && bits < 0) bits = 0;       // GE: [0, inf)
    else if (p.t == 2 && bits > 0) bits = 0;  // LE: (-inf, 0]
    const double yn = __longlong_as_double(bits);
    y[i] = yn;
    ybar[i] = fma(w, yn - p.yb, p.yb);
  }
};

struct StoreEpi {
  double *out;
  struct Pre {};
  __device__ __forceinline__ Pre load(int) const { return {}; }
  __device__ __forceinline__ double init(const Pre &) const { return 0.0; }
  __device__ __forceinline__ void store(int r, double a, double, const Pre &) const { out[r] = a; }
};

// Sign, magnitude and class tests on a double's bit pattern (integer pipe;
// GB300 issues 2 FP64 operations per cycle per SM, comparisons and min/max
// included).  For non-NaN v: pos(v) <=> v > 0, neg(v) <=> v < 0.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ bool pos_d(double v) { return dbits(v) > 0; }
__device__ __forceinline__ bool neg_d(double v) {
  const long long b = dbits(v);
  return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool nonzero_d(double v) { return (dbits(v) << 1) != 0; }
__device__ __forceinline__ bool finite_d(double v) {
  return (dbits(v) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
__device__ __forceinline__ double abs_d(double v) {
  return __longlong_as_double(dbits(v) & 0x7fffffffffffffffll);
}
// max(v, +0) for non-NaN v (-0 maps to +0)
__device__ __forceinline__ double pos_part(double v) { return dbits(v) < 0 ? 0.0 : v; }
constexpr long long kNegInfBits = (long long)0xfff0000000000000ull;
constexpr long long kPosInfBits = 0x7ff0000000000000ll;

// One coordinate of the linear trust region of Section 6.3 in the
// omega-rescaled space: objective component G, distance dist >= 0 to the
// bound it moves toward (INFINITY if none), scales sd (distance) and sg
// (objective).  Breakpoint lambda_hat = d / g; its bit pattern is the key.
struct GapOut {
  uint64_t *keys;
  double *d2, *g2, *gd;
};

__device__ __forceinline__ void gap_elem(double G, double dist, double sd, double sg, int64_t e,
                                         const GapOut &o, double &sum_d2, double &sum_gd,
                                         double &sum_g2inf) {
  uint64_t key = kNoKey;
  if (nonzero_d(G)) {
    const double g = abs_d(G) * sg;
    if (!finite_d(dist)) {
      sum_g2inf += g * g;
    } else {
      const double d = dist * sd;
      const double lam = d / g;
      if (!finite_d(lam)) {
        sum_g2inf += g * g;
      } else {
        key = (uint64_t)dbits(lam);
        const double vd2 = d * d, vg2 = g * g, vgd = d * g;
        sum_d2 += vd2;
        sum_gd += vgd;
        o.d2[e] = vd2;
        o.g2[e] = vg2;
        o.gd[e] = vgd;
      }
    }
  }
  o.keys[e] = key;
}

// Check epilogue over columns (x-space): reduced costs lam = c - A^T y for
// both candidates, dual residual, dual-objective bound terms, primal
// objective, and the x-part of the trust region with F_x = lam.
// Lambda_j (the reduced-cost cone of column j) is R with both bounds, [0,inf)
// with only l finite, (-inf,0] with only u finite, {0} if free: the
// projection of lam keeps lam when its sign is allowed and is 0 otherwise.
struct CheckColsEpi {
  // quantities the epilogue accumulates (the current iterate's gap data only
  // under the flexible scheme)
  static constexpr uint32_t kUsed =
      (1u << Q_RD2_A) | (1u << Q_RD2_C) | (1u << Q_POBJ_A) | (1u << Q_POBJ_C) |
      (1u << Q_DOBJ_A) | (1u << Q_DOBJ_C) | (1u << Q_RRX_A) | (1u << Q_D2_A) | (1u << Q_GD_A) |
      (1u << Q_G2INF_A) | (1u << Q_BAD);
  static constexpr uint32_t kUsedGapC =
      (1u << Q_RRX_C) | (1u << Q_D2_C) | (1u << Q_GD_C) | (1u << Q_G2INF_C);
  const double *__restrict__ c;
  const double *__restrict__ lb;
  const double *__restrict__ ub;
  const double *__restrict__ xbar;
  const double *__restrict__ x;
  const double *__restrict__ x0;
  GapOut ga, gc;
  double *lam_out0, *lam_out1;  // mixed precision: c - A^T y of both candidates, or null
  double sw, isw;
  int gap_a, gap_c;
  double q[NQ];
  // split rows: the reductions of each split row go to
  // split_slots[q * slot_stride + (slice of its first chunk)] (see
  // process_split_item); null when the matrix has no split rows
  static constexpr bool kSplitSlots = true;
  double *split_slots = nullptr;
  int slot_stride = 0;
  __device__ __forceinline__ void zero_split_slot(int item) const {
#pragma unroll
    for (int i = 0; i < NQ; ++i) split_slots[(size_t)i * slot_stride + item] = 0.0;
  }
  __device__ __forceinline__ void flush_split_slot(int first) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      split_slots[(size_t)i * slot_stride + first] = q[i];
      q[i] = 0.0;
    }
  }
  struct Pre { double c, lb, ub, xb, x, x0; };
  __device__ __forceinline__ Pre load(int j) const {
    return {c[j], lb[j], ub[j], xbar[j], x[j], x0[j]};
  }
  __device__ __forceinline__ double init(const Pre &) const { return 0.0; }
  __device__ __forceinline__ void candidate(int j, double lam, double xv, const Pre &p, bool lf,
                                            bool uf, int qrd, int qdobj, int qpobj, int qrrx,
                                            int qd2, int qgd, int qg2inf, bool gap,
                                            const GapOut &go) {
    const bool lp = pos_d(lam), ln = neg_d(lam);
    const bool keep = (lp && lf) || (ln && uf);    // lam inside Lambda_j
    const double off = keep ? 0.0 : lam;            // lam - proj(lam)
    q[qrd] += off * off;
    if (keep) q[qdobj] += (lp ? p.lb : p.ub) * lam;  // l proj(lam)^+ - u proj(lam)^-
    q[qpobj] += p.c * xv;
    if (gap) {
      const double dx = xv - p.x0;
      q[qrrx] += dx * dx;
      double dist = INFINITY;
      if (lp && lf) dist = pos_part(xv - p.lb);
      if (ln && uf) dist = pos_part(p.ub - xv);
      gap_elem(lam, dist, sw, isw, j, go, q[qd2], q[qgd], q[qg2inf]);
    }
  }
  __device__ __forceinline__ void store(int j, double aty_a, double aty_c, const Pre &p) {
    const bool lf = dbits(p.lb) != kNegInfBits, uf = dbits(p.ub) != kPosInfBits;
    const double lam_a = p.c - aty_a, lam_c = p.c - aty_c;
    if (lam_out0) {
      lam_out0[j] = lam_a;
      lam_out1[j] = lam_c;
    }
    candidate(j, lam_a, p.xb, p, lf, uf, Q_RD2_A, Q_DOBJ_A, Q_POBJ_A, Q_RRX_A, Q_D2_A, Q_GD_A,
              Q_G2INF_A, gap_a, ga);
    candidate(j, lam_c, p.x, p, lf, uf, Q_RD2_C, Q_DOBJ_C, Q_POBJ_C, Q_RRX_C, Q_D2_C, Q_GD_C,
              Q_G2INF_C, gap_c, gc);
    if (!(finite_d(lam_a) && finite_d(lam_c) && finite_d(p.xb) && finite_d(p.x))) q[Q_BAD] += 1.0;
  }
};

// Check epilogue over rows (y-space): primal residual by row sense, b^T y,
// and the y-part of the trust region with F_y = A x - b.
struct CheckRowsEpi {
  static constexpr uint32_t kUsed =
      (1u << Q_RP2_A) | (1u << Q_RP2_C) | (1u << Q_DOBJ_A) | (1u << Q_DOBJ_C) | (1u << Q_RRY_A) |
      (1u << Q_D2_A) | (1u << Q_GD_A) | (1u << Q_G2INF_A) | (1u << Q_BAD);
  static constexpr uint32_t kUsedGapC =
      (1u << Q_RRY_C) | (1u << Q_D2_C) | (1u << Q_GD_C) | (1u << Q_G2INF_C);
  const double *__restrict__ b;
  const int8_t *__restrict__ rt;
  const double *__restrict__ ybar;
  const double *__restrict__ y;
  const double *__restrict__ y0;
  GapOut ga, gc;
  double *gy_out0, *gy_out1;  // mixed precision: A x - b of both candidates, or null
  double sw, isw;
  int64_t off;  // element offset of the y-part in the search arrays (= n)
  int gap_a, gap_c;
  double q[NQ];
  // split rows: the reductions of each split row go to
  // split_slots[q * slot_stride + (slice of its first chunk)] (see
  // process_split_item); null when the matrix has no split rows
  static constexpr bool kSplitSlots = true;
  double *split_slots = nullptr;
  int slot_stride = 0;
  __device__ __forceinline__ void zero_split_slot(int item) const {
#pragma unroll
    for (int i = 0; i < NQ; ++i) split_slots[(size_t)i * slot_stride + item] = 0.0;
  }
  __device__ __forceinline__ void flush_split_slot(int first) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      split_slots[(size_t)i * slot_stride + first] = q[i];
      q[i] = 0.0;
    }
  }
  struct Pre { double b, yb, y, y0; int t; };
  __device__ __forceinline__ Pre load(int i) const { return {b[i], ybar[i], y[i], y0[i], (int)rt[i]}; }
  __device__ __forceinline__ double init(const Pre &) const { return 0.0; }
  __device__ __forceinline__ void candidate(int i, double G, double yv, const Pre &p, int qrp,
                                            int qdobj, int qrry, int qd2, int qgd, int qg2inf,
                                            bool gap, const GapOut &go) {
    const bool gp = pos_d(G), gn = neg_d(G);
    // residual of A x >= b (GE) counts only G < 0, of A x <= b (LE) only G > 0
    const double v = (p.t == 1 && !gn) || (p.t == 2 && !gp) ? 0.0 : G;
    q[qrp] += v * v;
    q[qdobj] += p.b * yv;
    if (gap) {
      const double dy = yv - p.y0;
      q[qrry] += dy * dy;
      double dist = INFINITY;
      if (gp && p.t == 1) dist = pos_part(yv);
      if (gn && p.t == 2) dist = pos_part(-yv);
      gap_elem(G, dist, isw, sw, off + i, go, q[qd2], q[qgd], q[qg2inf]);
    }
  }
  __device__ __forceinline__ void store(int i, double ax_a, double ax_c, const Pre &p) {
    const double va = ax_a - p.b, vc = ax_c - p.b;
    if (gy_out0) {
      gy_out0[i] = va;
      gy_out1[i] = vc;
    }
    candidate(i, va, p.yb, p, Q_RP2_A, Q_DOBJ_A, Q_RRY_A, Q_D2_A, Q_GD_A, Q_G2INF_A, gap_a, ga);
    candidate(i, vc, p.y, p, Q_RP2_C, Q_DOBJ_C, Q_RRY_C, Q_D2_C, Q_GD_C, Q_G2INF_C, gap_c, gc);
    if (!(finite_d(ax_a) && finite_d(ax_c) && finite_d(p.yb) && finite_d(p.y))) q[Q_BAD] += 1.0;
  }
};

// --------------------------------------------------- mixed precision
//
// FP32 PDHG step on the correction dz = s (z - z^{n,0}): the same update as
// Eq. (PDHG-update) with the correction's data (cf, bf, bounds lf/uf,
// ylo/yhi), FP32 matrix values and FP32 accumulation; the running average
// of the correction stays in FP64.
struct PrimalMixEpi {
  const float *__restrict__ cf;
  const float *__restrict__ lf;
  const float *__restrict__ uf;
  float *dx, *dxhat;
  double *dxbar;
  float tau;
  double w;
  struct Pre { float c, l, u, x; double xb; };
  __device__ __forceinline__ Pre load(int j) const { return {cf[j], lf[j], uf[j], dx[j], dxbar[j]}; }
  __device__ __forceinline__ float init(const Pre &p) const { return -p.c; }
  __device__ __forceinline__ void store(int j, float neg_g, float, const Pre &p) const {
    const float xn = fminf(fmaxf(fmaf(tau, neg_g, p.x), p.l), p.u);
    dx[j] = xn;
    dxhat[j] = fmaf(2.0f, xn, -p.x);
    dxbar[j] = fma(w, (double)xn - p.xb, p.xb);
  }
};

struct DualMixEpi {
  const float *__restrict__ bf;
  const float *__restrict__ lo;
  const float *__restrict__ hi;
  float *dy;
  double *dybar;
  float sigma;
  double w;
  struct Pre { float b, l, h, y; double yb; };
  __device__ __forceinline__ Pre load(int i) const { return {bf[i], lo[i], hi[i], dy[i], dybar[i]}; }
  __device__ __forceinline__ float init(const Pre &p) const { return -p.b; }
  __device__ __forceinline__ void store(int i, float r, float, const Pre &p) const {
    const float yn = fminf(fmaxf(fmaf(-sigma, r, p.y), p.l), p.h);
    dy[i] = yn;
    dybar[i] = fma(w, (double)yn - p.yb, p.yb);
  }
};

// Adjoint of one unrolled step (reverse mode, masks of the recomputed
// forward step, restart decisions held fixed).  With adjoints (ax, ay, axb,
// ayb) of the outputs (x, y, xbar, ybar) of step k:
//   u   = D_y (ay + w ayb),  grad_b += sigma u,  ayb <- (1 - w) ayb
//   v   = D_x (ax + w axb - 2 sigma A^T u),       grad_c -= tau v
//   ax <- v + sigma A^T u,   axb <- (1 - w) axb,  ay <- u + tau A v
struct AdjColsEpi {
  double *ax, *axb, *ac, *v;
  const uint8_t *__restrict__ mx;
  double tau, sigma, w;
  struct Pre { double ax, axb, ac; int m; };
  __device__ __forceinline__ Pre load(int j) const { return {ax[j], axb[j], ac[j], (int)mx[j]}; }
  __device__ __forceinline__ double init(const Pre &) const { return 0.0; }
  __device__ __forceinline__ void store(int j, double atu, double, const Pre &p) const {
    const double adj_xhat = -sigma * atu;
    const double adj_xp = fma(2.0, adj_xhat, fma(w, p.axb, p.ax));
    const double vv = p.m ? adj_xp : 0.0;
    ax[j] = vv - adj_xhat;
    ac[j] = fma(-tau, vv, p.ac);
    axb[j] = (1.0 - w) * p.axb;
    v[j] = vv;
  }
};

struct AdjRowsEpi {
  double *ay, *ayb, *ab, *u;
  const uint8_t *__restrict__ my_prev;
  double tau, sigma, w_prev;
  int has_prev;
  struct Pre { double u, ayb, ab; int mp; };
  __device__ __forceinline__ Pre load(int i) const {
    return {u[i], ayb[i], ab[i], has_prev ? (int)my_prev[i] : 0};
  }
  __device__ __forceinline__ double init(const Pre &) const { return 0.0; }
  __device__ __forceinline__ void store(int i, double av, double, const Pre &p) const {
    const double ayk = fma(tau, av, p.u);
    ay[i] = ayk;
    if (has_prev) {
      const double up = p.mp ? fma(w_prev, p.ayb, ayk) : 0.0;
      ab[i] = fma(sigma, up, p.ab);
      ayb[i] = (1.0 - w_prev) * p.ayb;
      u[i] = up;
    }
  }
};

// ------------------------------------------------------ check helpers

__device__ __forceinline__ void init_search(LSearch &L, double r, double d2, double gd, double g2inf) {
  L.r2 = r * r;
  L.f_lo = 0.0;
  L.e_lo = 0.0;
  L.f_hi = g2inf;
  L.prefix = 0ull;
  L.lambda = 0.0;
  L.rho_r = 0.0;
  L.done = 0;
  if (r == 0.0) {
    L.done = 1;  // zero radius: rho := 0 (Section 6.1)
  } else if (g2inf == 0.0 && d2 <= L.r2) {
    L.done = 1;  // the full clamp is inside the ball (Algorithm 2, first test)
    L.lambda = INFINITY;
    L.rho_r = gd;
  }
}

__device__ __forceinline__ void kkt_from(const double *t, int qp, int qd, int qpo, int qdo, double nb, double nc,
                         double *out) {
  const double rp = sqrt(t[qp]), rd = sqrt(t[qd]);
  const double p = t[qpo], d = t[qdo];
  double rel = fmax(rp / (1.0 + nb), rd / (1.0 + nc));
  rel = fmax(rel, fabs(p - d) / (1.0 + fabs(p) + fabs(d)));
  out[0] = rp; out[1] = rd; out[2] = p; out[3] = d; out[4] = rel;
}

// Fixed-order inclusive scan of 256 values held one per thread of the
// first 256 threads (8 warps): shuffle scan inside each warp, then the warp
// totals.  Returns the inclusive prefix for thread b.
__device__ __forceinline__ double scan256(double v, double *warp_tot) {
  const int b = threadIdx.x, lane = b & 31, w = b >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_tot[w] = v;
  __syncwarp();
  return v;
}


// ------------------------------------------------- Lanczos Ritz value
//
// Largest eigenvalue of the symmetric tridiagonal Lanczos matrix T_k
// (diagonal a[0..k-1], off-diagonal b[0..k-2]) by Sturm-sequence
// multisection (the bisection method for symmetric tridiagonal matrices,
// Golub & Van Loan, Matrix Computations, Section 8.4.1), run by one full
// warp: each round, lane l counts the eigenvalues below the l-th of 32
// interior points of the bracket [lo, hi] and the bracket shrinks to the
// interval where the count first reaches k.  lo starts at the largest
// diagonal entry (a lower bound on the largest eigenvalue), hi at the
// largest Gershgorin row bound (an upper bound).  Returns the bracket's
// midpoint (exactly lo when lo = hi, e.g. a 1 x 1 or zero matrix).
__device__ __forceinline__ int sturm_count_below(const double *a, const double *b, int k,
                                                 double x, double pivmin) {
  int c = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    d = (i == 0) ? a[0] - x : a[i] - x - b[i - 1] * b[i - 1] / d;
    if (fabs(d) < pivmin) d = -pivmin;
    c += d < 0.0;
  }
  return c;
}

__device__ double tridiag_top_eig(const double *a, const double *b, int k) {
  const int lane = threadIdx.x & (kWarp - 1);
  double lo = -INFINITY, hi = -INFINITY, bmax2 = 0.0;
  for (int i = lane; i < k; i += kWarp) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmax(lo, a[i]);
    hi = fmax(hi, a[i] + r);
    if (i + 1 < k) bmax2 = fmax(bmax2, b[i] * b[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmax(lo, __shfl_xor_sync(kFull, lo, o));
    hi = fmax(hi, __shfl_xor_sync(kFull, hi, o));
    bmax2 = fmax(bmax2, __shfl_xor_sync(kFull, bmax2, o));
  }
  // the largest eigenvalue lies in [lo, hi]; when no point of a round has all
  // k eigenvalues below it, it lies above the last point
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, bmax2);
  for (int round = 0; round < 24 && hi - lo > 2.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi));
       ++round) {
    const double w = (hi - lo) / 33.0;
    const double x = lo + w * (double)(lane + 1);
    const unsigned all = __ballot_sync(kFull, sturm_count_below(a, b, k, x, pivmin) >= k);
    if (all == 0u) {
      lo = lo + w * 32.0;
    } else {
      const int f = __ffs(all) - 1;
      const double nlo = lo + w * (double)f, nhi = lo + w * (double)(f + 1);
      lo = nlo;
      hi = nhi;
    }
  }
  return 0.5 * (lo + hi);
}

}  // namespace
}  // namespace lpg
