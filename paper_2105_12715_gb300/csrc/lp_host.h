// Host-side helpers shared by the single-problem API (lp_api.cu) and the
// batched API (lp_batch.cu): error reporting, input copies, option checks,
// and the construction of the sliced device layout of a sparse operator.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lp.h"
#include "lp_internal.h"

namespace lpg {

// Message of the last failed call on the calling thread.
inline std::string &err_msg() {
  static thread_local std::string s;
  return s;
}


inline lp_status fail(lp_status s, const std::string &msg) {
  err_msg() = msg;
  return s;
}

inline lp_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define LP_CU(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct HostSell {
  int32_t nrows = 0, ncols = 0, nslices = 0, n_warp_rows = 0;
  std::vector<SliceInfo> info;
  std::vector<int32_t> idx;
  std::vector<double> val;
};

// Lanes per row: rows of at most single_max elements get one lane (no
// cross-lane sum); longer rows get the fewest lanes G = 2^lg (<= 32) with
// ceil(len / G) <= lane_steps, so that no lane's chain of dependent
// gathers is long; rows of at least warp_threshold elements take a warp.
struct LanePolicy {
  int32_t warp_threshold, lane_steps, single_max;
};

inline int lanes_log2(int64_t len, const LanePolicy &p) {
  if (len >= p.warp_threshold) return 5;
  if (len <= p.single_max) return 0;
  int lg = 0;
  while (lg < 5 && (int64_t(p.lane_steps) << lg) < len) ++lg;
  return lg;
}

// Row limit of the slice starting at row r: the first break after r (rows
// where a slice must start, ascending; the starts of batched problems), or
// nrows.  *bi walks the breaks as r grows.
inline int32_t slice_limit(const std::vector<int32_t> &breaks, size_t *bi, int32_t r,
                           int32_t nrows) {
  while (*bi < breaks.size() && breaks[*bi] <= r) ++*bi;
  return *bi < breaks.size() ? std::min(breaks[*bi], nrows) : nrows;
}

// Number of slices the layout of rows perm[0..) (longest first within each
// segment between breaks) would have.
inline int64_t count_slices(const std::vector<int64_t> &ptr, const std::vector<int32_t> &perm,
                            const LanePolicy &p, const std::vector<int32_t> &breaks = {}) {
  const int32_t nrows = (int32_t)perm.size();
  int64_t ns = 0;
  int32_t r = 0;
  size_t bi = 0;
  while (r < nrows) {
    const int32_t lim = slice_limit(breaks, &bi, r, nrows);
    const int lg = lanes_log2(ptr[perm[r] + 1] - ptr[perm[r]], p);
    const int cap = kWarp >> lg;
    int32_t q = r;
    while (q < lim && q - r < cap && lanes_log2(ptr[perm[q] + 1] - ptr[perm[q]], p) == lg) ++q;
    ++ns;
    r = q;
  }
  return ns;
}

// Launch-shape tuning by a model: a pass runs one warp per slice, and
// fewer slices than `target` warps leave SMs idle while each warp walks a
// long chain of dependent gathers.  Starting from the given policy, give
// rows more lanes (halving single_max and lane_steps) until the layout
// has at least `target` slices or rows get one element per lane.
inline LanePolicy choose_policy(const std::vector<int64_t> &ptr, const std::vector<int32_t> &perm,
                                LanePolicy p, int64_t target,
                                const std::vector<int32_t> &breaks = {}) {
  if (target <= 0) return p;
  while (count_slices(ptr, perm, p, breaks) < target && (p.single_max > 1 || p.lane_steps > 1)) {
    p.single_max = p.single_max / 2;
    p.lane_steps = std::max(1, p.lane_steps / 2);
  }
  return p;
}

// Sliced layout (see SellMat) of the operator whose row r (permuted order)
// is original row perm[r] of the CSR (ptr, ind, v); column indices
// relabeled by relabel.  Rows come longest first, so a slice is closed when
// it is full (32 / G rows), when the next row wants another G, or at a
// break (no slice spans two batched problems).
inline void build_sell(int32_t nrows, int32_t ncols, const std::vector<int64_t> &ptr,
                       const std::vector<int32_t> &ind, const std::vector<double> &v,
                       const std::vector<int32_t> &perm, const std::vector<int32_t> &relabel,
                       const LanePolicy &policy, HostSell &S,
                       const std::vector<int32_t> &breaks = {}) {
  S.nrows = nrows;
  S.ncols = ncols;
  auto len = [&](int32_t r) { return ptr[perm[r] + 1] - ptr[perm[r]]; };
  S.info.clear();
  int64_t off = 0;
  int32_t r = 0;
  size_t bi = 0;
  while (r < nrows) {
    const int32_t lim = slice_limit(breaks, &bi, r, nrows);
    const int lg = lanes_log2(len(r), policy);
    const int cap = kWarp >> lg;
    int32_t q = r;
    int64_t mx = 0;
    while (q < lim && q - r < cap && lanes_log2(len(q), policy) == lg) {
      mx = std::max<int64_t>(mx, len(q));
      ++q;
    }
    const int64_t steps = (mx + (int64_t(1) << lg) - 1) >> lg;
    if (lg == 5) S.n_warp_rows += q - r;
    S.info.push_back(SliceInfo{off, r, (int32_t)((steps << 3) | lg)});
    off += steps * kWarp;
    r = q;
  }
  S.nslices = (int32_t)S.info.size();
  S.info.push_back(SliceInfo{off, nrows, 0});
  S.idx.assign(off, 0);
  S.val.assign(off, 0.0);
  for (int32_t s = 0; s < S.nslices; ++s) {
    const SliceInfo &a = S.info[s];
    const int lg = a.len_g & 7, G = 1 << lg;
    for (int32_t row = a.row0; row < S.info[s + 1].row0; ++row) {
      const int64_t src = ptr[perm[row]];
      const int64_t lane0 = (int64_t)(row - a.row0) * G;
      for (int64_t k = 0; k < len(row); ++k) {
        const int64_t dst = a.off + kWarp * (k >> lg) + lane0 + (k & (G - 1));
        S.idx[dst] = relabel[ind[src + k]];
        S.val[dst] = v[src + k];
      }
    }
  }
}

template <class T>
inline bool copy_in(std::vector<T> &dst, const T *src, int64_t count) {
  dst.resize(count);
  if (count == 0) return true;
  return cudaMemcpy(dst.data(), src, sizeof(T) * count, cudaMemcpyDefault) == cudaSuccess;
}

inline lp_status validate_options(const lp_options &o) {
  if (!(o.beta > 0.0 && o.beta < 1.0)) return fail(LP_ERR_INVALID_ARG, "beta must lie in (0, 1)");
  if (o.check_every < 1 || o.check_every > 65536)
    return fail(LP_ERR_INVALID_ARG, "check_every must lie in [1, 65536]");
  if (o.restart_scheme < LP_RESTART_NONE || o.restart_scheme > LP_RESTART_FLEXIBLE)
    return fail(LP_ERR_INVALID_ARG, "unknown restart_scheme");
  if (o.tau0 < 0 || o.fixed_len < 0) return fail(LP_ERR_INVALID_ARG, "tau0 and fixed_len must be >= 0");
  if (!(o.omega > 0.0) || !std::isfinite(o.omega)) return fail(LP_ERR_INVALID_ARG, "omega must be finite and > 0");
  if (!(o.eta >= 0.0) || !std::isfinite(o.eta)) return fail(LP_ERR_INVALID_ARG, "eta must be finite and >= 0");
  if (o.power_iters < 1) return fail(LP_ERR_INVALID_ARG, "power_iters must be >= 1");
  if (!(o.power_tol >= 0.0)) return fail(LP_ERR_INVALID_ARG, "power_tol must be >= 0");
  if (o.max_iter < 0) return fail(LP_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (o.long_row_threshold < 1) return fail(LP_ERR_INVALID_ARG, "long_row_threshold must be >= 1");
  if (o.trace_capacity < 0) return fail(LP_ERR_INVALID_ARG, "trace_capacity must be >= 0");
  for (int32_t u : {o.spmv_unroll, o.spmv_unroll_rows}) {
    const int32_t b = u % 100;
    if (u / 100 < -1 || u / 100 > 1 || (b != 2 && b != 4 && b != 8 && b != -2 && b != -4))
      return fail(LP_ERR_INVALID_ARG,
                  "spmv_unroll(_rows) must be 2, 4, 8, -2 or -4, or that +-100 (capped registers)");
  }
  if (o.lane_steps < 1 || o.lane_steps > 1024) return fail(LP_ERR_INVALID_ARG, "lane_steps must lie in [1, 1024]");
  if (o.single_lane_max < 0) return fail(LP_ERR_INVALID_ARG, "single_lane_max must be >= 0");
  if (o.spmv_mode != 0 && o.spmv_mode != 1) return fail(LP_ERR_INVALID_ARG, "spmv_mode must be 0 or 1");
  if (o.lane_auto < 0) return fail(LP_ERR_INVALID_ARG, "lane_auto must be >= 0");
  if (o.precision != LP_PRECISION_FP64 && o.precision != LP_PRECISION_MIXED)
    return fail(LP_ERR_INVALID_ARG, "precision must be LP_PRECISION_FP64 or LP_PRECISION_MIXED");
  return LP_OK;
}

}  // namespace lpg
