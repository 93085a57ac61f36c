// Host-side helpers shared by the single-problem API (lp_api.cu) and the
// batched API (lp_batch.cu): error reporting, input copies, option checks,
// and the construction of the sliced device layout of a sparse operator.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

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

// NVTX range around an entry point (header-only NVTX3: a no-op unless a
// profiler is attached), so a timeline shows the library's phases.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

#define LP_CU(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// ---- host parallelism for the set-up (deterministic: fixed partitions)

// Allocator whose construct() leaves elements uninitialized, so that
// resize() of a large array the caller fills completely costs nothing.
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U> &) {}
  template <class U>
  void construct(U *) noexcept {}
  template <class U, class... A>
  void construct(U *p, A &&...a) {
    ::new ((void *)p) U(std::forward<A>(a)...);
  }
};
template <class T>
using uvec = std::vector<T, UninitAlloc<T>>;

inline int host_threads() {
  static const int t = [] {
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h, 32u));
  }();
  return t;
}

// Runs f(t) for t = 0..nt-1, on nt threads (the calling thread takes the
// chunks whose thread could not be started).
template <class F>
inline void run_threads(int nt, F f) {
  if (nt <= 1) {
    f(0);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  int started = 1;
  try {
    for (int t = 1; t < nt; ++t) {
      th.emplace_back([&f, t] { f(t); });
      started = t + 1;
    }
  } catch (...) {
  }
  f(0);
  for (int t = started; t < nt; ++t) f(t);
  for (auto &x : th) x.join();
}

// f(begin, end) over [0, n) in contiguous chunks, one per thread.
template <class F>
inline void parallel_for(int64_t n, F f, int64_t grain = 16384) {
  const int nt = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / grain));
  run_threads(nt, [&](int t) { f(n * t / nt, n * (t + 1) / nt); });
}

// CSC copy (cp[n + 1], ri[nnz], cv[nnz]) of the CSR (rp[m + 1], ci, v) with
// rows ascending within each column: a stable counting sort in which thread t
// owns the columns [n t / T, n (t + 1) / T) and scans the whole CSR in row
// order.  Returns false if a column index lies outside [0, n).
inline bool build_csc(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                      std::vector<int64_t> &cp, uvec<int32_t> &ri, uvec<double> &cv) {
  const int64_t nnz = rp[m];
  cp.assign((size_t)n + 1, 0);
  ri.resize((size_t)nnz);
  cv.resize((size_t)nnz);
  std::atomic<int> bad{0};
  parallel_for(nnz, [&](int64_t lo, int64_t hi) {
    for (int64_t p = lo; p < hi; ++p)
      if (ci[p] < 0 || ci[p] >= n) bad.store(1, std::memory_order_relaxed);
  });
  if (bad.load()) return false;
  const int nt = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, nnz / 262144));
  run_threads(nt, [&](int t) {
    const int32_t lo = (int32_t)((int64_t)n * t / nt), hi = (int32_t)((int64_t)n * (t + 1) / nt);
    for (int64_t p = 0; p < nnz; ++p) {
      const int32_t j = ci[p];
      if (j >= lo && j < hi) cp[(size_t)j + 1]++;
    }
  });
  for (int32_t j = 0; j < n; ++j) cp[(size_t)j + 1] += cp[j];
  run_threads(nt, [&](int t) {
    const int32_t lo = (int32_t)((int64_t)n * t / nt), hi = (int32_t)((int64_t)n * (t + 1) / nt);
    std::vector<int64_t> pos(cp.begin() + lo, cp.begin() + hi);
    for (int32_t i = 0; i < m; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        const int32_t j = ci[p];
        if (j >= lo && j < hi) {
          const int64_t q = pos[j - lo]++;
          ri[q] = i;
          cv[q] = v[p];
        }
      }
  });
  return true;
}

// True if some column of the CSC lists a row twice (rows are ascending, so
// a repeat is adjacent): a column repeated within a row of the CSR.
inline bool csc_has_duplicates(int32_t n, const std::vector<int64_t> &cp, const uvec<int32_t> &ri) {
  std::atomic<int> dup{0};
  parallel_for(n, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j)
      for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p)
        if (ri[p] == ri[p - 1]) dup.store(1, std::memory_order_relaxed);
  });
  return dup.load() != 0;
}

// perm[begin..end) <- begin..end-1 ordered by decreasing ptr[i+1] - ptr[i],
// ties in index order (a stable counting sort on the length).
template <class P>
inline void sort_by_length_desc(const P *ptr, int32_t begin, int32_t end, int32_t *perm) {
  if (end <= begin) return;
  int64_t mx = 0;
  for (int32_t i = begin; i < end; ++i) mx = std::max<int64_t>(mx, ptr[i + 1] - ptr[i]);
  std::vector<int64_t> cnt((size_t)mx + 2, 0);
  for (int32_t i = begin; i < end; ++i) cnt[(size_t)(mx - (ptr[i + 1] - ptr[i])) + 1]++;
  for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
  for (int32_t i = begin; i < end; ++i) perm[begin + cnt[(size_t)(mx - (ptr[i + 1] - ptr[i]))]++] = i;
}

struct HostSell {
  int32_t nrows = 0, ncols = 0, nslices = 0, n_warp_rows = 0;
  std::vector<SliceInfo> info;
  std::vector<SplitSlice> split;  // chunk slices of split rows (slices 0 .. split.size() - 1)
  uvec<int32_t> idx;
  uvec<double> val;
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
// break (no slice spans two batched problems).  With split_len > 0 (no
// breaks), a whole-warp row longer than split_len becomes ceil(len /
// split_len) chunk slices of at most split_len elements; being the longest,
// these rows come first, so their chunk slices are slices 0 .. nsplit - 1.
inline void build_sell(int32_t nrows, int32_t ncols, const std::vector<int64_t> &ptr,
                       const int32_t *ind, const double *v,
                       const std::vector<int32_t> &perm, const std::vector<int32_t> &relabel,
                       const LanePolicy &policy, HostSell &S,
                       const std::vector<int32_t> &breaks = {}, int32_t split_len = 0) {
  S.nrows = nrows;
  S.ncols = ncols;
  auto len = [&](int32_t r) { return ptr[perm[r] + 1] - ptr[perm[r]]; };
  S.info.clear();
  S.split.clear();
  int64_t off = 0;
  int32_t r = 0;
  size_t bi = 0;
  while (r < nrows) {
    const int32_t lim = slice_limit(breaks, &bi, r, nrows);
    const int lg = lanes_log2(len(r), policy);
    if (split_len > 0 && breaks.empty() && lg == 5 && len(r) > split_len &&
        S.split.size() == S.info.size()) {
      const int64_t L = len(r);
      const int32_t nch = (int32_t)((L + split_len - 1) / split_len);
      const int32_t first = (int32_t)S.info.size();
      for (int32_t c = 0; c < nch; ++c) {
        const int64_t clen = std::min<int64_t>(split_len, L - (int64_t)c * split_len);
        const int64_t steps = (clen + kWarp - 1) / kWarp;
        S.info.push_back(SliceInfo{off, r, (int32_t)((steps << 3) | 5)});
        S.split.push_back(SplitSlice{c, nch, first, c * split_len});
        off += steps * kWarp;
      }
      S.n_warp_rows += 1;
      ++r;
      continue;
    }
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
  S.idx.resize((size_t)off);
  S.val.resize((size_t)off);
  // slices in parallel, in chunks of about equal element counts; each slice
  // zero-fills its region (padding) and writes its rows' elements
  const int nt = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, off / 65536));
  run_threads(nt, [&](int t) {
    const int64_t e_lo = off * t / nt, e_hi = off * (t + 1) / nt;
    auto first_slice = [&](int64_t e) {  // first slice starting at or after element e
      int32_t lo = 0, hi = S.nslices;
      while (lo < hi) {
        const int32_t mid = (lo + hi) / 2;
        if (S.info[mid].off < e) lo = mid + 1;
        else hi = mid;
      }
      return lo;
    };
    const int32_t s_lo = t == 0 ? 0 : first_slice(e_lo);
    const int32_t s_hi = t == nt - 1 ? S.nslices : first_slice(e_hi);
    for (int32_t sl = s_lo; sl < s_hi; ++sl) {
      const SliceInfo &a = S.info[sl];
      const int lg = a.len_g & 7, G = 1 << lg;
      std::fill(S.idx.begin() + a.off, S.idx.begin() + S.info[sl + 1].off, 0);
      std::fill(S.val.begin() + a.off, S.val.begin() + S.info[sl + 1].off, 0.0);
      if (sl < (int32_t)S.split.size()) {  // a chunk of a split row (G = 32)
        const SplitSlice &sp = S.split[sl];
        const int64_t src = ptr[perm[a.row0]] + sp.begin;
        const int64_t clen = std::min<int64_t>(split_len, len(a.row0) - sp.begin);
        for (int64_t k = 0; k < clen; ++k) {
          S.idx[a.off + k] = relabel[ind[src + k]];
          S.val[a.off + k] = v[src + k];
        }
        continue;
      }
      for (int32_t row = a.row0; row < S.info[sl + 1].row0; ++row) {
        const int64_t src = ptr[perm[row]];
        const int64_t lane0 = (int64_t)(row - a.row0) * G;
        for (int64_t k = 0; k < len(row); ++k) {
          const int64_t dst = a.off + kWarp * (k >> lg) + lane0 + (k & (G - 1));
          S.idx[dst] = relabel[ind[src + k]];
          S.val[dst] = v[src + k];
        }
      }
    }
  });
}

// A host-readable view of count elements at src: device memory is copied
// into storage, host memory (pageable, pinned or managed) is read in place.
// *ok becomes false if src cannot be read.
template <class T>
inline const T *host_view(const T *src, int64_t count, std::vector<T> &storage, bool *ok) {
  if (count <= 0) return src;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, src) != cudaSuccess) {
    cudaGetLastError();
    *ok = false;
    return nullptr;
  }
  if (at.type != cudaMemoryTypeDevice) return src;
  storage.resize((size_t)count);
  if (cudaMemcpy(storage.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    *ok = false;
    return nullptr;
  }
  return storage.data();
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
  if (o.spmv_mode != 0) return fail(LP_ERR_INVALID_ARG, "spmv_mode must be 0 (reserved)");
  if (o.lane_auto < 0) return fail(LP_ERR_INVALID_ARG, "lane_auto must be >= 0");
  if (o.autotune != 0 && o.autotune != 1) return fail(LP_ERR_INVALID_ARG, "autotune must be 0 or 1");
  if (o.sigma_method != LP_SIGMA_POWER && o.sigma_method != LP_SIGMA_LANCZOS)
    return fail(LP_ERR_INVALID_ARG, "sigma_method must be LP_SIGMA_POWER or LP_SIGMA_LANCZOS");
  if (o.device_layout != 0 && o.device_layout != 1)
    return fail(LP_ERR_INVALID_ARG, "device_layout must be 0 or 1");
  if (o.split_row_len < 0 || o.split_row_len % 32 != 0)
    return fail(LP_ERR_INVALID_ARG, "split_row_len must be 0 or a positive multiple of 32");
  if (o.precision != LP_PRECISION_FP64 && o.precision != LP_PRECISION_MIXED)
    return fail(LP_ERR_INVALID_ARG, "precision must be LP_PRECISION_FP64 or LP_PRECISION_MIXED");
  return LP_OK;
}

}  // namespace lpg
