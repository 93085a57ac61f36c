// Device-side construction of the library's layout (setup step of Section 7's
// method: the CSC copy of A, the length-sorted row and column orders and the
// two lane-grouped slice layouts), the same arrays, bit for bit, as the host
// construction in lp_host.h (build_csc, sort_by_length_desc, choose_policy,
// build_sell), so that both give identical iterates.  Every step is
// deterministic: integer histograms and scans, and stable sorts.
//
//   * validation of the inputs (flag bits, read back once);
//   * CSC: a stable LSD radix sort of the nonzeros by column (8 bits per
//     pass; within a column, CSR order, i.e. rows ascending), then a gather
//     of rows and values; repeated columns within a row show up as equal
//     adjacent (column, row) pairs;
//   * orders: stable radix sorts of rows and columns by decreasing length;
//   * slices: rows of equal lane count form contiguous runs of the sorted
//     order (the lane count is a nondecreasing function of the length), so a
//     slice is the k-th group of 32 / G rows of its run; its step count is
//     that of its first (longest) row; offsets are an exclusive scan;
//   * fill: one warp per slice writes its elements (and zero padding) with
//     relabeled indices; lane l writes element off + 32 t + l at step t.
#include <algorithm>
#include <cstdint>
#include <utility>

#include "lp_internal.h"

namespace lpg {
namespace {

constexpr int kLayBlock = 256;
constexpr int kTileItems = 16;                      // radix sort: items per thread and tile
constexpr int kTile = kLayBlock * kTileItems;       // elements per tile
constexpr int kScanChunk = kLayBlock * 16;          // scan: elements per block

__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

// ------------------------------------------------------------- validation

__global__ void __launch_bounds__(kLayBlock) lay_validate_kernel(
    const int32_t *__restrict__ rp, int32_t m, int64_t nnz, const int32_t *__restrict__ ci,
    int32_t n, const double *__restrict__ v, const double *__restrict__ c,
    const double *__restrict__ lb, const double *__restrict__ ub, const double *__restrict__ b,
    const int8_t *__restrict__ rt, int32_t *flags) {
  int f = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t0 == 0 && (rp[0] != 0 || (int64_t)rp[m] != nnz)) f |= kLayBadRowPtr;
  for (int64_t i = t0; i < m; i += stride) {
    if (rp[i + 1] < rp[i]) f |= kLayBadRowPtr;
    if (!finite_val(b[i])) f |= kLayBadB;
    if (rt[i] < 0 || rt[i] > 2) f |= kLayBadRowType;
  }
  for (int64_t p = t0; p < nnz; p += stride) {
    if (ci[p] < 0 || ci[p] >= n) f |= kLayBadColIdx;
    if (!finite_val(v[p])) f |= kLayBadVal;
  }
  for (int64_t j = t0; j < n; j += stride) {
    if (!finite_val(c[j])) f |= kLayBadC;
    const double l = lb[j], u = ub[j];
    if (isnan(l) || isnan(u) || l > u || l == INFINITY || u == -INFINITY) f |= kLayBadBounds;
  }
  if (f) atomicOr(flags, f);
}

// row_of[p]: the row of CSR position p (rp validated: nondecreasing, rp[0] = 0,
// rp[m] = nnz): the last i with rp[i] <= p, by binary search.
__global__ void __launch_bounds__(kLayBlock) lay_row_of_kernel(const int32_t *__restrict__ rp,
                                                               int32_t m, int64_t nnz,
                                                               int32_t *row_of) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = m;  // invariant: rp[lo] <= p < rp[hi]
    while (hi - lo > 1) {
      const int32_t mid = lo + (hi - lo) / 2;
      if ((int64_t)rp[mid] <= p) lo = mid;
      else hi = mid;
    }
    row_of[p] = lo;
  }
}

__global__ void __launch_bounds__(kLayBlock) lay_iota_kernel(int32_t *a, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// ----------------------------------------------------- radix sort (stable)

// Tile histogram of the 8-bit digit at shift: gh[d * ntiles + tile].
__global__ void __launch_bounds__(kLayBlock) rs_hist_kernel(const uint32_t *__restrict__ keys,
                                                            int64_t count, int shift,
                                                            int64_t *gh, int64_t ntiles) {
  __shared__ int32_t hist[256];
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = blockIdx.x * (int64_t)kTile;
  for (int r = 0; r < kTileItems; ++r) {
    const int64_t e = t0 + (int64_t)r * kLayBlock + threadIdx.x;
    if (e < count) atomicAdd(&hist[(keys[e] >> shift) & 255u], 1);
  }
  __syncthreads();
  gh[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter of one tile: elements are taken in tile order, 256 per
// round; an element's rank among equal digits is the count of equal digits
// in earlier rounds, in earlier warps of its round and in lower lanes of
// its warp.
__global__ void __launch_bounds__(kLayBlock) rs_scatter_kernel(
    const uint32_t *__restrict__ kin, const int32_t *__restrict__ pin, int64_t count, int shift,
    const int64_t *__restrict__ goff, int64_t ntiles, uint32_t *kout, int32_t *pout) {
  constexpr int W = kLayBlock / kWarp;
  __shared__ int32_t wcnt[W][256];
  __shared__ int64_t running[256];
  const int tid = threadIdx.x, lane = tid & (kWarp - 1), warp = tid >> 5;
  for (int w = 0; w < W; ++w) wcnt[w][tid] = 0;
  running[tid] = goff[(int64_t)tid * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t t0 = blockIdx.x * (int64_t)kTile;
  for (int r = 0; r < kTileItems; ++r) {
    const int64_t e = t0 + (int64_t)r * kLayBlock + tid;
    const bool act = e < count;
    uint32_t key = 0;
    int32_t pay = 0;
    int d = 256;  // inactive: a digit no active element has
    if (act) {
      key = kin[e];
      pay = pin[e];
      d = (int)((key >> shift) & 255u);
    }
    const unsigned same = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(same & ((1u << lane) - 1u));
    if (act && rank == 0) wcnt[warp][d] = __popc(same);
    __syncthreads();
    if (act) {
      int64_t pos = running[d] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      kout[pos] = key;
      pout[pos] = pay;
    }
    __syncthreads();
    int32_t tot = 0;
    for (int w = 0; w < W; ++w) {
      tot += wcnt[w][tid];
      wcnt[w][tid] = 0;
    }
    running[tid] += tot;
    __syncthreads();
  }
}

// ------------------------------------------------ exclusive scan (int64)

__global__ void __launch_bounds__(kLayBlock) scan_sums_kernel(const int64_t *__restrict__ in,
                                                              int64_t len, int64_t *sums) {
  __shared__ int64_t red[kLayBlock];
  int64_t s = 0;
  const int64_t b0 = blockIdx.x * (int64_t)kScanChunk;
  for (int r = 0; r < kScanChunk / kLayBlock; ++r) {
    const int64_t i = b0 + (int64_t)r * kLayBlock + threadIdx.x;
    if (i < len) s += in[i];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kLayBlock / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// Block-level exclusive scan of kLayBlock values (one per thread); returns
// the thread's exclusive prefix and sets *total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *sh, int64_t *total) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kLayBlock; o <<= 1) {
    const int64_t add = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += add;
    __syncthreads();
  }
  const int64_t incl = sh[threadIdx.x];
  *total = sh[kLayBlock - 1];
  __syncthreads();
  return incl - v;
}

// One block: sums[0..nb) <- exclusive prefix sums, in chunks of kLayBlock.
__global__ void __launch_bounds__(kLayBlock) scan_top_kernel(int64_t *sums, int64_t nb) {
  __shared__ int64_t sh[kLayBlock];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kLayBlock) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? sums[i] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan(v, sh, &total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
}

// out[i] = sums[block] + sum of in over the block's chunk before i.
__global__ void __launch_bounds__(kLayBlock) scan_apply_kernel(const int64_t *__restrict__ in,
                                                               int64_t len,
                                                               const int64_t *__restrict__ sums,
                                                               int64_t *out) {
  __shared__ int64_t sh[kLayBlock];
  constexpr int R = kScanChunk / kLayBlock;
  const int64_t b0 = blockIdx.x * (int64_t)kScanChunk;
  // thread t owns the R consecutive elements b0 + t R .. b0 + t R + R - 1
  int64_t loc[R];
  int64_t s = 0;
  for (int r = 0; r < R; ++r) {
    const int64_t i = b0 + (int64_t)threadIdx.x * R + r;
    loc[r] = i < len ? in[i] : 0;
    s += loc[r];
  }
  int64_t total;
  int64_t run = sums[blockIdx.x] + block_exclusive_scan(s, sh, &total);
  for (int r = 0; r < R; ++r) {
    const int64_t i = b0 + (int64_t)threadIdx.x * R + r;
    if (i < len) out[i] = run;
    run += loc[r];
  }
}

// ------------------------------------------------------------ CSC steps

__global__ void __launch_bounds__(kLayBlock) lay_col_count_kernel(const int32_t *__restrict__ ci,
                                                                  int64_t nnz, int64_t *cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[ci[p]]), 1ull);
}

__global__ void __launch_bounds__(kLayBlock) lay_csc_gather_kernel(
    const int32_t *__restrict__ pos, const int32_t *__restrict__ row_of,
    const double *__restrict__ v, int64_t nnz, int32_t *ri, double *cv) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pos[q];
    ri[q] = row_of[p];
    cv[q] = v[p];
  }
}

// A column listing a row twice (adjacent after the stable sort): a column
// repeated within a row of the CSR.
__global__ void __launch_bounds__(kLayBlock) lay_dup_kernel(const uint32_t *__restrict__ col,
                                                            const int32_t *__restrict__ ri,
                                                            int64_t nnz, int32_t *flags) {
  int f = 0;
  for (int64_t q = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
       q += (int64_t)gridDim.x * blockDim.x)
    if (col[q] == col[q - 1] && ri[q] == ri[q - 1]) f = kLayDuplicate;
  if (f) atomicOr(flags, f);
}

// ------------------------------------------------------------ orders

// len[i] = ptr[i + 1] - ptr[i]; key[i] = mx - len[i] once mx is known (second call).
template <class P>
__global__ void __launch_bounds__(kLayBlock) lay_len_kernel(const P *__restrict__ ptr,
                                                            int32_t count, int64_t *mx,
                                                            uint32_t *key, int64_t mxv,
                                                            int64_t *hist) {
  int64_t local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = (int64_t)ptr[i + 1] - (int64_t)ptr[i];
    if (key) {
      key[i] = (uint32_t)(mxv - len);
      atomicAdd(reinterpret_cast<unsigned long long *>(&hist[len]), 1ull);
    } else {
      local = len > local ? len : local;
    }
  }
  if (!key && local > 0) atomicMax(reinterpret_cast<unsigned long long *>(mx),
                                   (unsigned long long)local);
}

__global__ void __launch_bounds__(kLayBlock) lay_inverse_kernel(const int32_t *__restrict__ perm,
                                                                int32_t count, int32_t *inv) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < count;
       r += (int64_t)gridDim.x * blockDim.x)
    inv[perm[r]] = (int32_t)r;
}

// ------------------------------------------------------------ slices

// Slice s of run q (rows [g0, g0 + cnt) of the sorted order, 2^lg lanes per
// row, cap = 32 >> lg rows per slice): row0 = g0 + k cap for k = s - s0;
// steps from the slice's first (longest) row.
template <class P>
__global__ void __launch_bounds__(kLayBlock) lay_slices_kernel(LayRuns runs,
                                                               const int32_t *__restrict__ perm,
                                                               const P *__restrict__ ptr,
                                                               int64_t s_begin, int64_t nslices,
                                                               SliceInfo *info, int64_t *width) {
  for (int64_t s = s_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslices;
       s += (int64_t)gridDim.x * blockDim.x) {
    int q = 0;
    while (q + 1 < runs.count && s >= runs.s0[q + 1]) ++q;
    const int lg = runs.lg[q];
    const int64_t row0 = runs.g0[q] + (s - runs.s0[q]) * (int64_t)(kWarp >> lg);
    const int32_t r = perm[row0];
    const int64_t len = (int64_t)ptr[r + 1] - (int64_t)ptr[r];
    const int64_t steps = (len + (int64_t(1) << lg) - 1) >> lg;
    info[s].row0 = (int32_t)row0;
    info[s].len_g = (int32_t)((steps << 3) | lg);
    width[s] = steps * kWarp;
  }
}

// Split rows (the first nsr rows of the sorted order): chunk counts, then,
// from their exclusive scan cstart, each chunk's slice (G = 32, at most
// split_len elements) and its SplitSlice record.
template <class P>
__global__ void __launch_bounds__(kLayBlock) lay_split_count_kernel(
    const int32_t *__restrict__ perm, const P *__restrict__ ptr, int64_t nsr, int32_t split_len,
    int64_t *nch) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nsr;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = perm[r];
    const int64_t len = (int64_t)ptr[q + 1] - (int64_t)ptr[q];
    nch[r] = (len + split_len - 1) / split_len;
  }
}

template <class P>
__global__ void __launch_bounds__(kLayBlock) lay_split_slices_kernel(
    const int32_t *__restrict__ perm, const P *__restrict__ ptr, int64_t nsr, int32_t split_len,
    const int64_t *__restrict__ cstart, SliceInfo *info, int64_t *width, SplitSlice *split) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nsr;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = perm[r];
    const int64_t len = (int64_t)ptr[q + 1] - (int64_t)ptr[q];
    const int32_t nch = (int32_t)((len + split_len - 1) / split_len);
    const int64_t first = cstart[r];
    for (int32_t c = 0; c < nch; ++c) {
      const int64_t clen = min((int64_t)split_len, len - (int64_t)c * split_len);
      const int64_t steps = (clen + kWarp - 1) / kWarp;
      info[first + c].row0 = (int32_t)r;
      info[first + c].len_g = (int32_t)((steps << 3) | 5);
      width[first + c] = steps * kWarp;
      split[first + c] = SplitSlice{c, nch, (int32_t)first, c * split_len};
    }
  }
}

__global__ void lay_slice_offsets_kernel(SliceInfo *info, const int64_t *__restrict__ off,
                                         const int64_t *__restrict__ width, int64_t nslices,
                                         int32_t nrows) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= nslices;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (s < nslices) {
      info[s].off = off[s];
    } else {
      const int64_t end = nslices > 0 ? off[nslices - 1] + width[nslices - 1] : 0;
      info[s] = SliceInfo{end, nrows, 0};
    }
  }
}

// One warp per slice: lane l writes element off + 32 t + l for every step t
// (its row's element t G + (l mod G), or zero padding).
template <class P>
__global__ void __launch_bounds__(kLayBlock) lay_fill_kernel(
    const SliceInfo *__restrict__ info, int64_t nslices, const int32_t *__restrict__ perm,
    const P *__restrict__ ptr, const int32_t *__restrict__ ind, const double *__restrict__ val,
    const int32_t *__restrict__ relabel, int32_t *idx, double *vout, float *vf,
    const SplitSlice *__restrict__ split, int64_t nsplit, int32_t split_len) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; s < nslices; s += nw) {
    const SliceInfo a = info[s];
    const int32_t row_end = info[s + 1].row0;
    const int lg = a.len_g & 7, G = 1 << lg;
    const int64_t steps = a.len_g >> 3;
    const int32_t row = a.row0 + (lane >> lg);
    const int sub = lane & (G - 1);
    int64_t src = 0, len = 0;
    if (s < nsplit) {  // chunk of a split row (G = 32: every lane on row a.row0)
      const int32_t r = perm[a.row0];
      const int64_t begin = split[s].begin;
      src = ptr[r] + begin;
      len = min((int64_t)split_len, (int64_t)ptr[r + 1] - (int64_t)ptr[r] - begin);
    } else if (row < row_end) {
      const int32_t r = perm[row];
      src = ptr[r];
      len = (int64_t)ptr[r + 1] - src;
    }
    for (int64_t t = 0; t < steps; ++t) {
      const int64_t k = t * G + sub;
      const int64_t dst = a.off + kWarp * t + lane;
      int32_t j = 0;
      double x = 0.0;
      if (k < len) {
        j = relabel[ind[src + k]];
        x = val[src + k];
      }
      idx[dst] = j;
      vout[dst] = x;
      if (vf) vf[dst] = (float)x;
    }
  }
}

// ------------------------------------------------------------ vectors

__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 ? (b ^ 0x7fffffffffffffffll) : b;
}

__global__ void __launch_bounds__(kLayBlock) lay_cols_vectors_kernel(
    const int32_t *__restrict__ perm, int32_t n, const double *__restrict__ c,
    const double *__restrict__ lb, const double *__restrict__ ub, double *pc, double *pl,
    double *pu, long long *lk, long long *uk) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = perm[r];
    pc[r] = c[j];
    pl[r] = lb[j];
    pu[r] = ub[j];
    lk[r] = order_key(lb[j]);
    uk[r] = order_key(ub[j]);
  }
}

__global__ void __launch_bounds__(kLayBlock) lay_rows_vectors_kernel(
    const int32_t *__restrict__ perm, int32_t m, const double *__restrict__ b,
    const int8_t *__restrict__ rt, double *pb, int8_t *prt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = perm[r];
    pb[r] = b[i];
    prt[r] = rt[i];
  }
}

int lay_grid(int64_t work, int nsm) {
  int64_t g = (work + kLayBlock - 1) / kLayBlock;
  const int64_t cap = (int64_t)nsm * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ------------------------------------------------------------ launchers

void lay_validate(const int32_t *rp, int32_t m, int64_t nnz, const int32_t *ci, int32_t n,
                  const double *v, const double *c, const double *lb, const double *ub,
                  const double *b, const int8_t *rt, int32_t *flags, int nsm, cudaStream_t s) {
  const int64_t work = std::max<int64_t>(std::max<int64_t>(m, n), nnz);
  lay_validate_kernel<<<lay_grid(work, nsm), kLayBlock, 0, s>>>(rp, m, nnz, ci, n, v, c, lb, ub,
                                                                 b, rt, flags);
}

void lay_row_of(const int32_t *rp, int32_t m, int64_t nnz, int32_t *row_of, int nsm,
                cudaStream_t s) {
  if (nnz > 0) lay_row_of_kernel<<<lay_grid(nnz, nsm), kLayBlock, 0, s>>>(rp, m, nnz, row_of);
}

void lay_iota(int32_t *a, int64_t count, int nsm, cudaStream_t s) {
  if (count > 0) lay_iota_kernel<<<lay_grid(count, nsm), kLayBlock, 0, s>>>(a, count);
}

int64_t lay_scan_scratch(int64_t len) { return (len + kScanChunk - 1) / kScanChunk + 1; }

void lay_exclusive_scan(const int64_t *in, int64_t len, int64_t *out, int64_t *sums,
                        cudaStream_t s) {
  if (len <= 0) return;
  const int64_t nb = (len + kScanChunk - 1) / kScanChunk;
  scan_sums_kernel<<<(unsigned)nb, kLayBlock, 0, s>>>(in, len, sums);
  scan_top_kernel<<<1, kLayBlock, 0, s>>>(sums, nb);
  scan_apply_kernel<<<(unsigned)nb, kLayBlock, 0, s>>>(in, len, sums, out);
}

int64_t lay_radix_tiles(int64_t count) { return (count + kTile - 1) / kTile; }

void lay_radix_sort(uint32_t *keys, int32_t *pay, uint32_t *keys_alt, int32_t *pay_alt,
                    int64_t count, int bits, int64_t *gh, int64_t *goff, int64_t *sums,
                    cudaStream_t s, bool *in_alt) {
  *in_alt = false;
  if (count <= 1 || bits <= 0) return;
  const int64_t nt = lay_radix_tiles(count);
  uint32_t *k0 = keys, *k1 = keys_alt;
  int32_t *p0 = pay, *p1 = pay_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    rs_hist_kernel<<<(unsigned)nt, kLayBlock, 0, s>>>(k0, count, shift, gh, nt);
    lay_exclusive_scan(gh, 256 * nt, goff, sums, s);
    rs_scatter_kernel<<<(unsigned)nt, kLayBlock, 0, s>>>(k0, p0, count, shift, goff, nt, k1, p1);
    std::swap(k0, k1);
    std::swap(p0, p1);
    *in_alt = !*in_alt;
  }
}

void lay_col_count(const int32_t *ci, int64_t nnz, int64_t *cnt, int nsm, cudaStream_t s) {
  if (nnz > 0) lay_col_count_kernel<<<lay_grid(nnz, nsm), kLayBlock, 0, s>>>(ci, nnz, cnt);
}

void lay_csc_gather(const int32_t *pos, const int32_t *row_of, const double *v, int64_t nnz,
                    int32_t *ri, double *cv, int nsm, cudaStream_t s) {
  if (nnz > 0)
    lay_csc_gather_kernel<<<lay_grid(nnz, nsm), kLayBlock, 0, s>>>(pos, row_of, v, nnz, ri, cv);
}

void lay_dup(const uint32_t *col, const int32_t *ri, int64_t nnz, int32_t *flags, int nsm,
             cudaStream_t s) {
  if (nnz > 1) lay_dup_kernel<<<lay_grid(nnz, nsm), kLayBlock, 0, s>>>(col, ri, nnz, flags);
}

template <class P>
void lay_lengths(const P *ptr, int32_t count, int64_t *mx, uint32_t *key, int64_t mxv,
                 int64_t *hist, int nsm, cudaStream_t s) {
  if (count > 0)
    lay_len_kernel<P><<<lay_grid(count, nsm), kLayBlock, 0, s>>>(ptr, count, mx, key, mxv, hist);
}
template void lay_lengths<int32_t>(const int32_t *, int32_t, int64_t *, uint32_t *, int64_t,
                                   int64_t *, int, cudaStream_t);
template void lay_lengths<int64_t>(const int64_t *, int32_t, int64_t *, uint32_t *, int64_t,
                                   int64_t *, int, cudaStream_t);

void lay_inverse(const int32_t *perm, int32_t count, int32_t *inv, int nsm, cudaStream_t s) {
  if (count > 0) lay_inverse_kernel<<<lay_grid(count, nsm), kLayBlock, 0, s>>>(perm, count, inv);
}

template <class P>
void lay_slices(const LayRuns &runs, const int32_t *perm, const P *ptr, int64_t nslices,
                int32_t nrows, SliceInfo *info, int64_t *width, int64_t *off, int64_t *sums,
                int nsm, cudaStream_t s, int64_t nsr, int64_t nsplit, int32_t split_len,
                SplitSlice *split, int64_t *nch, int64_t *cstart) {
  if (nsr > 0) {
    lay_split_count_kernel<P><<<lay_grid(nsr, nsm), kLayBlock, 0, s>>>(perm, ptr, nsr, split_len,
                                                                       nch);
    lay_exclusive_scan(nch, nsr, cstart, sums, s);
    lay_split_slices_kernel<P><<<lay_grid(nsr, nsm), kLayBlock, 0, s>>>(
        perm, ptr, nsr, split_len, cstart, info, width, split);
  }
  if (nslices > nsplit)
    lay_slices_kernel<P><<<lay_grid(nslices - nsplit, nsm), kLayBlock, 0, s>>>(
        runs, perm, ptr, nsplit, nslices, info, width);
  if (nslices > 0) lay_exclusive_scan(width, nslices, off, sums, s);
  lay_slice_offsets_kernel<<<lay_grid(nslices + 1, nsm), kLayBlock, 0, s>>>(info, off, width,
                                                                            nslices, nrows);
}
template void lay_slices<int32_t>(const LayRuns &, const int32_t *, const int32_t *, int64_t,
                                  int32_t, SliceInfo *, int64_t *, int64_t *, int64_t *, int,
                                  cudaStream_t, int64_t, int64_t, int32_t, SplitSlice *, int64_t *,
                                  int64_t *);
template void lay_slices<int64_t>(const LayRuns &, const int32_t *, const int64_t *, int64_t,
                                  int32_t, SliceInfo *, int64_t *, int64_t *, int64_t *, int,
                                  cudaStream_t, int64_t, int64_t, int32_t, SplitSlice *, int64_t *,
                                  int64_t *);

template <class P>
void lay_fill(const SliceInfo *info, int64_t nslices, const int32_t *perm, const P *ptr,
              const int32_t *ind, const double *val, const int32_t *relabel, int32_t *idx,
              double *vout, float *vf, int nsm, cudaStream_t s, const SplitSlice *split,
              int64_t nsplit, int32_t split_len) {
  if (nslices > 0)
    lay_fill_kernel<P><<<lay_grid(nslices * kWarp, nsm), kLayBlock, 0, s>>>(
        info, nslices, perm, ptr, ind, val, relabel, idx, vout, vf, split, nsplit, split_len);
}
template void lay_fill<int32_t>(const SliceInfo *, int64_t, const int32_t *, const int32_t *,
                                const int32_t *, const double *, const int32_t *, int32_t *,
                                double *, float *, int, cudaStream_t, const SplitSlice *, int64_t,
                                int32_t);
template void lay_fill<int64_t>(const SliceInfo *, int64_t, const int32_t *, const int64_t *,
                                const int32_t *, const double *, const int32_t *, int32_t *,
                                double *, float *, int, cudaStream_t, const SplitSlice *, int64_t,
                                int32_t);

void lay_vectors(const int32_t *perm_x, int32_t n, const double *c, const double *lb,
                 const double *ub, double *pc, double *pl, double *pu, long long *lk,
                 long long *uk, const int32_t *perm_y, int32_t m, const double *b,
                 const int8_t *rt, double *pb, int8_t *prt, int nsm, cudaStream_t s) {
  if (n > 0)
    lay_cols_vectors_kernel<<<lay_grid(n, nsm), kLayBlock, 0, s>>>(perm_x, n, c, lb, ub, pc, pl,
                                                                   pu, lk, uk);
  if (m > 0)
    lay_rows_vectors_kernel<<<lay_grid(m, nsm), kLayBlock, 0, s>>>(perm_y, m, b, rt, pb, prt);
}

}  // namespace lpg
