// Batched restarted PDHG (include/lp_batch.h): many independent LPs of
// uneven sizes on one GPU, each running Algorithm 1 with its own step
// sizes, restart state and termination test.
//
// Layout.  The batch is stored as one block-diagonal LP in the sliced
// layout of the single-problem solver, with rows (and columns) permuted by
// length WITHIN each problem, so every problem keeps a contiguous range of
// rows, columns and slices, and no slice spans two problems.  A slice knows
// its problem (sinst), a problem knows its ranges (BInst).
//
// Per block of K_base iterations (one CUDA graph):
//   b_primal / b_dual (x K_base): one warp per slice of the running
//       problems' work list, with that problem's tau or sigma and averaging
//       weight 1 / (t + k + 1) -- the fused step and average of the
//       single-problem kernels (FP32 correction steps in mixed precision),
//       launched with programmatic dependent launch;
//   b_pre_check: counters; a problem is due for its check every K_k
//       iterations (K_k a multiple of K_base);
//   b_check (columns, rows): the check epilogues on the due problems'
//       slices, each warp a chunk of 8 slices of one problem, one
//       fixed-order partial sum per chunk and quantity;
//   b_finalize: one block per due problem: its sums, relative KKT,
//       termination, radius, search setup;
//   b_search: one block (or an 8-block cluster for large problems) per due
//       problem: the multiplier search of Section 6.3 (radix passes over
//       the breakpoints' bit patterns from their common prefix down,
//       per-warp histograms, per-warp candidate lists after the first pass,
//       bracket selection in-block);
//   b_decide: restart rule, counters, running count (one thread per problem);
//   b_restart_copy: z^{n+1,0} <- zbar, z <- zbar for restarting problems;
//   b_list_scan / b_list_fill: the next block's slice work lists and
//       averaging weights (running problems only).
// Also here: the batch tuner, mixed precision (combine / recenter per
// problem), and the recorded forward and adjoint of the unrolled maps.
// All reductions run in a fixed order: results are bitwise reproducible
// for a given batch and launch configuration.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "../../include/lp_batch.h"
#include "lp_host.h"
#include "lp_internal.h"
#include "spmv_core.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace lpg {
namespace {

constexpr int kMaxClasses = 8;
constexpr int kCheckChunk = 8;  // slices per warp and reduction in the check kernels
constexpr int kStatusIterLimit = 4;
constexpr int kListThreads = 1024;
constexpr int kSearchWarps = 8;
constexpr int kSearchThreads = kSearchWarps * kWarp;  // one thread per bucket
static_assert(kSearchThreads == kBuckets, "bracket selection uses one thread per bucket");
constexpr size_t kSearchHistBytes = sizeof(double) * kSearchWarps * kBuckets * 3;
constexpr size_t kSearchCntBytes = sizeof(unsigned) * kSearchWarps * kBuckets;
constexpr size_t kSearchSmem = kSearchHistBytes + kSearchCntBytes + sizeof(double) * kSearchWarps * kWarp * 3;

// Per-problem state (device, one per problem).
struct BInst {
  int32_t col0, ncol, row0, nrow;  // ranges in the permuted index spaces
  int32_t cs0, cs1, rs0, rs1;      // slice ranges in A^T and A
  int32_t cc0, cc1, rc0, rc1;      // check-chunk ranges in A^T and A
  int32_t wlc0, wlr0;              // this problem's offsets in the work lists (if running)
  int32_t K;                       // check period (multiple of K_base)
  int32_t status;                  // kRunning or a final lp_status
  int32_t returned, restart_now, use_cur, due;
  int32_t pw_done, pw_iters;
  int64_t t0;                      // inner iterations since the restart, at block start
  int64_t iters, checks, restarts;
  int64_t since;                   // iterations since the last check
  int64_t iter_cap;                // stop (iteration limit) once iters reaches it
  int64_t tau0, fixed_len;
  double tau, sigma, omega;
  double norm_b, norm_c;
  double rho_stored, last_rho, last_r;
  double kkt_a[5], kkt_c[5];
  double pw_est, pw_nw;
  double mix_s;                    // mixed precision: scale of the current correction
  LSearch ls[2];
};

// Batch-wide parameters and counters (device).
struct BGlobal {
  double tol, beta, pw_tol;
  int32_t count, Kb, scheme, pw_max;
  int32_t running;     // problems still iterating after the last check
  int32_t pw_running;  // problems still estimating sigma_max after the last step
  int32_t wl_n[2];     // work-list lengths: [0] column slices, [1] row slices
  int32_t mixed;       // 1: mixed-precision iterations
};

struct SearchArrays {
  uint64_t *keys[2];
  double *d2[2], *g2[2], *gd[2];
  int32_t *cand[2];  // per-warp candidate lists, [n + m + 256 count] each
};

// ---------------------------------------------------------------- iteration

template <int U, bool PIPE>
__global__ void __launch_bounds__(kBlock) b_primal_kernel(SellMat AT, const double *__restrict__ y,
                                                          PrimalEpi epi,
                                                          const BInst *__restrict__ I,
                                                          const int32_t *__restrict__ sinst,
                                                          const int32_t *__restrict__ wl,
                                                          const BGlobal *G,
                                                          const double *__restrict__ wtab, int k) {
  pdl_enter();
  const int nwl = G->wl_n[0], Kb = G->Kb;
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int it = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); it < nwl; it += nwarps) {
    const int s = wl[it];
    const int i = sinst[s];
    epi.tau = I[i].tau;
    epi.w = wtab[(size_t)i * Kb + k];
    process_item<1, U, PIPE>(AT, y, (const double *)nullptr, s, lane, epi);
  }
}

template <int U, bool PIPE>
__global__ void __launch_bounds__(kBlock) b_dual_kernel(SellMat A, const double *__restrict__ xhat,
                                                        DualEpi epi, const BInst *__restrict__ I,
                                                        const int32_t *__restrict__ sinst,
                                                        const int32_t *__restrict__ wl,
                                                        const BGlobal *G,
                                                        const double *__restrict__ wtab, int k) {
  pdl_enter();
  const int nwl = G->wl_n[1], Kb = G->Kb;
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int it = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); it < nwl; it += nwarps) {
    const int s = wl[it];
    const int i = sinst[s];
    epi.sigma = I[i].sigma;
    epi.w = wtab[(size_t)i * Kb + k];
    process_item<1, U, PIPE>(A, xhat, (const double *)nullptr, s, lane, epi);
  }
}

// Mixed precision: the FP32 step on each problem's scaled correction (the
// single-problem mixed kernels' epilogues), per-slice step and weight.
template <int U, bool PIPE>
__global__ void __launch_bounds__(kBlock) b_primal_mix_kernel(SellMat AT, const float *__restrict__ dy,
                                                              PrimalMixEpi epi,
                                                              const BInst *__restrict__ I,
                                                              const int32_t *__restrict__ sinst,
                                                              const int32_t *__restrict__ wl,
                                                              const BGlobal *G,
                                                              const double *__restrict__ wtab,
                                                              int k) {
  pdl_enter();
  const int nwl = G->wl_n[0], Kb = G->Kb;
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int it = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); it < nwl; it += nwarps) {
    const int s = wl[it];
    const int i = sinst[s];
    epi.tau = (float)I[i].tau;
    epi.w = wtab[(size_t)i * Kb + k];
    process_item<1, U, PIPE>(AT, dy, (const float *)nullptr, s, lane, epi);
  }
}

template <int U, bool PIPE>
__global__ void __launch_bounds__(kBlock) b_dual_mix_kernel(SellMat A, const float *__restrict__ dxhat,
                                                            DualMixEpi epi,
                                                            const BInst *__restrict__ I,
                                                            const int32_t *__restrict__ sinst,
                                                            const int32_t *__restrict__ wl,
                                                            const BGlobal *G,
                                                            const double *__restrict__ wtab,
                                                            int k) {
  pdl_enter();
  const int nwl = G->wl_n[1], Kb = G->Kb;
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int it = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); it < nwl; it += nwarps) {
    const int s = wl[it];
    const int i = sinst[s];
    epi.sigma = (float)I[i].sigma;
    epi.w = wtab[(size_t)i * Kb + k];
    process_item<1, U, PIPE>(A, dxhat, (const float *)nullptr, s, lane, epi);
  }
}

// ------------------------------------------------------------------- check

__global__ void b_pre_check_kernel(BInst *I, BGlobal *G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) G->running = 0;  // counted again by b_decide
  if (i >= G->count) return;
  BInst &B = I[i];
  B.due = 0;
  if (B.status != kRunning) return;
  B.iters += G->Kb;
  B.since += G->Kb;
  B.due = (B.since >= B.K) ? 1 : 0;
}

// Check epilogue over the due problems' slices.  A warp takes a chunk of
// up to kCheckChunk consecutive slices of one problem (chunk c covers slices
// [chunk[c], chunk[c + 1]) ), accumulates every quantity in its lanes over
// the whole chunk, and reduces once (warp butterfly, fixed order) into
// spart[q * pstride + poff + c]: the FP64 reductions (2 operations per cycle
// per SM on GB300) are paid per chunk, not per slice.
template <class Epi>
__global__ void __launch_bounds__(kBlock) b_check_kernel(SellMat A, const double *__restrict__ v0,
                                                         const double *__restrict__ v1, Epi epi,
                                                         const BInst *__restrict__ I,
                                                         const int32_t *__restrict__ sinst,
                                                         const int32_t *__restrict__ chunk,
                                                         int nchunks, const BGlobal *G,
                                                         double *spart, int64_t pstride, int poff) {
  const int scheme = G->scheme;
  epi.gap_a = (scheme == kSchemeAdaptive || scheme == kSchemeFlexible);
  epi.gap_c = (scheme == kSchemeFlexible);
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < nchunks; c += nwarps) {
    const int s0 = chunk[c], s1 = chunk[c + 1];
    const int i = sinst[s0];
    if (!I[i].due) continue;
    epi.sw = sqrt(I[i].omega);
    epi.isw = 1.0 / epi.sw;
#pragma unroll
    for (int q = 0; q < NQ; ++q) epi.q[q] = 0.0;
    for (int sl = s0; sl < s1; ++sl) process_item<2, kUnroll2, false>(A, v0, v1, sl, lane, epi);
    // only the quantities this epilogue accumulates are reduced (the others are 0)
    const uint32_t used = Epi::kUsed | (epi.gap_c ? Epi::kUsedGapC : 0u);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double v = epi.q[q];
      if ((used >> q) & 1u) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      }
      if (lane == 0) spart[(size_t)q * pstride + poff + c] = v;
    }
  }
}

// One block per problem: the due problem's check sums (warp q sums quantity
// q over its chunks in order), relative KKT, termination, search setup.
__global__ void __launch_bounds__(kBlock) b_finalize_kernel(BInst *I, const BGlobal *G,
                                                            const double *__restrict__ spart,
                                                            int64_t pstride, int ncc) {
  BInst &B = I[blockIdx.x];
  if (!B.due) return;
  __shared__ double tot[NQ];
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
  for (int q = warp; q < NQ; q += kBlock / kWarp) {
    const double *p = spart + (size_t)q * pstride;
    double acc = 0.0;
    for (int c = B.cc0 + lane; c < B.cc1; c += kWarp) acc += p[c];
    for (int c = B.rc0 + lane; c < B.rc1; c += kWarp) acc += p[ncc + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) tot[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int scheme = G->scheme;
  const double om = B.omega, tol = G->tol;
  B.checks += 1;
  kkt_from(tot, Q_RP2_A, Q_RD2_A, Q_POBJ_A, Q_DOBJ_A, B.norm_b, B.norm_c, B.kkt_a);
  kkt_from(tot, Q_RP2_C, Q_RD2_C, Q_POBJ_C, Q_DOBJ_C, B.norm_b, B.norm_c, B.kkt_c);
  const double ra = B.kkt_a[4], rc = B.kkt_c[4];
  B.ls[0].done = 1;
  B.ls[1].done = 1;
  if (tot[Q_BAD] > 0.0 || !isfinite(ra) || !isfinite(rc)) {
    B.status = kStatusNumerical;
    return;
  }
  if (ra <= tol) {
    B.status = kStatusOK;
    B.returned = 0;
    return;
  }
  if (rc <= tol) {
    B.status = kStatusOK;
    B.returned = 1;
    return;
  }
  B.returned = (ra <= rc) ? 0 : 1;
  if (scheme == kSchemeAdaptive || scheme == kSchemeFlexible) {
    const double r = sqrt(om * tot[Q_RRX_A] + tot[Q_RRY_A] / om);
    init_search(B.ls[0], r, tot[Q_D2_A], tot[Q_GD_A], tot[Q_G2INF_A]);
    B.last_r = r;
  }
  if (scheme == kSchemeFlexible) {
    const double r = sqrt(om * tot[Q_RRX_C] + tot[Q_RRY_C] / om);
    init_search(B.ls[1], r, tot[Q_D2_C], tot[Q_GD_C], tot[Q_G2INF_C]);
  }
}

// One block per (due problem, candidate): the multiplier search of
// Section 6.3 over the problem's breakpoints, with the bracket logic of the
// single-problem solver (radix passes of 8 bits over the bit patterns of the
// breakpoints, exact f at bucket edges, closed form on the final bracket),
// organised for one block:
//   * a first scan finds the smallest and largest breakpoint key; bits
//     above their first difference are common to every key, so the passes
//     start right below them (bracket [P, P + 2^(shift0+8)) with P the
//     common prefix); if f exceeds r^2 already at P, lambda* lies below
//     every breakpoint (closed form with all of them above it);
//   * pass 0 scans every element; afterwards each warp gathers the elements
//     of the chosen bucket into its own list (global scratch), and later
//     passes scan only these lists;
//   * full scans load four rounds of keys (and values) before using them.
// Warp w owns elements w*32 + 256 t + lane; within a warp, equal buckets are
// summed by their lowest lane in lane order; warps are combined in order:
// the result is deterministic.
constexpr int kScanUnroll = 4;
constexpr int kMaxCluster = 8;          // blocks per problem in the clustered search
constexpr int64_t kClusterMinElems = 8192;  // problems with at least n + m elements use it

__device__ __forceinline__ void hist_add(bool act, int bk, double vd, double vg, double ve,
                                         double (*hist)[kBuckets][3], unsigned (*cnt)[kBuckets],
                                         double (*stage)[kWarp][3], int warp, int lane) {
  if (__ballot_sync(kFull, act) == 0u) return;
  const unsigned grp = __match_any_sync(kFull, act ? bk : -1);
  const bool leader = act && (grp & ((1u << lane) - 1u)) == 0u;
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
  __syncwarp();
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int o) {
  return (unsigned long long)__shfl_xor_sync(kFull, (long long)v, o);
}

template <int CS>
__global__ void __launch_bounds__(kSearchThreads) b_search_kernel(BInst *I,
                                                                  const int32_t *__restrict__ plist,
                                                                  int64_t nx_total,
                                                                  SearchArrays sa) {
  const int pk = plist[blockIdx.x / CS];
  BInst &B = I[pk];
  const int sidx = blockIdx.y;
  __shared__ LSearch L;
  __shared__ double bc[kBuckets], bsd[kBuckets], bsg[kBuckets], bse[kBuckets];
  __shared__ double lb[CS > 1 ? 2 : 1][4][kBuckets];  // this block's bucket sums (cluster exchange)
  __shared__ double cum_d[kBuckets + 1], cum_e[kBuckets + 1], tail_g[kBuckets + 1];
  __shared__ double wt[3][8];
  __shared__ int kstar;
  __shared__ unsigned long long wmin[kSearchWarps], wmax[kSearchWarps];
  __shared__ int64_t wcnt[kSearchWarps];
  extern __shared__ __align__(16) unsigned char dsm[];
  double(*hist)[kBuckets][3] = reinterpret_cast<double(*)[kBuckets][3]>(dsm);
  unsigned(*cnt)[kBuckets] = reinterpret_cast<unsigned(*)[kBuckets]>(dsm + kSearchHistBytes);
  double(*stage)[kWarp][3] =
      reinterpret_cast<double(*)[kWarp][3]>(dsm + kSearchHistBytes + kSearchCntBytes);
  const int tid = threadIdx.x;
  if (tid == 0) L = B.ls[sidx];
  __syncthreads();
  // every block of a cluster reads the same state: the whole cluster leaves together
  if (!B.due || B.status != kRunning || L.done) return;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = CS > 1 ? (int)cluster.block_rank() : 0;
  const uint64_t *__restrict__ keys = sidx ? sa.keys[1] : sa.keys[0];
  const double *__restrict__ d2 = sidx ? sa.d2[1] : sa.d2[0];
  const double *__restrict__ g2 = sidx ? sa.g2[1] : sa.g2[0];
  const double *__restrict__ gd = sidx ? sa.gd[1] : sa.gd[0];
  const int64_t nx = B.ncol, N = nx + B.nrow;
  const int64_t xbase = B.col0, ybase = nx_total + B.row0 - nx;
  const int lane = tid & (kWarp - 1), warp = tid >> 5;
  const int gw = rank * kSearchWarps + warp;              // warp index in the cluster
  constexpr int64_t kRound = (int64_t)CS * kSearchThreads;  // elements per round of a cluster
  const int64_t cap = ((N + kRound - 1) / kRound) * kWarp;
  int32_t *list = (sidx ? sa.cand[1] : sa.cand[0]) + (int64_t)B.col0 + B.row0 +
                  (int64_t)kMaxCluster * kSearchThreads * pk + gw * cap;
  auto elem = [&](int64_t v) { return v < nx ? xbase + v : ybase + v; };

  // smallest and largest breakpoint key (over the cluster)
  {
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t base = (int64_t)gw * kWarp; base < N; base += kScanUnroll * kRound) {
      uint64_t k[kScanUnroll];
#pragma unroll
      for (int r = 0; r < kScanUnroll; ++r) {
        const int64_t v = base + r * kRound + lane;
        k[r] = v < N ? keys[elem(v)] : kNoKey;
      }
#pragma unroll
      for (int r = 0; r < kScanUnroll; ++r) {
        if (k[r] != kNoKey) {
          lo = k[r] < lo ? k[r] : lo;
          hi = k[r] > hi ? k[r] : hi;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long a = shfl_xor_u64(lo, o), b = shfl_xor_u64(hi, o);
      lo = a < lo ? a : lo;
      hi = b > hi ? b : hi;
    }
    if (lane == 0) {
      wmin[warp] = lo;
      wmax[warp] = hi;
    }
  }
  if (CS > 1) cluster.sync();
  else __syncthreads();
  unsigned long long kmin = ~0ull, kmax = 0ull;
  for (int r = 0; r < CS; ++r) {
    const unsigned long long *rmin = CS > 1 ? cluster.map_shared_rank(wmin, r) : wmin;
    const unsigned long long *rmax = CS > 1 ? cluster.map_shared_rank(wmax, r) : wmax;
    for (int w = 0; w < kSearchWarps; ++w) {
      kmin = rmin[w] < kmin ? rmin[w] : kmin;
      kmax = rmax[w] > kmax ? rmax[w] : kmax;
    }
  }
  if (kmin > kmax) {  // no finite breakpoint: every coordinate moves without bound
    if (tid == 0 && rank == 0) {
      L.lambda = sqrt(fmax(L.r2 - L.f_lo, 0.0) / L.f_hi);
      L.rho_r = L.e_lo + L.lambda * L.f_hi;
      L.done = 1;
      B.ls[sidx] = L;
    }
    if (CS > 1) cluster.sync();  // no block leaves while another may read its memory
    return;
  }
  const int cp = (kmin == kmax) ? 64 : __clzll((long long)(kmin ^ kmax));
  // bucket bits [shift0, shift0 + 8) hold the first differing bit (63 - cp);
  // every bit from shift0 + 8 up is common to all keys
  const int shift0 = (56 - cp) > 0 ? ((56 - cp + 7) / 8) * 8 : 0;
  if (tid == 0) L.prefix = (shift0 + 8 >= 64) ? 0ull : (kmin & ~((1ull << (shift0 + 8)) - 1ull));
  if (tid < kSearchWarps) wcnt[tid] = 0;
  __syncthreads();

  for (int shift = shift0, pass = 0; shift >= 0; shift -= 8, ++pass) {
    const uint64_t pre = L.prefix;
    for (int i = tid; i < kSearchWarps * kBuckets; i += kSearchThreads) {
      double *h = &hist[0][0][0] + 3 * i;
      h[0] = 0.0;
      h[1] = 0.0;
      h[2] = 0.0;
      (&cnt[0][0])[i] = 0u;
    }
    __syncthreads();
    const bool full_prefix = (shift + 8 >= 64);
    auto match = [&](uint64_t k) {
      return k != kNoKey && (full_prefix || (k >> (shift + 8)) == (pre >> (shift + 8)));
    };
    if (pass == 0) {
      for (int64_t base = (int64_t)gw * kWarp; base < N; base += kScanUnroll * kRound) {
        uint64_t k[kScanUnroll];
        double a[kScanUnroll], b[kScanUnroll], c[kScanUnroll];
#pragma unroll
        for (int r = 0; r < kScanUnroll; ++r) {
          const int64_t v = base + r * kRound + lane;
          k[r] = kNoKey;
          if (v < N) {
            const int64_t e = elem(v);
            k[r] = keys[e];
            a[r] = d2[e];
            b[r] = g2[e];
            c[r] = gd[e];
          }
        }
#pragma unroll
        for (int r = 0; r < kScanUnroll; ++r) {
          const bool act = match(k[r]);
          hist_add(act, act ? (int)((k[r] >> shift) & 255u) : -1, act ? a[r] : 0.0,
                   act ? b[r] : 0.0, act ? c[r] : 0.0, hist, cnt, stage, warp, lane);
        }
      }
    } else {
      const int64_t nl = wcnt[warp];
      for (int64_t base = 0; base < nl; base += kWarp) {
        const int64_t i = base + lane;
        uint64_t k = kNoKey;
        int32_t e = 0;
        if (i < nl) {
          e = list[i];
          k = keys[e];
        }
        const bool act = match(k);
        hist_add(act, act ? (int)((k >> shift) & 255u) : -1, act ? d2[e] : 0.0,
                 act ? g2[e] : 0.0, act ? gd[e] : 0.0, hist, cnt, stage, warp, lane);
      }
    }
    __syncthreads();
    const int b = tid;
    {
      double c = 0.0, sd = 0.0, sg = 0.0, se = 0.0;
      for (int w = 0; w < kSearchWarps; ++w) {
        c += (double)cnt[w][b];
        sd += hist[w][b][0];
        sg += hist[w][b][1];
        se += hist[w][b][2];
      }
      if (CS > 1) {
        double(*mine)[kBuckets] = lb[pass & 1];
        mine[0][b] = c;
        mine[1][b] = sd;
        mine[2][b] = sg;
        mine[3][b] = se;
        // lb is double-buffered by pass parity: a block rewrites this buffer two
        // passes later, after the next cluster barrier, which every reader of
        // this pass has reached
        cluster.sync();
        c = sd = sg = se = 0.0;
        for (int r = 0; r < CS; ++r) {  // blocks in rank order: the same sums in every block
          const double *rem = cluster.map_shared_rank(&lb[pass & 1][0][0], r);
          c += rem[b];
          sd += rem[kBuckets + b];
          sg += rem[2 * kBuckets + b];
          se += rem[3 * kBuckets + b];
        }
      }
      bc[b] = c;
      bsd[b] = sd;
      bsg[b] = sg;
      bse[b] = se;
      if (b == 0) kstar = -1;
    }
    __syncthreads();
    const double pd = scan256(bsd[b], wt[0]);
    const double pe = scan256(bse[b], wt[1]);
    const double pg = scan256(bsg[kBuckets - 1 - b], wt[2]);  // reversed: suffix sums
    __syncthreads();
    {
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
    {
      const uint64_t edge_bits = pre | ((uint64_t)b << shift);
      const double edge = __longlong_as_double((long long)edge_bits);
      bool ok = false;
      if ((edge_bits >> 63) == 0ull && isfinite(edge)) {  // nonnegative finite edges only
        const double f = L.f_lo + cum_d[b] + edge * edge * (L.f_hi + tail_g[b]);
        ok = f <= L.r2;
      }
      if (ok) atomicMax(&kstar, b);
    }
    __syncthreads();
    if (tid == 0) {
      if (kstar < 0) {
        // f > r^2 at the bracket's lower end (only possible in the first pass,
        // at the common prefix): lambda* lies below every breakpoint
        L.f_hi += tail_g[0];
        L.lambda = sqrt(fmax(L.r2 - L.f_lo, 0.0) / L.f_hi);
        L.rho_r = L.e_lo + L.lambda * L.f_hi;
        L.done = 1;
      } else {
        const int k = kstar;
        L.f_lo += cum_d[k];
        L.e_lo += cum_e[k];
        L.f_hi += tail_g[k + 1];
        L.prefix = pre | ((uint64_t)k << shift);
        if (bc[k] == 0.0 || shift == 0) {
          if (bc[k] != 0.0) {  // last pass: breakpoints equal to the edge are clamped
            L.f_lo += bsd[k];
            L.e_lo += bse[k];
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
    }
    __syncthreads();
    if (L.done) break;  // the same decision in every block of the cluster
    if (pass == 0) {
      // gather the chosen bucket's elements (keys matching the new prefix
      // down to bit shift) into this warp's list, in scan order
      const uint64_t np = L.prefix;
      int64_t n_out = 0;
      for (int64_t base = (int64_t)gw * kWarp; base < N; base += kScanUnroll * kRound) {
        uint64_t k[kScanUnroll];
        int64_t e[kScanUnroll];
#pragma unroll
        for (int r = 0; r < kScanUnroll; ++r) {
          const int64_t v = base + r * kRound + lane;
          k[r] = kNoKey;
          e[r] = 0;
          if (v < N) {
            e[r] = elem(v);
            k[r] = keys[e[r]];
          }
        }
#pragma unroll
        for (int r = 0; r < kScanUnroll; ++r) {
          const bool keep = k[r] != kNoKey && (k[r] >> shift) == (np >> shift);
          const unsigned bal = __ballot_sync(kFull, keep);
          if (keep) list[n_out + __popc(bal & ((1u << lane) - 1u))] = (int32_t)e[r];
          n_out += __popc(bal);
        }
      }
      if (lane == 0) wcnt[warp] = n_out;
      __syncthreads();
    }
  }
  if (tid == 0 && rank == 0) B.ls[sidx] = L;
  if (CS > 1) cluster.sync();  // no block leaves while another may read its memory
}

// Restart rule per due problem (Eq. adaptive-restart-scheme, flexible,
// fixed), counters and iteration limits, and the running count (one thread
// per problem; integer atomics, so the count is exact).
__global__ void __launch_bounds__(kBlock) b_decide_kernel(BInst *I, BGlobal *G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int count = G->count, Kb = G->Kb, scheme = G->scheme;
  bool run = false;
  if (i < count) {
    BInst &B = I[i];
    B.restart_now = 0;
    B.use_cur = 0;
    if (B.status == kRunning) {
      if (B.due) {
        double rho = NAN, r = B.last_r;
        int use_cur = 0;
        if (scheme == kSchemeAdaptive || scheme == kSchemeFlexible) {
          const LSearch &La = B.ls[0];
          r = sqrt(La.r2);
          rho = (La.r2 > 0.0) ? La.rho_r / r : 0.0;
          if (scheme == kSchemeFlexible) {
            const LSearch &Lc = B.ls[1];
            const double rc = sqrt(Lc.r2);
            const double rho_c = (Lc.r2 > 0.0) ? Lc.rho_r / rc : 0.0;
            if (rho_c < rho) {
              use_cur = 1;
              rho = rho_c;
              r = rc;
            }
          }
        }
        const int64_t t = B.t0 + Kb;
        int restart = 0;
        if (scheme == kSchemeAdaptive || scheme == kSchemeFlexible)
          restart = (B.restarts == 0) ? (t >= B.tau0) : (rho <= G->beta * B.rho_stored);
        else if (scheme == kSchemeFixed)
          restart = (t >= B.fixed_len);
        B.last_rho = rho;
        B.last_r = r;
        B.use_cur = use_cur;
        B.restart_now = restart;
        if (restart) {
          B.rho_stored = rho;
          B.restarts += 1;
          B.t0 = 0;
          // mixed precision: the next correction is scaled by the distance moved
          if (G->mixed && r > 0.0 && isfinite(r)) B.mix_s = fmin(1.0 / r, 1e12);
        } else {
          B.t0 = t;
        }
        B.since = 0;
      } else {
        B.t0 += Kb;
      }
      if (B.iters >= B.iter_cap) B.status = kStatusIterLimit;  // the check's restart still happens
      else run = true;
    }
  }
  const unsigned bal = __ballot_sync(kFull, run);
  if ((threadIdx.x & (kWarp - 1)) == 0 && bal) atomicAdd(&G->running, __popc(bal));
}

// Grid (chunks, problems): block (x, k) copies elements x*kCopyChunk + ...
// of problem k.
constexpr int kCopyChunk = 4096;
__global__ void __launch_bounds__(kBlock) b_restart_copy_kernel(DevVecs v, const BInst *I) {
  const BInst &B = I[blockIdx.y];
  const int rs = B.restart_now, uc = B.use_cur;
  if (!rs && !uc) return;
  const int64_t lo = (int64_t)blockIdx.x * kCopyChunk;
  const int64_t nx = B.ncol, N = nx + B.nrow;
  if (lo >= N) return;
  const int64_t hi = lo + kCopyChunk < N ? lo + kCopyChunk : N;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (t < nx) {
      const int64_t j = B.col0 + t;
      const double s = uc ? v.x[j] : v.xbar[j];
      if (rs) {
        v.x0[j] = s;
        v.x[j] = s;
      }
      v.xbar[j] = s;
    } else {
      const int64_t i = B.row0 + (t - nx);
      const double s = uc ? v.y[i] : v.ybar[i];
      if (rs) {
        v.y0[i] = s;
        v.y[i] = s;
      }
      v.ybar[i] = s;
    }
  }
}

// Mixed precision, grid (chunks, problems) like the restart copy.
// b_combine: the FP64 iterate and average z = z^{n,0} + dz / s of each due
// problem (every problem when forced), projected onto X x Y.
__global__ void __launch_bounds__(kBlock) b_combine_kernel(DevVecs v, MixVecs mv, const BInst *I,
                                                           int force) {
  const BInst &B = I[blockIdx.y];
  if (!force && !B.due) return;
  const int64_t lo = (int64_t)blockIdx.x * kCopyChunk;
  const int64_t nx = B.ncol, N = nx + B.nrow;
  if (lo >= N) return;
  const int64_t hi = lo + kCopyChunk < N ? lo + kCopyChunk : N;
  const double inv = 1.0 / B.mix_s;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (t < nx) {
      const int64_t j = B.col0 + t;
      const double x0 = v.x0[j], l = v.lb[j], u = v.ub[j];
      v.x[j] = fmin(fmax(fma((double)mv.dx[j], inv, x0), l), u);
      v.xbar[j] = fmin(fmax(fma(mv.dxbar[j], inv, x0), l), u);
    } else {
      const int64_t r = B.row0 + (t - nx);
      const int rt = v.row_type[r];
      const double ylo = (rt == 1) ? 0.0 : -INFINITY, yhi = (rt == 2) ? 0.0 : INFINITY;
      const double y0 = v.y0[r];
      v.y[r] = fmin(fmax(fma((double)mv.dy[r], inv, y0), ylo), yhi);
      v.ybar[r] = fmin(fmax(fma(mv.dybar[r], inv, y0), ylo), yhi);
    }
  }
}

// b_recenter: after a restart the correction data are re-formed in FP64 --
// s times the residuals (from the check) of the chosen candidate at the new
// restart point -- and dz restarts at 0; the flexible scheme's replacement
// of the average by the current iterate is applied to dz.  Forced: every
// problem, candidate 0 (set-up).
__global__ void __launch_bounds__(kBlock) b_recenter_kernel(DevVecs v, MixVecs mv, const BInst *I,
                                                            int force) {
  const BInst &B = I[blockIdx.y];
  const int rs = force ? 1 : B.restart_now, uc = force ? 0 : B.use_cur;
  if (!rs && !uc) return;
  const int64_t lo = (int64_t)blockIdx.x * kCopyChunk;
  const int64_t nx = B.ncol, N = nx + B.nrow;
  if (lo >= N) return;
  const int64_t hi = lo + kCopyChunk < N ? lo + kCopyChunk : N;
  const double sc = B.mix_s;
  const double *lam = uc ? mv.lam[1] : mv.lam[0];
  const double *gy = uc ? mv.gy[1] : mv.gy[0];
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (t < nx) {
      const int64_t j = B.col0 + t;
      if (rs) {
        const double x0 = v.x0[j];
        mv.cf[j] = (float)(sc * lam[j]);
        mv.lf[j] = (float)(sc * (v.lb[j] - x0));
        mv.uf[j] = (float)(sc * (v.ub[j] - x0));
        mv.dx[j] = 0.0f;
        mv.dxhat[j] = 0.0f;
        mv.dxbar[j] = 0.0;
      } else {
        mv.dxbar[j] = (double)mv.dx[j];
      }
    } else {
      const int64_t r = B.row0 + (t - nx);
      if (rs) {
        const int rt = v.row_type[r];
        const double ylo = (rt == 1) ? 0.0 : -INFINITY, yhi = (rt == 2) ? 0.0 : INFINITY;
        const double y0 = v.y0[r];
        mv.bf[r] = (float)(-sc * gy[r]);
        mv.ylo[r] = (float)(sc * (ylo - y0));
        mv.yhi[r] = (float)(sc * (yhi - y0));
        mv.dy[r] = 0.0f;
        mv.dybar[r] = 0.0;
      } else {
        mv.dybar[r] = (double)mv.dy[r];
      }
    }
  }
}

// ------------------------------------------------------------- adjoint
//
// Recording of the unrolled forward (lp_batch_solve_recorded): before each
// block, every problem's inner count t0 and restart count; after it, whether
// the block's check restarted the problem.
__global__ void b_rec_pre_kernel(const BInst *I, int count, int64_t *t0, int64_t *restarts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  t0[i] = I[i].t0;
  restarts[i] = I[i].restarts;
}

__global__ void b_rec_post_kernel(const BInst *I, int count, const int64_t *restarts_before,
                                  int8_t *restarted, int *stopped) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  restarted[i] = I[i].restarts > restarts_before[i] ? 1 : 0;
  if (I[i].status != kRunning) atomicOr(stopped, 1);
}

// Averaging weights of a recorded block: w[i][k] = 1 / (t0_i + k + 1).
__global__ void b_rec_weights_kernel(const int64_t *t0, int count, int K, double *wtab) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)count * K) return;
  const int i = (int)(e / K), k = (int)(e - (int64_t)i * K);
  wtab[e] = 1.0 / (double)(t0[i] + k + 1);
}

// Adjoint steps over every slice, with the slice's problem's tau, sigma and
// weights of steps k and k - 1 (epilogues AdjColsEpi / AdjRowsEpi).
__global__ void __launch_bounds__(kBlock) b_adj_cols_kernel(SellMat AT, const double *__restrict__ u,
                                                            AdjColsEpi epi,
                                                            const BInst *__restrict__ I,
                                                            const int32_t *__restrict__ sinst,
                                                            const double *__restrict__ wtab, int K,
                                                            int k) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < AT.nslices; s += nwarps) {
    const int i = sinst[s];
    epi.tau = I[i].tau;
    epi.sigma = I[i].sigma;
    epi.w = wtab[(size_t)i * K + k];
    process_item<1, 2, true>(AT, u, (const double *)nullptr, s, lane, epi);
  }
}

__global__ void __launch_bounds__(kBlock) b_adj_rows_kernel(SellMat A, const double *__restrict__ v,
                                                            AdjRowsEpi epi,
                                                            const BInst *__restrict__ I,
                                                            const int32_t *__restrict__ sinst,
                                                            const double *__restrict__ wtab, int K,
                                                            int k) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
  for (int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < A.nslices; s += nwarps) {
    const int i = sinst[s];
    epi.tau = I[i].tau;
    epi.sigma = I[i].sigma;
    epi.w_prev = k > 0 ? wtab[(size_t)i * K + k - 1] : 0.0;
    process_item<1, 4, true>(A, v, (const double *)nullptr, s, lane, epi);
  }
}

// Start of a reverse block, grid (chunks, problems): the restart after the
// block (if problem k restarted there: ax moves into axb, ay into ayb), then
// u of the block's last step.
__global__ void __launch_bounds__(kBlock) b_adj_block_start_kernel(AdjVecs a, const BInst *I,
                                                                   const int8_t *restarted,
                                                                   const uint8_t *my_last,
                                                                   const double *wtab, int K) {
  const int p = blockIdx.y;
  const BInst &B = I[p];
  const int64_t lo = (int64_t)blockIdx.x * kCopyChunk;
  const int64_t nx = B.ncol, N = nx + B.nrow;
  if (lo >= N) return;
  const int64_t hi = lo + kCopyChunk < N ? lo + kCopyChunk : N;
  const int rs = restarted[p];
  const double sigma = B.sigma, w = wtab[(size_t)p * K + K - 1];
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (t < nx) {
      const int64_t j = B.col0 + t;
      if (rs) {
        a.axb[j] += a.ax[j];
        a.ax[j] = 0.0;
      }
    } else {
      const int64_t r = B.row0 + (t - nx);
      double ay = a.ay[r], yb = a.ayb[r];
      if (rs) {
        yb += ay;
        ay = 0.0;
        a.ay[r] = 0.0;
      }
      const double up = my_last[r] ? fma(w, yb, ay) : 0.0;
      a.ab[r] = fma(sigma, up, a.ab[r]);
      a.ayb[r] = (1.0 - w) * yb;
      a.u[r] = up;
    }
  }
}

// z <- zbar for the problems whose recorded check restarted (replay of the
// final block after the reverse sweep), grid (chunks, problems).
__global__ void __launch_bounds__(kBlock) b_rec_restart_kernel(DevVecs v, const BInst *I,
                                                               const int8_t *restarted) {
  const int p = blockIdx.y;
  if (!restarted[p]) return;
  const BInst &B = I[p];
  const int64_t lo = (int64_t)blockIdx.x * kCopyChunk;
  const int64_t nx = B.ncol, N = nx + B.nrow;
  if (lo >= N) return;
  const int64_t hi = lo + kCopyChunk < N ? lo + kCopyChunk : N;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (t < nx) v.x[B.col0 + t] = v.xbar[B.col0 + t];
    else v.y[B.row0 + (t - nx)] = v.ybar[B.row0 + (t - nx)];
  }
}

// Block-wide exclusive scan of one int per thread (kListThreads threads);
// returns the exclusive prefix, *total receives the block total.
__device__ __forceinline__ int block_exscan(int v, int *warp_tot, int *total) {
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int u = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += u;
  }
  if (lane == kWarp - 1) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
      const int u = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += u;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const int before = (warp == 0 ? 0 : warp_tot[warp - 1]) + x - v;
  *total = warp_tot[kWarp - 1];
  __syncthreads();
  return before;
}

// Work lists of the next block (slices of the running problems, in problem
// order): one block scans the running problems' slice counts into offsets;
// then one block per running problem writes its slice ids and the averaging
// weights w[k][kk] = 1 / (t0_k + kk + 1) of its next block.
__global__ void __launch_bounds__(kListThreads) b_list_scan_kernel(BInst *I, BGlobal *G) {
  __shared__ int wt[kWarp];
  const int count = G->count;
  int carry_c = 0, carry_r = 0;
  for (int base = 0; base < count; base += kListThreads) {
    const int i = base + (int)threadIdx.x;
    int nc = 0, nr = 0;
    if (i < count && I[i].status == kRunning) {
      nc = I[i].cs1 - I[i].cs0;
      nr = I[i].rs1 - I[i].rs0;
    }
    int tc = 0, tr = 0;
    const int oc = carry_c + block_exscan(nc, wt, &tc);
    const int orr = carry_r + block_exscan(nr, wt, &tr);
    if (i < count) {
      I[i].wlc0 = oc;
      I[i].wlr0 = orr;
    }
    carry_c += tc;
    carry_r += tr;
  }
  if (threadIdx.x == 0) {
    G->wl_n[0] = carry_c;
    G->wl_n[1] = carry_r;
  }
}

__global__ void __launch_bounds__(kBlock) b_list_fill_kernel(const BInst *I, const BGlobal *G,
                                                             int32_t *wl_c, int32_t *wl_r,
                                                             double *wtab) {
  const BInst &B = I[blockIdx.x];
  if (B.status != kRunning) return;
  const int Kb = G->Kb;
  for (int t = threadIdx.x; t < B.cs1 - B.cs0; t += blockDim.x) wl_c[B.wlc0 + t] = B.cs0 + t;
  for (int t = threadIdx.x; t < B.rs1 - B.rs0; t += blockDim.x) wl_r[B.wlr0 + t] = B.rs0 + t;
  for (int k = threadIdx.x; k < Kb; k += blockDim.x)
    wtab[(size_t)blockIdx.x * Kb + k] = 1.0 / (double)(B.t0 + k + 1);
}

// --------------------------------------------------------- setup kernels

__device__ double block_sum_sq(const double *p, int64_t begin, int64_t end, double *red) {
  double s = 0.0;
  for (int64_t j = begin + threadIdx.x; j < end; j += blockDim.x) s += p[j] * p[j];
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

__device__ double block_sum(double s, double *red) {
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

// One Lanczos step on A_k^T A_k per problem still running (one block per
// problem), after w = A^T (A v) over the whole batch: alpha = v . w,
// w <- w - alpha v - beta_prev v_prev, beta = ||w||, then v_next = w / beta.
// alpha and beta go to the problem's row of the coefficient tables
// (cap entries each); every few steps, at beta = 0 (invariant subspace) or
// at the cap, warp 0 evaluates the largest Ritz value (tridiag_top_eig) and
// the problem stops when it changed by at most pw_tol relative since the
// previous evaluation.  The same recurrence as the single-problem kernels.
__global__ void __launch_bounds__(kBlock) b_lanczos_kernel(BInst *I, BGlobal *G,
                                                           const double *vprev, const double *v,
                                                           double *w, double *alpha,
                                                           double *beta, int cap, int k,
                                                           int evaluate) {
  BInst &B = I[blockIdx.x];
  if (B.pw_done) return;
  __shared__ double red[kBlock];
  __shared__ int stop;
  const int64_t c0 = B.col0, c1 = (int64_t)B.col0 + B.ncol;
  double s = 0.0;
  for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) s += v[j] * w[j];
  const double a = block_sum(s, red);
  double *al = alpha + (size_t)blockIdx.x * cap, *be = beta + (size_t)blockIdx.x * cap;
  const double bprev = k > 0 ? be[k - 1] : 0.0;
  double q = 0.0;
  for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
    double r = w[j] - a * v[j];
    if (k > 0) r -= bprev * vprev[j];
    w[j] = r;
    q += r * r;
  }
  const double bk = sqrt(block_sum(q, red));
  if (threadIdx.x == 0) {
    al[k] = a;
    be[k] = bk;
    stop = 0;
  }
  __syncthreads();
  const bool last = (k + 1 >= cap) || !(bk > 0.0);
  if ((evaluate || last) && threadIdx.x < kWarp) {
    const double theta = tridiag_top_eig(al, be, k + 1);
    if (threadIdx.x == 0) {
      const int conv = (B.pw_iters > 0 && fabs(theta - B.pw_est) <= G->pw_tol * theta);
      B.pw_est = theta;
      B.pw_iters = k + 1;
      stop = (conv || last) ? 1 : 0;
    }
  }
  __syncthreads();
  if (stop) {
    if (threadIdx.x == 0) B.pw_done = 1;
    return;
  }
  if (threadIdx.x == 0) atomicAdd(&G->pw_running, 1);
  for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) w[j] = w[j] / bk;
}

// One power-iteration step per problem (Section 7: sigma_max(A_k)^2 as the
// Rayleigh quotient of A_k^T A_k), after av = A v and w = A^T av over the
// whole batch: ray = ||A v||^2 (||v|| = 1), stop when |ray - est| <= tol ray
// after the first step, or A^T A v = 0, or at the step cap; otherwise
// v <- w / ||w||.
__global__ void __launch_bounds__(kBlock) b_power_kernel(BInst *I, BGlobal *G, double *v,
                                                         const double *av, const double *w) {
  BInst &B = I[blockIdx.x];
  if (B.pw_done) return;
  __shared__ double red[kBlock];
  __shared__ int stop;
  const double ray = block_sum_sq(av, B.row0, (int64_t)B.row0 + B.nrow, red);
  const double nw2 = block_sum_sq(w, B.col0, (int64_t)B.col0 + B.ncol, red);
  const double nw = sqrt(nw2);
  if (threadIdx.x == 0) {
    const int done = (B.pw_iters > 0 && fabs(ray - B.pw_est) <= G->pw_tol * ray);
    B.pw_est = ray;
    B.pw_iters += 1;
    B.pw_nw = nw;
    stop = (nw == 0.0 || done || B.pw_iters >= G->pw_max) ? 1 : 0;
    if (stop) B.pw_done = 1;
    else atomicAdd(&G->pw_running, 1);
  }
  __syncthreads();
  if (stop) return;
  for (int j = B.col0 + threadIdx.x; j < B.col0 + B.ncol; j += blockDim.x) v[j] = w[j] / nw;
}

__global__ void __launch_bounds__(kBlock) b_norms_kernel(BInst *I, const double *b,
                                                         const double *c) {
  BInst &B = I[blockIdx.x];
  __shared__ double red[kBlock];
  const double b2 = block_sum_sq(b, B.row0, (int64_t)B.row0 + B.nrow, red);
  const double c2 = block_sum_sq(c, B.col0, (int64_t)B.col0 + B.ncol, red);
  if (threadIdx.x == 0) {
    B.norm_b = sqrt(b2);
    B.norm_c = sqrt(c2);
  }
}

// Each problem's solution candidate (average or current iterate).
__global__ void __launch_bounds__(kBlock) b_select_kernel(const BInst *I, const double *cur,
                                                          const double *avg, double *out,
                                                          int rows) {
  const BInst &B = I[blockIdx.x];
  const int lo = rows ? B.row0 : B.col0, len = rows ? B.nrow : B.ncol;
  const double *src = B.returned ? cur : avg;
  for (int j = lo + threadIdx.x; j < lo + len; j += blockDim.x) out[j] = src[j];
}

// ------------------------------------------------------------- launchers

int blocks_for_slices(int nslices) { return std::max(1, (nslices + kWarpsPerBlock - 1) / kWarpsPerBlock); }

template <int U, bool PIPE>
void b_primal_launch(int g, cudaStream_t s, const SellMat &AT, const double *y, const PrimalEpi &epi,
                     const BInst *I, const int32_t *sinst, const int32_t *wl, const BGlobal *G,
                     const double *wtab, int k) {
  launch_pdl(b_primal_kernel<U, PIPE>, g, kBlock, s, AT, y, epi, I, sinst, wl, G, wtab, k);
}

template <int U, bool PIPE>
void b_dual_launch(int g, cudaStream_t s, const SellMat &A, const double *xhat, const DualEpi &epi,
                   const BInst *I, const int32_t *sinst, const int32_t *wl, const BGlobal *G,
                   const double *wtab, int k) {
  launch_pdl(b_dual_kernel<U, PIPE>, g, kBlock, s, A, xhat, epi, I, sinst, wl, G, wtab, k);
}

template <int U, bool PIPE>
void b_primal_mix_launch(int g, cudaStream_t s, const SellMat &AT, const float *dy,
                         const PrimalMixEpi &epi, const BInst *I, const int32_t *sinst,
                         const int32_t *wl, const BGlobal *G, const double *wtab, int k) {
  launch_pdl(b_primal_mix_kernel<U, PIPE>, g, kBlock, s, AT, dy, epi, I, sinst, wl, G, wtab, k);
}

template <int U, bool PIPE>
void b_dual_mix_launch(int g, cudaStream_t s, const SellMat &A, const float *dxhat,
                       const DualMixEpi &epi, const BInst *I, const int32_t *sinst,
                       const int32_t *wl, const BGlobal *G, const double *wtab, int k) {
  launch_pdl(b_dual_mix_kernel<U, PIPE>, g, kBlock, s, A, dxhat, epi, I, sinst, wl, G, wtab, k);
}

}  // namespace
}  // namespace lpg

using namespace lpg;

struct lp_batch {
  int32_t count = 0, m = 0, n = 0;
  int64_t nnz = 0;
  lp_options opt{};
  lp_batch_tuning tune{};
  int device = 0, nsm = 0;
  std::vector<void *> allocs;
  SellMat A{}, AT{};
  int32_t *sinst_a = nullptr, *sinst_at = nullptr;
  int32_t *chunk_a = nullptr, *chunk_at = nullptr;  // check chunks: first slice, + end
  int nchunk_a = 0, nchunk_at = 0;
  int64_t max_elems = 0;  // largest n_k + m_k
  DevVecs v{};
  bool mixed = false;
  MixVecs mv{};
  BInst *I = nullptr;
  BGlobal *G = nullptr;
  double *wtab = nullptr;
  double *spart = nullptr;
  int64_t pstride = 0;
  SearchArrays sa{};
  int nsearch = 0;
  int32_t *wl[2] = {nullptr, nullptr};
  int32_t *perm_x = nullptr, *perm_y = nullptr;
  double *tmp = nullptr, *tmp2 = nullptr;
  int32_t *plist_big = nullptr, *plist_small = nullptr;  // search: clustered / one block
  int n_big = 0, n_small = 0;
  std::vector<int32_t> row_start, col_start;
  std::vector<int32_t> size_class;
  int32_t class_k[kMaxClasses] = {0};
  int32_t unroll_cols = -2, unroll_rows = -4;
  int grid_cols = 1, grid_rows = 1;
  double tune_ms = 0.0, setup_ms = 0.0;
  double tune_iter_ms[kMaxClasses] = {0}, tune_check_ms[kMaxClasses] = {0};
  std::vector<double> eta, sigma_max;
  std::vector<int32_t> sigma_steps;  // steps of the sigma_max estimator per problem
  int64_t blocks = 0;
  // unrolled-forward recording for lp_batch_backward
  double *ckpt = nullptr;            // [blocks][2n + 2m]: x, y, xbar, ybar at block start
  int64_t rec_blocks = 0;
  int64_t *rec_t0 = nullptr;         // [blocks][count] inner count at block start
  int64_t *rec_r0 = nullptr;         // [count] restart count before the current block
  int8_t *rec_rs = nullptr;          // [blocks][count] the block's check restarted the problem
  int *rec_stopped = nullptr;        // a problem left the running state while recording
  double *wrec = nullptr;            // [count][K] weights of the block being recomputed
  uint8_t *mask_x = nullptr, *mask_y = nullptr;  // [K][n], [K][m]
  AdjVecs adj{};
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t *h_running = nullptr;  // pinned [2]
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool solved = false;

  ~lp_batch() {
    if (ckpt) cudaFree(ckpt);
    if (rec_t0) cudaFree(rec_t0);
    if (rec_rs) cudaFree(rec_rs);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (h_running) cudaFreeHost(h_running);
    for (void *p : allocs) cudaFree(p);
  }

  template <class T>
  lp_status alloc(T **p, int64_t count_) {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(16, sizeof(T) * (size_t)std::max<int64_t>(count_, 1));
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    allocs.push_back(q);
    *p = static_cast<T *>(q);
    return LP_OK;
  }

  template <class T, class Al>
  lp_status upload(T **p, const std::vector<T, Al> &h) {
    lp_status s = alloc(p, (int64_t)h.size());
    if (s != LP_OK) return s;
    if (!h.empty()) LP_CU(cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return LP_OK;
  }

  lp_status upload_sell(const HostSell &H, SellMat &M, bool with_f32) {
    SliceInfo *info = nullptr;
    int32_t *ix = nullptr;
    double *vv = nullptr;
    float *vf = nullptr;
    lp_status s;
    if ((s = upload(&info, H.info)) != LP_OK) return s;
    if ((s = upload(&ix, H.idx)) != LP_OK) return s;
    if ((s = upload(&vv, H.val)) != LP_OK) return s;
    if (with_f32) {
      uvec<float> hf(H.val.size());
      parallel_for((int64_t)hf.size(), [&](int64_t lo, int64_t hi) {
        for (int64_t q = lo; q < hi; ++q) hf[q] = (float)H.val[q];
      });
      if ((s = upload(&vf, hf)) != LP_OK) return s;
    }
    M.nrows = H.nrows;
    M.ncols = H.ncols;
    M.nslices = H.nslices;
    M.n_warp_rows = H.n_warp_rows;
    M.info = info;
    M.idx = ix;
    M.val = vv;
    M.valf = vf;
    return LP_OK;
  }

  void launch_primal(int k, cudaStream_t s) {
    const int g = grid_cols;
    if (mixed) {
      PrimalMixEpi me{mv.cf, mv.lf, mv.uf, mv.dx, mv.dxhat, mv.dxbar, 0.0f, 0.0};
      switch (unroll_cols) {
        case 2: b_primal_mix_launch<2, false>(g, s, AT, mv.dy, me, I, sinst_at, wl[0], G, wtab, k); break;
        case 4: b_primal_mix_launch<4, false>(g, s, AT, mv.dy, me, I, sinst_at, wl[0], G, wtab, k); break;
        case -4: b_primal_mix_launch<4, true>(g, s, AT, mv.dy, me, I, sinst_at, wl[0], G, wtab, k); break;
        default: b_primal_mix_launch<2, true>(g, s, AT, mv.dy, me, I, sinst_at, wl[0], G, wtab, k); break;
      }
      return;
    }
    PrimalEpi epi{v.c, v.lbk, v.ubk, v.x, v.xhat, v.xbar, 0.0, 0.0, nullptr};
    switch (unroll_cols) {
      case 2: b_primal_launch<2, false>(g, s, AT, v.y, epi, I, sinst_at, wl[0], G, wtab, k); break;
      case 4: b_primal_launch<4, false>(g, s, AT, v.y, epi, I, sinst_at, wl[0], G, wtab, k); break;
      case -4: b_primal_launch<4, true>(g, s, AT, v.y, epi, I, sinst_at, wl[0], G, wtab, k); break;
      default: b_primal_launch<2, true>(g, s, AT, v.y, epi, I, sinst_at, wl[0], G, wtab, k); break;
    }
  }

  void launch_dual(int k, cudaStream_t s) {
    const int g = grid_rows;
    if (mixed) {
      DualMixEpi me{mv.bf, mv.ylo, mv.yhi, mv.dy, mv.dybar, 0.0f, 0.0};
      switch (unroll_rows) {
        case 2: b_dual_mix_launch<2, false>(g, s, A, mv.dxhat, me, I, sinst_a, wl[1], G, wtab, k); break;
        case 4: b_dual_mix_launch<4, false>(g, s, A, mv.dxhat, me, I, sinst_a, wl[1], G, wtab, k); break;
        case -2: b_dual_mix_launch<2, true>(g, s, A, mv.dxhat, me, I, sinst_a, wl[1], G, wtab, k); break;
        default: b_dual_mix_launch<4, true>(g, s, A, mv.dxhat, me, I, sinst_a, wl[1], G, wtab, k); break;
      }
      return;
    }
    DualEpi epi{v.b, v.row_type, v.y, v.ybar, 0.0, 0.0, nullptr};
    switch (unroll_rows) {
      case 2: b_dual_launch<2, false>(g, s, A, v.xhat, epi, I, sinst_a, wl[1], G, wtab, k); break;
      case 4: b_dual_launch<4, false>(g, s, A, v.xhat, epi, I, sinst_a, wl[1], G, wtab, k); break;
      case -2: b_dual_launch<2, true>(g, s, A, v.xhat, epi, I, sinst_a, wl[1], G, wtab, k); break;
      default: b_dual_launch<4, true>(g, s, A, v.xhat, epi, I, sinst_a, wl[1], G, wtab, k); break;
    }
  }

  // work lists and averaging weights of the next block
  // one forward step of the recorded iteration, writing the clamp and
  // projection masks (weights from wtab_rec)
  void launch_masked_step(int k, const double *wtab_rec, cudaStream_t s) {
    const int K = opt.check_every;
    PrimalEpi pe{v.c, v.lbk, v.ubk, v.x, v.xhat, v.xbar, 0.0, 0.0, mask_x + (int64_t)k * n};
    b_primal_launch<2, true>(blocks_for_slices(AT.nslices), s, AT, v.y, pe, I, sinst_at, wl[0], G,
                             wtab_rec, k);
    DualEpi de{v.b, v.row_type, v.y, v.ybar, 0.0, 0.0, mask_y + (int64_t)k * std::max(m, 1)};
    b_dual_launch<4, true>(blocks_for_slices(A.nslices), s, A, v.xhat, de, I, sinst_a, wl[1], G,
                           wtab_rec, k);
    (void)K;
  }

  void launch_worklist(cudaStream_t s) {
    b_list_scan_kernel<<<1, kListThreads, 0, s>>>(I, G);
    b_list_fill_kernel<<<count, kBlock, 0, s>>>(I, G, wl[0], wl[1], wtab);
  }

  dim3 chunk_grid() const {
    return dim3((unsigned)((max_elems + kCopyChunk - 1) / kCopyChunk), (unsigned)count);
  }

  void launch_combine(int force, cudaStream_t s) {
    b_combine_kernel<<<chunk_grid(), kBlock, 0, s>>>(v, mv, I, force);
  }

  void launch_check(cudaStream_t s) {
    b_pre_check_kernel<<<(count + kBlock - 1) / kBlock, kBlock, 0, s>>>(I, G);
    if (mixed) launch_combine(0, s);
    CheckColsEpi ce{};
    if (mixed) {
      ce.lam_out0 = mv.lam[0];
      ce.lam_out1 = mv.lam[1];
    }
    ce.c = v.c; ce.lb = v.lb; ce.ub = v.ub; ce.xbar = v.xbar; ce.x = v.x; ce.x0 = v.x0;
    ce.ga = GapOut{sa.keys[0], sa.d2[0], sa.g2[0], sa.gd[0]};
    ce.gc = GapOut{sa.keys[1], sa.d2[1], sa.g2[1], sa.gd[1]};
    CheckRowsEpi re{};
    re.b = v.b; re.rt = v.row_type; re.ybar = v.ybar; re.y = v.y; re.y0 = v.y0;
    re.ga = ce.ga;
    re.gc = ce.gc;
    re.off = n;
    if (mixed) {
      re.gy_out0 = mv.gy[0];
      re.gy_out1 = mv.gy[1];
    }
    b_check_kernel<CheckColsEpi><<<blocks_for_slices(nchunk_at), kBlock, 0, s>>>(
        AT, v.ybar, v.y, ce, I, sinst_at, chunk_at, nchunk_at, G, spart, pstride, 0);
    b_check_kernel<CheckRowsEpi><<<blocks_for_slices(nchunk_a), kBlock, 0, s>>>(
        A, v.xbar, v.x, re, I, sinst_a, chunk_a, nchunk_a, G, spart, pstride, nchunk_at);
    b_finalize_kernel<<<count, kBlock, 0, s>>>(I, G, spart, pstride, nchunk_at);
    if (nsearch > 0 && n_small > 0)
      b_search_kernel<1><<<dim3(n_small, nsearch), kSearchThreads, kSearchSmem, s>>>(
          I, plist_small, n, sa);
    if (nsearch > 0 && n_big > 0) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      cfg.gridDim = dim3((unsigned)(n_big * kMaxCluster), (unsigned)nsearch);
      cfg.blockDim = dim3(kSearchThreads);
      cfg.dynamicSmemBytes = kSearchSmem;
      cfg.stream = s;
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kMaxCluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, b_search_kernel<kMaxCluster>, I, (const int32_t *)plist_big,
                         (int64_t)n, sa);
    }
    b_decide_kernel<<<(count + kBlock - 1) / kBlock, kBlock, 0, s>>>(I, G);
    b_restart_copy_kernel<<<chunk_grid(), kBlock, 0, s>>>(v, I);
    if (mixed) b_recenter_kernel<<<chunk_grid(), kBlock, 0, s>>>(v, mv, I, 0);
    launch_worklist(s);
  }
};

namespace {

lp_status batch_build_graph(lp_batch *h) {
  if (h->exec) return LP_OK;
  cudaStream_t s = h->cap_stream;
  LP_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < h->opt.check_every; ++k) {
    h->launch_primal(k, s);
    h->launch_dual(k, s);
  }
  h->launch_check(s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  h->graph = g;
  LP_CU(cudaGraphInstantiate(&h->exec, g, 0));
  return LP_OK;
}

// Resets every problem's Algorithm-1 state to z^{0,0} = proj(0) (status
// running, counters zero), the averaging weights and the work lists.
lp_status batch_reset(lp_batch *h, cudaStream_t s, const double *x_start = nullptr,
                      const double *y_start = nullptr) {
  std::vector<BInst> hi(h->count);
  LP_CU(cudaMemcpyAsync(hi.data(), h->I, sizeof(BInst) * h->count, cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  for (BInst &B : hi) {
    B.status = kRunning;
    B.returned = B.restart_now = B.use_cur = B.due = 0;
    B.t0 = B.iters = B.checks = B.restarts = B.since = 0;
    B.iter_cap = h->opt.max_iter;
    B.tau0 = h->opt.tau0 > 0 ? h->opt.tau0 : B.K;
    B.fixed_len = h->opt.fixed_len;
    B.rho_stored = B.last_rho = B.last_r = NAN;
    for (int q = 0; q < 5; ++q) B.kkt_a[q] = B.kkt_c[q] = NAN;
    B.kkt_a[4] = B.kkt_c[4] = INFINITY;
    B.ls[0].done = B.ls[1].done = 1;
    B.mix_s = 1.0;
  }
  LP_CU(cudaMemcpyAsync(h->I, hi.data(), sizeof(BInst) * h->count, cudaMemcpyHostToDevice, s));
  // z^{0,0} = proj(start): the caller's point (caller order, host or device) or zero
  if (x_start) {
    LP_CU(cudaMemcpyAsync(h->tmp, x_start, sizeof(double) * h->n, cudaMemcpyDefault, s));
    launch_gather(h->v.x, h->tmp, h->perm_x, h->n, s);
  } else {
    launch_fill(h->v.x, 0.0, h->n, s);
  }
  if (y_start && h->m > 0) {
    LP_CU(cudaMemcpyAsync(h->tmp, y_start, sizeof(double) * h->m, cudaMemcpyDefault, s));
    launch_gather(h->v.y, h->tmp, h->perm_y, h->m, s);
  } else {
    launch_fill(h->v.y, 0.0, h->m, s);
  }
  launch_project(h->v, h->n, h->m, s);
  if (h->mixed) {  // correction data at the starting point, dz = 0, s = 1
    launch_residuals(h->A, h->AT, h->v, h->mv, h->n, h->m, s);
    b_recenter_kernel<<<h->chunk_grid(), kBlock, 0, s>>>(h->v, h->mv, h->I, 1);
  }
  h->launch_worklist(s);
  LP_CU(cudaGetLastError());
  LP_CU(cudaStreamSynchronize(s));
  h->blocks = 0;
  h->solved = false;
  return LP_OK;
}

// Status <- running for every problem that has not failed; iteration cap
// <- iters + max_iter; tol.  Then the work lists.
lp_status batch_start(lp_batch *h, double tol, cudaStream_t s) {
  std::vector<BInst> hi(h->count);
  LP_CU(cudaMemcpyAsync(hi.data(), h->I, sizeof(BInst) * h->count, cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  for (BInst &B : hi) {
    if (B.status == kStatusNumerical) continue;
    B.status = kRunning;
    B.iter_cap = B.iters + h->opt.max_iter;
  }
  LP_CU(cudaMemcpyAsync(h->I, hi.data(), sizeof(BInst) * h->count, cudaMemcpyHostToDevice, s));
  LP_CU(cudaMemcpyAsync(&h->G->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
  h->launch_worklist(s);
  LP_CU(cudaGetLastError());
  return LP_OK;
}

// Milliseconds per call of f (enqueued `reps` times on s after one warm-up
// call), by CUDA events on s.
template <class F>
lp_status time_ms(cudaStream_t s, int reps, F f, double *out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LP_CU(cudaEventCreate(&e0));
  LP_CU(cudaEventCreate(&e1));
  f();
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) f();
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "tuner timing");
  LP_CU(cudaGetLastError());
  *out = ms / reps;
  return LP_OK;
}

// The batch's tuner (run at create on the batch itself, from z = proj(0)):
//  (1) kernel variants: for each pass, every unroll code of {2, 4, -2, -4}
//      with one warp per slice or a grid of 8 blocks per SM (grid-stride
//      over the work list), timed over 5 launches; the fastest is kept;
//  (2) check period per size class: with only that class running, the
//      cost of one iteration (both passes) and of one check (the whole
//      chain, every problem due) are timed; the class gets the smallest
//      K = K_base 2^s (s <= max_k_shift) with check <= budget x K x iteration.
// Leaves the state dirty: the caller resets it.
lp_status batch_tune(lp_batch *h, cudaStream_t s) {
  lp_status e;
  const int cands[4] = {2, 4, -2, -4};
  const int g_full[2] = {blocks_for_slices(h->AT.nslices), blocks_for_slices(h->A.nslices)};
  for (int pass = 0; pass < 2; ++pass) {
    double best = 1e300;
    int bu = pass ? h->unroll_rows : h->unroll_cols, bg = g_full[pass];
    for (int u : cands) {
      for (int gm = 0; gm < 2; ++gm) {
        const int g = gm ? std::min(g_full[pass], 8 * h->nsm) : g_full[pass];
        if (gm && g == g_full[pass]) continue;
        (pass ? h->unroll_rows : h->unroll_cols) = u;
        (pass ? h->grid_rows : h->grid_cols) = g;
        double t = 0.0;
        if (pass == 0) e = time_ms(s, 5, [&] { h->launch_primal(0, s); }, &t);
        else e = time_ms(s, 5, [&] { h->launch_dual(0, s); }, &t);
        if (e != LP_OK) return e;
        if (t < best) {
          best = t;
          bu = u;
          bg = g;
        }
      }
    }
    (pass ? h->unroll_rows : h->unroll_cols) = bu;
    (pass ? h->grid_rows : h->grid_cols) = bg;
  }
  // check period per size class
  std::vector<BInst> hi(h->count), run(h->count);
  LP_CU(cudaMemcpy(hi.data(), h->I, sizeof(BInst) * h->count, cudaMemcpyDeviceToHost));
  const int Kb = h->opt.check_every;
  for (int c = 0; c < kMaxClasses; ++c) {
    bool any = false;
    for (int32_t q = 0; q < h->count; ++q) any |= (h->size_class[q] == c);
    if (!any) continue;
    for (int32_t q = 0; q < h->count; ++q) {
      run[q] = hi[q];
      run[q].status = (h->size_class[q] == c) ? kRunning : LP_ERR_NOT_SOLVED;
      run[q].K = Kb;
      run[q].since = 0;
      run[q].iter_cap = INT64_MAX;
    }
    LP_CU(cudaMemcpyAsync(h->I, run.data(), sizeof(BInst) * h->count, cudaMemcpyHostToDevice, s));
    h->launch_worklist(s);
    double t_it = 0.0, t_ck = 0.0;
    if ((e = time_ms(s, 4, [&] { h->launch_primal(0, s); h->launch_dual(0, s); }, &t_it)) != LP_OK)
      return e;
    if ((e = time_ms(s, 3, [&] { h->launch_check(s); }, &t_ck)) != LP_OK) return e;
    int sh = 0;
    while (sh < h->tune.max_k_shift && t_ck > h->tune.check_budget * (double)(Kb << sh) * t_it) ++sh;
    h->class_k[c] = Kb << sh;
    h->tune_iter_ms[c] = t_it;
    h->tune_check_ms[c] = t_ck;
  }
  for (int32_t q = 0; q < h->count; ++q) hi[q].K = h->class_k[h->size_class[q]];
  LP_CU(cudaMemcpy(h->I, hi.data(), sizeof(BInst) * h->count, cudaMemcpyHostToDevice));
  return LP_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int class_of(int64_t nnz) {
  int c = 0;
  int64_t lim = 256;  // 64 * 4
  while (c < kMaxClasses - 1 && nnz >= lim) {
    ++c;
    lim *= 4;
  }
  return c;
}

}  // namespace

extern "C" {

void lp_batch_default_tuning(lp_batch_tuning *t) {
  if (!t) return;
  t->autotune = 1;
  t->max_k_shift = 2;
  t->check_budget = 0.05;
}

lp_status lp_batch_create(int32_t count, const int32_t *host_row_start,
                          const int32_t *host_col_start, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, const double *val, const double *c,
                          const double *b, const double *lb, const double *ub,
                          const int8_t *row_type, const lp_options *opt_in,
                          const lp_batch_tuning *tuning, void *cuda_stream,
                          lp_batch_handle *out) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_create");
  const auto t_start = std::chrono::steady_clock::now();
  if (!out) return fail(LP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1) return fail(LP_ERR_INVALID_ARG, "count must be >= 1");
  if (!host_row_start || !host_col_start) return fail(LP_ERR_INVALID_ARG, "NULL problem boundaries");
  std::vector<int32_t> rs(host_row_start, host_row_start + count + 1);
  std::vector<int32_t> cs(host_col_start, host_col_start + count + 1);
  if (rs[0] != 0 || cs[0] != 0) return fail(LP_ERR_INVALID_ARG, "problem boundaries must start at 0");
  for (int32_t k = 0; k < count; ++k) {
    if (rs[k + 1] < rs[k]) return fail(LP_ERR_INVALID_ARG, "host_row_start must be nondecreasing");
    if (cs[k + 1] <= cs[k]) return fail(LP_ERR_INVALID_ARG, "every problem needs at least one column");
  }
  const int32_t m = rs[count], n = cs[count];
  if ((int64_t)m + n + (int64_t)kMaxCluster * kSearchThreads * count >= (int64_t(1) << 31))
    return fail(LP_ERR_INVALID_ARG, "the batch needs m + n + 2048 count < 2^31");
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return fail(LP_ERR_INVALID_ARG, "nnz must lie in [0, 2^31)");
  if (!row_ptr || !c || !lb || !ub || (m > 0 && (!b || !row_type)) ||
      (nnz > 0 && (!col_idx || !val)))
    return fail(LP_ERR_INVALID_ARG, "NULL array argument");
  lp_options opt;
  if (opt_in) opt = *opt_in;
  else lp_default_options(&opt);
  lp_status st = validate_options(opt);
  if (st != LP_OK) return st;
  if (opt.spmv_mode != 0) return fail(LP_ERR_INVALID_ARG, "the batched solver has spmv_mode 0 only");
  lp_batch_tuning tune{};
  tune.autotune = 0;
  tune.max_k_shift = 0;
  tune.check_budget = 0.05;
  if (tuning) tune = *tuning;
  if (tune.max_k_shift < 0 || tune.max_k_shift > 8) return fail(LP_ERR_INVALID_ARG, "max_k_shift must lie in [0, 8]");
  if (!(tune.check_budget > 0.0)) return fail(LP_ERR_INVALID_ARG, "check_budget must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // ---- inputs (host arrays read in place, device arrays copied) and validation
  std::vector<int32_t> s_rp, s_ci;
  std::vector<double> s_v, s_c, s_b, s_l, s_u;
  std::vector<int8_t> s_rt;
  LP_CU(cudaStreamSynchronize(s));
  bool readable = true;
  const int32_t *hrp32 = host_view(row_ptr, (int64_t)m + 1, s_rp, &readable);
  const int32_t *hci = host_view(col_idx, nnz, s_ci, &readable);
  const double *hv = host_view(val, nnz, s_v, &readable);
  const double *hc = host_view(c, n, s_c, &readable);
  const double *hb = host_view(b, m, s_b, &readable);
  const double *hl = host_view(lb, n, s_l, &readable);
  const double *hu = host_view(ub, n, s_u, &readable);
  const int8_t *hrt = host_view(row_type, m, s_rt, &readable);
  if (!readable) return fail(LP_ERR_INVALID_ARG, "could not read an input array (bad pointer?)");
  if (hrp32[0] != 0) return fail(LP_ERR_INVALID_ARG, "row_ptr[0] must be 0");
  for (int32_t i = 0; i < m; ++i)
    if (hrp32[i + 1] < hrp32[i]) return fail(LP_ERR_INVALID_ARG, "row_ptr must be nondecreasing");
  if (hrp32[m] != nnz) return fail(LP_ERR_INVALID_ARG, "row_ptr[m] must equal nnz");
  {
    std::atomic<int> outside{0}, nonfinite{0};
    parallel_for(count, [&](int64_t k0, int64_t k1) {
      for (int64_t k = k0; k < k1; ++k)
        for (int64_t p = hrp32[rs[k]]; p < hrp32[rs[k + 1]]; ++p) {
          if (hci[p] < cs[k] || hci[p] >= cs[k + 1]) outside.store(1, std::memory_order_relaxed);
          if (!std::isfinite(hv[p])) nonfinite.store(1, std::memory_order_relaxed);
        }
    }, 1);
    if (outside.load()) return fail(LP_ERR_INVALID_ARG, "col_idx outside its problem's columns");
    if (nonfinite.load()) return fail(LP_ERR_INVALID_ARG, "non-finite matrix value");
  }
  for (int32_t j = 0; j < n; ++j) {
    if (!std::isfinite(hc[j])) return fail(LP_ERR_INVALID_ARG, "non-finite objective c");
    if (std::isnan(hl[j]) || std::isnan(hu[j]) || hl[j] > hu[j] || hl[j] == INFINITY ||
        hu[j] == -INFINITY)
      return fail(LP_ERR_INVALID_ARG, "invalid bounds (need lb <= ub, lb < inf, ub > -inf)");
  }
  for (int32_t i = 0; i < m; ++i) {
    if (!std::isfinite(hb[i])) return fail(LP_ERR_INVALID_ARG, "non-finite right-hand side b");
    if (hrt[i] < LP_ROW_EQ || hrt[i] > LP_ROW_LE) return fail(LP_ERR_INVALID_ARG, "row_type must be 0, 1 or 2");
  }
  std::vector<int64_t> cp;
  uvec<int32_t> ri;
  uvec<double> cv;
  if (!build_csc(m, n, hrp32, hci, hv, cp, ri, cv)) return fail(LP_ERR_INVALID_ARG, "col_idx out of range");
  if (csc_has_duplicates(n, cp, ri)) return fail(LP_ERR_INVALID_ARG, "duplicate column in a row");

  std::unique_ptr<lp_batch> h(new lp_batch());
  h->count = count;
  h->m = m;
  h->n = n;
  h->nnz = nnz;
  h->opt = opt;
  h->tune = tune;
  h->row_start = rs;
  h->col_start = cs;
  LP_CU(cudaGetDevice(&h->device));
  LP_CU(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
  h->nsearch = (opt.restart_scheme == LP_RESTART_ADAPTIVE) ? 1
               : (opt.restart_scheme == LP_RESTART_FLEXIBLE) ? 2 : 0;
  h->unroll_cols = opt.spmv_unroll % 100;
  h->unroll_rows = opt.spmv_unroll_rows % 100;

  // ---- per-problem permutations by length (stable counting sorts), sliced layouts
  std::vector<int64_t> rp((size_t)m + 1);
  for (int32_t i = 0; i <= m; ++i) rp[i] = hrp32[i];
  std::vector<int32_t> perm_y(m), perm_x(n), inv_y(m), inv_x(n);
  parallel_for(count, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      sort_by_length_desc(rp.data(), rs[k], rs[k + 1], perm_y.data());
      sort_by_length_desc(cp.data(), cs[k], cs[k + 1], perm_x.data());
    }
  }, 1);
  for (int32_t r = 0; r < m; ++r) inv_y[perm_y[r]] = r;
  for (int32_t r = 0; r < n; ++r) inv_x[perm_x[r]] = r;
  const std::vector<int32_t> brk_rows(rs.begin() + 1, rs.end() - 1);
  const std::vector<int32_t> brk_cols(cs.begin() + 1, cs.end() - 1);
  HostSell HA, HAT;
  const LanePolicy policy{opt.long_row_threshold, opt.lane_steps, opt.single_lane_max};
  const int64_t target = (int64_t)opt.lane_auto * h->nsm;
  const LanePolicy pa = choose_policy(rp, perm_y, policy, target, brk_rows);
  const LanePolicy pat = choose_policy(cp, perm_x, policy, target, brk_cols);
  build_sell(m, n, rp, hci, hv, perm_y, inv_x, pa, HA, brk_rows);
  build_sell(n, m, cp, ri.data(), cv.data(), perm_x, inv_y, pat, HAT, brk_cols);

  // slice -> problem, problem -> slice ranges
  std::vector<BInst> hi(count);
  std::vector<int32_t> sa_host(HA.nslices), sat_host(HAT.nslices);
  std::vector<int32_t> chk_a, chk_at;
  {
    int32_t k = 0;
    for (int32_t sl = 0; sl < HA.nslices; ++sl) {
      while (HA.info[sl].row0 >= rs[k + 1]) ++k;
      sa_host[sl] = k;
    }
    k = 0;
    for (int32_t sl = 0; sl < HAT.nslices; ++sl) {
      while (HAT.info[sl].row0 >= cs[k + 1]) ++k;
      sat_host[sl] = k;
    }
    for (int32_t q = 0; q < count; ++q) {
      hi[q].rs0 = hi[q].rs1 = -1;
      hi[q].cs0 = hi[q].cs1 = -1;
    }
    for (int32_t sl = 0; sl < HA.nslices; ++sl) {
      BInst &B = hi[sa_host[sl]];
      if (B.rs0 < 0) B.rs0 = sl;
      B.rs1 = sl + 1;
    }
    for (int32_t sl = 0; sl < HAT.nslices; ++sl) {
      BInst &B = hi[sat_host[sl]];
      if (B.cs0 < 0) B.cs0 = sl;
      B.cs1 = sl + 1;
    }
    h->size_class.resize(count);
    for (int32_t q = 0; q < count; ++q) {
      BInst &B = hi[q];
      if (B.rs0 < 0) B.rs0 = B.rs1 = 0;
      if (B.cs0 < 0) B.cs0 = B.cs1 = 0;
      // check chunks: consecutive runs of at most kCheckChunk slices of this problem
      B.cc0 = (int32_t)chk_at.size();
      for (int32_t sl = B.cs0; sl < B.cs1; sl += kCheckChunk) chk_at.push_back(sl);
      B.cc1 = (int32_t)chk_at.size();
      B.rc0 = (int32_t)chk_a.size();
      for (int32_t sl = B.rs0; sl < B.rs1; sl += kCheckChunk) chk_a.push_back(sl);
      B.rc1 = (int32_t)chk_a.size();
      B.col0 = cs[q];
      B.ncol = cs[q + 1] - cs[q];
      B.row0 = rs[q];
      B.nrow = rs[q + 1] - rs[q];
      B.K = opt.check_every;
      B.omega = opt.omega;
      B.status = kRunning;
      h->size_class[q] = class_of(rp[rs[q + 1]] - rp[rs[q]]);
      h->max_elems = std::max<int64_t>(h->max_elems, (int64_t)B.ncol + B.nrow);
    }
    chk_at.push_back(HAT.nslices);
    chk_a.push_back(HA.nslices);
    h->nchunk_at = (int)chk_at.size() - 1;
    h->nchunk_a = (int)chk_a.size() - 1;
  }

  // permuted vectors
  std::vector<double> pc(n), pl(n), pu(n), pb(m);
  std::vector<int8_t> prt(m);
  std::vector<long long> lk(n), uk(n);
  for (int32_t r = 0; r < n; ++r) {
    pc[r] = hc[perm_x[r]];
    pl[r] = hl[perm_x[r]];
    pu[r] = hu[perm_x[r]];
    long long bl, bu;
    std::memcpy(&bl, &pl[r], 8);
    std::memcpy(&bu, &pu[r], 8);
    lk[r] = bl < 0 ? (bl ^ 0x7fffffffffffffffll) : bl;
    uk[r] = bu < 0 ? (bu ^ 0x7fffffffffffffffll) : bu;
  }
  for (int32_t r = 0; r < m; ++r) {
    pb[r] = hb[perm_y[r]];
    prt[r] = hrt[perm_y[r]];
  }

  // ---- device buffers
  lp_status e;
  h->mixed = (opt.precision == LP_PRECISION_MIXED);
  if ((e = h->upload_sell(HA, h->A, h->mixed)) != LP_OK) return e;
  if ((e = h->upload_sell(HAT, h->AT, h->mixed)) != LP_OK) return e;
  if ((e = h->upload(&h->sinst_a, sa_host)) != LP_OK) return e;
  if ((e = h->upload(&h->sinst_at, sat_host)) != LP_OK) return e;
  if ((e = h->upload(&h->chunk_a, chk_a)) != LP_OK) return e;
  if ((e = h->upload(&h->chunk_at, chk_at)) != LP_OK) return e;
  if ((e = h->upload(&h->v.c, pc)) != LP_OK) return e;
  if ((e = h->upload(&h->v.lb, pl)) != LP_OK) return e;
  if ((e = h->upload(&h->v.ub, pu)) != LP_OK) return e;
  if ((e = h->upload(&h->v.lbk, lk)) != LP_OK) return e;
  if ((e = h->upload(&h->v.ubk, uk)) != LP_OK) return e;
  if ((e = h->upload(&h->v.b, pb)) != LP_OK) return e;
  if ((e = h->upload(&h->v.row_type, prt)) != LP_OK) return e;
  if ((e = h->upload(&h->perm_x, perm_x)) != LP_OK) return e;
  if ((e = h->upload(&h->perm_y, perm_y)) != LP_OK) return e;
  double **xs[] = {&h->v.x, &h->v.xhat, &h->v.xbar, &h->v.x0};
  for (double **p : xs)
    if ((e = h->alloc(p, n)) != LP_OK) return e;
  double **ys[] = {&h->v.y, &h->v.ybar, &h->v.y0};
  for (double **p : ys)
    if ((e = h->alloc(p, m)) != LP_OK) return e;
  if ((e = h->alloc(&h->tmp, std::max(n, m))) != LP_OK) return e;
  if ((e = h->alloc(&h->tmp2, std::max(n, m))) != LP_OK) return e;
  if (h->mixed) {
    MixVecs &mv = h->mv;
    float **fn[] = {&mv.cf, &mv.lf, &mv.uf, &mv.dx, &mv.dxhat};
    for (float **p : fn)
      if ((e = h->alloc(p, n)) != LP_OK) return e;
    float **fm[] = {&mv.bf, &mv.ylo, &mv.yhi, &mv.dy};
    for (float **p : fm)
      if ((e = h->alloc(p, m)) != LP_OK) return e;
    double **dn[] = {&mv.dxbar, &mv.lam[0], &mv.lam[1]};
    for (double **p : dn)
      if ((e = h->alloc(p, n)) != LP_OK) return e;
    double **dm[] = {&mv.dybar, &mv.gy[0], &mv.gy[1]};
    for (double **p : dm)
      if ((e = h->alloc(p, m)) != LP_OK) return e;
  }
  if ((e = h->alloc(&h->I, count)) != LP_OK) return e;
  if ((e = h->alloc(&h->G, 1)) != LP_OK) return e;
  if ((e = h->alloc(&h->wtab, (int64_t)count * opt.check_every)) != LP_OK) return e;
  h->pstride = (int64_t)h->nchunk_a + h->nchunk_at;
  if ((e = h->alloc(&h->spart, (int64_t)NQ * h->pstride)) != LP_OK) return e;
  if ((e = h->alloc(&h->wl[0], HAT.nslices)) != LP_OK) return e;
  if ((e = h->alloc(&h->wl[1], HA.nslices)) != LP_OK) return e;
  const int64_t N = (int64_t)n + m;
  for (int k = 0; k < 2; ++k) {
    if (k == 1 && h->nsearch < 2) {
      h->sa.keys[1] = h->sa.keys[0];
      h->sa.d2[1] = h->sa.d2[0];
      h->sa.g2[1] = h->sa.g2[0];
      h->sa.gd[1] = h->sa.gd[0];
      h->sa.cand[1] = h->sa.cand[0];
      break;
    }
    if ((e = h->alloc(&h->sa.cand[k], N + (int64_t)kMaxCluster * kSearchThreads * count)) != LP_OK)
      return e;
    if ((e = h->alloc(&h->sa.keys[k], N)) != LP_OK) return e;
    if ((e = h->alloc(&h->sa.d2[k], N)) != LP_OK) return e;
    if ((e = h->alloc(&h->sa.g2[k], N)) != LP_OK) return e;
    if ((e = h->alloc(&h->sa.gd[k], N)) != LP_OK) return e;
  }
  LP_CU(cudaFuncSetAttribute(b_search_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSearchSmem));
  LP_CU(cudaFuncSetAttribute(b_search_kernel<kMaxCluster>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSearchSmem));
  {
    // problems with many elements search with a cluster of kMaxCluster blocks,
    // if the device can hold such a cluster (else every problem uses one block)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(kMaxCluster);
    cfg.blockDim = dim3(kSearchThreads);
    cfg.dynamicSmemBytes = kSearchSmem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kMaxCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, b_search_kernel<kMaxCluster>, &cfg) !=
        cudaSuccess)
      nclusters = 0;
    cudaGetLastError();
    std::vector<int32_t> big, small;
    for (int32_t q = 0; q < count; ++q) {
      const int64_t ne = (int64_t)hi[q].ncol + hi[q].nrow;
      if (nclusters > 0 && ne >= kClusterMinElems) big.push_back(q);
      else small.push_back(q);
    }
    h->n_big = (int)big.size();
    h->n_small = (int)small.size();
    if ((e = h->upload(&h->plist_big, big)) != LP_OK) return e;
    if ((e = h->upload(&h->plist_small, small)) != LP_OK) return e;
  }
  LP_CU(cudaMallocHost(&h->h_running, 2 * sizeof(int32_t)));
  LP_CU(cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming));
  LP_CU(cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming));
  LP_CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  h->grid_cols = blocks_for_slices(HAT.nslices);
  h->grid_rows = blocks_for_slices(HA.nslices);

  BGlobal hg{};
  hg.tol = 1e-8;
  hg.beta = opt.beta;
  hg.pw_tol = opt.power_tol;
  hg.count = count;
  hg.Kb = opt.check_every;
  hg.scheme = opt.restart_scheme;
  hg.pw_max = opt.power_iters;
  hg.running = count;
  hg.mixed = h->mixed ? 1 : 0;
  LP_CU(cudaMemcpy(h->G, &hg, sizeof(BGlobal), cudaMemcpyHostToDevice));
  LP_CU(cudaMemcpy(h->I, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice));
  b_norms_kernel<<<count, kBlock, 0, s>>>(h->I, h->v.b, h->v.c);
  LP_CU(cudaGetLastError());

  // ---- step sizes (Section 7): eta_k = 0.9 / sigma_max(A_k) per problem
  h->eta.assign(count, opt.eta);
  h->sigma_max.assign(count, NAN);
  h->sigma_steps.assign(count, 0);
  if (!(opt.eta > 0.0)) {
    // start vector per problem: v_j = 0.5 + u_j, u_j from SplitMix64 at the
    // problem-local original column index j, normalized per problem
    std::vector<double> v0(n);
    std::vector<double> nv(count, 0.0);
    int32_t k = 0;
    for (int32_t r = 0; r < n; ++r) {
      while (r >= cs[k + 1]) ++k;
      const uint64_t j = (uint64_t)(perm_x[r] - cs[k]);
      uint64_t z = (j + 1) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      v0[r] = 0.5 + (double)(z >> 11) * 0x1.0p-53;
      nv[k] += v0[r] * v0[r];
    }
    k = 0;
    for (int32_t r = 0; r < n; ++r) {
      while (r >= cs[k + 1]) ++k;
      v0[r] /= std::sqrt(nv[k]);
    }
    double *pv = h->v.x, *pav = h->v.y, *pw = h->v.xhat;
    LP_CU(cudaMemcpy(pv, v0.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    if (opt.sigma_method == LP_SIGMA_LANCZOS) {
      // coefficient tables of count x cap doubles (cap shrinks for very large
      // batches so that the two tables stay within 1 GiB)
      const int cap = (int)std::min<int64_t>(
          std::min<int64_t>(opt.power_iters, kLanczosMax),
          std::max<int64_t>(64, ((int64_t)1 << 26) / std::max<int32_t>(count, 1)));
      double *coef = nullptr;
      if (cudaMalloc(&coef, sizeof(double) * 2 * (size_t)count * cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(LP_ERR_OOM, "cudaMalloc of the Lanczos coefficients failed");
      }
      struct Free {
        double *p;
        ~Free() { cudaFree(p); }
      } free_coef{coef};
      double *P[3] = {pv, pw, h->v.xbar};
      for (int k = 0; k < cap; ++k) {
        LP_CU(cudaMemsetAsync(&h->G->pw_running, 0, sizeof(int32_t), s));
        launch_spmv(h->A, P[k % 3], pav, s, nullptr);
        launch_spmv(h->AT, pav, P[(k + 1) % 3], s, nullptr);
        b_lanczos_kernel<<<count, kBlock, 0, s>>>(h->I, h->G, P[(k + 2) % 3], P[k % 3],
                                                  P[(k + 1) % 3], coef,
                                                  coef + (size_t)count * cap, cap, k,
                                                  (k + 1) % 4 == 0 ? 1 : 0);
        if ((k + 1) % 16 != 0 && k + 1 != cap) continue;
        LP_CU(cudaGetLastError());
        int32_t left = 0;
        LP_CU(cudaMemcpyAsync(&left, &h->G->pw_running, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LP_CU(cudaStreamSynchronize(s));
        if (left == 0) break;
      }
      LP_CU(cudaStreamSynchronize(s));
    } else {
      const int chunk = 25;
      for (int it = 0; it < opt.power_iters; it += chunk) {
        for (int q = 0; q < chunk; ++q) {
          LP_CU(cudaMemsetAsync(&h->G->pw_running, 0, sizeof(int32_t), s));
          launch_spmv(h->A, pv, pav, s, nullptr);
          launch_spmv(h->AT, pav, pw, s, nullptr);
          b_power_kernel<<<count, kBlock, 0, s>>>(h->I, h->G, pv, pav, pw);
        }
        LP_CU(cudaGetLastError());
        int32_t left = 0;
        LP_CU(cudaMemcpyAsync(&left, &h->G->pw_running, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LP_CU(cudaStreamSynchronize(s));
        if (left == 0) break;
      }
    }
    LP_CU(cudaStreamSynchronize(s));
    LP_CU(cudaMemcpy(hi.data(), h->I, sizeof(BInst) * count, cudaMemcpyDeviceToHost));
    for (int32_t q = 0; q < count; ++q) {
      h->sigma_max[q] = std::sqrt(hi[q].pw_est);
      h->sigma_steps[q] = hi[q].pw_iters;
      if (!(h->sigma_max[q] > 0.0) || !std::isfinite(h->sigma_max[q]))
        return fail(LP_ERR_NUMERICAL, "sigma_max of problem " + std::to_string(q) +
                                          " is zero or not finite; pass eta explicitly");
      h->eta[q] = 0.9 / h->sigma_max[q];
    }
  } else {
    LP_CU(cudaStreamSynchronize(s));
    LP_CU(cudaMemcpy(hi.data(), h->I, sizeof(BInst) * count, cudaMemcpyDeviceToHost));
  }
  for (int32_t q = 0; q < count; ++q) {
    hi[q].tau = h->eta[q] / opt.omega;
    hi[q].sigma = h->eta[q] * opt.omega;
  }
  LP_CU(cudaMemcpy(h->I, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice));
  for (int q = 0; q < kMaxClasses; ++q) h->class_k[q] = 0;
  for (int32_t q = 0; q < count; ++q) h->class_k[h->size_class[q]] = opt.check_every;
  if (tune.autotune) {
    const auto t_tune = std::chrono::steady_clock::now();
    if ((e = batch_reset(h.get(), s)) != LP_OK) return e;
    if ((e = batch_tune(h.get(), s)) != LP_OK) return e;
    h->tune_ms = ms_since(t_tune);
  }
  if ((e = batch_reset(h.get(), s)) != LP_OK) return e;
  h->setup_ms = ms_since(t_start);
  *out = h.release();
  return LP_OK;
}

lp_status lp_batch_set_state(lp_batch_handle h, const double *x, const double *y,
                             void *cuda_stream) {
  err_msg().clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  return batch_reset(h, static_cast<cudaStream_t>(cuda_stream), x, y);
}

lp_status lp_batch_select_omega(lp_batch_handle h, const double *host_omegas, int32_t n_omegas,
                                int64_t iters, double *host_kkt, double *host_best,
                                void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_select_omega");
  if (!h || !host_omegas || n_omegas < 1) return fail(LP_ERR_INVALID_ARG, "bad arguments");
  const int K = h->opt.check_every;
  if (iters < K || iters % K != 0)
    return fail(LP_ERR_INVALID_ARG, "iters must be a positive multiple of check_every");
  for (int32_t k = 0; k < n_omegas; ++k)
    if (!(host_omegas[k] > 0.0) || !std::isfinite(host_omegas[k]))
      return fail(LP_ERR_INVALID_ARG, "every omega must be finite and > 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  lp_status e = batch_build_graph(h);
  if (e != LP_OK) return e;
  const int count = h->count;
  auto set_scheme = [&](int32_t sch) -> lp_status {
    LP_CU(cudaMemcpyAsync(&h->G->scheme, &sch, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    return LP_OK;
  };
  // every problem gets omega_k (or its own choice), tau = eta/omega, sigma = eta*omega
  auto set_weights = [&](const std::vector<double> &om, bool unlimited) -> lp_status {
    std::vector<BInst> hi(count);
    LP_CU(cudaMemcpyAsync(hi.data(), h->I, sizeof(BInst) * count, cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    for (int32_t q = 0; q < count; ++q) {
      hi[q].omega = om[q];
      hi[q].tau = h->eta[q] / om[q];
      hi[q].sigma = h->eta[q] * om[q];
      if (unlimited) hi[q].iter_cap = INT64_MAX;
    }
    LP_CU(cudaMemcpyAsync(h->I, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, s));
    LP_CU(cudaStreamSynchronize(s));
    return LP_OK;
  };
  std::vector<double> kkt((size_t)count * n_omegas, INFINITY);
  if ((e = set_scheme(LP_RESTART_NONE)) != LP_OK) return e;
  const double tiny = 1e-300;
  for (int32_t k = 0; k < n_omegas; ++k) {
    if ((e = batch_reset(h, s)) != LP_OK) return e;
    if ((e = set_weights(std::vector<double>(count, host_omegas[k]), true)) != LP_OK) return e;
    LP_CU(cudaMemcpyAsync(&h->G->tol, &tiny, sizeof(double), cudaMemcpyHostToDevice, s));
    for (int64_t b = 0; b < iters / K; ++b) LP_CU(cudaGraphLaunch(h->exec, s));
    std::vector<BInst> hi(count);
    LP_CU(cudaMemcpyAsync(hi.data(), h->I, sizeof(BInst) * count, cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    for (int32_t q = 0; q < count; ++q) {
      const double v = std::fmin(hi[q].kkt_a[4], hi[q].kkt_c[4]);
      kkt[(size_t)q * n_omegas + k] = std::isfinite(v) ? v : INFINITY;
    }
  }
  std::vector<double> best(count);
  for (int32_t q = 0; q < count; ++q) {
    int32_t b = 0;
    for (int32_t k = 1; k < n_omegas; ++k)
      if (kkt[(size_t)q * n_omegas + k] < kkt[(size_t)q * n_omegas + b]) b = k;
    best[q] = host_omegas[b];
  }
  if ((e = set_scheme(h->opt.restart_scheme)) != LP_OK) return e;
  if ((e = batch_reset(h, s)) != LP_OK) return e;
  if ((e = set_weights(best, false)) != LP_OK) return e;
  if (host_kkt) std::copy(kkt.begin(), kkt.end(), host_kkt);
  if (host_best) std::copy(best.begin(), best.end(), host_best);
  return LP_OK;
}

lp_status lp_batch_set_check_every(lp_batch_handle h, const int32_t *host_k, void *cuda_stream) {
  err_msg().clear();
  if (!h || !host_k) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int Kb = h->opt.check_every;
  for (int32_t q = 0; q < h->count; ++q)
    if (host_k[q] < Kb || host_k[q] % Kb != 0)
      return fail(LP_ERR_INVALID_ARG, "check periods must be positive multiples of check_every");
  std::vector<BInst> hi(h->count);
  LP_CU(cudaMemcpyAsync(hi.data(), h->I, sizeof(BInst) * h->count, cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  for (int32_t q = 0; q < h->count; ++q) hi[q].K = host_k[q];
  LP_CU(cudaMemcpyAsync(h->I, hi.data(), sizeof(BInst) * h->count, cudaMemcpyHostToDevice, s));
  for (int q = 0; q < kMaxClasses; ++q) h->class_k[q] = 0;
  for (int32_t q = 0; q < h->count; ++q)
    h->class_k[h->size_class[q]] = std::max(h->class_k[h->size_class[q]], host_k[q]);
  return batch_reset(h, s);
}

lp_status lp_batch_iterate(lp_batch_handle h, int32_t n_blocks, double tol, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_iterate");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!(tol > 0.0)) return fail(LP_ERR_INVALID_ARG, "tol must be > 0");
  if (n_blocks < 0) return fail(LP_ERR_INVALID_ARG, "n_blocks must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  lp_status e = batch_build_graph(h);
  if (e != LP_OK) return e;
  if ((e = batch_start(h, tol, s)) != LP_OK) return e;
  for (int32_t i = 0; i < n_blocks; ++i) LP_CU(cudaGraphLaunch(h->exec, s));
  h->blocks += n_blocks;
  h->solved = true;
  return LP_OK;
}

lp_status lp_batch_solve(lp_batch_handle h, double tol, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_solve");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!(tol > 0.0)) return fail(LP_ERR_INVALID_ARG, "tol must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  lp_status e = batch_build_graph(h);
  if (e != LP_OK) return e;
  if ((e = batch_start(h, tol, s)) != LP_OK) return e;
  const int Kb = h->opt.check_every;
  // every problem stops within max_iter iterations (+ one block): bound the loop
  int64_t remaining = h->opt.max_iter / Kb + 2;
  int32_t running = 1;
  int inflight = 0, head = 0;  // ring of two (event, running-count slot)
  while (true) {
    while (inflight < 2 && remaining > 0) {
      const int slot = (head + inflight) & 1;
      LP_CU(cudaGraphLaunch(h->exec, s));
      LP_CU(cudaMemcpyAsync(&h->h_running[slot], &h->G->running, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
      LP_CU(cudaEventRecord(h->ev[slot], s));
      --remaining;
      ++h->blocks;
      ++inflight;
    }
    if (inflight == 0) break;
    LP_CU(cudaEventSynchronize(h->ev[head]));
    running = h->h_running[head];
    head ^= 1;
    --inflight;
    if (running == 0) break;
  }
  LP_CU(cudaStreamSynchronize(s));
  h->solved = true;
  std::vector<BInst> hi(h->count);
  LP_CU(cudaMemcpy(hi.data(), h->I, sizeof(BInst) * h->count, cudaMemcpyDeviceToHost));
  bool numerical = false, limit = false;
  for (const BInst &B : hi) {
    if (B.status == kStatusNumerical) numerical = true;
    else if (B.status != kStatusOK) limit = true;
  }
  if (numerical) return fail(LP_ERR_NUMERICAL, "NaN or Inf in a problem's iterates or residuals");
  if (limit) return fail(LP_ITER_LIMIT, "iteration limit reached by some problem");
  return LP_OK;
}

lp_status lp_batch_get_solution(lp_batch_handle h, double *x, double *y, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_get_solution");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "no solve has run on this batch");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (h->mixed) h->launch_combine(1, s);
  if (x) {
    b_select_kernel<<<h->count, kBlock, 0, s>>>(h->I, h->v.x, h->v.xbar, h->tmp2, 0);
    launch_scatter(h->tmp, h->tmp2, h->perm_x, h->n, s);
    LP_CU(cudaMemcpyAsync(x, h->tmp, sizeof(double) * h->n, cudaMemcpyDefault, s));
    LP_CU(cudaStreamSynchronize(s));
  }
  if (y && h->m > 0) {
    b_select_kernel<<<h->count, kBlock, 0, s>>>(h->I, h->v.y, h->v.ybar, h->tmp2, 1);
    launch_scatter(h->tmp, h->tmp2, h->perm_y, h->m, s);
    LP_CU(cudaMemcpyAsync(y, h->tmp, sizeof(double) * h->m, cudaMemcpyDefault, s));
    LP_CU(cudaStreamSynchronize(s));
  }
  LP_CU(cudaGetLastError());
  return LP_OK;
}

lp_status lp_batch_get_state(lp_batch_handle h, double *x, double *y, double *xbar, double *ybar,
                             double *x0, double *y0, void *cuda_stream) {
  err_msg().clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (h->mixed) h->launch_combine(1, s);
  struct Item { double *dst; const double *src; const int32_t *perm; int32_t len; };
  const Item items[] = {{x, h->v.x, h->perm_x, h->n},       {y, h->v.y, h->perm_y, h->m},
                        {xbar, h->v.xbar, h->perm_x, h->n}, {ybar, h->v.ybar, h->perm_y, h->m},
                        {x0, h->v.x0, h->perm_x, h->n},     {y0, h->v.y0, h->perm_y, h->m}};
  for (const Item &it : items) {
    if (!it.dst || it.len == 0) continue;
    launch_scatter(h->tmp, it.src, it.perm, it.len, s);
    LP_CU(cudaMemcpyAsync(it.dst, h->tmp, sizeof(double) * it.len, cudaMemcpyDefault, s));
    LP_CU(cudaStreamSynchronize(s));
  }
  LP_CU(cudaGetLastError());
  return LP_OK;
}

lp_status lp_batch_get_info(lp_batch_handle h, lp_batch_info *info,
                            lp_batch_problem_info *probs, int32_t capacity) {
  err_msg().clear();
  if (!h || !info) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  if (probs && capacity < 0) return fail(LP_ERR_INVALID_ARG, "capacity must be >= 0");
  std::vector<BInst> hi(h->count);
  BGlobal hg{};
  LP_CU(cudaMemcpy(hi.data(), h->I, sizeof(BInst) * h->count, cudaMemcpyDeviceToHost));
  LP_CU(cudaMemcpy(&hg, h->G, sizeof(BGlobal), cudaMemcpyDeviceToHost));
  std::memset(info, 0, sizeof(*info));
  info->count = h->count;
  int32_t running = 0;
  for (const BInst &B : hi) running += (B.status == kRunning);
  info->running = h->solved ? running : h->count;
  info->m = h->m;
  info->n = h->n;
  info->nnz = h->nnz;
  info->blocks = h->blocks;
  info->k_base = h->opt.check_every;
  info->spmv_unroll = h->unroll_cols;
  info->spmv_unroll_rows = h->unroll_rows;
  info->grid_cols = h->grid_cols;
  info->grid_rows = h->grid_rows;
  int nc = 0;
  for (int q = 0; q < kMaxClasses; ++q) {
    info->class_k[q] = h->class_k[q];
    info->class_iter_ms[q] = h->tune_iter_ms[q];
    info->class_check_ms[q] = h->tune_check_ms[q];
    nc += h->class_k[q] > 0;
  }
  info->n_classes = nc;
  info->tune_ms = h->tune_ms;
  info->setup_ms = h->setup_ms;
  if (probs) {
    const int32_t k = std::min(capacity, h->count);
    for (int32_t q = 0; q < k; ++q) {
      const BInst &B = hi[q];
      lp_batch_problem_info &P = probs[q];
      std::memset(&P, 0, sizeof(P));
      P.iters = B.iters;
      P.restarts = B.restarts;
      P.checks = B.checks;
      P.status = (B.status == kRunning) ? (h->solved ? LP_ITER_LIMIT : LP_ERR_NOT_SOLVED) : B.status;
      P.returned = B.returned;
      P.check_every = B.K;
      P.size_class = h->size_class[q];
      for (int i = 0; i < 5; ++i) {
        P.kkt_avg[i] = B.kkt_a[i];
        P.kkt_cur[i] = B.kkt_c[i];
      }
      P.eta = h->eta[q];
      P.sigma_max = h->sigma_max[q];
      P.sigma_steps = h->sigma_steps.empty() ? 0 : h->sigma_steps[q];
      P.tau = B.tau;
      P.sigma = B.sigma;
      P.rho_stored = B.rho_stored;
      P.last_rho = B.last_rho;
      P.omega = B.omega;
    }
  }
  return LP_OK;
}

lp_status lp_batch_solve_recorded(lp_batch_handle h, int64_t iters, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_solve_recorded");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  const int K = h->opt.check_every;
  if (iters < K || iters % K != 0) return fail(LP_ERR_INVALID_ARG, "iters must be a positive multiple of check_every");
  if (h->mixed) return fail(LP_ERR_INVALID_ARG, "recording needs LP_PRECISION_FP64");
  if (h->opt.restart_scheme == LP_RESTART_FLEXIBLE)
    return fail(LP_ERR_INVALID_ARG, "recording supports the adaptive, fixed and no-restart schemes");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  lp_status e = batch_build_graph(h);
  if (e != LP_OK) return e;
  const int64_t blocks = iters / K, slot = 2 * (int64_t)h->n + 2 * (int64_t)h->m;
  const int count = h->count, n = h->n, m = h->m;
  // every problem runs (no tolerance, no iteration cap) for exactly `iters`
  std::vector<BInst> hi(count);
  LP_CU(cudaMemcpyAsync(hi.data(), h->I, sizeof(BInst) * count, cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  for (BInst &B : hi) {
    if (B.status == kStatusNumerical) return fail(LP_ERR_NUMERICAL, "a problem has failed; reset the batch");
    B.status = kRunning;
    B.iter_cap = INT64_MAX;
  }
  LP_CU(cudaMemcpyAsync(h->I, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, s));
  const double tiny = 1e-300;
  LP_CU(cudaMemcpyAsync(&h->G->tol, &tiny, sizeof(double), cudaMemcpyHostToDevice, s));
  h->launch_worklist(s);
  // recording buffers
  if (h->ckpt) cudaFree(h->ckpt);
  if (h->rec_t0) cudaFree(h->rec_t0);
  if (h->rec_rs) cudaFree(h->rec_rs);
  h->ckpt = nullptr;
  h->rec_t0 = nullptr;
  h->rec_rs = nullptr;
  h->rec_blocks = 0;
  LP_CU(cudaMalloc(&h->ckpt, sizeof(double) * std::max<int64_t>(1, blocks * slot)));
  LP_CU(cudaMalloc(&h->rec_t0, sizeof(int64_t) * blocks * count));
  LP_CU(cudaMalloc(&h->rec_rs, sizeof(int8_t) * blocks * count));
  if (!h->mask_x) {  // masks, adjoint vectors and small records, once per batch
    if ((e = h->alloc(&h->mask_x, (int64_t)K * n)) != LP_OK) return e;
    if ((e = h->alloc(&h->mask_y, (int64_t)K * std::max(m, 1))) != LP_OK) return e;
    if ((e = h->alloc(&h->rec_r0, count)) != LP_OK) return e;
    if ((e = h->alloc(&h->rec_stopped, 1)) != LP_OK) return e;
    if ((e = h->alloc(&h->wrec, (int64_t)count * K)) != LP_OK) return e;
    double **xs[] = {&h->adj.ax, &h->adj.axb, &h->adj.ac, &h->adj.v};
    for (double **p : xs)
      if ((e = h->alloc(p, n)) != LP_OK) return e;
    double **ys[] = {&h->adj.ay, &h->adj.ayb, &h->adj.ab, &h->adj.u};
    for (double **p : ys)
      if ((e = h->alloc(p, std::max(m, 1))) != LP_OK) return e;
  }
  LP_CU(cudaMemsetAsync(h->rec_stopped, 0, sizeof(int), s));
  const int pg = (count + kBlock - 1) / kBlock;
  for (int64_t b = 0; b < blocks; ++b) {
    double *c = h->ckpt + b * slot;
    LP_CU(cudaMemcpyAsync(c, h->v.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(c + n, h->v.y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(c + n + m, h->v.xbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(c + 2 * n + m, h->v.ybar, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    b_rec_pre_kernel<<<pg, kBlock, 0, s>>>(h->I, count, h->rec_t0 + b * count, h->rec_r0);
    LP_CU(cudaGraphLaunch(h->exec, s));
    b_rec_post_kernel<<<pg, kBlock, 0, s>>>(h->I, count, h->rec_r0, h->rec_rs + b * count,
                                            h->rec_stopped);
    LP_CU(cudaGetLastError());
  }
  h->blocks += blocks;
  int stopped = 0;
  LP_CU(cudaMemcpyAsync(&stopped, h->rec_stopped, sizeof(int), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  if (stopped) return fail(LP_ERR_NUMERICAL, "a problem stopped during recording");
  h->rec_blocks = blocks;
  h->solved = true;
  return LP_OK;
}

lp_status lp_batch_backward(lp_batch_handle h, const double *dl_dx, const double *dl_dy,
                            double *dl_dc, double *dl_db, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_batch_backward");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (h->rec_blocks == 0) return fail(LP_ERR_NOT_SOLVED, "no recorded solve (lp_batch_solve_recorded)");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int n = h->n, m = h->m, K = h->opt.check_every, count = h->count;
  const int64_t slot = 2 * (int64_t)n + 2 * (int64_t)m;
  const int wg = (int)std::max<int64_t>(1, ((int64_t)count * K + kBlock - 1) / kBlock);
  AdjVecs &a = h->adj;
  launch_fill(a.ax, 0.0, n, s);
  launch_fill(a.ac, 0.0, n, s);
  launch_fill(a.ay, 0.0, m, s);
  launch_fill(a.ab, 0.0, m, s);
  if (dl_dx) {
    LP_CU(cudaMemcpyAsync(h->tmp, dl_dx, sizeof(double) * n, cudaMemcpyDefault, s));
    launch_gather(a.axb, h->tmp, h->perm_x, n, s);
  } else {
    launch_fill(a.axb, 0.0, n, s);
  }
  if (dl_dy && m > 0) {
    LP_CU(cudaMemcpyAsync(h->tmp, dl_dy, sizeof(double) * m, cudaMemcpyDefault, s));
    launch_gather(a.ayb, h->tmp, h->perm_y, m, s);
  } else {
    launch_fill(a.ayb, 0.0, m, s);
  }
  auto restore = [&](int64_t b) -> lp_status {
    const double *c = h->ckpt + b * slot;
    LP_CU(cudaMemcpyAsync(h->v.x, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.y, c + n, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.xbar, c + n + m, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.ybar, c + 2 * n + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    b_rec_weights_kernel<<<wg, kBlock, 0, s>>>(h->rec_t0 + b * count, count, K, h->wrec);
    for (int k = 0; k < K; ++k) h->launch_masked_step(k, h->wrec, s);
    return LP_OK;
  };
  const int ga = blocks_for_slices(h->A.nslices), gat = blocks_for_slices(h->AT.nslices);
  const int64_t mstride = std::max(m, 1);
  for (int64_t b = h->rec_blocks - 1; b >= 0; --b) {
    lp_status e = restore(b);  // recompute the block's steps with their masks
    if (e != LP_OK) return e;
    b_adj_block_start_kernel<<<h->chunk_grid(), kBlock, 0, s>>>(
        a, h->I, h->rec_rs + b * count, h->mask_y + (int64_t)(K - 1) * mstride, h->wrec, K);
    for (int k = K - 1; k >= 0; --k) {
      AdjColsEpi ce{a.ax, a.axb, a.ac, a.v, h->mask_x + (int64_t)k * n, 0.0, 0.0, 0.0};
      b_adj_cols_kernel<<<gat, kBlock, 0, s>>>(h->AT, a.u, ce, h->I, h->sinst_at, h->wrec, K, k);
      AdjRowsEpi re{a.ay, a.ayb, a.ab, a.u, k > 0 ? h->mask_y + (int64_t)(k - 1) * mstride : nullptr,
                    0.0, 0.0, 0.0, k > 0 ? 1 : 0};
      b_adj_rows_kernel<<<ga, kBlock, 0, s>>>(h->A, a.v, re, h->I, h->sinst_a, h->wrec, K, k);
    }
    LP_CU(cudaGetLastError());
  }
  // restore the final state of the recorded solve: replay the last block
  {
    lp_status e = restore(h->rec_blocks - 1);
    if (e != LP_OK) return e;
    b_rec_restart_kernel<<<h->chunk_grid(), kBlock, 0, s>>>(h->v, h->I,
                                                            h->rec_rs + (h->rec_blocks - 1) * count);
  }
  if (dl_dc) {
    launch_scatter(h->tmp, a.ac, h->perm_x, n, s);
    LP_CU(cudaMemcpyAsync(dl_dc, h->tmp, sizeof(double) * n, cudaMemcpyDefault, s));
    LP_CU(cudaStreamSynchronize(s));
  }
  if (dl_db && m > 0) {
    launch_scatter(h->tmp, a.ab, h->perm_y, m, s);
    LP_CU(cudaMemcpyAsync(dl_db, h->tmp, sizeof(double) * m, cudaMemcpyDefault, s));
  }
  LP_CU(cudaGetLastError());
  LP_CU(cudaStreamSynchronize(s));
  return LP_OK;
}

void lp_batch_destroy(lp_batch_handle h) { delete h; }

}  // extern "C"
