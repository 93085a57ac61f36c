// C ABI of liblp.so (declared in include/lp.h): problem setup, the
// restarted-PDHG driver around CUDA graphs, and state I/O.
//
// Setup (lp_create) builds the library's device layout on the host:
//   * a CSC copy of A by a stable counting sort (rows ascending per column);
//   * row and column permutations sorting rows of A and rows of A^T by
//     length, longest first (stable), so that each slice (one warp) holds
//     rows of nearly equal length, with 1-32 lanes per row by length;
//   * both operators relabeled into the permuted index spaces, so every
//     vector (x, xhat, xbar, x0, c, l, u and y, ybar, y0, b, row sense) is
//     stored permuted and accessed with unit stride; only the gathered
//     operand of each SpMV is indexed.
// The solve (lp_solve / lp_iterate) replays one captured CUDA graph per
// block of K iterations + check; lp_solve keeps two blocks in flight and
// reads a 4-byte status per check.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lp.h"
#include "lp_internal.h"
#include "lp_host.h"

using namespace lpg;


namespace {

double now_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

struct lp_problem {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  lp_options opt{};
  int device = 0;
  int nsm = 0;
  std::vector<void *> allocs;
  SellMat A{}, AT{};
  DevVecs v{};
  MixVecs mv{};
  bool mixed = false;
  // unrolled-forward recording for lp_backward
  double *ckpt = nullptr;              // [blocks][2n + 2m]: x, y, xbar, ybar at block start
  std::vector<int64_t> ckpt_t0;        // inner iteration count at each block start
  std::vector<int8_t> ckpt_restart;    // restart decision of each block's check
  int64_t rec_blocks = 0;
  AdjVecs adj{};
  uint8_t *mask_x = nullptr, *mask_y = nullptr;  // [K][n], [K][m]
  DevState *st = nullptr;
  double *w = nullptr;
  CheckScratch cs{};
  double *trace = nullptr;
  int32_t *perm_x = nullptr, *perm_y = nullptr;
  double *tmp = nullptr;
  int64_t nnz_padded = 0;
  double eta = 0, sigma_max = NAN;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t *h_status = nullptr;  // pinned [2]
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool solved = false;
  cudaStream_t last_stream = nullptr;  // stream of the latest call that enqueued work
  bool stream_used = false;
  void use_stream(cudaStream_t s) {
    last_stream = s;
    stream_used = true;
  }
  int nsearch = 1;
  int grid_cap = 0;  // blocks of the per-slice iteration kernels (0: one warp per slice)
  double setup_ms[4] = {0, 0, 0, 0};  // lp_create phases (lp_info.setup_ms)
  int32_t sigma_steps = 0;            // Lanczos / power-iteration steps taken for sigma_max
  int32_t graph_kernels = 0;          // kernel nodes of the K-iteration graph

  ~lp_problem() {
    if (ckpt) cudaFree(ckpt);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (h_status) cudaFreeHost(h_status);
    for (void *p : allocs) cudaFree(p);
  }

  template <class T>
  lp_status alloc(T **p, int64_t count) {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(16, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
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
        for (int64_t i = lo; i < hi; ++i) hf[i] = (float)H.val[i];
      });
      if ((s = upload(&vf, hf)) != LP_OK) return s;
    }
    M.valf = vf;
    M.nrows = H.nrows;
    M.ncols = H.ncols;
    M.nslices = H.nslices;
    M.n_warp_rows = H.n_warp_rows;
    M.info = info;
    M.idx = ix;
    M.val = vv;
    SplitSlice *split = nullptr;
    if (!H.split.empty() && (s = upload(&split, H.split)) != LP_OK) return s;
    return attach_split(M, split, (int64_t)H.split.size());
  }

  // Chunk-slice table of split rows, their partial sums and arrival counters
  // (zero between passes).
  lp_status attach_split(SellMat &M, const SplitSlice *split, int64_t nsplit) {
    M.nsplit = (int32_t)nsplit;
    M.split = split;
    M.split_part = nullptr;
    M.split_cnt = nullptr;
    if (nsplit == 0) return LP_OK;
    lp_status s;
    if ((s = alloc(&M.split_part, 2 * nsplit)) != LP_OK) return s;
    if ((s = alloc(&M.split_cnt, nsplit)) != LP_OK) return s;
    LP_CU(cudaMemset(M.split_cnt, 0, sizeof(int32_t) * (size_t)nsplit));
    return LP_OK;
  }
};

namespace {

// Resets Algorithm 1's counters on the device (status running).
lp_status reset_state(lp_problem *h, cudaStream_t s) {
  DevState hs{};
  LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  hs.t0 = 0;
  hs.iters = 0;
  hs.checks = 0;
  hs.restarts = 0;
  hs.status = kRunning;
  hs.returned = 0;
  hs.restart_now = 0;
  hs.use_cur = 0;
  hs.rho_stored = NAN;
  hs.last_rho = NAN;
  hs.last_r = NAN;
  for (int i = 0; i < 5; ++i) hs.kkt_a[i] = hs.kkt_c[i] = NAN;
  hs.kkt_a[4] = hs.kkt_c[4] = INFINITY;
  hs.ls[0].done = hs.ls[1].done = 1;
  hs.trace_count = 0;
  hs.given_radius = 0;
  hs.mix_s = 1.0;
  LP_CU(cudaMemcpyAsync(h->st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, s));
  LP_CU(cudaStreamSynchronize(s));
  launch_weights(h->st, h->w, s);
  if (h->mixed) {  // correction data at the starting point, dz = 0
    launch_residuals(h->A, h->AT, h->v, h->mv, h->n, h->m, s);
    launch_recenter(h->v, h->mv, h->st, h->n, h->m, 1, s);
  }
  LP_CU(cudaGetLastError());
  return LP_OK;
}

void launch_iteration(lp_problem *h, int k, cudaStream_t s) {
  if (h->mixed) {
    launch_primal_mix(h->AT, h->mv, h->st, h->w, k, h->opt.spmv_unroll, s);
    launch_dual_mix(h->A, h->mv, h->v, h->st, h->w, k, h->opt.spmv_unroll_rows, s);
  } else {
    launch_primal_step(h->AT, h->v, h->st, h->w, k, h->opt.spmv_unroll, h->grid_cap, s);
    launch_dual_step(h->A, h->v, h->st, h->w, k, h->opt.spmv_unroll_rows, h->grid_cap, s);
  }
}

lp_status build_graph(lp_problem *h) {
  if (h->exec) return LP_OK;
  cudaStream_t s = h->cap_stream;
  LP_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < h->opt.check_every; ++k) launch_iteration(h, k, s);
  launch_check(h->A, h->AT, h->v, h->st, h->w, h->cs, h->n, h->m, h->nsearch, h->trace, true, s,
               h->mixed ? &h->mv : nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  h->graph = g;
  LP_CU(cudaGraphInstantiate(&h->exec, g, 0));
  // kernel launches per replay (lp_info.graph_kernels)
  size_t count = 0;
  LP_CU(cudaGraphGetNodes(g, nullptr, &count));
  std::vector<cudaGraphNode_t> nodes(count);
  if (count > 0) LP_CU(cudaGraphGetNodes(g, nodes.data(), &count));
  int32_t kernels = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    LP_CU(cudaGraphNodeGetType(nd, &t));
    kernels += (t == cudaGraphNodeTypeKernel);
  }
  h->graph_kernels = kernels;
  return LP_OK;
}

lp_status set_run_params(lp_problem *h, double tol, cudaStream_t s) {
  // status <- running, tol <- tol (two small host-to-device copies)
  const int32_t running = kRunning;
  LP_CU(cudaMemcpyAsync(&h->st->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
  LP_CU(cudaMemcpyAsync(&h->st->status, &running, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  return LP_OK;
}

// Kernel-variant tuner (lp_options.autotune): on this problem, times every
// unroll variant of the column pass, then of the row pass (three rounds, each
// a warm-up and three timed launches per variant, CUDA events on the stream)
// and keeps the fastest.  Every variant sums each row in the same order, so the choice
// changes speed, not results.  The launches advance the iterate: the caller
// resets the state afterwards.
lp_status tune_variants(lp_problem *h, cudaStream_t s) {
  constexpr int kCands = 4, kRounds = 3, kReps = 3;
  const int cands[kCands] = {-2, -4, 2, 4};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LP_CU(cudaEventCreate(&e0));
  LP_CU(cudaEventCreate(&e1));
  lp_status st = LP_OK;
  // Rounds visit the candidates in rotated order (no candidate always runs
  // first after the previous pass); each candidate keeps its best time.
  for (int pass = 0; pass < 2 && st == LP_OK; ++pass) {
    int32_t &u = pass ? h->opt.spmv_unroll_rows : h->opt.spmv_unroll;
    float best[kCands];
    for (float &b : best) b = 1e30f;
    for (int round = 0; round < kRounds && st == LP_OK; ++round) {
      for (int i = 0; i < kCands; ++i) {
        const int ci = (i + round) % kCands;
        u = cands[ci];
        for (int r = 0; r <= kReps; ++r) {
          if (r == 1) cudaEventRecord(e0, s);
          if (h->mixed) {
            if (pass == 0) launch_primal_mix(h->AT, h->mv, h->st, h->w, 0, u, s);
            else launch_dual_mix(h->A, h->mv, h->v, h->st, h->w, 0, u, s);
          } else if (pass == 0) {
            launch_primal_step(h->AT, h->v, h->st, h->w, 0, u, h->grid_cap, s);
          } else {
            launch_dual_step(h->A, h->v, h->st, h->w, 0, u, h->grid_cap, s);
          }
        }
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        cudaError_t err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) {
          st = cuda_fail(err, "variant tuning");
          break;
        }
        best[ci] = std::min(best[ci], ms);
      }
    }
    int pick = 0;
    for (int ci = 1; ci < kCands; ++ci)
      if (best[ci] < best[pick]) pick = ci;
    u = cands[pick];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// Layout built on the host cores (lp_host.h) from host-readable views of the
// inputs, then uploaded: the CSC copy, the length orders, both slice layouts,
// the permuted vectors and the orders themselves.
lp_status host_layout(lp_problem *h, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *val, const double *c, const double *b, const double *lb,
                      const double *ub, const int8_t *row_type, cudaStream_t s,
                      double *t_copied, double *t_layout) {
  const int32_t m = h->m, n = h->n;
  const int64_t nnz = h->nnz;
  const lp_options &opt = h->opt;
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
    std::atomic<int> bad{0};
    parallel_for(nnz, [&](int64_t lo, int64_t hi) {
      for (int64_t p = lo; p < hi; ++p)
        if (!std::isfinite(hv[p])) bad.store(1, std::memory_order_relaxed);
    });
    if (bad.load()) return fail(LP_ERR_INVALID_ARG, "non-finite matrix value");
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
  // CSC copy (also checks the column indices and finds repeated columns in a row)
  std::vector<int64_t> cp;
  uvec<int32_t> ri;
  uvec<double> cv;
  if (!build_csc(m, n, hrp32, hci, hv, cp, ri, cv)) return fail(LP_ERR_INVALID_ARG, "col_idx out of range");
  if (csc_has_duplicates(n, cp, ri)) return fail(LP_ERR_INVALID_ARG, "duplicate column in a row");

  *t_copied = now_seconds();

  // ---- permutations by length (stable counting sorts), SELL layouts
  std::vector<int64_t> rp((size_t)m + 1);
  for (int32_t i = 0; i <= m; ++i) rp[i] = hrp32[i];
  std::vector<int32_t> perm_y(m), perm_x(n), inv_y(m), inv_x(n);
  sort_by_length_desc(rp.data(), 0, m, perm_y.data());
  sort_by_length_desc(cp.data(), 0, n, perm_x.data());
  for (int32_t r = 0; r < m; ++r) inv_y[perm_y[r]] = r;
  parallel_for(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) inv_x[perm_x[r]] = (int32_t)r;
  });
  HostSell HA, HAT;
  const LanePolicy policy{opt.long_row_threshold, opt.lane_steps, opt.single_lane_max};
  const int64_t target = (int64_t)opt.lane_auto * h->nsm;
  const LanePolicy pa = choose_policy(rp, perm_y, policy, target);
  const LanePolicy pat = choose_policy(cp, perm_x, policy, target);
  const int32_t split_len = opt.split_row_len;
  build_sell(m, n, rp, hci, hv, perm_y, inv_x, pa, HA, {}, split_len);
  build_sell(n, m, cp, ri.data(), cv.data(), perm_x, inv_y, pat, HAT, {}, split_len);
  h->nnz_padded = (int64_t)HA.idx.size();

  // permuted vectors
  std::vector<double> pc(n), pl(n), pu(n), pb(m);
  std::vector<int8_t> prt(m);
  for (int32_t r = 0; r < n; ++r) {
    pc[r] = hc[perm_x[r]];
    pl[r] = hl[perm_x[r]];
    pu[r] = hu[perm_x[r]];
  }
  for (int32_t r = 0; r < m; ++r) {
    pb[r] = hb[perm_y[r]];
    prt[r] = hrt[perm_y[r]];
  }

  *t_layout = now_seconds();

  // ---- device buffers
  lp_status e;
  if ((e = h->upload_sell(HA, h->A, h->mixed)) != LP_OK) return e;
  if ((e = h->upload_sell(HAT, h->AT, h->mixed)) != LP_OK) return e;
  if ((e = h->upload(&h->v.c, pc)) != LP_OK) return e;
  if ((e = h->upload(&h->v.lb, pl)) != LP_OK) return e;
  if ((e = h->upload(&h->v.ub, pu)) != LP_OK) return e;
  {
    // order keys of the bounds: the bit pattern, with all bits but the sign
    // flipped for negative values (monotone as signed 64-bit integers)
    std::vector<long long> lk(n), uk(n);
    for (int32_t r = 0; r < n; ++r) {
      long long bl, bu;
      std::memcpy(&bl, &pl[r], 8);
      std::memcpy(&bu, &pu[r], 8);
      lk[r] = bl < 0 ? (bl ^ 0x7fffffffffffffffll) : bl;
      uk[r] = bu < 0 ? (bu ^ 0x7fffffffffffffffll) : bu;
    }
    if ((e = h->upload(&h->v.lbk, lk)) != LP_OK) return e;
    if ((e = h->upload(&h->v.ubk, uk)) != LP_OK) return e;
  }
  if ((e = h->upload(&h->v.b, pb)) != LP_OK) return e;
  if ((e = h->upload(&h->v.row_type, prt)) != LP_OK) return e;
  if ((e = h->upload(&h->perm_x, perm_x)) != LP_OK) return e;
  if ((e = h->upload(&h->perm_y, perm_y)) != LP_OK) return e;
  return LP_OK;
}

// Layout built on the GPU (lp_layout.cu): the same arrays as host_layout,
// from device copies of the inputs (host inputs are copied in; device inputs
// are read in place).  Scratch is freed on return.
lp_status device_layout(lp_problem *h, const int32_t *row_ptr, const int32_t *col_idx,
                        const double *val, const double *c, const double *b, const double *lb,
                        const double *ub, const int8_t *row_type, cudaStream_t s,
                        double *t_copied, double *t_layout) {
  const int32_t m = h->m, n = h->n;
  const int64_t nnz = h->nnz;
  const lp_options &opt = h->opt;
  const int nsm = h->nsm;
  std::vector<void *> scratch;
  struct Guard {
    std::vector<void *> &v;
    ~Guard() {
      for (void *p : v) cudaFree(p);
    }
  } guard{scratch};
  auto tmp = [&](auto **p, int64_t count) -> lp_status {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(16, sizeof(**p) * (size_t)std::max<int64_t>(count, 1));
    const cudaError_t err = cudaMalloc(&q, bytes);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMalloc (layout scratch)");
    scratch.push_back(q);
    *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    return LP_OK;
  };
  // device views of the inputs
  auto dview = [&](const auto *src, int64_t count, const auto **out) -> lp_status {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(src)>>;
    *out = src;
    if (count <= 0) return LP_OK;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, src) != cudaSuccess) {
      cudaGetLastError();
      return fail(LP_ERR_INVALID_ARG, "could not read an input array (bad pointer?)");
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return LP_OK;
    T *d = nullptr;
    lp_status e = tmp(&d, count);
    if (e != LP_OK) return e;
    LP_CU(cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
    *out = d;
    return LP_OK;
  };
  lp_status e;
  const int32_t *drp = nullptr, *dci = nullptr;
  const double *dv = nullptr, *dc = nullptr, *db = nullptr, *dl = nullptr, *du = nullptr;
  const int8_t *drt = nullptr;
  if ((e = dview(row_ptr, (int64_t)m + 1, &drp)) != LP_OK) return e;
  if ((e = dview(col_idx, nnz, &dci)) != LP_OK) return e;
  if ((e = dview(val, nnz, &dv)) != LP_OK) return e;
  if ((e = dview(c, n, &dc)) != LP_OK) return e;
  if ((e = dview(b, m, &db)) != LP_OK) return e;
  if ((e = dview(lb, n, &dl)) != LP_OK) return e;
  if ((e = dview(ub, n, &du)) != LP_OK) return e;
  if ((e = dview(row_type, m, &drt)) != LP_OK) return e;

  // validation (before anything indexes by row_ptr or col_idx)
  int64_t *small = nullptr;  // [0] flags (int32), [1] max row length, [2] max column length
  if ((e = tmp(&small, 4)) != LP_OK) return e;
  int32_t *flags = reinterpret_cast<int32_t *>(small);
  LP_CU(cudaMemsetAsync(small, 0, sizeof(int64_t) * 4, s));
  lay_validate(drp, m, nnz, dci, n, dv, dc, dl, du, db, drt, flags, nsm, s);
  LP_CU(cudaGetLastError());
  auto check_flags = [&](int32_t f) -> lp_status {
    if (f & kLayBadRowPtr)
      return fail(LP_ERR_INVALID_ARG, "row_ptr must start at 0, be nondecreasing and end at nnz");
    if (f & kLayBadVal) return fail(LP_ERR_INVALID_ARG, "non-finite matrix value");
    if (f & kLayBadC) return fail(LP_ERR_INVALID_ARG, "non-finite objective c");
    if (f & kLayBadBounds)
      return fail(LP_ERR_INVALID_ARG, "invalid bounds (need lb <= ub, lb < inf, ub > -inf)");
    if (f & kLayBadB) return fail(LP_ERR_INVALID_ARG, "non-finite right-hand side b");
    if (f & kLayBadRowType) return fail(LP_ERR_INVALID_ARG, "row_type must be 0, 1 or 2");
    if (f & kLayBadColIdx) return fail(LP_ERR_INVALID_ARG, "col_idx out of range");
    if (f & kLayDuplicate) return fail(LP_ERR_INVALID_ARG, "duplicate column in a row");
    return LP_OK;
  };
  int64_t hsmall[4] = {0, 0, 0, 0};
  LP_CU(cudaMemcpyAsync(hsmall, small, sizeof(hsmall), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  if ((e = check_flags((int32_t)hsmall[0])) != LP_OK) return e;
  *t_copied = now_seconds();

  // radix-sort scratch for the largest sort (nnz, m or n elements)
  const int64_t most = std::max<int64_t>(std::max<int64_t>(nnz, m), n);
  const int64_t ntiles = lay_radix_tiles(most);
  int64_t *gh = nullptr, *goff = nullptr, *sums = nullptr;
  const int64_t scan_len = std::max<int64_t>(256 * ntiles, most + 1);
  if ((e = tmp(&gh, 256 * ntiles)) != LP_OK) return e;
  if ((e = tmp(&goff, 256 * ntiles)) != LP_OK) return e;
  if ((e = tmp(&sums, lay_scan_scratch(scan_len))) != LP_OK) return e;
  uint32_t *k0 = nullptr, *k1 = nullptr;
  int32_t *p0 = nullptr, *p1 = nullptr;
  if ((e = tmp(&k0, most)) != LP_OK) return e;
  if ((e = tmp(&k1, most)) != LP_OK) return e;
  if ((e = tmp(&p0, most)) != LP_OK) return e;
  if ((e = tmp(&p1, most)) != LP_OK) return e;
  auto bitlen = [](uint64_t v) {
    int b = 0;
    while (v) {
      ++b;
      v >>= 1;
    }
    return b;
  };

  // CSC: stable sort of the CSR positions by column
  int32_t *row_of = nullptr, *ri = nullptr;
  double *cv = nullptr;
  int64_t *cnt = nullptr, *cp = nullptr;
  if ((e = tmp(&row_of, nnz)) != LP_OK) return e;
  if ((e = tmp(&ri, nnz)) != LP_OK) return e;
  if ((e = tmp(&cv, nnz)) != LP_OK) return e;
  if ((e = tmp(&cnt, (int64_t)n + 1)) != LP_OK) return e;
  if ((e = tmp(&cp, (int64_t)n + 1)) != LP_OK) return e;
  lay_row_of(drp, m, nnz, row_of, nsm, s);
  if (nnz > 0) LP_CU(cudaMemcpyAsync(k0, dci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
  lay_iota(p0, nnz, nsm, s);
  bool alt = false;
  lay_radix_sort(k0, p0, k1, p1, nnz, bitlen((uint64_t)(n - 1)), gh, goff, sums, s, &alt);
  const uint32_t *col_sorted = alt ? k1 : k0;
  const int32_t *pos_sorted = alt ? p1 : p0;
  LP_CU(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * ((size_t)n + 1), s));
  lay_col_count(dci, nnz, cnt, nsm, s);
  lay_exclusive_scan(cnt, (int64_t)n + 1, cp, sums, s);
  lay_csc_gather(pos_sorted, row_of, dv, nnz, ri, cv, nsm, s);
  lay_dup(col_sorted, ri, nnz, flags, nsm, s);
  // lengths: maxima first
  lay_lengths<int32_t>(drp, m, &small[1], nullptr, 0, nullptr, nsm, s);
  lay_lengths<int64_t>(cp, n, &small[2], nullptr, 0, nullptr, nsm, s);
  LP_CU(cudaGetLastError());
  LP_CU(cudaMemcpyAsync(hsmall, small, sizeof(hsmall), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  if ((e = check_flags((int32_t)hsmall[0])) != LP_OK) return e;
  const int64_t mx_r = hsmall[1], mx_c = hsmall[2];

  // orders by decreasing length (stable), their inverses, length histograms
  int32_t *perm_y = nullptr, *perm_x = nullptr, *inv_y = nullptr, *inv_x = nullptr;
  int64_t *hist_r = nullptr, *hist_c = nullptr;
  if ((e = h->alloc(&perm_y, m)) != LP_OK) return e;
  if ((e = h->alloc(&perm_x, n)) != LP_OK) return e;
  if ((e = tmp(&inv_y, m)) != LP_OK) return e;
  if ((e = tmp(&inv_x, n)) != LP_OK) return e;
  if ((e = tmp(&hist_r, mx_r + 1)) != LP_OK) return e;
  if ((e = tmp(&hist_c, mx_c + 1)) != LP_OK) return e;
  auto order = [&](auto *ptr, int32_t count, int64_t mx, int64_t *hist, int32_t *perm) -> lp_status {
    LP_CU(cudaMemsetAsync(hist, 0, sizeof(int64_t) * ((size_t)mx + 1), s));
    if (count == 0) return LP_OK;
    lay_lengths(ptr, count, nullptr, k0, mx, hist, nsm, s);
    lay_iota(p0, count, nsm, s);
    bool a = false;
    lay_radix_sort(k0, p0, k1, p1, count, bitlen((uint64_t)mx), gh, goff, sums, s, &a);
    LP_CU(cudaMemcpyAsync(perm, a ? p1 : p0, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, s));
    return LP_OK;
  };
  if ((e = order(drp, m, mx_r, hist_r, perm_y)) != LP_OK) return e;
  if ((e = order(cp, n, mx_c, hist_c, perm_x)) != LP_OK) return e;
  lay_inverse(perm_y, m, inv_y, nsm, s);
  lay_inverse(perm_x, n, inv_x, nsm, s);
  std::vector<int64_t> hr((size_t)mx_r + 1), hc((size_t)mx_c + 1);
  LP_CU(cudaMemcpyAsync(hr.data(), hist_r, sizeof(int64_t) * hr.size(), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaMemcpyAsync(hc.data(), hist_c, sizeof(int64_t) * hc.size(), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));

  // lane policy (the host layout's choose_policy, from the length histogram)
  // and the runs of equal lane count in the sorted order
  // (the lane count is nondecreasing in the length, so each of the at most 6
  // lane counts forms one run; false if that ever failed)
  auto runs_of = [](const std::vector<int64_t> &hist, const LanePolicy &p, LayRuns *runs,
                    int64_t *nslices, int64_t *warp_rows) {
    LayRuns R{};
    int64_t g = 0, ns = 0, wr = 0;
    for (int64_t len = (int64_t)hist.size() - 1; len >= 0; --len) {
      if (hist[(size_t)len] == 0) continue;
      const int lg = lanes_log2(len, p);
      if (R.count == 0 || R.lg[R.count - 1] != lg) {
        if (R.count == 6) return false;
        R.lg[R.count] = lg;
        R.g0[R.count] = g;
        R.s0[R.count] = 0;
        ++R.count;
      }
      g += hist[(size_t)len];
      if (lg == 5) wr += hist[(size_t)len];
    }
    for (int q = 0; q < R.count; ++q) {  // slices: ceil(rows / (32 >> lg)) per run
      const int64_t rows = (q + 1 < R.count ? R.g0[q + 1] : g) - R.g0[q];
      R.s0[q] = ns;
      ns += (rows + (kWarp >> R.lg[q]) - 1) / (kWarp >> R.lg[q]);
    }
    if (runs) *runs = R;
    *nslices = ns;
    if (warp_rows) *warp_rows = wr;
    return true;
  };
  auto choose = [&](const std::vector<int64_t> &hist, LanePolicy p) {
    const int64_t target = (int64_t)opt.lane_auto * nsm;
    if (target <= 0) return p;
    int64_t ns = 0;
    for (;;) {
      if (!runs_of(hist, p, nullptr, &ns, nullptr)) break;
      if (ns >= target || !(p.single_max > 1 || p.lane_steps > 1)) break;
      p.single_max = p.single_max / 2;
      p.lane_steps = std::max(1, p.lane_steps / 2);
    }
    return p;
  };
  const LanePolicy policy{opt.long_row_threshold, opt.lane_steps, opt.single_lane_max};
  const int32_t split_len = opt.split_row_len;

  // slices and fill of one operator
  auto make = [&](auto *ptr, int32_t nrows, int32_t ncols, const std::vector<int64_t> &hist,
                  const int32_t *perm, const int32_t *ind, const double *vals,
                  const int32_t *relabel, SellMat &M) -> lp_status {
    const LanePolicy pol = choose(hist, policy);
    // split rows: whole-warp rows longer than split_len, the longest rows, so
    // the first nsr of the sorted order; the ordinary runs follow them
    std::vector<int64_t> rest = hist;
    int64_t nsr = 0, nsplit = 0;
    if (split_len > 0)
      for (int64_t len = (int64_t)hist.size() - 1; len > split_len; --len)
        if (hist[(size_t)len] > 0 && lanes_log2(len, pol) == 5) {
          nsr += hist[(size_t)len];
          nsplit += hist[(size_t)len] * ((len + split_len - 1) / split_len);
          rest[(size_t)len] = 0;
        }
    LayRuns runs{};
    int64_t ns = 0, wr = 0;
    if (!runs_of(rest, pol, &runs, &ns, &wr))
      return fail(LP_ERR_INVALID_ARG, "lane policy gives more than 6 runs");
    for (int q = 0; q < runs.count; ++q) {
      runs.g0[q] += nsr;
      runs.s0[q] += nsplit;
    }
    ns += nsplit;
    wr += nsr;
    SliceInfo *info = nullptr;
    SplitSlice *split = nullptr;
    int64_t *width = nullptr, *off = nullptr, *nch = nullptr, *cstart = nullptr;
    if ((e = h->alloc(&info, ns + 1)) != LP_OK) return e;
    if ((e = h->alloc(&split, nsplit)) != LP_OK) return e;
    if ((e = tmp(&width, ns)) != LP_OK) return e;
    if ((e = tmp(&off, ns)) != LP_OK) return e;
    if ((e = tmp(&nch, nsr)) != LP_OK) return e;
    if ((e = tmp(&cstart, nsr)) != LP_OK) return e;
    lay_slices(runs, perm, ptr, ns, nrows, info, width, off, sums, nsm, s, nsr, nsplit, split_len,
               split, nch, cstart);
    SliceInfo last{};
    LP_CU(cudaMemcpyAsync(&last, info + ns, sizeof(SliceInfo), cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    int32_t *ix = nullptr;
    double *vv = nullptr;
    float *vf = nullptr;
    if ((e = h->alloc(&ix, last.off)) != LP_OK) return e;
    if ((e = h->alloc(&vv, last.off)) != LP_OK) return e;
    if (h->mixed && (e = h->alloc(&vf, last.off)) != LP_OK) return e;
    lay_fill(info, ns, perm, ptr, ind, vals, relabel, ix, vv, vf, nsm, s, split, nsplit,
             split_len);
    LP_CU(cudaGetLastError());
    M.nrows = nrows;
    M.ncols = ncols;
    M.nslices = (int32_t)ns;
    M.n_warp_rows = (int32_t)wr;
    M.info = info;
    M.idx = ix;
    M.val = vv;
    M.valf = vf;
    return h->attach_split(M, split, nsplit);
  };
  if ((e = make(drp, m, n, hr, perm_y, dci, dv, inv_x, h->A)) != LP_OK) return e;
  if ((e = make(cp, n, m, hc, perm_x, ri, cv, inv_y, h->AT)) != LP_OK) return e;
  {
    SliceInfo last{};
    LP_CU(cudaMemcpyAsync(&last, h->A.info + h->A.nslices, sizeof(SliceInfo),
                          cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    h->nnz_padded = last.off;
  }
  *t_layout = now_seconds();

  // permuted vectors and the orders
  if ((e = h->alloc(&h->v.c, n)) != LP_OK) return e;
  if ((e = h->alloc(&h->v.lb, n)) != LP_OK) return e;
  if ((e = h->alloc(&h->v.ub, n)) != LP_OK) return e;
  if ((e = h->alloc(&h->v.lbk, n)) != LP_OK) return e;
  if ((e = h->alloc(&h->v.ubk, n)) != LP_OK) return e;
  if ((e = h->alloc(&h->v.b, m)) != LP_OK) return e;
  if ((e = h->alloc(&h->v.row_type, m)) != LP_OK) return e;
  lay_vectors(perm_x, n, dc, dl, du, h->v.c, h->v.lb, h->v.ub, h->v.lbk, h->v.ubk, perm_y, m, db,
              drt, h->v.b, h->v.row_type, nsm, s);
  LP_CU(cudaGetLastError());
  h->perm_x = perm_x;
  h->perm_y = perm_y;
  LP_CU(cudaStreamSynchronize(s));  // scratch is freed on return
  return LP_OK;
}
}  // namespace

extern "C" {

void lp_default_options(lp_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->beta = std::exp(-1.0);
  o->check_every = 64;
  o->restart_scheme = LP_RESTART_ADAPTIVE;
  o->tau0 = 0;
  o->fixed_len = 0;
  o->omega = 1.0;
  o->eta = 0.0;
  o->power_iters = 5000;
  o->power_tol = 1e-10;
  o->max_iter = 10000000;
  o->long_row_threshold = 512;
  o->trace_capacity = 65536;
  o->spmv_unroll = -2;
  o->spmv_unroll_rows = -4;
  o->lane_steps = 16;
  o->single_lane_max = 64;
  o->spmv_mode = 0;
  o->lane_auto = 32;
  o->autotune = 1;
  o->sigma_method = LP_SIGMA_LANCZOS;
  o->device_layout = 1;
  o->split_row_len = 512;
}

const char *lp_last_error(void) { return err_msg().c_str(); }

lp_status lp_create(int32_t m, int32_t n, int64_t nnz, const int32_t *row_ptr,
                    const int32_t *col_idx, const double *val, const double *c, const double *b,
                    const double *lb, const double *ub, const int8_t *row_type,
                    const lp_options *opt_in, void *cuda_stream, lp_handle *out) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_create");
  if (!out) return fail(LP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (m < 0 || n < 1) return fail(LP_ERR_INVALID_ARG, "need m >= 0 and n >= 1");
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return fail(LP_ERR_INVALID_ARG, "nnz must lie in [0, 2^31)");
  if (!row_ptr || !c || !lb || !ub || (m > 0 && (!b || !row_type)) ||
      (nnz > 0 && (!col_idx || !val)))
    return fail(LP_ERR_INVALID_ARG, "NULL array argument");
  lp_options opt;
  if (opt_in) opt = *opt_in;
  else lp_default_options(&opt);
  lp_status st = validate_options(opt);
  if (st != LP_OK) return st;
  if (opt.tau0 == 0) opt.tau0 = opt.check_every;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const double t_start = now_seconds();

  std::unique_ptr<lp_problem> h(new lp_problem());
  h->m = m;
  h->n = n;
  h->nnz = nnz;
  h->opt = opt;
  LP_CU(cudaGetDevice(&h->device));
  LP_CU(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
  h->nsearch = (opt.restart_scheme == LP_RESTART_ADAPTIVE) ? 1
               : (opt.restart_scheme == LP_RESTART_FLEXIBLE) ? 2 : 0;
  h->mixed = (opt.precision == LP_PRECISION_MIXED);
  double t_copied = t_start, t_layout = t_start;
  lp_status e = opt.device_layout
                    ? device_layout(h.get(), row_ptr, col_idx, val, c, b, lb, ub, row_type, s,
                                    &t_copied, &t_layout)
                    : host_layout(h.get(), row_ptr, col_idx, val, c, b, lb, ub, row_type, s,
                                  &t_copied, &t_layout);
  if (e != LP_OK) return e;
  double **xs[] = {&h->v.x, &h->v.xhat, &h->v.xbar, &h->v.x0};
  for (double **p : xs)
    if ((e = h->alloc(p, n)) != LP_OK) return e;
  double **ys[] = {&h->v.y, &h->v.ybar, &h->v.y0};
  for (double **p : ys)
    if ((e = h->alloc(p, m)) != LP_OK) return e;
  if ((e = h->alloc(&h->tmp, std::max(n, m))) != LP_OK) return e;
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
  if ((e = h->alloc(&h->st, 1)) != LP_OK) return e;
  if ((e = h->alloc(&h->w, opt.check_every)) != LP_OK) return e;
  if ((e = h->alloc(&h->trace, (int64_t)6 * std::max(1, opt.trace_capacity))) != LP_OK) return e;

  // check scratch
  CheckScratch &cs = h->cs;
  cs.cols_grid = check_grid_for(h->AT, h->nsm);
  cs.rows_grid = check_grid_for(h->A, h->nsm);
  // one slot per block of the check passes, then one per chunk slice of split rows
  cs.pstride = std::max(cs.cols_grid + cs.rows_grid + split_grid(h->A) + split_grid(h->AT) +
                            h->A.nsplit + h->AT.nsplit,
                        8 * h->nsm);
  if ((e = h->alloc(&cs.partials, (int64_t)NQ * cs.pstride)) != LP_OK) return e;
  const int64_t N = (int64_t)n + m;
  for (int k = 0; k < 2; ++k) {
    if (k == 1 && h->nsearch < 2) {
      cs.keys[1] = cs.keys[0];
      cs.d2[1] = cs.d2[0];
      cs.g2[1] = cs.g2[0];
      cs.gd[1] = cs.gd[0];
      break;
    }
    if ((e = h->alloc(&cs.keys[k], N)) != LP_OK) return e;
    if ((e = h->alloc(&cs.d2[k], N)) != LP_OK) return e;
    if ((e = h->alloc(&cs.g2[k], N)) != LP_OK) return e;
    if ((e = h->alloc(&cs.gd[k], N)) != LP_OK) return e;
  }
  cs.hist_grid = (int)std::min<int64_t>(std::max<int64_t>(1, (N + 2047) / 2048), 4 * h->nsm);
  if ((e = h->alloc(&cs.hpart, (int64_t)2 * cs.hist_grid * 4 * kBuckets)) != LP_OK) return e;
  {
    // a histogram warp scans at most kWarp * ceil(N / stride) elements
    const int64_t nw = (int64_t)cs.hist_grid * kHistWarps, stride = nw * kWarp;
    cs.cand_cap = (int64_t)kWarp * ((N + stride - 1) / stride);
    for (int k = 0; k < 2; ++k) {
      if (k == 1 && h->nsearch < 2) {
        cs.cand[1] = cs.cand[0];
        cs.ccnt[1] = cs.ccnt[0];
        break;
      }
      if ((e = h->alloc(&cs.cand[k], nw * cs.cand_cap)) != LP_OK) return e;
      if ((e = h->alloc(&cs.ccnt[k], nw)) != LP_OK) return e;
    }
  }
  if ((e = h->alloc(&cs.btot, (int64_t)2 * 4 * kBuckets)) != LP_OK) return e;
  if ((e = h->alloc(&cs.pair_x, (int64_t)2 * n)) != LP_OK) return e;
  if ((e = h->alloc(&cs.pair_y, (int64_t)2 * m)) != LP_OK) return e;
  LP_CU(cudaMallocHost(&h->h_status, 2 * sizeof(int32_t)));
  LP_CU(cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming));
  LP_CU(cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming));
  LP_CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));

  LP_CU(cudaStreamSynchronize(s));
  const double t_uploaded = now_seconds();

  // ---- device state: step sizes, norms, sigma_max estimate
  DevState hs{};
  hs.omega = opt.omega;
  hs.beta = opt.beta;
  hs.tol = 1e-8;
  hs.K = opt.check_every;
  hs.scheme = opt.restart_scheme;
  hs.tau0 = opt.tau0;
  hs.fixed_len = opt.fixed_len;
  hs.status = kRunning;
  hs.trace_cap = opt.trace_capacity;
  hs.pw_tol = opt.power_tol;
  hs.pw_max = opt.power_iters;
  hs.mixed = h->mixed ? 1 : 0;
  hs.mix_s = 1.0;
  LP_CU(cudaMemcpy(h->st, &hs, sizeof(DevState), cudaMemcpyHostToDevice));
  const int rgrid = std::min(std::max(1, (int)((std::max(n, m) + kBlock - 1) / kBlock)), 8 * h->nsm);
  launch_norms(h->v, h->st, cs.partials, cs.pstride, rgrid, n, m, s);
  LP_CU(cudaGetLastError());
  if (opt.eta > 0.0) {
    h->eta = opt.eta;
  } else {
    // Section 7: eta = 0.9 / sigma_max(A); sigma_max^2 is the largest eigenvalue of
    // A^T A, estimated by Lanczos (default) or Section 7's power iteration
    double *pv = h->v.x, *pav = h->v.y, *pw = h->v.xhat;
    // start vector v_j = 0.5 + u_j (u_j in [0,1) from SplitMix64 at counter j, the
    // original column index), normalized; the all-ones vector can be orthogonal
    // to the top singular vector (symmetric network matrices)
    launch_start_vector(h->perm_x, pv, n, cs.partials, cs.pstride, rgrid, s);
    LP_CU(cudaGetLastError());
    if (opt.sigma_method == LP_SIGMA_LANCZOS) {
      // three rotating n-vectors: v_{k-1}, v_k and w (which becomes v_{k+1})
      LanczosT T{nullptr, nullptr, std::min<int32_t>(opt.power_iters, kLanczosMax)};
      double *coef = nullptr;
      if (cudaMalloc(&coef, sizeof(double) * 2 * T.cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(LP_ERR_OOM, "cudaMalloc of the Lanczos coefficients failed");
      }
      struct Free {
        double *p;
        ~Free() { cudaFree(p); }
      } free_coef{coef};
      T.alpha = coef;
      T.beta = coef + T.cap;
      double *P[3] = {pv, pw, h->v.xbar};
      for (int k = 0; k < T.cap; ++k) {
        launch_lanczos_step(h->A, h->AT, P[k % 3], pav, P[(k + 1) % 3], P[(k + 2) % 3], h->st, T,
                            k, (k + 1) % 4 == 0, cs.partials, cs.pstride, rgrid, n, s);
        if ((k + 1) % 16 != 0 && k + 1 != T.cap) continue;
        LP_CU(cudaGetLastError());
        int32_t done = 0;
        LP_CU(cudaMemcpyAsync(&done, &h->st->pw_done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LP_CU(cudaStreamSynchronize(s));
        if (done) break;
      }
      LP_CU(cudaStreamSynchronize(s));
    } else {
      const int chunk = 25;
      for (int it = 0; it < opt.power_iters; it += chunk) {
        for (int k = 0; k < chunk; ++k)
          launch_power_iteration_step(h->A, h->AT, pv, pav, pw, h->st, cs.partials, cs.pstride,
                                      rgrid, n, m, s);
        LP_CU(cudaGetLastError());
        int32_t done = 0;
        LP_CU(cudaMemcpyAsync(&done, &h->st->pw_done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LP_CU(cudaStreamSynchronize(s));
        if (done) break;
      }
    }
    {
      int32_t steps = 0;
      LP_CU(cudaMemcpyAsync(&steps, &h->st->pw_iters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      LP_CU(cudaStreamSynchronize(s));
      h->sigma_steps = steps;
    }
    double est = 0.0;
    LP_CU(cudaMemcpyAsync(&est, &h->st->pw_est, sizeof(double), cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    h->sigma_max = std::sqrt(est);
    if (!(h->sigma_max > 0.0)) return fail(LP_ERR_NUMERICAL, "sigma_max(A) is zero or not finite; pass eta explicitly");
    h->eta = 0.9 / h->sigma_max;
  }
  const double t_power = now_seconds();
  h->setup_ms[0] = 1e3 * (t_copied - t_start);
  h->setup_ms[1] = 1e3 * (t_layout - t_copied);
  h->setup_ms[2] = 1e3 * (t_uploaded - t_layout);
  h->setup_ms[3] = 1e3 * (t_power - t_uploaded);
  const double tau = h->eta / opt.omega, sigma = h->eta * opt.omega;
  LP_CU(cudaMemcpyAsync(&h->st->tau, &tau, sizeof(double), cudaMemcpyHostToDevice, s));
  LP_CU(cudaMemcpyAsync(&h->st->sigma, &sigma, sizeof(double), cudaMemcpyHostToDevice, s));
  if (opt.autotune && (e = tune_variants(h.get(), s)) != LP_OK) return e;
  // z^{0,0} = proj(0)
  launch_fill(h->v.x, 0.0, n, s);
  launch_fill(h->v.y, 0.0, m, s);
  launch_project(h->v, n, m, s);
  LP_CU(cudaGetLastError());
  if ((e = reset_state(h.get(), s)) != LP_OK) return e;
  LP_CU(cudaStreamSynchronize(s));
  *out = h.release();
  return LP_OK;
}

lp_status lp_set_state(lp_handle h, const double *x, const double *y, void *cuda_stream) {
  err_msg().clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  if (x) {
    LP_CU(cudaMemcpyAsync(h->tmp, x, sizeof(double) * h->n, cudaMemcpyDefault, s));
    launch_gather(h->v.x, h->tmp, h->perm_x, h->n, s);
  } else {
    launch_fill(h->v.x, 0.0, h->n, s);
  }
  if (y) {
    LP_CU(cudaMemcpyAsync(h->tmp, y, sizeof(double) * h->m, cudaMemcpyDefault, s));
    launch_gather(h->v.y, h->tmp, h->perm_y, h->m, s);
  } else {
    launch_fill(h->v.y, 0.0, h->m, s);
  }
  launch_project(h->v, h->n, h->m, s);
  LP_CU(cudaGetLastError());
  h->solved = false;
  return reset_state(h, s);
}

lp_status lp_iterate(lp_handle h, int32_t n_checks, double tol, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_iterate");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!(tol > 0.0)) return fail(LP_ERR_INVALID_ARG, "tol must be > 0");
  if (n_checks < 0) return fail(LP_ERR_INVALID_ARG, "n_checks must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  lp_status e = build_graph(h);
  if (e != LP_OK) return e;
  if ((e = set_run_params(h, tol, s)) != LP_OK) return e;
  for (int32_t i = 0; i < n_checks; ++i) LP_CU(cudaGraphLaunch(h->exec, s));
  h->solved = true;
  return LP_OK;
}

lp_status lp_solve(lp_handle h, double tol, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_solve");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!(tol > 0.0)) return fail(LP_ERR_INVALID_ARG, "tol must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  lp_status e = build_graph(h);
  if (e != LP_OK) return e;
  if ((e = set_run_params(h, tol, s)) != LP_OK) return e;
  const int K = h->opt.check_every;
  int64_t remaining = h->opt.max_iter;
  int32_t status = kRunning;
  int inflight = 0, head = 0;  // ring of two (event, status slot)
  while (true) {
    while (inflight < 2 && remaining >= K) {
      const int slot = (head + inflight) & 1;
      LP_CU(cudaGraphLaunch(h->exec, s));
      LP_CU(cudaMemcpyAsync(&h->h_status[slot], &h->st->status, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
      LP_CU(cudaEventRecord(h->ev[slot], s));
      remaining -= K;
      ++inflight;
    }
    if (inflight == 0) break;
    LP_CU(cudaEventSynchronize(h->ev[head]));
    status = h->h_status[head];
    head ^= 1;
    --inflight;
    if (status != kRunning) break;
  }
  LP_CU(cudaStreamSynchronize(s));
  if (status == kRunning && remaining > 0) {
    const int r = (int)remaining;
    for (int k = 0; k < r; ++k) launch_iteration(h, k, s);
    launch_advance(h->st, h->w, r, s);
    LP_CU(cudaGetLastError());
  }
  LP_CU(cudaMemcpyAsync(&status, &h->st->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  h->solved = true;
  if (status == kRunning) return fail(LP_ITER_LIMIT, "iteration limit reached");
  if (status == LP_ERR_NUMERICAL) return fail(LP_ERR_NUMERICAL, "NaN or Inf in the iterates or residuals");
  return static_cast<lp_status>(status);
}

lp_status lp_get_solution(lp_handle h, double *x, double *y, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_get_solution");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "no solve has run on this handle");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  if (h->mixed) launch_combine(h->v, h->mv, h->st, h->n, h->m, 1, s);
  int32_t returned = 0;
  LP_CU(cudaMemcpyAsync(&returned, &h->st->returned, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  if (x) {
    launch_scatter(h->tmp, returned ? h->v.x : h->v.xbar, h->perm_x, h->n, s);
    LP_CU(cudaMemcpyAsync(x, h->tmp, sizeof(double) * h->n, cudaMemcpyDefault, s));
  }
  if (y) {
    LP_CU(cudaStreamSynchronize(s));
    launch_scatter(h->tmp, returned ? h->v.y : h->v.ybar, h->perm_y, h->m, s);
    LP_CU(cudaMemcpyAsync(y, h->tmp, sizeof(double) * h->m, cudaMemcpyDefault, s));
  }
  LP_CU(cudaGetLastError());
  LP_CU(cudaStreamSynchronize(s));
  return LP_OK;
}

lp_status lp_get_state(lp_handle h, double *x, double *y, double *xbar, double *ybar, double *x0,
                       double *y0, void *cuda_stream) {
  err_msg().clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  if (h->mixed) launch_combine(h->v, h->mv, h->st, h->n, h->m, 1, s);
  struct Item { double *dst; const double *src; const int32_t *perm; int32_t len; };
  const Item items[] = {{x, h->v.x, h->perm_x, h->n},       {y, h->v.y, h->perm_y, h->m},
                        {xbar, h->v.xbar, h->perm_x, h->n}, {ybar, h->v.ybar, h->perm_y, h->m},
                        {x0, h->v.x0, h->perm_x, h->n},     {y0, h->v.y0, h->perm_y, h->m}};
  for (const Item &it : items) {
    if (!it.dst) continue;
    launch_scatter(h->tmp, it.src, it.perm, it.len, s);
    LP_CU(cudaMemcpyAsync(it.dst, h->tmp, sizeof(double) * it.len, cudaMemcpyDefault, s));
    LP_CU(cudaStreamSynchronize(s));
  }
  LP_CU(cudaGetLastError());
  return LP_OK;
}

lp_status lp_get_info(lp_handle h, lp_info *info) {
  err_msg().clear();
  if (!h || !info) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  DevState hs{};
  LP_CU(cudaMemcpy(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  std::memset(info, 0, sizeof(*info));
  info->iters = hs.iters;
  info->restarts = hs.restarts;
  info->checks = hs.checks;
  info->status = (hs.status == kRunning) ? (h->solved ? LP_ITER_LIMIT : LP_ERR_NOT_SOLVED) : hs.status;
  info->returned = hs.returned;
  for (int i = 0; i < 5; ++i) {
    info->kkt_avg[i] = hs.kkt_a[i];
    info->kkt_cur[i] = hs.kkt_c[i];
  }
  info->eta = h->eta;
  info->sigma_max = h->sigma_max;
  info->omega = hs.omega;
  info->tau = hs.tau;
  info->sigma = hs.sigma;
  info->rho_stored = hs.rho_stored;
  info->last_rho = hs.last_rho;
  info->last_radius = hs.last_r;
  info->nnz_padded = h->nnz_padded;
  info->n_long_rows = h->A.n_warp_rows;
  info->n_long_cols = h->AT.n_warp_rows;
  info->spmv_unroll = h->opt.spmv_unroll;
  info->spmv_unroll_rows = h->opt.spmv_unroll_rows;
  for (int i = 0; i < 4; ++i) info->setup_ms[i] = h->setup_ms[i];
  info->sigma_steps = h->sigma_steps;
  info->graph_kernels = h->graph_kernels;
  info->n_split_slices = h->A.nsplit + h->AT.nsplit;
  return LP_OK;
}

lp_status lp_get_trace(lp_handle h, double *rows, int64_t capacity, int64_t *count) {
  err_msg().clear();
  if (!h || !count || (capacity > 0 && !rows)) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  int64_t tc = 0;
  LP_CU(cudaMemcpy(&tc, &h->st->trace_count, sizeof(int64_t), cudaMemcpyDeviceToHost));
  tc = std::min<int64_t>(tc, h->opt.trace_capacity);
  const int64_t k = std::min(tc, capacity);
  if (k > 0) LP_CU(cudaMemcpy(rows, h->trace, sizeof(double) * 6 * k, cudaMemcpyDeviceToHost));
  *count = k;
  return LP_OK;
}

lp_status lp_normalized_gap(lp_handle h, const double *x, const double *y, double r,
                            double *host_rho, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_normalized_gap");
  if (!h || !host_rho || !x || (h->m > 0 && !y)) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  if (!(r >= 0.0) || !std::isfinite(r)) return fail(LP_ERR_INVALID_ARG, "radius must be finite and >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  const int n = h->n, m = h->m;
  const int64_t N = (int64_t)n + m;
  // scratch owned by this call
  std::vector<void *> mine;
  struct Guard {
    std::vector<void *> &v;
    ~Guard() { for (void *p : v) cudaFree(p); }
  } guard{mine};
  auto get = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    mine.push_back(p);
    return p;
  };
  DevVecs v = h->v;
  double *xp = (double *)get(sizeof(double) * n), *yp = (double *)get(sizeof(double) * std::max(m, 1));
  DevState *st = (DevState *)get(sizeof(DevState));
  CheckScratch cs = h->cs;
  cs.partials = (double *)get(sizeof(double) * NQ * cs.pstride);
  cs.keys[0] = (uint64_t *)get(sizeof(uint64_t) * N);
  cs.d2[0] = (double *)get(sizeof(double) * N);
  cs.g2[0] = (double *)get(sizeof(double) * N);
  cs.gd[0] = (double *)get(sizeof(double) * N);
  cs.keys[1] = cs.keys[0];
  cs.d2[1] = cs.d2[0];
  cs.g2[1] = cs.g2[0];
  cs.gd[1] = cs.gd[0];
  cs.hpart = (double *)get(sizeof(double) * 2 * cs.hist_grid * 4 * kBuckets);
  cs.btot = (double *)get(sizeof(double) * 2 * 4 * kBuckets);
  double *tmpx = (double *)get(sizeof(double) * std::max(n, m));
  // split-row partial sums and arrival counters of this call (the handle's
  // belong to its solves); the counters start at zero
  SellMat A = h->A, AT = h->AT;
  bool split_ok = true;
  for (SellMat *M : {&A, &AT}) {
    if (M->nsplit == 0) continue;
    M->split_part = (double *)get(sizeof(double) * 2 * (size_t)M->nsplit);
    M->split_cnt = (int32_t *)get(sizeof(int32_t) * (size_t)M->nsplit);
    split_ok = split_ok && M->split_part && M->split_cnt;
  }
  if (!xp || !yp || !st || !cs.partials || !cs.keys[0] || !cs.d2[0] || !cs.g2[0] || !cs.gd[0] ||
      !cs.hpart || !cs.btot || !tmpx || !split_ok) {
    cudaGetLastError();
    return fail(LP_ERR_OOM, "cudaMalloc of gap scratch failed");
  }
  for (SellMat *M : {&A, &AT})
    if (M->nsplit > 0) LP_CU(cudaMemsetAsync(M->split_cnt, 0, sizeof(int32_t) * (size_t)M->nsplit, s));
  LP_CU(cudaMemcpyAsync(tmpx, x, sizeof(double) * n, cudaMemcpyDefault, s));
  launch_gather(xp, tmpx, h->perm_x, n, s);
  if (m > 0) {
    LP_CU(cudaMemcpyAsync(tmpx, y, sizeof(double) * m, cudaMemcpyDefault, s));
    launch_gather(yp, tmpx, h->perm_y, m, s);
  }
  v.x = v.xbar = v.x0 = xp;
  v.y = v.ybar = v.y0 = yp;
  DevState hs{};
  LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  hs.status = kRunning;
  hs.given_radius = 1;
  hs.r_given = r;
  LP_CU(cudaMemcpyAsync(st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, s));
  LP_CU(cudaStreamSynchronize(s));
  cs.pair_x = cs.pair_y = nullptr;  // the handle's pair buffers belong to its solve
  cs.cand[0] = cs.cand[1] = nullptr;  // and so do its candidate lists: full scans
  launch_check(A, AT, v, st, nullptr, cs, n, m, 1, nullptr, false, s);
  LP_CU(cudaGetLastError());
  LSearch L{};
  LP_CU(cudaMemcpyAsync(&L, &st->ls[0], sizeof(LSearch), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  *host_rho = (r == 0.0) ? 0.0 : L.rho_r / r;
  return LP_OK;
}

lp_status lp_select_omega(lp_handle h, const double *omegas, int32_t count, int64_t iters,
                          double *kkt_out, double *best_out, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_select_omega");
  if (!h || !omegas || !kkt_out || count < 1) return fail(LP_ERR_INVALID_ARG, "bad arguments");
  if (iters < h->opt.check_every) return fail(LP_ERR_INVALID_ARG, "iters must be >= check_every");
  for (int32_t k = 0; k < count; ++k)
    if (!(omegas[k] > 0.0) || !std::isfinite(omegas[k]))
      return fail(LP_ERR_INVALID_ARG, "every omega must be finite and > 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  lp_status e = build_graph(h);
  if (e != LP_OK) return e;
  const int32_t scheme = h->opt.restart_scheme;
  const int K = h->opt.check_every;
  auto set_weight = [&](double om, int32_t sch) -> lp_status {
    const double tau = h->eta / om, sigma = h->eta * om;
    LP_CU(cudaMemcpyAsync(&h->st->omega, &om, sizeof(double), cudaMemcpyHostToDevice, s));
    LP_CU(cudaMemcpyAsync(&h->st->tau, &tau, sizeof(double), cudaMemcpyHostToDevice, s));
    LP_CU(cudaMemcpyAsync(&h->st->sigma, &sigma, sizeof(double), cudaMemcpyHostToDevice, s));
    LP_CU(cudaMemcpyAsync(&h->st->scheme, &sch, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    LP_CU(cudaStreamSynchronize(s));
    return LP_OK;
  };
  int32_t best = 0;
  for (int32_t k = 0; k < count; ++k) {
    if ((e = set_weight(omegas[k], LP_RESTART_NONE)) != LP_OK) return e;
    if ((e = lp_set_state(h, nullptr, nullptr, cuda_stream)) != LP_OK) return e;
    if ((e = set_run_params(h, 1e-300, s)) != LP_OK) return e;
    const int64_t blocks = iters / K, rem = iters % K;
    for (int64_t b = 0; b < blocks; ++b) LP_CU(cudaGraphLaunch(h->exec, s));
    for (int64_t r = 0; r < rem; ++r) launch_iteration(h, (int)r, s);
    if (rem) launch_advance(h->st, h->w, (int)rem, s);
    LP_CU(cudaGetLastError());
    DevState hs{};
    LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    double v = std::fmin(hs.kkt_a[4], hs.kkt_c[4]);
    if (!std::isfinite(v)) v = INFINITY;
    kkt_out[k] = v;
    if (v < kkt_out[best]) best = k;
  }
  h->opt.omega = omegas[best];
  if ((e = set_weight(omegas[best], scheme)) != LP_OK) return e;
  if (best_out) *best_out = omegas[best];
  h->solved = false;
  return lp_set_state(h, nullptr, nullptr, cuda_stream);
}

lp_status lp_solve_recorded(lp_handle h, int64_t iters, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_solve_recorded");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  const int K = h->opt.check_every;
  if (iters < K || iters % K != 0) return fail(LP_ERR_INVALID_ARG, "iters must be a positive multiple of check_every");
  if (h->mixed) return fail(LP_ERR_INVALID_ARG, "recording needs LP_PRECISION_FP64");
  if (h->opt.restart_scheme == LP_RESTART_FLEXIBLE)
    return fail(LP_ERR_INVALID_ARG, "recording supports the adaptive, fixed and no-restart schemes");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  lp_status e = build_graph(h);
  if (e != LP_OK) return e;
  const int n = h->n, m = h->m;
  const int64_t blocks = iters / K, slot = 2 * (int64_t)n + 2 * (int64_t)m;
  if (h->ckpt) {
    cudaFree(h->ckpt);
    h->ckpt = nullptr;
  }
  LP_CU(cudaMalloc(&h->ckpt, sizeof(double) * std::max<int64_t>(1, blocks * slot)));
  if (!h->mask_x) {  // masks and adjoint vectors, allocated once per handle
    if ((e = h->alloc(&h->mask_x, (int64_t)K * n)) != LP_OK) return e;
    if ((e = h->alloc(&h->mask_y, (int64_t)K * std::max(m, 1))) != LP_OK) return e;
    double **xs[] = {&h->adj.ax, &h->adj.axb, &h->adj.ac, &h->adj.v};
    for (double **p : xs)
      if ((e = h->alloc(p, n)) != LP_OK) return e;
    double **ys[] = {&h->adj.ay, &h->adj.ayb, &h->adj.ab, &h->adj.u};
    for (double **p : ys)
      if ((e = h->alloc(p, m)) != LP_OK) return e;
  }
  h->ckpt_t0.assign(blocks, 0);
  h->ckpt_restart.assign(blocks, 0);
  h->rec_blocks = 0;
  if ((e = set_run_params(h, 1e-300, s)) != LP_OK) return e;
  for (int64_t b = 0; b < blocks; ++b) {
    double *c = h->ckpt + b * slot;
    LP_CU(cudaMemcpyAsync(c, h->v.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(c + n, h->v.y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(c + n + m, h->v.xbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(c + 2 * n + m, h->v.ybar, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    DevState hs{};
    LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    if (hs.status != kRunning) return fail(LP_ERR_NUMERICAL, "solve stopped during recording");
    h->ckpt_t0[b] = hs.t0;
    const int64_t restarts_before = hs.restarts;
    LP_CU(cudaGraphLaunch(h->exec, s));
    LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LP_CU(cudaStreamSynchronize(s));
    h->ckpt_restart[b] = (hs.restarts > restarts_before) ? 1 : 0;
  }
  h->rec_blocks = blocks;
  h->solved = true;
  return LP_OK;
}

lp_status lp_backward(lp_handle h, const double *dl_dx, const double *dl_dy, double *dl_dc,
                      double *dl_db, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_backward");
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (h->rec_blocks == 0) return fail(LP_ERR_NOT_SOLVED, "no recorded solve (lp_solve_recorded)");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  const int n = h->n, m = h->m, K = h->opt.check_every;
  const int64_t slot = 2 * (int64_t)n + 2 * (int64_t)m;
  DevState hs{};
  LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  const double tau = hs.tau, sigma = hs.sigma;
  // adjoint seeds: gradients of the loss with respect to the final averages
  launch_fill(h->adj.ax, 0.0, n, s);
  launch_fill(h->adj.ac, 0.0, n, s);
  launch_fill(h->adj.ay, 0.0, m, s);
  launch_fill(h->adj.ab, 0.0, m, s);
  if (dl_dx) {
    LP_CU(cudaMemcpyAsync(h->tmp, dl_dx, sizeof(double) * n, cudaMemcpyDefault, s));
    launch_gather(h->adj.axb, h->tmp, h->perm_x, n, s);
  } else {
    launch_fill(h->adj.axb, 0.0, n, s);
  }
  if (dl_dy && m > 0) {
    LP_CU(cudaMemcpyAsync(h->tmp, dl_dy, sizeof(double) * m, cudaMemcpyDefault, s));
    launch_gather(h->adj.ayb, h->tmp, h->perm_y, m, s);
  } else {
    launch_fill(h->adj.ayb, 0.0, m, s);
  }
  for (int64_t b = h->rec_blocks - 1; b >= 0; --b) {
    // recompute the block's forward steps with their masks
    const double *c = h->ckpt + b * slot;
    LP_CU(cudaMemcpyAsync(h->v.x, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.y, c + n, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.xbar, c + n + m, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.ybar, c + 2 * n + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    const int64_t t0 = h->ckpt_t0[b];
    auto wk = [&](int k) { return 1.0 / (double)(t0 + k + 1); };
    for (int k = 0; k < K; ++k)
      launch_forward_masked(h->A, h->AT, h->v, tau, sigma, wk(k), h->mask_x + (int64_t)k * n,
                            h->mask_y + (int64_t)k * m, s);
    // reverse through the block
    launch_adjoint_block_start(h->adj, h->mask_y + (int64_t)(K - 1) * m, h->ckpt_restart[b],
                               sigma, wk(K - 1), n, m, s);
    for (int k = K - 1; k >= 0; --k)
      launch_adjoint_step(h->A, h->AT, h->adj, h->mask_x + (int64_t)k * n,
                          k > 0 ? h->mask_y + (int64_t)(k - 1) * m : nullptr, tau, sigma, wk(k),
                          k > 0 ? wk(k - 1) : 0.0, k > 0 ? 1 : 0, s);
    LP_CU(cudaGetLastError());
  }
  // restore the final state of the recorded solve: replay the last block
  {
    const int64_t b = h->rec_blocks - 1;
    const double *c = h->ckpt + b * slot;
    LP_CU(cudaMemcpyAsync(h->v.x, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.y, c + n, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.xbar, c + n + m, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    LP_CU(cudaMemcpyAsync(h->v.ybar, c + 2 * n + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    const int64_t t0 = h->ckpt_t0[b];
    for (int k = 0; k < K; ++k)
      launch_forward_masked(h->A, h->AT, h->v, tau, sigma, 1.0 / (double)(t0 + k + 1),
                            h->mask_x + (int64_t)k * n, h->mask_y + (int64_t)k * m, s);
    if (h->ckpt_restart[b]) {  // the recorded check restarted: z <- zbar
      LP_CU(cudaMemcpyAsync(h->v.x, h->v.xbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      LP_CU(cudaMemcpyAsync(h->v.y, h->v.ybar, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (dl_dc) {
    launch_scatter(h->tmp, h->adj.ac, h->perm_x, n, s);
    LP_CU(cudaMemcpyAsync(dl_dc, h->tmp, sizeof(double) * n, cudaMemcpyDefault, s));
    LP_CU(cudaStreamSynchronize(s));
  }
  if (dl_db && m > 0) {
    launch_scatter(h->tmp, h->adj.ab, h->perm_y, m, s);
    LP_CU(cudaMemcpyAsync(dl_db, h->tmp, sizeof(double) * m, cudaMemcpyDefault, s));
  }
  LP_CU(cudaGetLastError());
  LP_CU(cudaStreamSynchronize(s));
  return LP_OK;
}

lp_status lp_profile_kernel(lp_handle h, int32_t which, int32_t reps, void *cuda_stream) {
  err_msg().clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (which < 0 || which > 1 || reps < 0) return fail(LP_ERR_INVALID_ARG, "which must be 0 or 1, reps >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  for (int32_t r = 0; r < reps; ++r) {
    if (h->mixed) {
      if (which == 0) launch_primal_mix(h->AT, h->mv, h->st, h->w, 0, h->opt.spmv_unroll, s);
      else launch_dual_mix(h->A, h->mv, h->v, h->st, h->w, 0, h->opt.spmv_unroll_rows, s);
    } else {
      if (which == 0) launch_primal_step(h->AT, h->v, h->st, h->w, 0, h->opt.spmv_unroll, h->grid_cap, s);
      else launch_dual_step(h->A, h->v, h->st, h->w, 0, h->opt.spmv_unroll_rows, h->grid_cap, s);
    }
  }
  LP_CU(cudaGetLastError());
  return LP_OK;
}

void lp_destroy(lp_handle h) {
  if (!h) return;
  // the handle's work is stream-ordered: wait for the stream of its latest
  // call and for its own capture stream, not for the whole device
  if (h->stream_used) cudaStreamSynchronize(h->last_stream);
  if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// lp_normalized_gap_static: the normalized duality gap without any device
// allocation.
//
// Some callers cannot let a library call cudaMalloc/cudaFree: a host loop
// with a latency budget (cudaFree synchronizes the whole device), a process
// whose framework has already reserved nearly all device memory for its own
// pool, or code that must not change the device's allocation state while
// other work is queued.  For them this entry point keeps its scratch in a
// file-scope device array of fixed size, loaded with the library on every
// GPU that uses it and held until the process exits.
//
// Scratch budget: 16 MiB per device, enough for n + m <= 262,144.  Larger
// problems are rejected with LP_ERR_INVALID_ARG.
//
// Host code cannot use the array's name as a device address (it names a
// host-side shadow), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device.  Make that first call before any stream
// capture begins.  Every call reuses the same array: two calls whose work
// overlaps on the GPU (different streams, different host threads) race on
// it and must be serialized by the caller.  A call writes nothing that the
// handle's own calls use (its split-row counters and partial sums come from
// the array too), so it may overlap a solve on the same handle.  The
// split-row arrival counters are cleared at the start of every call; every
// other region is fully written by a call before the same call reads it.
// The histogram grid is the handle's (at most 129 blocks for n + m within
// the limit), so the result is that of lp_normalized_gap bit for bit.
namespace {

constexpr size_t kGapScratchBytes = size_t(16) << 20;
constexpr int64_t kGapScratchMaxElems = int64_t(1) << 18;  // n + m
constexpr int32_t kGapScratchMaxParts = 65536;              // partial-sum slots per quantity
constexpr int kGapScratchMaxDevices = 256;

static __device__ __align__(256) unsigned char g_gap_scratch[kGapScratchBytes];

std::mutex g_gap_scratch_mu;
void *g_gap_scratch_addr[kGapScratchMaxDevices] = {};

struct ScratchCarver {
  unsigned char *base;
  size_t off;
  size_t cap;
  void *take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    if (off + bytes > cap) return nullptr;
    void *p = base + off;
    off += bytes;
    return p;
  }
};

}  // namespace

extern "C" lp_status lp_normalized_gap_static(lp_handle h, const double *x, const double *y,
                                              double r, double *host_rho, void *cuda_stream) {
  err_msg().clear();
  NvtxRange nvtx_range("lp_normalized_gap_static");
  if (!h || !host_rho || !x || (h->m > 0 && !y)) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  if (!(r >= 0.0) || !std::isfinite(r)) return fail(LP_ERR_INVALID_ARG, "radius must be finite and >= 0");
  const int n = h->n, m = h->m;
  const int64_t N = (int64_t)n + m;
  if (N > kGapScratchMaxElems)
    return fail(LP_ERR_INVALID_ARG, "lp_normalized_gap_static: n + m = " + std::to_string(N) +
                                        " exceeds the static scratch limit of " +
                                        std::to_string(kGapScratchMaxElems));
  if (h->cs.pstride > kGapScratchMaxParts)
    return fail(LP_ERR_INVALID_ARG, "lp_normalized_gap_static: too many partial sums for the static scratch");
  int dev = 0;
  LP_CU(cudaGetDevice(&dev));
  if (dev != h->device) return fail(LP_ERR_INVALID_ARG, "the handle's device is not current");
  if (dev < 0 || dev >= kGapScratchMaxDevices) return fail(LP_ERR_INVALID_ARG, "device index out of range");
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_gap_scratch_mu);
    if (!g_gap_scratch_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_gap_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_gap_scratch)");
      g_gap_scratch_addr[dev] = p;
    }
    base = g_gap_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->use_stream(s);
  ScratchCarver sc{static_cast<unsigned char *>(base), 0, kGapScratchBytes};
  double *xp = (double *)sc.take(sizeof(double) * std::max(n, 1));
  double *yp = (double *)sc.take(sizeof(double) * std::max(m, 1));
  double *tmpx = (double *)sc.take(sizeof(double) * std::max(std::max(n, m), 1));
  DevState *st = (DevState *)sc.take(sizeof(DevState));
  CheckScratch cs = h->cs;  // same histogram grid as lp_normalized_gap: same reduction order
  cs.partials = (double *)sc.take(sizeof(double) * NQ * cs.pstride);
  cs.keys[0] = (uint64_t *)sc.take(sizeof(uint64_t) * N);
  cs.d2[0] = (double *)sc.take(sizeof(double) * N);
  cs.g2[0] = (double *)sc.take(sizeof(double) * N);
  cs.gd[0] = (double *)sc.take(sizeof(double) * N);
  cs.hpart = (double *)sc.take(sizeof(double) * 2 * cs.hist_grid * 4 * kBuckets);
  cs.btot = (double *)sc.take(sizeof(double) * 2 * 4 * kBuckets);
  // split-row partial sums and arrival counters of this call (the handle's
  // belong to its solves); the counters start at zero
  SellMat A = h->A, AT = h->AT;
  bool split_ok = true;
  for (SellMat *M : {&A, &AT}) {
    if (M->nsplit == 0) continue;
    M->split_part = (double *)sc.take(sizeof(double) * 2 * (size_t)M->nsplit);
    M->split_cnt = (int32_t *)sc.take(sizeof(int32_t) * (size_t)M->nsplit);
    split_ok = split_ok && M->split_part && M->split_cnt;
  }
  if (!xp || !yp || !tmpx || !st || !cs.partials || !cs.keys[0] || !cs.d2[0] || !cs.g2[0] ||
      !cs.gd[0] || !cs.hpart || !cs.btot || !split_ok)
    return fail(LP_ERR_INVALID_ARG, "lp_normalized_gap_static: problem does not fit the static scratch");
  for (SellMat *M : {&A, &AT})
    if (M->nsplit > 0) LP_CU(cudaMemsetAsync(M->split_cnt, 0, sizeof(int32_t) * (size_t)M->nsplit, s));
  cs.keys[1] = cs.keys[0];
  cs.d2[1] = cs.d2[0];
  cs.g2[1] = cs.g2[0];
  cs.gd[1] = cs.gd[0];
  LP_CU(cudaMemcpyAsync(tmpx, x, sizeof(double) * n, cudaMemcpyDefault, s));
  launch_gather(xp, tmpx, h->perm_x, n, s);
  if (m > 0) {
    LP_CU(cudaMemcpyAsync(tmpx, y, sizeof(double) * m, cudaMemcpyDefault, s));
    launch_gather(yp, tmpx, h->perm_y, m, s);
  }
  DevVecs v = h->v;
  v.x = v.xbar = v.x0 = xp;
  v.y = v.ybar = v.y0 = yp;
  DevState hs{};
  LP_CU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  hs.status = kRunning;
  hs.given_radius = 1;
  hs.r_given = r;
  LP_CU(cudaMemcpyAsync(st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, s));
  cs.pair_x = cs.pair_y = nullptr;  // the handle's pair buffers belong to its solve
  cs.cand[0] = cs.cand[1] = nullptr;  // and so do its candidate lists: full scans
  launch_check(A, AT, v, st, nullptr, cs, n, m, 1, nullptr, false, s);
  LP_CU(cudaGetLastError());
  LSearch L{};
  LP_CU(cudaMemcpyAsync(&L, &st->ls[0], sizeof(LSearch), cudaMemcpyDeviceToHost, s));
  LP_CU(cudaStreamSynchronize(s));
  *host_rho = (r == 0.0) ? 0.0 : L.rho_r / r;
  return LP_OK;
}
