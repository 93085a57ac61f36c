// Host layout builder check (compiled and run by tests/test_layout_cpu.py; no
// GPU needed).  Random matrices and lane policies, with and without split
// rows: build_csc against a plain transpose, sort_by_length_desc against a
// stable sort, csc_has_duplicates, and build_sell rebuilt row by row from its
// slices (every element once, in order, relabeled; zero padding; chunk
// records of split rows).  Prints "ok" or the first failure.
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <random>

#include "lp_host.h"

using namespace lpg;

static int fails = 0;
#define CHECK(c, msg)                                   \
  do {                                                  \
    if (!(c)) {                                         \
      std::printf("FAIL %s (trial %d)\n", msg, trial); \
      ++fails;                                          \
      return;                                           \
    }                                                   \
  } while (0)

static void one(int trial, std::mt19937_64 &rng) {
  const int m = 1 + (int)(rng() % 300), n = 1 + (int)(rng() % 3000);
  std::vector<int32_t> rp(m + 1, 0), ci;
  std::vector<double> v;
  for (int i = 0; i < m; ++i) {
    int64_t len = (rng() % 8 == 0) ? (int64_t)(rng() % 3000) : (int64_t)(rng() % 30);
    if (len > n) len = n;
    std::vector<int32_t> cols(n);
    std::iota(cols.begin(), cols.end(), 0);
    std::shuffle(cols.begin(), cols.end(), rng);
    for (int64_t k = 0; k < len; ++k) {
      ci.push_back(cols[k]);
      v.push_back((double)ci.size());
    }
    rp[i + 1] = (int32_t)ci.size();
  }
  // CSC against a plain transpose (rows ascending in every column)
  std::vector<int64_t> cp;
  uvec<int32_t> ri;
  uvec<double> cv;
  CHECK(build_csc(m, n, rp.data(), ci.data(), v.data(), cp, ri, cv), "build_csc range");
  std::vector<std::vector<std::pair<int32_t, double>>> col(n);
  for (int i = 0; i < m; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) col[ci[p]].push_back({i, v[p]});
  for (int j = 0; j < n; ++j) {
    CHECK(cp[j + 1] - cp[j] == (int64_t)col[j].size(), "csc column length");
    for (size_t k = 0; k < col[j].size(); ++k)
      CHECK(ri[cp[j] + k] == col[j][k].first && cv[cp[j] + k] == col[j][k].second, "csc entry");
  }
  CHECK(!csc_has_duplicates(n, cp, ri), "no duplicates");
  // stable order by decreasing length
  std::vector<int32_t> perm(n), ref(n);
  sort_by_length_desc(cp.data(), 0, n, perm.data());
  std::iota(ref.begin(), ref.end(), 0);
  std::stable_sort(ref.begin(), ref.end(), [&](int32_t a, int32_t b) {
    return cp[a + 1] - cp[a] > cp[b + 1] - cp[b];
  });
  CHECK(perm == ref, "length order");
  // slices of A^T (rows = columns of A), relabeled by a permutation of the rows of A
  std::vector<int32_t> relabel(m);
  std::iota(relabel.begin(), relabel.end(), 0);
  std::shuffle(relabel.begin(), relabel.end(), rng);
  const int32_t split_len = (rng() % 3 == 0) ? 0 : 32 * (int32_t)(1 + rng() % 16);
  const LanePolicy pol{int32_t(16 + rng() % 600), int32_t(1 + rng() % 16), int32_t(rng() % 80)};
  HostSell S;
  build_sell(n, m, cp, ri.data(), cv.data(), perm, relabel, pol, S, {}, split_len);
  const int nsplit = (int)S.split.size();
  std::vector<std::vector<std::pair<int32_t, double>>> got(n);
  for (int s = 0; s < S.nslices; ++s) {
    const SliceInfo &a = S.info[s];
    const int lg = a.len_g & 7, G = 1 << lg;
    const int64_t steps = a.len_g >> 3;
    CHECK(S.info[s + 1].off - a.off == steps * 32, "slice width");
    if (s < nsplit) {
      const SplitSlice &sp = S.split[s];
      const int64_t L = cp[perm[a.row0] + 1] - cp[perm[a.row0]];
      CHECK(lg == 5 && L > split_len, "chunk of a long whole-warp row");
      CHECK(sp.first + sp.chunk == s && sp.begin == (int64_t)sp.chunk * split_len &&
                sp.nchunks == (L + split_len - 1) / split_len,
            "chunk record");
      const int64_t clen = std::min<int64_t>(split_len, L - sp.begin);
      CHECK(steps == (clen + 31) / 32, "chunk steps");
      for (int64_t k = 0; k < clen; ++k) got[a.row0].push_back({S.idx[a.off + k], S.val[a.off + k]});
      for (int64_t k = clen; k < steps * 32; ++k) CHECK(S.val[a.off + k] == 0.0, "chunk padding");
      continue;
    }
    for (int32_t row = a.row0; row < S.info[s + 1].row0; ++row) {
      const int64_t L = cp[perm[row] + 1] - cp[perm[row]];
      CHECK(split_len == 0 || lg < 5 || L <= split_len, "long row left unsplit");
      CHECK(lanes_log2(L, pol) == lg, "lane count");
      for (int64_t k = 0; k < L; ++k) {
        const int64_t dst = a.off + 32 * (k >> lg) + (int64_t)(row - a.row0) * G + (k & (G - 1));
        got[row].push_back({S.idx[dst], S.val[dst]});
      }
    }
  }
  for (int r = 0; r < n; ++r) {
    const int32_t j = perm[r];
    CHECK((int64_t)got[r].size() == cp[j + 1] - cp[j], "row element count");
    for (int64_t k = 0; k < cp[j + 1] - cp[j]; ++k)
      CHECK(got[r][k].first == relabel[ri[cp[j] + k]] && got[r][k].second == cv[cp[j] + k],
            "row element");
  }
}

int main() {
  std::mt19937_64 rng(11);
  for (int trial = 0; trial < 150 && fails == 0; ++trial) one(trial, rng);
  std::printf("%s\n", fails ? "FAIL" : "ok");
  return fails != 0;
}
