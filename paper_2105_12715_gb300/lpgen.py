"""Seeded synthetic LP generators.

This module only draws random LP data.  It holds none of the solver's
arithmetic, and both the CUDA path and the CPU oracle take its output as
input.  Every instance has a *planted* optimum: a primal-dual pair
``(x*, y*)`` that satisfies the LP optimality conditions by construction.
The LP form is the one of Eq. (LP-Lag) widened to box bounds on ``x`` and
sign-typed rows:

    min c^T x   s.t.   (A x)_i = b_i  (row type EQ),
                       (A x)_i >= b_i (row type GE),
                       (A x)_i <= b_i (row type LE),
                       lb <= x <= ub.

The planted pair is optimal because ``c - A^T y* = s`` with ``s`` chosen
complementary to ``x*`` (``s_j >= 0`` where ``x*_j`` sits at its lower bound,
``s_j <= 0`` at its upper bound, ``s_j = 0`` in the interior or for free
columns), and ``y*_i = 0`` on inequality rows that are slack at ``x*``.

Workloads (the paper's Mittelmann QAP relaxations, Table 4, are not shipped;
these seeded instances stand in for them):

* ``tiny_standard_form``: m equality rows, n columns with x >= 0, a fixed
  number of distinct uniform rows per column, N(0,1) values.
* ``large_mixed``: 70% equality / 30% >= rows, bounds 40% [0,inf),
  40% [0,U(1,10)], 20% free, power-law column degree on 2..200 (exponent
  1.82, mean ~10), uniform rows, N(0,1) values.
* ``batch_standard_form``: batches of uneven standard-form LPs (m log-uniform,
  n = 2m, 3-12 rows per column) for the batched solver.
* ``adversarial``: small LPs with empty rows/columns, one dense row, one
  dense column, LE rows and every bound kind, for edge-case coverage.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ROW_EQ, ROW_GE, ROW_LE = 0, 1, 2


@dataclass
class LPData:
    """An LP in CSR form plus its planted optimum (when one is known)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int32 [m+1]
    col_idx: np.ndarray  # int32 [nnz], sorted within each row
    val: np.ndarray  # float64 [nnz]
    c: np.ndarray  # float64 [n]
    b: np.ndarray  # float64 [m]
    lb: np.ndarray  # float64 [n], -inf = no lower bound
    ub: np.ndarray  # float64 [n], +inf = no upper bound
    row_type: np.ndarray  # int8 [m] in {ROW_EQ, ROW_GE, ROW_LE}
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def obj_star(self) -> float | None:
        if self.x_star is None:
            return None
        return float(np.dot(self.c, self.x_star))

    def dense(self) -> np.ndarray:
        """Dense copy of A (small instances only)."""
        a = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            a[i, self.col_idx[s:e]] += self.val[s:e]
        return a


def _coo_to_csr(m: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """Sort COO entries row-major and build int32 CSR arrays."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    assert row_ptr[-1] < 2**31
    return row_ptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def _distinct_rows_per_column(rng, m: int, degree: np.ndarray):
    """For column j draw degree[j] distinct rows uniformly from [0, m).

    Returns (rows, cols) in column-major order.  Duplicates inside a column
    are redrawn until none remain.
    """
    n = degree.shape[0]
    cols = np.repeat(np.arange(n, dtype=np.int64), degree)
    rows = rng.integers(0, m, size=cols.shape[0], dtype=np.int64)
    while True:
        key = cols * m + rows
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ks.shape[0], dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            return rows[order], cols[order]
        rows, cols = rows[order], cols[order]
        rows[dup] = rng.integers(0, m, size=int(dup.sum()), dtype=np.int64)


def _matvec(m, rows, cols, vals, x):
    out = np.zeros(m)
    np.add.at(out, rows, vals * x[cols])
    return out


def _rmatvec(n, rows, cols, vals, y):
    out = np.zeros(n)
    np.add.at(out, cols, vals * y[rows])
    return out


def tiny_standard_form(seed: int = 0, m: int = 200, n: int = 400, per_col: int = 5) -> LPData:
    """Standard-form LP (Ax = b, x >= 0) with a planted optimum.

    x* is zero on a random half of the columns and U(0,1) elsewhere; y* is
    N(0,1); s_j = 0 where x*_j > 0 and U(0,1) elsewhere; b = A x*,
    c = A^T y* + s.
    """
    rng = np.random.default_rng(seed)
    per_col = min(per_col, m)
    degree = np.full(n, per_col, dtype=np.int64)
    rows, cols = _distinct_rows_per_column(rng, m, degree)
    vals = rng.standard_normal(rows.shape[0])
    x_star = np.zeros(n)
    pos = rng.permutation(n)[: n // 2]
    x_star[pos] = rng.random(pos.shape[0])
    y_star = rng.standard_normal(m)
    s = rng.random(n)
    s[pos] = 0.0
    b = _matvec(m, rows, cols, vals, x_star)
    c = _rmatvec(n, rows, cols, vals, y_star) + s
    row_ptr, col_idx, val = _coo_to_csr(m, rows, cols, vals)
    return LPData(m, n, row_ptr, col_idx, val, c, b,
                  np.zeros(n), np.full(n, np.inf), np.zeros(m, dtype=np.int8),
                  x_star, y_star, name=f"tiny_standard_form(m={m},n={n},seed={seed})")


def batch_standard_form(seed: int = 2, count: int = 512, m_lo: int = 50, m_hi: int = 20000,
                        k_lo: int = 3, k_hi: int = 12) -> list:
    """A batch of uneven standard-form LPs (Ax = b, x >= 0), each with a planted optimum.

    Problem k has m_k rows with log(m_k) ~ U(log m_lo, log m_hi), n_k = 2 m_k
    columns, U{k_lo..k_hi} distinct uniform rows per column, N(0,1) values,
    and the planted pair of ``tiny_standard_form``.  Problem k is drawn from
    its own stream (seed, k), so a prefix of a batch is the smaller batch.
    """
    out = []
    for k in range(count):
        rng = np.random.default_rng([seed, k])
        m = int(round(float(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))))
        n = 2 * m
        degree = rng.integers(min(k_lo, m), min(k_hi, m) + 1, size=n).astype(np.int64)
        rows, cols = _distinct_rows_per_column(rng, m, degree)
        vals = rng.standard_normal(rows.shape[0])
        x_star = np.zeros(n)
        pos = rng.permutation(n)[: n // 2]
        x_star[pos] = rng.random(pos.shape[0])
        y_star = rng.standard_normal(m)
        sv = rng.random(n)
        sv[pos] = 0.0
        b = _matvec(m, rows, cols, vals, x_star)
        c = _rmatvec(n, rows, cols, vals, y_star) + sv
        row_ptr, col_idx, val = _coo_to_csr(m, rows, cols, vals)
        out.append(LPData(m, n, row_ptr, col_idx, val, c, b, np.zeros(n), np.full(n, np.inf),
                          np.zeros(m, dtype=np.int8), x_star, y_star,
                          name=f"batch_standard_form(seed={seed},k={k},m={m})"))
    return out


def power_law_degrees(rng, n: int, kmin: int = 2, kmax: int = 200, exponent: float = 1.82):
    """Discrete power law P(k) ~ k^-exponent on [kmin, kmax]."""
    k = np.arange(kmin, kmax + 1)
    p = k.astype(np.float64) ** (-exponent)
    p /= p.sum()
    return rng.choice(k, size=n, p=p).astype(np.int64)


def large_mixed(seed: int = 1, m: int = 200_000, n: int = 1_000_000,
                eq_frac: float = 0.7, exponent: float = 1.82,
                kmin: int = 2, kmax: int = 200) -> LPData:
    """Mixed-bound, mixed-row LP with power-law column degrees and a planted optimum.

    Rows: the first ``eq_frac`` share are EQ, the rest GE (half active with
    y*_i = |N(0,1)|, half slack by U(0,1) with y*_i = 0); EQ rows take
    y* ~ N(0,1).  Columns: 40% [0,inf) (half at 0 with s ~ U(0,1), half
    U(0,1) with s = 0), 40% [0,U], U ~ U(1,10) (thirds at 0 with s > 0,
    interior with s = 0, at U with s < 0), 20% free (x* ~ N(0,1), s = 0).
    Row and column kinds are assigned by a seeded shuffle.
    """
    rng = np.random.default_rng(seed)
    kmax = min(kmax, m)
    degree = power_law_degrees(rng, n, kmin, kmax, exponent)
    rows, cols = _distinct_rows_per_column(rng, m, degree)
    vals = rng.standard_normal(rows.shape[0])

    # column kinds
    kind = np.zeros(n, dtype=np.int8)  # 0: [0,inf), 1: [0,U], 2: free
    perm = rng.permutation(n)
    n0, n1 = int(0.4 * n), int(0.4 * n)
    kind[perm[n0:n0 + n1]] = 1
    kind[perm[n0 + n1:]] = 2
    lb = np.zeros(n)
    ub = np.full(n, np.inf)
    lb[kind == 2] = -np.inf
    ub_box = rng.uniform(1.0, 10.0, size=n)
    ub[kind == 1] = ub_box[kind == 1]

    x_star = np.zeros(n)
    s = np.zeros(n)
    u01 = rng.random(n)
    sel = rng.random(n)
    # [0, inf): half at zero with positive reduced cost, half interior
    k0 = kind == 0
    at0 = k0 & (sel < 0.5)
    x_star[k0 & ~at0] = u01[k0 & ~at0]
    s[at0] = rng.random(int(at0.sum()))
    # [0, U]: thirds at 0, interior, at U
    k1 = kind == 1
    lo_t = k1 & (sel < 1 / 3)
    hi_t = k1 & (sel >= 2 / 3)
    mid_t = k1 & ~lo_t & ~hi_t
    s[lo_t] = rng.random(int(lo_t.sum()))
    x_star[mid_t] = u01[mid_t] * ub[mid_t]
    x_star[hi_t] = ub[hi_t]
    s[hi_t] = -rng.random(int(hi_t.sum()))
    # free
    k2 = kind == 2
    x_star[k2] = rng.standard_normal(int(k2.sum()))

    # row kinds
    row_type = np.full(m, ROW_EQ, dtype=np.int8)
    rperm = rng.permutation(m)
    n_eq = int(round(eq_frac * m))
    ge_rows = rperm[n_eq:]
    row_type[ge_rows] = ROW_GE
    y_star = rng.standard_normal(m)
    ax = _matvec(m, rows, cols, vals, x_star)
    b = ax.copy()
    ge_sel = rng.random(m)
    ge = row_type == ROW_GE
    active = ge & (ge_sel < 0.5)
    slack = ge & ~active
    y_star[active] = np.abs(y_star[active])
    y_star[slack] = 0.0
    b[slack] = ax[slack] - rng.random(int(slack.sum()))
    c = _rmatvec(n, rows, cols, vals, y_star) + s
    row_ptr, col_idx, val = _coo_to_csr(m, rows, cols, vals)
    return LPData(m, n, row_ptr, col_idx, val, c, b, lb, ub, row_type,
                  x_star, y_star, name=f"large_mixed(m={m},n={n},seed={seed})",
                  meta={"col_kind": kind})


def adversarial(seed: int = 7, m: int = 70, n: int = 150, dense_row: bool = True,
                dense_col: bool = True, empty: bool = True) -> LPData:
    """Small LP exercising edge cases of the sparse layouts.

    Contains empty rows and columns (when ``empty``), one row touching every
    column (when ``dense_row``), one column touching every row (when
    ``dense_col``), EQ/GE/LE rows, and all four bound kinds ([0,inf),
    [l,u], (-inf,u], free).  A planted optimum is built as in
    ``large_mixed``; LE rows are mirrored versions of GE rows.
    """
    rng = np.random.default_rng(seed)
    degree = rng.integers(1, 6, size=n)
    if empty:
        degree[rng.choice(n, size=3, replace=False)] = 0
    rows, cols = _distinct_rows_per_column(rng, m, degree)
    if empty:
        # clear a few rows entirely
        dead = rng.choice(m, size=3, replace=False)
        keep = ~np.isin(rows, dead)
        rows, cols = rows[keep], cols[keep]
    extra_r, extra_c = [], []
    if dense_row:
        r0 = int(rng.integers(0, m))
        if empty:
            while r0 in dead:
                r0 = int(rng.integers(0, m))
        extra_r.append(np.full(n, r0))
        extra_c.append(np.arange(n))
    if dense_col:
        c0 = int(rng.integers(0, n))
        live = np.setdiff1d(np.arange(m), dead) if empty else np.arange(m)
        extra_r.append(live)
        extra_c.append(np.full(live.shape[0], c0))
    if extra_r:
        rows = np.concatenate([rows] + extra_r)
        cols = np.concatenate([cols] + extra_c)
        key = np.unique(cols.astype(np.int64) * m + rows)
        cols, rows = key // m, key % m
    vals = rng.standard_normal(rows.shape[0])

    kind = rng.integers(0, 4, size=n)  # 0 [0,inf) 1 [l,u] 2 (-inf,u] 3 free
    lb = np.where(kind == 0, 0.0, np.where(kind == 1, rng.uniform(-2, 0, n), -np.inf))
    ub = np.where(kind == 1, rng.uniform(0.5, 3, n), np.where(kind == 2, rng.uniform(-1, 2, n), np.inf))
    x_star = np.zeros(n)
    s = np.zeros(n)
    sel = rng.random(n)
    for j in range(n):
        if kind[j] == 0:
            if sel[j] < 0.5:
                x_star[j], s[j] = 0.0, rng.random()
            else:
                x_star[j] = rng.random()
        elif kind[j] == 1:
            if sel[j] < 1 / 3:
                x_star[j], s[j] = lb[j], rng.random()
            elif sel[j] < 2 / 3:
                x_star[j] = lb[j] + rng.random() * (ub[j] - lb[j])
            else:
                x_star[j], s[j] = ub[j], -rng.random()
        elif kind[j] == 2:
            if sel[j] < 0.5:
                x_star[j], s[j] = ub[j], -rng.random()
            else:
                x_star[j] = ub[j] - rng.random()
        else:
            x_star[j] = rng.standard_normal()
    row_type = rng.integers(0, 3, size=m).astype(np.int8)
    ax = _matvec(m, rows, cols, vals, x_star)
    b = ax.copy()
    y_star = rng.standard_normal(m)
    act = rng.random(m) < 0.5
    for i in range(m):
        if row_type[i] == ROW_GE:
            if act[i]:
                y_star[i] = abs(y_star[i])
            else:
                y_star[i] = 0.0
                b[i] = ax[i] - rng.random()
        elif row_type[i] == ROW_LE:
            if act[i]:
                y_star[i] = -abs(y_star[i])
            else:
                y_star[i] = 0.0
                b[i] = ax[i] + rng.random()
    c = _rmatvec(n, rows, cols, vals, y_star) + s
    row_ptr, col_idx, val = _coo_to_csr(m, rows, cols, vals)
    return LPData(m, n, row_ptr, col_idx, val, c, b, lb.astype(np.float64), ub.astype(np.float64),
                  row_type, x_star, y_star, name=f"adversarial(m={m},n={n},seed={seed})",
                  meta={"col_kind": kind})


def random_state(lp: LPData, seed: int, scale: float = 1.0):
    """A random primal-dual point inside X x Y (for step-level parity tests)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(lp.n) * scale
    x = np.minimum(np.maximum(x, lp.lb), lp.ub)
    y = rng.standard_normal(lp.m) * scale
    y = np.where(lp.row_type == ROW_GE, np.abs(y), np.where(lp.row_type == ROW_LE, -np.abs(y), y))
    return x, y


CONFIGS = {
    "tiny": lambda seed=0: tiny_standard_form(seed),
    "large": lambda seed=1: large_mixed(seed),
}


def multicommodity_grid(seed: int = 4, side: int = 300, commodities: int = 8) -> LPData:
    """Multicommodity min-cost flow on a side x side directed grid.

    Arcs join 4-neighbours in both directions (2 * 2 * side * (side - 1)
    arcs); cost U(1,10) and capacity U(5,50) per arc; each commodity has one
    random source != sink with demand U(1,20).  Variables f[k, a] >= 0
    (column k * arcs + a).  Rows: node balance (out - in = demand at the
    source, -demand at the sink, 0 elsewhere; EQ), one per commodity and
    node, then one capacity row per arc (sum_k f[k, a] <= cap_a; LE).  Every
    value is +-1.  No planted optimum: the optimum is certified by KKT and
    an LP solver.
    """
    rng = np.random.default_rng(seed)
    V = side * side
    idx = np.arange(V).reshape(side, side)
    tails = [idx[:, :-1].ravel(), idx[:, 1:].ravel(), idx[:-1, :].ravel(), idx[1:, :].ravel()]
    heads = [idx[:, 1:].ravel(), idx[:, :-1].ravel(), idx[1:, :].ravel(), idx[:-1, :].ravel()]
    tail = np.concatenate(tails).astype(np.int64)
    head = np.concatenate(heads).astype(np.int64)
    n_arcs = tail.shape[0]
    cost = rng.uniform(1.0, 10.0, n_arcs)
    cap = rng.uniform(5.0, 50.0, n_arcs)
    K = commodities
    m = K * V + n_arcs
    n = K * n_arcs
    rows, cols, vals = [], [], []
    b = np.zeros(m)
    for k in range(K):
        col = k * n_arcs + np.arange(n_arcs)
        rows += [k * V + tail, k * V + head, K * V + np.arange(n_arcs)]
        cols += [col, col, col]
        vals += [np.ones(n_arcs), -np.ones(n_arcs), np.ones(n_arcs)]
        s, t = rng.choice(V, size=2, replace=False)
        d = rng.uniform(1.0, 20.0)
        b[k * V + s] += d
        b[k * V + t] -= d
    b[K * V:] = cap
    row_type = np.zeros(m, dtype=np.int8)
    row_type[K * V:] = ROW_LE
    row_ptr, col_idx, val = _coo_to_csr(m, np.concatenate(rows), np.concatenate(cols),
                                        np.concatenate(vals))
    c = np.tile(cost, K)
    return LPData(m, n, row_ptr, col_idx, val, c, b, np.zeros(n), np.full(n, np.inf), row_type,
                  None, None, name=f"multicommodity_grid(side={side},K={K},seed={seed})",
                  meta={"arcs": n_arcs, "nodes": V})


def box_standard_form(seed: int = 3, m: int = 2000, n: int = 5000, per_col: int = 10) -> LPData:
    """Standard-form LP with box bounds [0, 1] and a planted optimum (x* zero
    on half the columns with s > 0, U(0,1) interior elsewhere with s = 0),
    the shape of the differentiable-LP workload (m = 2000, n = 5000,
    nnz = 50k)."""
    d = tiny_standard_form(seed, m=m, n=n, per_col=per_col)
    d.ub = np.ones(n)
    d.name = f"box_standard_form(m={m},n={n},seed={seed})"
    return d


def with_dense_lines(base: LPData, seed: int = 0, row_frac: float = 1.0,
                     col_frac: float = 1.0) -> LPData:
    """``base`` plus one dense EQ row and one dense column, keeping the planted
    optimum optimal: the new row has N(0,1) entries on a random ``row_frac``
    share of the columns, b = a x* and y* = 0 (so c is unchanged); the new
    column (x >= 0, x* = 0) has N(0,1) entries on a random ``col_frac`` share
    of the rows (the new row included) and reduced cost s ~ U(0,1) > 0.
    Rows and columns this long take a whole warp and, past the split length,
    several (the layout's split rows)."""
    rng = np.random.default_rng(seed)
    m, n = base.m, base.n
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(base.row_ptr).astype(np.int64))
    cols = base.col_idx.astype(np.int64)
    vals = base.val.astype(np.float64)
    # dense row m over the old columns
    rc = np.sort(rng.choice(n, size=max(1, int(round(row_frac * n))), replace=False))
    rv = rng.standard_normal(rc.shape[0])
    # dense column n over the old rows and the new one
    cr = np.sort(rng.choice(m + 1, size=max(1, int(round(col_frac * (m + 1)))), replace=False))
    cv = rng.standard_normal(cr.shape[0])
    rows = np.concatenate([rows, np.full(rc.shape[0], m, dtype=rows.dtype), cr.astype(rows.dtype)])
    cols = np.concatenate([cols, rc.astype(cols.dtype), np.full(cr.shape[0], n, dtype=cols.dtype)])
    vals = np.concatenate([vals, rv, cv])
    x_star = np.concatenate([base.x_star, [0.0]])
    y_star = np.concatenate([base.y_star, [0.0]])
    b = np.concatenate([base.b, [float(np.dot(rv, base.x_star[rc]))]])
    s_new = rng.random() + 0.1
    c = np.concatenate([base.c, [float(np.dot(cv, y_star[cr])) + s_new]])
    lb = np.concatenate([base.lb, [0.0]])
    ub = np.concatenate([base.ub, [np.inf]])
    row_type = np.concatenate([base.row_type, np.array([ROW_EQ], dtype=np.int8)])
    row_ptr, col_idx, val = _coo_to_csr(m + 1, rows, cols, vals)
    return LPData(m + 1, n + 1, row_ptr, col_idx, val, c, b, lb, ub, row_type, x_star, y_star,
                  name=f"{base.name}+dense row/column(seed={seed})")
