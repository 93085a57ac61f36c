"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each expected value comes from
a closed form, an independent brute force, a library routine, or an
invariant the paper proves.
"""
import itertools

import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen


def _lp_from_dense(A, c, b, lb, ub, row_type):
    m, n = A.shape
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return lpgen.LPData(m, n, row_ptr, cols.astype(np.int32), A[rows, cols].astype(np.float64),
                        np.asarray(c, float), np.asarray(b, float), np.asarray(lb, float),
                        np.asarray(ub, float), np.asarray(row_type, np.int8))


# ---------------------------------------------------------------- PDHG step

def _bilinear_lp(sig):
    """L(x, y) = -y^T diag(sig) x over R^m x R^m (c = b = 0, free, EQ rows)."""
    m = len(sig)
    A = np.diag(sig)
    return _lp_from_dense(A, np.zeros(m), np.zeros(m), np.full(m, -np.inf), np.full(m, np.inf),
                          np.zeros(m))


def test_bilinear_closed_form_iterates(oracle_mod):
    """Section 5 bilinear dynamics, Eq. (PDHG_simple) / (2d-dynamic).

    For L = y^T A x the paper's per-coordinate map is
    P_i = [[1, -eta s_i], [eta s_i, 1 - 2 eta^2 s_i^2]].  This package's
    Lagrangian carries -y^T A x (Eq. LP-Lag), i.e. s_i -> -s_i.
    """
    rng = np.random.default_rng(3)
    sig = np.array([0.3, 0.7, 1.0, 1.6, 2.5])
    lp = _bilinear_lp(sig)
    eta = 0.9 / sig.max()
    x = rng.standard_normal(5)
    y = rng.standard_normal(5)
    z0 = np.stack([x, y], axis=1)
    for t in range(1, 41):
        x, y = oracle_mod.pdhg_step(lp, eta, eta, x, y)
        for i, s in enumerate(-sig):
            P = np.array([[1.0, -eta * s], [eta * s, 1.0 - 2.0 * eta**2 * s**2]])
            want = np.linalg.matrix_power(P, t) @ z0[i]
            np.testing.assert_allclose([x[i], y[i]], want, rtol=1e-12, atol=1e-13)


def test_bilinear_eigen_contraction(oracle_mod):
    """Eq. (lin-converge) with (lambda-i-abs): ||Q_i^{-1} z_i^t||^2 = (1 - eta^2 s_i^2)^t ||Q_i^{-1} z_i^0||^2."""
    sig = np.array([0.4, 1.1, 2.0])
    lp = _bilinear_lp(sig)
    eta = 0.45
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(3), rng.standard_normal(3)
    z0 = np.stack([x, y], axis=1).astype(complex)
    Qinv = []
    for s in -sig:
        w = np.sqrt(1 - eta**2 * s**2)
        Q = np.array([[eta * s - 1j * w, eta * s + 1j * w], [1.0, 1.0]])
        Qinv.append(np.linalg.inv(Q))
    for t in range(1, 31):
        x, y = oracle_mod.pdhg_step(lp, eta, eta, x, y)
        for i, s in enumerate(sig):
            lhs = np.linalg.norm(Qinv[i] @ np.array([x[i], y[i]])) ** 2
            rhs = (1 - eta**2 * s**2) ** t * np.linalg.norm(Qinv[i] @ z0[i]) ** 2
            assert lhs == pytest.approx(rhs, rel=1e-10)


def test_pdhg_nonexpansive_in_M_norm(oracle_mod):
    """Proposition (PDHG) of Section 2 / Property 1: ||z^{t+1} - z*||_M <= ||z^t - z*||_M.

    For L = c^T x - y^T A x + b^T y with primal step tau, dual step sigma,
    M = [[I/tau, A^T], [A, I/sigma]] (the paper's M for +y^T A x with the
    sign of A flipped, scaled by 1/eta).
    """
    for lp in [lpgen.tiny_standard_form(5, m=30, n=60), lpgen.adversarial(11, m=25, n=50)]:
        A = lp.dense()
        smax = np.linalg.norm(A, 2)
        for omega in [0.5, 1.0, 3.0]:
            eta = 0.95 / smax
            tau, sigma = eta / omega, eta * omega
            M = np.block([[np.eye(lp.n) / tau, A.T], [A, np.eye(lp.m) / sigma]])
            assert np.linalg.eigvalsh(M).min() > 0
            zs = np.concatenate([lp.x_star, lp.y_star])
            x, y = lpgen.random_state(lp, 1, scale=2.0)
            prev = None
            for _ in range(60):
                d = np.concatenate([x, y]) - zs
                cur = d @ M @ d
                if prev is not None:
                    assert cur <= prev * (1 + 1e-12) + 1e-12
                prev = cur
                x, y = oracle_mod.pdhg_step(lp, tau, sigma, x, y)


def test_pdhg_step_projects(oracle_mod):
    lp = lpgen.adversarial(3)
    x, y = lpgen.random_state(lp, 2, scale=5.0)
    for _ in range(5):
        x, y = oracle_mod.pdhg_step(lp, 0.1, 0.2, x, y)
        assert np.all(x >= lp.lb) and np.all(x <= lp.ub)
        assert np.all(y[lp.row_type == lpgen.ROW_GE] >= 0)
        assert np.all(y[lp.row_type == lpgen.ROW_LE] <= 0)


# ------------------------------------------------------------ trust region

def _trust_region_bruteforce(z, lo, hi, g, r):
    """Minimum of g^T zt over the box and the ball by enumerating clamped sets."""
    idx = [i for i in range(len(z)) if g[i] != 0]
    bound = np.where(g > 0, lo, hi)
    best = np.inf
    for mask in range(1 << len(idx)):
        S = [idx[k] for k in range(len(idx)) if mask >> k & 1]
        F = [i for i in idx if i not in S]
        d2 = sum((bound[i] - z[i]) ** 2 for i in S)
        if not np.isfinite(d2) or d2 > r * r * (1 + 1e-12):
            continue
        g2 = sum(g[i] ** 2 for i in F)
        cand = z.copy()
        for i in S:
            cand[i] = bound[i]
        if g2 > 0:
            lam = np.sqrt(max(r * r - d2, 0.0) / g2)
            for i in F:
                cand[i] = z[i] - lam * g[i]
        if np.any(cand < lo - 1e-12) or np.any(cand > hi + 1e-12):
            continue
        best = min(best, g @ cand)
    return best


def test_trust_region_vs_enumeration(oracle_mod):
    """Algorithm 2 (two-sided form, Section 6.3) against 2^N enumeration, N <= 10."""
    rng = np.random.default_rng(0)
    for _ in range(250):
        N = int(rng.integers(1, 11))
        z = rng.standard_normal(N)
        lo = z - np.where(rng.random(N) < 0.3, np.inf, rng.random(N) * 2)
        hi = z + np.where(rng.random(N) < 0.3, np.inf, rng.random(N) * 2)
        at = rng.random(N) < 0.15  # coordinates sitting on a bound
        lo[at] = z[at]
        g = rng.standard_normal(N)
        g[rng.random(N) < 0.15] = 0.0
        if rng.random() < 0.2:  # ties in the breakpoints
            g = np.round(g, 1)
            lo = z - np.round(z - lo, 1)
        r = float(rng.random() * 3)
        zt, lam = oracle_mod.trust_region(z, lo, hi, g, r)
        assert np.linalg.norm(zt - z) <= r * (1 + 1e-12) + 1e-15
        assert np.all(zt >= lo - 1e-12) and np.all(zt <= hi + 1e-12)
        assert g @ zt == pytest.approx(_trust_region_bruteforce(z, lo, hi, g, r), abs=1e-12)


def test_trust_region_lower_vs_sorted_scan(oracle_mod):
    """Algorithm 2 against a sorted scan of Eq. (lp-trust-region:summation) (N up to 5000)."""
    rng = np.random.default_rng(1)
    for N in [1, 2, 17, 500, 5000]:
        z = rng.standard_normal(N)
        l = z - rng.exponential(1.0, N)
        l[rng.random(N) < 0.2] = -np.inf
        g = rng.exponential(1.0, N) + 1e-3
        full = np.sum(np.where(np.isinf(l), 0, (l - z) ** 2))
        for r in [0.0, 1e-3, 0.5, 3.0, np.sqrt(full) * 0.5]:
            zt, lam = oracle_mod.trust_region_lower(z, l, g, r)
            lam_hat = np.where(np.isinf(l), np.inf, (z - l) / g)
            order = np.argsort(lam_hat)
            lh, d2, g2 = lam_hat[order], ((l - z) ** 2)[order], (g**2)[order]
            # f(lambda) at breakpoint k: clamped = first k+1 entries
            want = None
            cum_d2 = 0.0
            tail_g2 = g2.sum()
            prev = 0.0
            for k in range(N + 1):
                # lambda in [prev, lh[k]) : clamped = first k entries
                if want is None:
                    hi_k = lh[k] if k < N else np.inf
                    f_hi = cum_d2 + (hi_k**2 * tail_g2 if np.isfinite(hi_k) else (np.inf if tail_g2 > 0 else 0))
                    if f_hi >= r * r:
                        want = np.sqrt((r * r - cum_d2) / tail_g2)
                        break
                if k < N:
                    cum_d2 += d2[k]
                    tail_g2 -= g2[k]
            if want is None:
                want = np.inf
            if np.isinf(want):
                assert np.isinf(lam)
            else:
                assert lam == pytest.approx(want, rel=1e-9, abs=1e-14)


def test_trust_region_special_cases(oracle_mod):
    z = np.array([1.0, 2.0, -1.0])
    lo = np.array([0.0, -np.inf, -3.0])
    hi = np.array([np.inf, 5.0, 0.0])
    # r = 0: no movement
    zt, _ = oracle_mod.trust_region(z, lo, hi, np.array([1.0, -1.0, 2.0]), 0.0)
    np.testing.assert_allclose(zt, z)
    # g = 0: nothing moves
    zt, _ = oracle_mod.trust_region(z, lo, hi, np.zeros(3), 1.0)
    np.testing.assert_allclose(zt, z)
    # radius beyond the full clamp: every coordinate at its bound
    g = np.array([1.0, -1.0, 2.0])
    zt, lam = oracle_mod.trust_region(z, lo, hi, g, 100.0)
    assert np.isinf(lam)
    np.testing.assert_allclose(zt, [0.0, 5.0, -3.0])


# ---------------------------------------------------- normalized duality gap

def test_gap_unconstrained_is_norm_of_F(oracle_mod):
    """Eq. (bilinear-1): with Z = R^{m+n}, rho_r(z) = ||F(z)|| for every r > 0."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((6, 9)) * (rng.random((6, 9)) < 0.5)
    c, b = rng.standard_normal(9), rng.standard_normal(6)
    lp = _lp_from_dense(A, c, b, np.full(9, -np.inf), np.full(9, np.inf), np.zeros(6))
    x, y = rng.standard_normal(9), rng.standard_normal(6)
    F = np.concatenate([c - A.T @ y, A @ x - b])
    for r in [1e-3, 0.1, 1.0, 10.0, 1e4]:
        assert oracle_mod.normalized_gap(lp, x, y, r) == pytest.approx(np.linalg.norm(F), rel=1e-12)
    # weighted norm: the dual norm of F in the omega-space
    for om in [0.25, 4.0]:
        Fw = np.concatenate([(c - A.T @ y) / np.sqrt(om), (A @ x - b) * np.sqrt(om)])
        assert oracle_mod.normalized_gap(lp, x, y, 0.7, omega=om) == pytest.approx(
            np.linalg.norm(Fw), rel=1e-12)


def test_gap_monotone_in_r(oracle_mod):
    """Proposition (basic properties): rho_r nonincreasing; Fact: r rho_r nondecreasing."""
    for lp in [lpgen.tiny_standard_form(1, m=40, n=80), lpgen.adversarial(5)]:
        x, y = lpgen.random_state(lp, 3)
        rs = np.geomspace(1e-4, 1e3, 40)
        rho = np.array([oracle_mod.normalized_gap(lp, x, y, r) for r in rs])
        assert np.all(rho > 0)
        assert np.all(np.diff(rho) <= 1e-12 * rho[:-1])
        assert np.all(np.diff(rs * rho) >= -1e-12 * (rs * rho)[1:])


def test_gap_zero_at_planted_optimum(oracle_mod):
    """Proposition (rho-duality-gap): rho_r(z*) = 0 at a saddle point."""
    for lp in [lpgen.tiny_standard_form(0), lpgen.adversarial(9)]:
        scale = 1 + np.abs(lp.c).max() + np.abs(lp.b).max()
        for r in [1e-2, 1.0, 50.0]:
            assert abs(oracle_mod.normalized_gap(lp, lp.x_star, lp.y_star, r)) < 1e-12 * scale


def _K_and_h(A, b, c):
    m, n = A.shape
    K = np.block([[np.eye(n), np.zeros((n, m))],
                  [-A, np.zeros((m, m))],
                  [A, np.zeros((m, m))],
                  [np.zeros((n, n)), -A.T],
                  [-c[None, :], b[None, :]]])
    h = np.concatenate([np.zeros(n), -b, b, -c, [0.0]])
    return K, h


def test_kkt_bounded_by_gap_lemma(oracle_mod):
    """Lemma (bound-kkt-error): ||(h - K z)^+|| <= rho_r(z) sqrt(1 + R^2), z in W_R(0), r <= R."""
    rng = np.random.default_rng(6)
    lp = lpgen.tiny_standard_form(2, m=12, n=25, per_col=3)
    A = lp.dense()
    K, h = _K_and_h(A, lp.b, lp.c)
    for _ in range(60):
        x = np.abs(rng.standard_normal(lp.n)) * (rng.random(lp.n) < 0.6)
        y = rng.standard_normal(lp.m)
        z = np.concatenate([x, y]) * rng.uniform(0.05, 3)
        R = np.linalg.norm(z) * rng.uniform(1.0, 2.0) + 1e-9
        r = R * rng.uniform(0.01, 1.0)
        lhs = np.linalg.norm(np.maximum(h - K @ z, 0))
        rho = oracle_mod.normalized_gap(lp, z[:lp.n], z[lp.n:], r)
        assert lhs <= rho * np.sqrt(1 + R * R) * (1 + 1e-10)


# ------------------------------------------------------------------ KKT

def test_kkt_standard_form_matches_K_blocks(oracle_mod):
    """For Ax = b, x >= 0 the primal and dual residuals are blocks of (h - K z)^+."""
    rng = np.random.default_rng(8)
    lp = lpgen.tiny_standard_form(3, m=15, n=30, per_col=3)
    A = lp.dense()
    K, h = _K_and_h(A, lp.b, lp.c)
    n, m = lp.n, lp.m
    for _ in range(20):
        x = np.abs(rng.standard_normal(n))
        y = rng.standard_normal(m)
        v = np.maximum(h - K @ np.concatenate([x, y]), 0)
        k = oracle_mod.kkt(lp, x, y)
        assert k["rp"] == pytest.approx(np.linalg.norm(v[n:n + 2 * m]), rel=1e-12)
        assert k["rd"] == pytest.approx(np.linalg.norm(v[n + 2 * m:n + 2 * m + n]), rel=1e-12, abs=1e-15)
        assert max(k["pobj"] - k["dobj"], 0) == pytest.approx(v[-1], rel=1e-12, abs=1e-13)


def test_kkt_planted_optimum_zero(oracle_mod):
    for lp in [lpgen.tiny_standard_form(0), lpgen.adversarial(2), lpgen.large_mixed(4, m=300, n=1500)]:
        k = oracle_mod.kkt(lp, lp.x_star, lp.y_star)
        assert k["rel"] < 1e-13


def test_planted_objective_is_lp_optimum():
    """The planted objective equals the LP optimum from an independent LP solver (HiGHS)."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    for lp in [lpgen.tiny_standard_form(1, m=40, n=80), lpgen.adversarial(4),
               lpgen.with_dense_lines(lpgen.large_mixed(2, m=60, n=200), seed=3)]:
        A = lp.dense()
        eq, ge, le = (lp.row_type == 0), (lp.row_type == 1), (lp.row_type == 2)
        A_ub = np.vstack([-A[ge], A[le]])
        b_ub = np.concatenate([-lp.b[ge], lp.b[le]])
        bounds = [(None if np.isinf(l) else l, None if np.isinf(u) else u) for l, u in zip(lp.lb, lp.ub)]
        res = linprog(lp.c, A_ub=A_ub if A_ub.size else None, b_ub=b_ub if A_ub.size else None,
                      A_eq=A[eq], b_eq=lp.b[eq], bounds=bounds, method="highs")
        assert res.status == 0
        assert res.fun == pytest.approx(lp.obj_star, rel=1e-7, abs=1e-7)


def test_dense_lines_keep_the_planted_optimum(oracle_mod):
    """with_dense_lines adds a full row and a full column and keeps (x*, y*) optimal:
    zero KKT error at the planted pair (complementary reduced costs, y* = 0 on the
    new row, x* = 0 with a positive reduced cost on the new column)."""
    base = lpgen.large_mixed(5, m=400, n=1500)
    d = lpgen.with_dense_lines(base, seed=2)
    assert (d.m, d.n) == (base.m + 1, base.n + 1)
    assert np.diff(d.row_ptr)[-1] == d.n  # the new row: every old column and the new one
    assert np.bincount(d.col_idx, minlength=d.n)[-1] == d.m  # the new column every row
    k = oracle_mod.kkt(d, d.x_star, d.y_star)
    assert k["rel"] < 1e-13
    assert d.obj_star == pytest.approx(base.obj_star, rel=1e-14)


def test_sigma_max_power_iteration(oracle_mod):
    for lp in [lpgen.tiny_standard_form(0), lpgen.adversarial(1)]:
        assert oracle_mod.sigma_max(lp) == pytest.approx(np.linalg.norm(lp.dense(), 2), rel=1e-6)


# ------------------------------------------------------------- Algorithm 1

def _vertex_enumeration_opt(A, b, c):
    """min c^T x, Ax = b, x >= 0 by enumerating all bases (tiny LPs)."""
    m, n = A.shape
    best = np.inf
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-10:
            continue
        xB = np.linalg.solve(AB, b)
        if np.all(xB >= -1e-10):
            best = min(best, c[list(B)] @ xB)
    return best


def test_solve_matches_vertex_enumeration(oracle_mod):
    rng = np.random.default_rng(12)
    done = 0
    for trial in range(40):
        m, n = 3, 7
        A = rng.standard_normal((m, n))
        x_feas = np.abs(rng.standard_normal(n))
        b = A @ x_feas
        c = np.abs(rng.standard_normal(n)) + A.T @ rng.standard_normal(m) * 0.3
        opt = _vertex_enumeration_opt(A, b, c)
        if not np.isfinite(opt):
            continue
        lp = _lp_from_dense(A, c, b, np.zeros(n), np.full(n, np.inf), np.zeros(m))
        eta = 0.9 / np.linalg.norm(A, 2)
        res = oracle_mod.solve(lp, eta, tol=1e-10, max_iter=400000, check_every=30)
        if res.status != 0:
            continue
        p = c @ res.x_sol
        assert p == pytest.approx(opt, rel=1e-7, abs=1e-7)
        done += 1
    assert done >= 20


def test_solve_reaches_planted_objective(oracle_mod):
    lp = lpgen.tiny_standard_form(2)
    eta = 0.9 / oracle_mod.sigma_max(lp)
    res = oracle_mod.solve(lp, eta, tol=1e-8, max_iter=200000, check_every=64)
    assert res.status == 0
    k = oracle_mod.kkt(lp, res.x_sol, res.y_sol)
    assert k["rel"] <= 1e-8
    assert k["pobj"] == pytest.approx(lp.obj_star, rel=1e-7)


def test_adaptive_restart_gap_sequence_contracts(oracle_mod):
    """Eq. (adaptive-restart-scheme): each stored restart gap is <= beta times the previous one."""
    lp = lpgen.tiny_standard_form(1)
    eta = 0.9 / oracle_mod.sigma_max(lp)
    beta = np.exp(-1)
    res = oracle_mod.solve(lp, eta, tol=1e-9, max_iter=60000, check_every=32, beta=beta)
    tr = res.trace
    rest = tr[tr[:, 2] == 1]
    assert len(rest) >= 5
    rho = rest[:, 1]
    assert np.all(rho[1:] <= beta * rho[:-1] * (1 + 1e-15))
    # between restarts the rule did not fire: rho > beta * stored
    stored = None
    for row in tr:
        if stored is not None and row[2] == 0:
            assert row[1] > beta * stored
        if row[2] == 1:
            stored = row[1]


def test_fixed_restart_lengths(oracle_mod):
    lp = lpgen.tiny_standard_form(0, m=30, n=60)
    eta = 0.9 / oracle_mod.sigma_max(lp)
    res = oracle_mod.solve(lp, eta, tol=1e-14, max_iter=1000, check_every=25,
                           restart_scheme=oracle_mod.RESTART_FIXED, fixed_len=100)
    rest = res.trace[res.trace[:, 2] == 1][:, 0]
    np.testing.assert_array_equal(rest, np.arange(100, 1001, 100))


def test_figure1_restarted_average_beats_plain(oracle_mod):
    """Figure 1: L(x, y) = x y, eta = 0.2, fixed restart length 25, 50 iterations.

    The restarted average ends closer to the solution (0, 0) than both the
    last and the average iterate of plain PDHG.  x y = -y^T A x with A = [-1].
    """
    lp = _lp_from_dense(np.array([[-1.0]]), [0.0], [0.0], [-np.inf], [np.inf], [0])
    z0x, z0y = np.array([1.0]), np.array([1.0])
    plain = oracle_mod.solve(lp, 0.2, tol=1e-300, max_iter=50, check_every=25,
                             restart_scheme=oracle_mod.RESTART_NONE, x_init=z0x, y_init=z0y)
    rest = oracle_mod.solve(lp, 0.2, tol=1e-300, max_iter=50, check_every=25,
                            restart_scheme=oracle_mod.RESTART_FIXED, fixed_len=25,
                            x_init=z0x, y_init=z0y)
    d_last = np.hypot(plain.x[0], plain.y[0])
    d_avg = np.hypot(plain.xbar[0], plain.ybar[0])
    d_rest = np.hypot(rest.x0[0], rest.y0[0])  # z^{2,0}: average restarted twice
    assert rest.restarts == 2
    assert d_rest < d_last and d_rest < d_avg


def test_multicommodity_oracle_matches_highs(oracle_mod):
    """Multicommodity grid LPs (no planted optimum): the oracle's solve reaches
    relative KKT 1e-8 and HiGHS's optimal objective; power iteration finds
    sigma_max although the top singular vector is orthogonal to the all-ones
    vector on these symmetric network matrices."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    for side, K, seed in [(5, 2, 4), (6, 2, 1)]:
        d = lpgen.multicommodity_grid(seed, side=side, commodities=K)
        A = d.dense()
        assert oracle_mod.sigma_max(d) == pytest.approx(np.linalg.norm(A, 2), rel=1e-6)
        eq, le = d.row_type == 0, d.row_type == 2
        res = linprog(d.c, A_ub=A[le], b_ub=d.b[le], A_eq=A[eq], b_eq=d.b[eq], bounds=(0, None),
                      method="highs")
        r = oracle_mod.solve(d, 0.9 / oracle_mod.sigma_max(d), tol=1e-8, max_iter=200000,
                             check_every=64)
        assert r.status == 0
        k = oracle_mod.kkt(d, r.x_sol, r.y_sol)
        assert k["rel"] <= 1e-8
        assert k["pobj"] == pytest.approx(res.fun, rel=1e-7)
