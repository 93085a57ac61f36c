"""Pins of the oracle's restart schemes and of its primal weight.

Each test fixes a branch of ``orc_solve`` by a property the paper states, not
by a second copy of the branch:

* the primal weight omega (Section 7: tau = eta/omega, sigma = eta*omega) and
  the omega-weighted norm of the normalized gap are a change of variables
  (the rescaling of the Section 2 footnote): a run with weight omega equals,
  after x' = sqrt(omega) x and y' = y / sqrt(omega), the omega = 1 run on the
  LP with c' = c / sqrt(omega), b' = sqrt(omega) b and bounds
  sqrt(omega) (l, u), whose steps and gaps are pinned elsewhere;
* the flexible scheme (Remark "Flexible restarts", Eq. flexible-restart-
  scheme) replaces the average by the last iterate exactly when the last
  iterate has the strictly smaller normalized gap, at every check, and then
  applies the adaptive test to the chosen candidate;
* the first restart of the adaptive scheme (Eq. adaptive-restart-scheme,
  n = 0) fires at the first check with t >= tau^0, whatever the gaps;
* a schedule of restart flags (the unrolled map the adjoint differentiates)
  reproduces the run whose decisions it copies, and an all-zero schedule is
  the run without restarts;
* restart points never move away from an optimum in the norm in which the
  PDHG step is non-expansive, so they stay within twice the starting
  distance of the starting point (the boundedness proposition of Section 4).
"""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

NEVER = -1.0  # a tolerance no relative KKT error meets: runs end at max_iter


def _mixed_lp(seed=5):
    """A small LP with EQ/GE/LE rows, every bound kind, empty lines."""
    return lpgen.adversarial(seed, m=40, n=90, dense_row=True)


def _eta(oracle_mod, lp):
    return 0.9 / oracle_mod.sigma_max(lp)


def _scaled_lp(lp, omega):
    s = np.sqrt(omega)
    return lpgen.LPData(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.c / s, lp.b * s,
                        lp.lb * s, lp.ub * s, lp.row_type)


@pytest.mark.parametrize("omega,rtol", [(4.0, 0.0), (0.25, 0.0), (0.3, 1e-11), (7.5, 1e-11)])
@pytest.mark.parametrize("scheme", ["adaptive", "flexible"])
def test_primal_weight_is_the_footnote_rescaling(oracle_mod, omega, rtol, scheme):
    """omega != 1 against the omega = 1 run of the rescaled LP.

    For omega = 4 and 1/4 (sqrt(omega) a power of two) every scaling is exact
    in binary floating point, so the two runs agree bit for bit; otherwise to
    rounding.  A swapped omega in tau/sigma, in the weighted radius or in the
    gap's rescaling changes the iterates, the radii or the restart flags."""
    lp = _mixed_lp()
    eta = _eta(oracle_mod, lp)
    sch = {"adaptive": oracle_mod.RESTART_ADAPTIVE, "flexible": oracle_mod.RESTART_FLEXIBLE}[scheme]
    rng = np.random.default_rng(11)
    x_init = np.clip(rng.standard_normal(lp.n), lp.lb, lp.ub)
    y_init = rng.standard_normal(lp.m)
    y_init[lp.row_type == 1] = np.abs(y_init[lp.row_type == 1])
    y_init[lp.row_type == 2] = -np.abs(y_init[lp.row_type == 2])
    s = np.sqrt(omega)
    K, iters = 8, 480
    a = oracle_mod.solve(lp, eta, omega=omega, tol=NEVER, max_iter=iters, check_every=K,
                         restart_scheme=sch, x_init=x_init, y_init=y_init)
    b = oracle_mod.solve(_scaled_lp(lp, omega), eta, omega=1.0, tol=NEVER, max_iter=iters,
                         check_every=K, restart_scheme=sch, x_init=s * x_init, y_init=y_init / s)
    assert a.iters == b.iters == iters
    assert a.restarts == b.restarts and a.restarts >= 3
    np.testing.assert_array_equal(a.trace[:, 2], b.trace[:, 2])  # restart flags
    for col, name in [(1, "rho"), (5, "radius")]:
        np.testing.assert_allclose(a.trace[:, col], b.trace[:, col], rtol=rtol, atol=0, err_msg=name)
    for k, sc in [("x", s), ("xbar", s), ("x0", s), ("y", 1 / s), ("ybar", 1 / s), ("y0", 1 / s)]:
        want = getattr(b, k)
        got = getattr(a, k) * sc
        tol = rtol * max(1.0, float(np.abs(want).max()))
        np.testing.assert_allclose(got, want, rtol=0, atol=tol, err_msg=k)


def test_weighted_radius_scales_as_the_footnote(oracle_mod):
    """||z - z0||_omega of a run with weight omega is the Euclidean distance in
    the rescaled variables; at omega = 1 it is the Euclidean norm."""
    rng = np.random.default_rng(2)
    x, x0 = rng.standard_normal(7), rng.standard_normal(7)
    y, y0 = rng.standard_normal(4), rng.standard_normal(4)
    e = np.linalg.norm(np.concatenate([x - x0, y - y0]))
    assert oracle_mod.weighted_dist(x, y, x0, y0, 1.0) == pytest.approx(e, rel=1e-15)
    for omega in (4.0, 0.25):  # exact: sqrt(omega) is a power of two
        s = np.sqrt(omega)
        e = np.linalg.norm(np.concatenate([s * (x - x0), (y - y0) / s]))
        assert oracle_mod.weighted_dist(x, y, x0, y0, omega) == pytest.approx(e, rel=1e-15)
    # only the primal part grows with omega
    assert oracle_mod.weighted_dist(x, y0, x0, y0, 4.0) == pytest.approx(
        2.0 * np.linalg.norm(x - x0), rel=1e-15)
    assert oracle_mod.weighted_dist(x0, y, x0, y0, 4.0) == pytest.approx(
        0.5 * np.linalg.norm(y - y0), rel=1e-15)


def _state_before_check(oracle_mod, lp, eta, K, c, sch, **kw):
    """The candidates of check c: run to K c - 1 iterations, take one more
    PDHG step (pinned) and the uniform average of Algorithm 1 by hand."""
    r = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=K * c - 1, check_every=K,
                         restart_scheme=sch, **kw)
    t = r.inner_t  # iterations averaged since the last restart
    x, y = oracle_mod.pdhg_step(lp, eta / kw.get("omega", 1.0), eta * kw.get("omega", 1.0), r.x, r.y)
    xbar = (t * r.xbar + x) / (t + 1)
    ybar = (t * r.ybar + y) / (t + 1)
    return r, x, y, xbar, ybar


@pytest.mark.parametrize("seed,omega", [(3, 1.0), (8, 1.0), (3, 4.0)])
def test_flexible_restart_takes_the_smaller_gap(oracle_mod, seed, omega):
    """Eq. (flexible-restart-scheme) at every check of a run: the candidate is
    the last iterate iff its normalized gap (Eq. rhorz, pinned) at radius
    ||z - z^{n,0}|| is strictly below the average's; the adaptive test then
    runs on the candidate, and a restart moves z^{n,0} and z to it."""
    lp = _mixed_lp(seed)
    eta = _eta(oracle_mod, lp)
    K, checks = 8, 24
    kw = dict(omega=omega, x_init=np.clip(np.zeros(lp.n), lp.lb, lp.ub))
    picked_current = restarted_to_current = 0
    for c in range(1, checks + 1):
        r, x, y, xbar, ybar = _state_before_check(oracle_mod, lp, eta, K, c,
                                                  oracle_mod.RESTART_FLEXIBLE, **kw)
        ra = oracle_mod.weighted_dist(xbar, ybar, r.x0, r.y0, omega)
        rc = oracle_mod.weighted_dist(x, y, r.x0, r.y0, omega)
        ga = oracle_mod.normalized_gap(lp, xbar, ybar, ra, omega=omega) if ra > 0 else 0.0
        gc = oracle_mod.normalized_gap(lp, x, y, rc, omega=omega) if rc > 0 else 0.0
        take_current = gc < ga
        cand_x, cand_y = (x, y) if take_current else (xbar, ybar)
        rho, rad = (gc, rc) if take_current else (ga, ra)
        after = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=K * c, check_every=K,
                                 restart_scheme=oracle_mod.RESTART_FLEXIBLE, **kw)
        row = after.trace[c - 1]
        assert row[0] == K * c
        assert row[1] == pytest.approx(rho, rel=1e-12, abs=1e-300), c
        assert row[5] == pytest.approx(rad, rel=1e-12), c
        # the average after the check is the candidate (restart or not)
        np.testing.assert_allclose(after.xbar, cand_x, rtol=0, atol=1e-13 * max(1, np.abs(cand_x).max()))
        np.testing.assert_allclose(after.ybar, cand_y, rtol=0, atol=1e-13 * max(1, np.abs(cand_y).max()))
        if r.restarts == 0:
            want_restart = r.inner_t + 1 >= K  # tau^0 = K (first check)
        else:
            want_restart = rho <= np.exp(-1.0) * r.rho_stored
        assert bool(row[2]) == want_restart, c
        if want_restart:
            np.testing.assert_allclose(after.x0, cand_x, rtol=0, atol=1e-13 * max(1, np.abs(cand_x).max()))
            np.testing.assert_allclose(after.y0, cand_y, rtol=0, atol=1e-13 * max(1, np.abs(cand_y).max()))
            np.testing.assert_array_equal(after.x, after.x0)
            np.testing.assert_array_equal(after.y, after.y0)
            assert after.rho_stored == row[1]
        else:
            np.testing.assert_array_equal(after.x0, r.x0)
        picked_current += take_current
        restarted_to_current += take_current and want_restart
    # the run exercises both branches of the choice
    assert 0 < picked_current < checks
    assert restarted_to_current > 0


def test_adaptive_restart_compares_the_average(oracle_mod):
    """The adaptive scheme keeps the average as its candidate even when the
    last iterate has the smaller gap (that choice is the flexible scheme's)."""
    lp = _mixed_lp(3)
    eta = _eta(oracle_mod, lp)
    K = 8
    seen = 0
    for c in range(1, 25):
        r, x, y, xbar, ybar = _state_before_check(oracle_mod, lp, eta, K, c,
                                                  oracle_mod.RESTART_ADAPTIVE)
        ra = oracle_mod.weighted_dist(xbar, ybar, r.x0, r.y0)
        after = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=K * c, check_every=K,
                                 restart_scheme=oracle_mod.RESTART_ADAPTIVE)
        row = after.trace[c - 1]
        assert row[5] == pytest.approx(ra, rel=1e-12)
        if ra > 0:
            assert row[1] == pytest.approx(oracle_mod.normalized_gap(lp, xbar, ybar, ra), rel=1e-12)
        if row[2]:
            np.testing.assert_allclose(after.x0, xbar, rtol=0, atol=1e-13 * max(1, np.abs(xbar).max()))
            seen += 1
    assert seen >= 2


@pytest.mark.parametrize("tau0_mult,first", [(None, 1), (0, 1), (3, 3), (2.5, 3), (5, 5)])
def test_first_restart_at_tau0(oracle_mod, tau0_mult, first):
    """Eq. (adaptive-restart-scheme), n = 0: restart at the first check with
    t >= tau^0 (tau^0 = 1 fires at the first check; the default is K),
    never earlier whatever the gap; the stored gap is that check's."""
    lp = _mixed_lp(4)
    eta = _eta(oracle_mod, lp)
    K = 8
    tau0 = None if tau0_mult is None else (1 if tau0_mult == 0 else int(tau0_mult * K))
    r = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=K * 12, check_every=K, tau0=tau0,
                         restart_scheme=oracle_mod.RESTART_ADAPTIVE)
    flags = r.trace[:, 2].astype(bool)
    assert not flags[:first - 1].any()
    assert flags[first - 1]
    assert np.all(np.isfinite(r.trace[:first, 1]))  # gaps are evaluated before the first restart
    # the rule of n >= 1 takes over after the first restart: later restarts
    # need the gap to fall by beta against the stored one
    stored = r.trace[first - 1, 1]
    for row in r.trace[first:]:
        assert bool(row[2]) == (row[1] <= np.exp(-1.0) * stored)
        if row[2]:
            stored = row[1]


def test_schedule_reproduces_the_runs_it_copies(oracle_mod):
    """SCHEDULE (decisions given from outside) with an adaptive run's restart
    flags is that run; with no flags it is the run without restarts."""
    lp = _mixed_lp(6)
    eta = _eta(oracle_mod, lp)
    K, iters = 8, 400
    for sch in (oracle_mod.RESTART_ADAPTIVE, oracle_mod.RESTART_FLEXIBLE,
                oracle_mod.RESTART_FIXED):
        if sch == oracle_mod.RESTART_FLEXIBLE:
            continue  # a flexible swap without a restart is not a restart flag
        a = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=iters, check_every=K, restart_scheme=sch,
                             fixed_len=3 * K)
        assert a.restarts >= 2
        s = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=iters, check_every=K,
                             restart_scheme=oracle_mod.RESTART_SCHEDULE,
                             schedule=a.trace[:, 2].astype(np.int8))
        assert s.restarts == a.restarts
        for k in ("x", "y", "xbar", "ybar", "x0", "y0"):
            np.testing.assert_array_equal(getattr(s, k), getattr(a, k), err_msg=k)
    none = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=iters, check_every=K,
                            restart_scheme=oracle_mod.RESTART_NONE)
    zero = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=iters, check_every=K,
                            restart_scheme=oracle_mod.RESTART_SCHEDULE,
                            schedule=np.zeros(iters // K, np.int8))
    assert none.restarts == zero.restarts == 0
    for k in ("x", "y", "xbar", "ybar"):
        np.testing.assert_array_equal(getattr(zero, k), getattr(none, k), err_msg=k)
    # a schedule shorter than the run restarts nowhere after its end
    short = oracle_mod.solve(lp, eta, tol=NEVER, max_iter=iters, check_every=K,
                             restart_scheme=oracle_mod.RESTART_SCHEDULE,
                             schedule=np.ones(3, np.int8))
    assert short.restarts == 3
    assert list(np.nonzero(short.trace[:, 2])[0]) == [0, 1, 2]


@pytest.mark.parametrize("scheme", ["adaptive", "flexible", "fixed"])
def test_restart_points_stay_in_the_ball(oracle_mod, scheme):
    """Proposition (restart points stay bounded) of Section 4, for PDHG: with
    z* optimal and ||.||_M the norm in which the PDHG step is non-expansive,
    every average satisfies ||z* - zbar^{n,t}|| <= ||z* - z^{n,0}||, so
    ||z* - z^{n,0}|| never grows from one restart to the next and every
    restart point lies within 2 ||z^{0,0} - z*|| of z^{0,0}.  Checked at
    every one of 40 checks (the average before the decision and the restart
    point after it) on a planted LP with EQ/GE/LE rows and every bound kind."""
    lp = lpgen.adversarial(11, m=25, n=50)
    A = lp.dense()
    eta = 0.95 / np.linalg.norm(A, 2)
    omega = 2.0
    tau, sigma = eta / omega, eta * omega
    M = np.block([[np.eye(lp.n) / tau, A.T], [A, np.eye(lp.m) / sigma]])
    zs = np.concatenate([lp.x_star, lp.y_star])

    def norm(d):
        return float(np.sqrt(d @ M @ d))

    sch = {"adaptive": oracle_mod.RESTART_ADAPTIVE, "flexible": oracle_mod.RESTART_FLEXIBLE,
           "fixed": oracle_mod.RESTART_FIXED}[scheme]
    x_init, y_init = lpgen.random_state(lp, 4, scale=3.0)
    z00 = np.concatenate([x_init, y_init])
    d0 = norm(z00 - zs)
    K = 8
    prev = d0
    restarts = 0
    for c in range(1, 41):
        r = oracle_mod.solve(lp, eta, omega=omega, tol=NEVER, max_iter=K * c, check_every=K,
                             restart_scheme=sch, fixed_len=3 * K, x_init=x_init, y_init=y_init)
        zbar = np.concatenate([r.xbar, r.ybar])
        z0 = np.concatenate([r.x0, r.y0])
        dn = norm(z0 - zs)
        assert norm(zbar - zs) <= prev * (1 + 1e-12) + 1e-12, c
        assert dn <= prev * (1 + 1e-12) + 1e-12, c
        assert norm(z0 - z00) <= 2 * d0 * (1 + 1e-12), c
        prev = dn
        restarts = r.restarts
    assert restarts >= 4
