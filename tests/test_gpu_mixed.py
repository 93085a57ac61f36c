"""Mixed precision (FP32 iterations on scaled corrections re-formed in FP64 at
every restart) against the FP64 oracle.

Stated error: over the first iterations the mixed iterates differ from the
FP64 oracle's by FP32 rounding, bounded here by 1e-5 relative (max-abs
difference over max(1, max|oracle|)); full solves must reach the same FP64
relative KKT tolerance as the FP64 path (checked with the oracle's KKT),
with the planted objective to 1e-7.
"""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

pytestmark = pytest.mark.gpu

MIX_TOL = 1e-5


@pytest.fixture(scope="module")
def lpm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2105_12715_gb300 import lp

    lp.load()
    return lp


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


@pytest.mark.parametrize("data", [lpgen.tiny_standard_form(0), lpgen.adversarial(7),
                                  lpgen.large_mixed(11, m=3001, n=15007)],
                         ids=["tiny", "adversarial", "mixed3k"])
def test_mixed_iterates_track_fp64_oracle(lpm, oracle_mod, data):
    eta = 0.9 / oracle_mod.sigma_max(data)
    iters = 200
    with lpm.LP(data, eta=eta, check_every=32, max_iter=iters, precision=lpm.LP_PRECISION_MIXED,
                long_row_threshold=16) as g:
        assert g.solve(1e-300) == lpm.LP_ITER_LIMIT
        st = g.state()
        tr = g.trace()
    # both sides start at the projection of zero onto X x Y
    x_start = np.clip(np.zeros(data.n), data.lb, data.ub)
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=iters, check_every=32, x_init=x_start)
    for k in ("x", "y", "xbar", "ybar", "x0", "y0"):
        assert rel_err(st[k], getattr(ref, k)) <= MIX_TOL, k
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_full_solve_reaches_fp64_tolerance(lpm, oracle_mod, seed):
    data = lpgen.tiny_standard_form(seed)
    eta = 0.9 / oracle_mod.sigma_max(data)
    with lpm.LP(data, eta=eta, check_every=64, max_iter=400000,
                precision=lpm.LP_PRECISION_MIXED) as g:
        status = g.solve(1e-8)
        info = g.info()
        x, y = g.solution()
    assert status == lpm.LP_OK, info
    k = oracle_mod.kkt(data, x, y)
    assert k["rel"] <= 1e-8
    assert k["pobj"] == pytest.approx(data.obj_star, rel=1e-7)
    assert np.all(x >= data.lb) and np.all(x <= data.ub)


def test_mixed_warm_start_and_bounds(lpm, oracle_mod):
    data = lpgen.adversarial(3)
    eta = 0.9 / oracle_mod.sigma_max(data)
    x0, y0 = lpgen.random_state(data, 9)
    with lpm.LP(data, eta=eta, check_every=16, max_iter=96,
                precision=lpm.LP_PRECISION_MIXED) as g:
        g.set_state(x0, y0)
        g.solve(1e-300)
        st = g.state()
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=96, check_every=16, x_init=x0, y_init=y0)
    for k in ("x", "y", "xbar", "ybar"):
        assert rel_err(st[k], getattr(ref, k)) <= MIX_TOL, k
    assert np.all(st["x"] >= data.lb) and np.all(st["x"] <= data.ub)


@pytest.mark.parametrize("precision", [0, 1])
def test_multicommodity_solve_matches_highs(lpm, oracle_mod, precision):
    """Multicommodity grid LP (all values +-1, no planted optimum): FP64 and
    mixed GPU solves reach relative KKT 1e-8 (oracle's KKT) and HiGHS's
    optimal objective; the first 128 FP64 iterations match the oracle."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    d = lpgen.multicommodity_grid(2, side=8, commodities=3)
    A = d.dense()
    eq, le = d.row_type == 0, d.row_type == 2
    res = linprog(d.c, A_ub=A[le], b_ub=d.b[le], A_eq=A[eq], b_eq=d.b[eq], bounds=(0, None),
                  method="highs")
    with lpm.LP(d, check_every=64, max_iter=400000, precision=precision) as g:
        assert g.info().sigma_max == pytest.approx(np.linalg.norm(A, 2), rel=1e-6)
        assert g.solve(1e-8) == lpm.LP_OK
        x, y = g.solution()
    k = oracle_mod.kkt(d, x, y)
    assert k["rel"] <= 1e-8
    assert k["pobj"] == pytest.approx(res.fun, rel=1e-7)
    if precision == 0:
        eta = 0.9 / oracle_mod.sigma_max(d)
        with lpm.LP(d, eta=eta, check_every=64, max_iter=128) as g:
            g.solve(1e-300)
            st = g.state()
        ref = oracle_mod.solve(d, eta, tol=1e-300, max_iter=128, check_every=64)
        for key in ("x", "y", "xbar", "ybar"):
            assert rel_err(st[key], getattr(ref, key)) <= 1e-9, key
