"""Failure paths of lp_solve, induced from the host (no device fault).

* Divergence: PDHG needs eta <= 1/sigma_max(A) (Section 2); with
  eta = 5/sigma_max the iterates grow geometrically until the relative KKT
  error of a check is no longer finite, and lp_solve must stop with
  LP_ERR_NUMERICAL at that check -- the one where the oracle stops too.
* Iteration limit: lp_solve returns LP_ITER_LIMIT, and lp_get_solution
  returns the candidate with the smaller relative KKT error at the last
  check (the average wins ties; Table 3 counts either candidate), as the
  oracle does.
"""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lpm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2105_12715_gb300 import lp

    lp.load()
    return lp


@pytest.mark.parametrize("precision", [0, 1])
def test_divergent_step_stops_numerical(lpm, oracle_mod, precision):
    data = lpgen.tiny_standard_form(1)
    eta = 5.0 / oracle_mod.sigma_max(data)
    K = 32
    with lpm.LP(data, eta=eta, check_every=K, max_iter=200 * K, precision=precision) as g:
        status = g.solve(1e-8)
        info = g.info()
    ref = oracle_mod.solve(data, eta, tol=1e-8, max_iter=200 * K, check_every=K)
    assert ref.status == oracle_mod.STATUS_NUMERICAL
    assert status == lpm.LP_ERR_NUMERICAL
    assert info.status == lpm.LP_ERR_NUMERICAL
    # stopped at a check, within a few checks of the oracle's (FMA rounding and,
    # for mixed precision, FP32 overflow move the first non-finite check)
    assert info.iters % K == 0
    assert abs(info.iters - ref.iters) <= (K if precision == 0 else 8 * K)
    assert info.iters < 200 * K
    # the handle stays usable: a fresh solve with a valid step runs
    with lpm.LP(data, eta=0.9 / oracle_mod.sigma_max(data), check_every=K, max_iter=4 * K) as g:
        assert g.solve(1e-8) == lpm.LP_ITER_LIMIT


def test_iteration_limit_returns_best_candidate(lpm, oracle_mod):
    data = lpgen.large_mixed(3, m=600, n=2500)
    eta = 0.9 / oracle_mod.sigma_max(data)
    K, iters = 32, 6 * 32
    with lpm.LP(data, eta=eta, check_every=K, max_iter=iters, autotune=0) as g:
        status = g.solve(1e-12)
        info = g.info()
        st = g.state()
        x, y = g.solution()
    ref = oracle_mod.solve(data, eta, tol=1e-12, max_iter=iters, check_every=K)
    assert status == lpm.LP_ITER_LIMIT and ref.status == oracle_mod.STATUS_ITER_LIMIT
    assert info.iters == ref.iters == iters
    want_ret = 0 if info.kkt_avg[4] <= info.kkt_cur[4] else 1
    assert info.returned == want_ret == ref.returned
    xs, ys = (st["xbar"], st["ybar"]) if want_ret == 0 else (st["x"], st["y"])
    np.testing.assert_array_equal(x, xs)
    np.testing.assert_array_equal(y, ys)
    scale = max(1.0, float(np.abs(ref.x_sol).max()))
    assert float(np.abs(x - ref.x_sol).max()) <= 1e-9 * scale
    assert float(np.abs(y - ref.y_sol).max()) <= 1e-9 * max(1.0, float(np.abs(ref.y_sol).max()))
    # its relative KKT error is the smaller of the two the last check reported
    k = oracle_mod.kkt(data, x, y)
    assert k["rel"] == pytest.approx(min(info.kkt_avg[4], info.kkt_cur[4]), rel=1e-8)
