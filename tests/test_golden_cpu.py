"""The oracle against the hand-derived worked examples under tests/golden.

Normalized duality gap on the linear trust region (Section 6.3), the relative
KKT error, and PDHG iterates on the bilinear example of Section 5.2.  The
expected values are closed forms written out in the fixtures.
"""
import numpy as np
import pytest

import golden

GAP = golden.load("normalized_gap_hand.json")["cases"]
KKT = golden.load("kkt_hand.json")["cases"]
BIL = golden.load("bilinear_pdhg_hand.json")


@pytest.mark.parametrize("case", GAP, ids=[c["name"] for c in GAP])
def test_normalized_gap_hand(oracle_mod, case):
    lp = golden.lp_data(case)
    got = oracle_mod.normalized_gap(lp, case["x"], case["y"], case["r"], omega=case["omega"])
    assert got == pytest.approx(golden.value(case["rho"]), rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("case", KKT, ids=[c["name"] for c in KKT])
def test_kkt_hand(oracle_mod, case):
    got = oracle_mod.kkt(golden.lp_data(case), case["x"], case["y"])
    for k in ["rp", "rd", "pobj", "dobj", "rel"]:
        assert got[k] == pytest.approx(golden.value(case[k]), rel=1e-14, abs=1e-15), k


def _bilinear():
    return golden.lp_data({"A": [[-1.0]], "b": [0.0], "row_type": [0], "c": [0.0],
                           "lb": [None], "ub": [None]})


def test_bilinear_pdhg_hand(oracle_mod):
    lp = _bilinear()
    eta = BIL["eta"]
    x, y = np.array([BIL["x0"]]), np.array([BIL["y0"]])
    for it in BIL["iterates"]:
        x, y = oracle_mod.pdhg_step(lp, eta, eta, x, y)
        assert x[0] == pytest.approx(golden.value(it["x"]), rel=1e-15), it["t"]
        assert y[0] == pytest.approx(golden.value(it["y"]), rel=1e-15), it["t"]


def test_bilinear_average_hand(oracle_mod):
    """Algorithm 1 with no restarts: the average of iterates 1..3."""
    res = oracle_mod.solve(_bilinear(), BIL["eta"], tol=1e-300, max_iter=3, check_every=1,
                           restart_scheme=oracle_mod.RESTART_NONE,
                           x_init=np.array([BIL["x0"]]), y_init=np.array([BIL["y0"]]))
    assert res.iters == 3
    assert res.x[0] == pytest.approx(golden.value(BIL["iterates"][-1]["x"]), rel=1e-15)
    assert res.xbar[0] == pytest.approx(golden.value(BIL["average_t3"]["x"]), rel=1e-15)
    assert res.ybar[0] == pytest.approx(golden.value(BIL["average_t3"]["y"]), rel=1e-15)


FLEX = golden.load("flexible_restart_hand.json")


@pytest.mark.parametrize("case", FLEX["cases"], ids=[c["name"] for c in FLEX["cases"]])
def test_flexible_restart_hand(oracle_mod, case):
    """Remark (Flexible restarts): check by check, the chosen candidate's gap
    and radius, the restart flag and the restart point, then the end state."""
    lp = golden.lp_data(FLEX["lp"])
    scheme = {"flexible": oracle_mod.RESTART_FLEXIBLE,
              "adaptive": oracle_mod.RESTART_ADAPTIVE}[case["scheme"]]
    kw = dict(tol=FLEX["tol"], check_every=FLEX["check_every"], tau0=FLEX["tau0"],
              restart_scheme=scheme, x_init=np.array([FLEX["x_init"]]), y_init=np.zeros(0))
    for i, ck in enumerate(case["checks"]):
        r = oracle_mod.solve(lp, case["eta"], max_iter=ck["iter"], **kw)
        row = r.trace[i]
        assert row[0] == ck["iter"]
        assert row[1] == pytest.approx(golden.value(ck["rho"]), rel=1e-15), ck
        assert row[5] == pytest.approx(golden.value(ck["radius"]), rel=1e-15), ck
        assert row[2] == ck["restarted"], ck
        assert r.x0[0] == pytest.approx(golden.value(ck["x0_after"]), rel=1e-15), ck
    r = oracle_mod.solve(lp, case["eta"], max_iter=1000, **kw)
    f = case["final"]
    assert r.status == oracle_mod.STATUS_OK
    assert (r.iters, r.restarts, r.returned) == (f["iters"], f["restarts"], f["returned"])
    for k in ("x", "xbar", "x0"):
        assert getattr(r, k)[0] == pytest.approx(golden.value(f[k]), rel=1e-15, abs=1e-300), k


def test_openmp_build_is_bitwise_the_default_build(oracle_mod):
    """The OpenMP build (used only to time the oracle on all cores) splits
    loops without dependences between iterations: same bits as the default build."""
    from paper_2105_12715_gb300 import lpgen

    try:
        oracle_mod.build(openmp=True)
    except Exception as e:  # noqa: BLE001
        pytest.skip(f"no OpenMP toolchain: {e}")
    d = lpgen.adversarial(5, m=40, n=90, dense_row=True)
    eta = 0.9 / oracle_mod.sigma_max(d)
    a = oracle_mod.solve(d, eta, tol=1e-300, max_iter=320, check_every=16)
    b = oracle_mod.solve(d, eta, tol=1e-300, max_iter=320, check_every=16, openmp=True)
    for k in ("x", "y", "xbar", "ybar", "x0", "y0", "trace"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)
