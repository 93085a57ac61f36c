"""The CUDA path (through the C ABI) against the hand-derived worked examples
under tests/golden: normalized duality gap (Section 6.3) and the PDHG
iterates and average on the bilinear example of Section 5.2.

Tolerance 1e-12 relative: these are a handful of FP64 operations on each
side, far inside the 1e-9 of the iterate parity tests.
"""
import numpy as np
import pytest

import golden

pytestmark = pytest.mark.gpu

GAP = golden.load("normalized_gap_hand.json")["cases"]
BIL = golden.load("bilinear_pdhg_hand.json")


@pytest.fixture(scope="module")
def lpm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2105_12715_gb300 import lp

    lp.load()
    return lp


@pytest.mark.parametrize("case", GAP, ids=[c["name"] for c in GAP])
def test_normalized_gap_hand(lpm, case):
    data = golden.lp_data(case)
    want = golden.value(case["rho"])
    with lpm.LP(data, eta=0.5, omega=case["omega"], autotune=0) as g:
        got = g.gap(np.array(case["x"], float), np.array(case["y"], float), case["r"])
        got_static = lpm.lp_normalized_gap_static(
            g.h, np.array(case["x"], float), np.array(case["y"], float), case["r"], g.stream)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-15)
    assert got_static == pytest.approx(want, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("t", [1, 2, 3])
def test_bilinear_iterates_hand(lpm, t):
    data = golden.lp_data({"A": [[-1.0]], "b": [0.0], "row_type": [0], "c": [0.0],
                           "lb": [None], "ub": [None]})
    with lpm.LP(data, eta=BIL["eta"], omega=1.0, check_every=1,
                restart_scheme=lpm.LP_RESTART_NONE, max_iter=t, autotune=0) as g:
        g.set_state(np.array([BIL["x0"]]), np.array([BIL["y0"]]))
        g.solve(1e-300)
        st = g.state()
        assert g.info().iters == t
    it = BIL["iterates"][t - 1]
    assert st["x"][0] == pytest.approx(golden.value(it["x"]), rel=1e-12)
    assert st["y"][0] == pytest.approx(golden.value(it["y"]), rel=1e-12)
    if t == 3:
        assert st["xbar"][0] == pytest.approx(golden.value(BIL["average_t3"]["x"]), rel=1e-12)
        assert st["ybar"][0] == pytest.approx(golden.value(BIL["average_t3"]["y"]), rel=1e-12)


FLEX = golden.load("flexible_restart_hand.json")


@pytest.mark.parametrize("case", FLEX["cases"], ids=[c["name"] for c in FLEX["cases"]])
def test_flexible_restart_hand(lpm, case):
    """Remark (Flexible restarts) through the C ABI: per check the chosen
    candidate's gap and radius, the restart flag and the restart point
    (lp_get_trace, lp_get_state), then the end state."""
    data = golden.lp_data(FLEX["lp"])
    scheme = {"flexible": lpm.LP_RESTART_FLEXIBLE,
              "adaptive": lpm.LP_RESTART_ADAPTIVE}[case["scheme"]]
    opts = dict(eta=case["eta"], omega=1.0, check_every=FLEX["check_every"], tau0=FLEX["tau0"],
                restart_scheme=scheme, autotune=0)
    x_init = np.array([FLEX["x_init"]])
    for i, ck in enumerate(case["checks"]):
        with lpm.LP(data, max_iter=ck["iter"], **opts) as g:
            g.set_state(x_init, np.zeros(0))
            g.solve(FLEX["tol"])
            tr = g.trace()
            st = g.state()
        row = tr[i]
        assert row[0] == ck["iter"]
        assert row[1] == pytest.approx(golden.value(ck["rho"]), rel=1e-12), ck
        assert row[5] == pytest.approx(golden.value(ck["radius"]), rel=1e-12), ck
        assert row[2] == ck["restarted"], ck
        assert st["x0"][0] == pytest.approx(golden.value(ck["x0_after"]), rel=1e-12), ck
    with lpm.LP(data, max_iter=1000, **opts) as g:
        g.set_state(x_init, np.zeros(0))
        assert g.solve(FLEX["tol"]) == lpm.LP_OK
        info = g.info()
        st = g.state()
    f = case["final"]
    assert (info.iters, info.restarts, info.returned) == (f["iters"], f["restarts"], f["returned"])
    for k in ("x", "xbar", "x0"):
        assert st[k][0] == pytest.approx(golden.value(f[k]), rel=1e-12, abs=1e-300), k
