"""The check's FP64 reductions against long-double sums.

The library reduces the check's quantities (primal and dual residuals,
primal and dual objectives) in FP64 in a fixed order.  Here the same
quantities are formed from the library's own state vectors (lp_get_state) in
numpy's long double (80-bit extended on x86, 128-bit quad on Arm) and the
reported values (lp_get_info) must agree to FP64 rounding of the sums:
relative 1e-12 for the residual norms (sums of squares), and, for the
objectives, 1e-13 of the sum of the terms' magnitudes.  Definitions: the
relative KKT error of Section 7's termination test as this library reads it
(primal residual by row sense, dual residual from the reduced costs' sign
cone, dual objective with the bound terms of finite bounds).
"""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

pytestmark = pytest.mark.gpu

LD = np.longdouble


def _kkt_ld(d, x, y):
    x, y = x.astype(LD), y.astype(LD)
    val = d.val.astype(LD)
    rows = np.repeat(np.arange(d.m), np.diff(d.row_ptr))
    ax = np.zeros(d.m, LD)
    np.add.at(ax, rows, val * x[d.col_idx])
    aty = np.zeros(d.n, LD)
    np.add.at(aty, d.col_idx, val * y[rows])
    r = ax - d.b.astype(LD)
    r[d.row_type == 1] = np.minimum(r[d.row_type == 1], 0)
    r[d.row_type == 2] = np.maximum(r[d.row_type == 2], 0)
    lam = d.c.astype(LD) - aty
    lf, uf = np.isfinite(d.lb), np.isfinite(d.ub)
    proj = lam.copy()
    proj[lf & ~uf] = np.maximum(lam[lf & ~uf], 0)
    proj[uf & ~lf] = np.minimum(lam[uf & ~lf], 0)
    proj[~lf & ~uf] = 0
    bt = np.zeros(d.n, LD)
    pos, neg = lf & (proj > 0), uf & (proj < 0)
    bt[pos] = d.lb[pos].astype(LD) * proj[pos]
    bt[neg] = d.ub[neg].astype(LD) * proj[neg]
    pterms = d.c.astype(LD) * x
    dterms = np.concatenate([d.b.astype(LD) * y, bt])
    return {"rp": np.sqrt(np.sum(r * r)), "rd": np.sqrt(np.sum((lam - proj) ** 2)),
            "pobj": np.sum(pterms), "dobj": np.sum(dterms),
            "pmag": np.sum(np.abs(pterms)), "dmag": np.sum(np.abs(dterms))}


@pytest.mark.parametrize("which", ["mixed3k", "adversarial"])
def test_check_reductions_against_long_double(oracle_mod, which):
    from paper_2105_12715_gb300 import lp

    d = lpgen.large_mixed(11, m=3001, n=15007) if which == "mixed3k" else lpgen.adversarial(7)
    eta = 0.9 / oracle_mod.sigma_max(d)
    K = 32
    for iters in (3 * K, 7 * K):
        with lp.LP(d, eta=eta, check_every=K, max_iter=iters, restart_scheme=lp.LP_RESTART_NONE,
                   autotune=0) as g:
            g.solve(1e-300)
            info, st = g.info(), g.state()
        # no restarts: the last check saw the current average and iterate
        for got, (x, y) in ((info.kkt_avg, (st["xbar"], st["ybar"])),
                            (info.kkt_cur, (st["x"], st["y"]))):
            want = _kkt_ld(d, x, y)
            assert float(got[0]) == pytest.approx(float(want["rp"]), rel=1e-12, abs=1e-300)
            assert float(got[1]) == pytest.approx(float(want["rd"]), rel=1e-12, abs=1e-300)
            assert abs(got[2] - float(want["pobj"])) <= 1e-13 * float(want["pmag"]) + 1e-300
            assert abs(got[3] - float(want["dobj"])) <= 1e-13 * float(want["dmag"]) + 1e-300
