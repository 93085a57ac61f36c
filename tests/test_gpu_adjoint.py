"""Adjoint of the unrolled restarted PDHG map (lp_backward) against central
finite differences of the oracle's unrolled map with the same restart
decisions (h = 1e-6, FP64), and through the torch.autograd.Function."""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

pytestmark = pytest.mark.gpu


def _box_lp(seed):
    d = lpgen.tiny_standard_form(seed, m=60, n=150, per_col=4)
    d.ub = np.ones(d.n)  # box [0, 1]; the planted optimum (x* in [0, 1)) stays optimal
    return d


def test_backward_matches_oracle_finite_differences(oracle_mod):
    import torch

    assert torch.cuda.is_available()
    from paper_2105_12715_gb300 import lp

    data = _box_lp(3)
    eta = 0.9 / oracle_mod.sigma_max(data)
    K, iters = 32, 320
    rng = np.random.default_rng(0)
    wx = rng.standard_normal(data.n)
    wy = rng.standard_normal(data.m) * 0.5
    with lp.LP(data, eta=eta, check_every=K) as g:
        lp.lp_solve_recorded(g.h, iters)
        st = g.state()
        flags = g.trace()[:, 2].astype(np.int8)
        dc, db = np.empty(data.n), np.empty(data.m)
        lp.lp_backward(g.h, wx, wy, dc, db)
        st_after = g.state()
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=iters, check_every=K)
    np.testing.assert_array_equal(flags, ref.trace[:, 2].astype(np.int8))
    assert flags.sum() >= 2  # the map contains restarts
    np.testing.assert_allclose(st["xbar"], ref.xbar, rtol=0, atol=1e-9)
    for k in st:  # lp_backward leaves the recorded state
        np.testing.assert_array_equal(st[k], st_after[k])

    def loss(c, b):
        d = lpgen.LPData(**{**data.__dict__})
        d.c, d.b = c, b
        r = oracle_mod.solve(d, eta, tol=1e-300, max_iter=iters, check_every=K,
                             restart_scheme=oracle_mod.RESTART_SCHEDULE, schedule=flags)
        return wx @ r.xbar + wy @ r.ybar

    h = 1e-6
    for j in rng.choice(data.n, size=8, replace=False):
        e = np.zeros(data.n)
        e[j] = h
        fd = (loss(data.c + e, data.b) - loss(data.c - e, data.b)) / (2 * h)
        assert dc[j] == pytest.approx(fd, rel=1e-4, abs=1e-6), ("c", j)
    for i in rng.choice(data.m, size=8, replace=False):
        e = np.zeros(data.m)
        e[i] = h
        fd = (loss(data.c, data.b + e) - loss(data.c, data.b - e)) / (2 * h)
        assert db[i] == pytest.approx(fd, rel=1e-4, abs=1e-6), ("b", i)


def test_autograd_function_gradient(oracle_mod):
    import torch

    from paper_2105_12715_gb300.autodiff import unrolled_pdhg

    data = _box_lp(4)
    eta = 0.9 / oracle_mod.sigma_max(data)
    c = torch.tensor(data.c, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(data.b, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.randn(data.n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    xbar, ybar = unrolled_pdhg(c, b, data, 256, eta=eta, check_every=32)
    loss = (w * xbar).sum()
    loss.backward()
    # directional derivative along a random direction vs central differences (oracle)
    rng = np.random.default_rng(2)
    dcv, dbv = rng.standard_normal(data.n), rng.standard_normal(data.m)
    with torch.no_grad():
        from paper_2105_12715_gb300 import lp

        with lp.LP(data, eta=eta, check_every=32) as g:
            lp.lp_solve_recorded(g.h, 256)
            flags = g.trace()[:, 2].astype(np.int8)
    h = 1e-6

    def L(cc, bb):
        d = lpgen.LPData(**{**data.__dict__})
        d.c, d.b = cc, bb
        r = oracle_mod.solve(d, eta, tol=1e-300, max_iter=256, check_every=32,
                             restart_scheme=oracle_mod.RESTART_SCHEDULE, schedule=flags)
        return w.cpu().numpy() @ r.xbar

    fd = (L(data.c + h * dcv, data.b + h * dbv) - L(data.c - h * dcv, data.b - h * dbv)) / (2 * h)
    got = float(c.grad.cpu().numpy() @ dcv + b.grad.cpu().numpy() @ dbv)
    assert got == pytest.approx(fd, rel=1e-4, abs=1e-6)


def test_backward_matches_implicit_kkt_gradient_on_the_face(oracle_mod):
    """Implicit-KKT active-set check.  At the converged face of a box LP
    (interior set B from the oracle's solution), A_B x_B = b - A_N x_N, so the
    loss w^T x with w = A_B^T u on B (0 elsewhere) has d/db = u whichever
    point of the face the method reaches.  The adjoint of the unrolled map run
    to convergence must return u."""
    import torch

    assert torch.cuda.is_available()
    from paper_2105_12715_gb300 import lp

    data = lpgen.box_standard_form(5, m=100, n=250, per_col=6)
    eta = 0.9 / oracle_mod.sigma_max(data)
    K = 64
    ref = oracle_mod.solve(data, eta, tol=1e-10, max_iter=400000, check_every=K)
    assert ref.status == 0
    x = ref.x_sol
    B = (x > 1e-7) & (x < 1 - 1e-7)
    A = data.dense()
    assert np.linalg.matrix_rank(A[:, B]) == data.m
    u = np.random.default_rng(0).standard_normal(data.m)
    w = np.zeros(data.n)
    w[B] = A[:, B].T @ u
    iters = ((ref.iters + 4 * K) // K) * K
    with lp.LP(data, eta=eta, check_every=K) as g:
        lp.lp_solve_recorded(g.h, iters)
        dc, db = np.empty(data.n), np.empty(data.m)
        lp.lp_backward(g.h, w, None, dc, db)
    assert np.linalg.norm(db - u) <= 1e-6 * np.linalg.norm(u)
