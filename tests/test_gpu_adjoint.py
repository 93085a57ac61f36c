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


def _batch_boxes():
    return [_box_lp(3), _box_lp(5), lpgen.box_standard_form(7, m=40, n=90, per_col=3)]


def test_batch_backward_matches_oracle_finite_differences(oracle_mod):
    """lp_batch_backward: every problem's gradient against central differences
    of the oracle's unrolled map of that problem alone (its own restart
    schedule), h = 1e-6."""
    import torch

    assert torch.cuda.is_available()
    from paper_2105_12715_gb300 import lp

    probs = _batch_boxes()
    eta = 0.9 / max(oracle_mod.sigma_max(d) for d in probs)
    K, iters = 32, 320
    rng = np.random.default_rng(1)
    wx = [rng.standard_normal(d.n) for d in probs]
    wy = [0.5 * rng.standard_normal(d.m) for d in probs]
    with lp.LPBatch(probs, eta=eta, check_every=K) as g:
        g.solve_recorded(iters)
        _, per = g.info()
        st = g.state()
        dc, db = g.backward(np.concatenate(wx), np.concatenate(wy))
        st_after = g.state()
    for key in st:  # the recorded state is left in place
        np.testing.assert_array_equal(st[key], st_after[key])
    co, ro = 0, 0
    for k, d in enumerate(probs):
        ref = oracle_mod.solve(d, eta, tol=1e-300, max_iter=iters, check_every=K)
        flags = ref.trace[:, 2].astype(np.int8)
        assert per[k]["restarts"] == ref.restarts == flags.sum() >= 1
        np.testing.assert_allclose(st["xbar"][co:co + d.n], ref.xbar, rtol=0, atol=1e-9)

        def loss(c, b):
            dd = lpgen.LPData(**{**d.__dict__})
            dd.c, dd.b = c, b
            r = oracle_mod.solve(dd, eta, tol=1e-300, max_iter=iters, check_every=K,
                                 restart_scheme=oracle_mod.RESTART_SCHEDULE, schedule=flags)
            return wx[k] @ r.xbar + wy[k] @ r.ybar

        h = 1e-6
        for j in rng.choice(d.n, size=4, replace=False):
            e = np.zeros(d.n)
            e[j] = h
            fd = (loss(d.c + e, d.b) - loss(d.c - e, d.b)) / (2 * h)
            assert dc[co + j] == pytest.approx(fd, rel=1e-4, abs=1e-6), (k, "c", j)
        for i in rng.choice(d.m, size=4, replace=False):
            e = np.zeros(d.m)
            e[i] = h
            fd = (loss(d.c, d.b + e) - loss(d.c, d.b - e)) / (2 * h)
            assert db[ro + i] == pytest.approx(fd, rel=1e-4, abs=1e-6), (k, "b", i)
        co += d.n
        ro += d.m


def test_batch_backward_equals_single_problem_backward(oracle_mod):
    """Each problem's batched gradient equals lp_backward on that problem alone."""
    import torch

    assert torch.cuda.is_available()
    from paper_2105_12715_gb300 import lp

    probs = _batch_boxes()
    eta = 0.9 / max(oracle_mod.sigma_max(d) for d in probs)
    K, iters = 32, 256
    rng = np.random.default_rng(4)
    wx = [rng.standard_normal(d.n) for d in probs]
    with lp.LPBatch(probs, eta=eta, check_every=K) as g:
        g.solve_recorded(iters)
        dc, db = g.backward(np.concatenate(wx), None)
    co, ro = 0, 0
    for k, d in enumerate(probs):
        with lp.LP(d, eta=eta, check_every=K) as s1:
            lp.lp_solve_recorded(s1.h, iters)
            c1, b1 = np.empty(d.n), np.empty(d.m)
            lp.lp_backward(s1.h, wx[k], None, c1, b1)
        np.testing.assert_allclose(dc[co:co + d.n], c1, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(db[ro:ro + d.m], b1, rtol=1e-11, atol=1e-13)
        co += d.n
        ro += d.m


def test_batch_autograd_function(oracle_mod):
    import torch

    from paper_2105_12715_gb300.autodiff import unrolled_pdhg_batch

    probs = _batch_boxes()
    eta = 0.9 / max(oracle_mod.sigma_max(d) for d in probs)
    c = torch.tensor(np.concatenate([d.c for d in probs]), dtype=torch.float64, device="cuda",
                     requires_grad=True)
    b = torch.tensor(np.concatenate([d.b for d in probs]), dtype=torch.float64, device="cuda",
                     requires_grad=True)
    w = torch.randn(c.shape[0], dtype=torch.float64, device="cuda",
                    generator=torch.Generator("cuda").manual_seed(3))
    xbar, ybar = unrolled_pdhg_batch(c, b, probs, 192, eta=eta, check_every=32)
    (w * xbar).sum().backward()
    # against the single-problem autograd path, problem by problem
    from paper_2105_12715_gb300.autodiff import unrolled_pdhg

    co, ro = 0, 0
    for d in probs:
        ck = torch.tensor(d.c, dtype=torch.float64, device="cuda", requires_grad=True)
        bk = torch.tensor(d.b, dtype=torch.float64, device="cuda", requires_grad=True)
        xk, _ = unrolled_pdhg(ck, bk, d, 192, eta=eta, check_every=32)
        (w[co:co + d.n] * xk).sum().backward()
        torch.testing.assert_close(c.grad[co:co + d.n], ck.grad, rtol=1e-11, atol=1e-13)
        torch.testing.assert_close(b.grad[ro:ro + d.m], bk.grad, rtol=1e-11, atol=1e-13)
        co += d.n
        ro += d.m


def test_backward_finite_differences_at_full_size(oracle_mod):
    """The differentiable-LP workload at its full size: m = 2000, n = 5000,
    50k nonzeros, box [0, 1], K = 100, 2000 unrolled iterations (checkpoints
    every 100).  Eight sampled coordinates of c and eight of b against
    central differences (h = 1e-6, FP64) of the oracle's unrolled map with
    the recorded restart schedule.  Over 2000 steps some clamp decisions may
    sit within the perturbation of their bound; the map is continuous and
    piecewise affine, so such a kink moves the difference quotient by a
    fraction of one coordinate's slope change, which the tolerance
    (1e-4 of the gradient's largest sampled entry) covers."""
    from paper_2105_12715_gb300 import lp

    data = lpgen.box_standard_form(100)
    assert (data.m, data.n, data.nnz) == (2000, 5000, 50000)
    eta = 0.9 / oracle_mod.sigma_max(data)
    K, iters = 100, 2000
    rng = np.random.default_rng(5)
    wx = rng.standard_normal(data.n)
    with lp.LP(data, eta=eta, check_every=K) as g:
        lp.lp_solve_recorded(g.h, iters)
        flags = g.trace()[:, 2].astype(np.int8)
        st = g.state()
        dc, db = np.empty(data.n), np.empty(data.m)
        lp.lp_backward(g.h, wx, None, dc, db)
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=iters, check_every=K)
    np.testing.assert_array_equal(flags, ref.trace[:, 2].astype(np.int8))
    assert flags.sum() >= 2
    np.testing.assert_allclose(st["xbar"], ref.xbar, rtol=0, atol=1e-9)

    def loss(c, b):
        d = lpgen.LPData(**{**data.__dict__})
        d.c, d.b = c, b
        r = oracle_mod.solve(d, eta, tol=1e-300, max_iter=iters, check_every=K,
                             restart_scheme=oracle_mod.RESTART_SCHEDULE, schedule=flags)
        return wx @ r.xbar

    h = 1e-6
    got, fds = [], []
    for j in rng.choice(data.n, size=8, replace=False):
        e = np.zeros(data.n)
        e[j] = h
        fds.append((loss(data.c + e, data.b) - loss(data.c - e, data.b)) / (2 * h))
        got.append(dc[j])
    for i in rng.choice(data.m, size=8, replace=False):
        e = np.zeros(data.m)
        e[i] = h
        fds.append((loss(data.c, data.b + e) - loss(data.c, data.b - e)) / (2 * h))
        got.append(db[i])
    got, fds = np.array(got), np.array(fds)
    scale = float(np.abs(fds).max())
    assert scale > 0
    np.testing.assert_allclose(got, fds, rtol=1e-4, atol=1e-4 * scale)


def test_autograd_loss_on_ybar_only(oracle_mod):
    """A loss that reads only ybar: backward gets no gradient for xbar (None)."""
    import torch

    from paper_2105_12715_gb300 import lp
    from paper_2105_12715_gb300.autodiff import unrolled_pdhg

    data = _box_lp(6)
    eta = 0.9 / oracle_mod.sigma_max(data)
    c = torch.tensor(data.c, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(data.b, dtype=torch.float64, device="cuda", requires_grad=True)
    wy = torch.linspace(-1.0, 1.0, data.m, dtype=torch.float64, device="cuda")
    _, ybar = unrolled_pdhg(c, b, data, 128, eta=eta, check_every=32)
    (wy * ybar).sum().backward()
    assert c.grad.device.type == "cuda" and b.grad.device.type == "cuda"
    with lp.LP(data, eta=eta, check_every=32) as g:
        lp.lp_solve_recorded(g.h, 128)
        dc, db = np.empty(data.n), np.empty(data.m)
        lp.lp_backward(g.h, None, wy.cpu().numpy(), dc, db)
    np.testing.assert_array_equal(c.grad.cpu().numpy(), dc)
    np.testing.assert_array_equal(b.grad.cpu().numpy(), db)
