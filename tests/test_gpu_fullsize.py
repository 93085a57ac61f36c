"""Parity at the benchmark's full size (m = 200,000 rows, n = 1,000,000
columns, ~10M nonzeros; mixed bounds and row senses, power-law column
degrees) in the benchmark's launch configuration (K = 64, adaptive
restarts): 128 iterations (two checks) of the CUDA path against the
oracle, every state vector compared element by element, in FP64 (1e-9) and
in mixed precision (1e-5)."""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

pytestmark = pytest.mark.gpu


def _sigma_estimate(data, iters=60):
    """Independent sigma_max estimate with SciPy's sparse product (power iteration)."""
    import scipy.sparse as sp

    A = sp.csr_matrix((data.val, data.col_idx, data.row_ptr), shape=(data.m, data.n))
    v = np.ones(data.n) / np.sqrt(data.n)
    s = 0.0
    for _ in range(iters):
        w = A.T @ (A @ v)
        s = np.linalg.norm(w)
        v = w / s
    return np.sqrt(s)


def _sigma_svds(data):
    """sigma_max(A) by SciPy's sparse SVD (ARPACK)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    A = sp.csr_matrix((data.val, data.col_idx, data.row_ptr), shape=(data.m, data.n))
    return float(sla.svds(A, k=1, tol=1e-14, return_singular_vectors=False, random_state=0)[0])


def test_full_size_two_checks(oracle_mod):
    import torch

    assert torch.cuda.is_available()
    from paper_2105_12715_gb300 import lp

    data = lpgen.large_mixed(1)
    eta = 0.9 / (1.02 * _sigma_estimate(data))
    iters = 128
    with lp.LP(data, eta=eta, check_every=64, max_iter=iters) as g:
        assert g.solve(1e-300) == lp.LP_ITER_LIMIT
        st = g.state()
        info = g.info()
        tr = g.trace()
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=iters, check_every=64)
    assert info.iters == ref.iters == iters
    for k in ["x", "y", "xbar", "ybar", "x0", "y0"]:
        want = getattr(ref, k)
        scale = max(1.0, float(np.abs(want).max()))
        err = float(np.abs(st[k] - want).max())
        assert err <= 1e-9 * scale, (k, err, scale)
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])
    np.testing.assert_allclose(tr[:, 1], ref.trace[:, 1], rtol=1e-8)
    # FP32-mixed iterations (FP64 averages, checks and refinement) on the same LP against the
    # same FP64 oracle run: FP32 rounding, bounded by 1e-5 relative, same restart decisions
    with lp.LP(data, eta=eta, check_every=64, max_iter=iters,
               precision=lp.LP_PRECISION_MIXED) as g:
        assert g.solve(1e-300) == lp.LP_ITER_LIMIT
        st = g.state()
        tr = g.trace()
    for k in ["x", "y", "xbar", "ybar", "x0", "y0"]:
        want = getattr(ref, k)
        scale = max(1.0, float(np.abs(want).max()))
        err = float(np.abs(st[k] - want).max())
        assert err <= 1e-5 * scale, ("mixed", k, err, scale)
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])


def test_full_size_batch_512_problems(oracle_mod):
    """The batched solver on 512 uneven standard-form LPs (m log-uniform in
    [50, 20000], n = 2m, 3-12 nonzeros per column; ~27.6M nonzeros) in the
    benchmark's launch configuration (tuned kernel variants and check
    periods): sigma_max and 128+ iterations of sampled problems against the
    oracle run on each problem alone."""
    import torch

    assert torch.cuda.is_available()
    from paper_2105_12715_gb300 import lp

    probs = lpgen.batch_standard_form(2, 512)
    ms = np.array([d.m for d in probs])
    order = np.argsort(ms, kind="stable")
    sample = [int(order[0]), int(order[len(order) // 2]), int(order[-1]), 77]
    with lp.LPBatch(probs, check_every=64, tuning={"autotune": 1}) as g:
        summary, per = g.info()
    for k in sample:  # the default estimator (Lanczos) against SciPy's sparse SVD
        assert per[k]["sigma_max"] == pytest.approx(_sigma_svds(probs[k]), rel=1e-9), k
    # iterates: one step size for every problem (an upper bound on every sigma_max),
    # per-problem check periods as in the tuned launch
    eta = 0.9 / max(_sigma_bound(d) for d in probs)
    ks = [p["check_every"] for p in per]
    iters = 2 * max(ks)
    with lp.LPBatch(probs, check_every=64, eta=eta, max_iter=iters,
                    tuning={"autotune": 1}) as g:
        g.set_check_every(ks)
        g.solve(1e-300)
        st = g.state()
        _, per2 = g.info()
    for k in sample:
        d = probs[k]
        ref = oracle_mod.solve(d, eta, tol=1e-300, max_iter=iters, check_every=ks[k],
                               x_init=np.zeros(d.n), y_init=np.zeros(d.m))
        assert per2[k]["iters"] == ref.iters == iters
        assert per2[k]["restarts"] == ref.restarts
        for key, st0 in [("x", g.col_start), ("xbar", g.col_start), ("x0", g.col_start),
                         ("y", g.row_start), ("ybar", g.row_start), ("y0", g.row_start)]:
            got = st[key][st0[k]:st0[k + 1]]
            want = getattr(ref, key)
            scale = max(1.0, float(np.abs(want).max()))
            assert float(np.abs(got - want).max()) <= 1e-9 * scale, (k, key)


def _sigma_bound(d):
    """sqrt(||A||_1 ||A||_inf), an upper bound on sigma_max(A)."""
    a = np.abs(d.val)
    rows = np.add.reduceat(a, d.row_ptr[:-1])
    rows[np.diff(d.row_ptr) == 0] = 0.0
    cols = np.bincount(d.col_idx, weights=a, minlength=d.n)
    return float(np.sqrt(rows.max() * cols.max()))
