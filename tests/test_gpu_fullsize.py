"""Parity at the benchmark's full size (m = 200,000 rows, n = 1,000,000
columns, ~10M nonzeros; mixed bounds and row senses, power-law column
degrees) in the benchmark's launch configuration (K = 64, adaptive
restarts): 128 iterations (two checks) of the CUDA path against the
oracle, every state vector compared element by element."""
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
