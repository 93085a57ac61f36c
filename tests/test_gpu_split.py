"""Split rows (lp_options.split_row_len): a whole-warp row of A or A^T longer
than the split length is cut into chunks of at most that many elements, one
warp each; the last chunk to finish adds the partial sums in chunk order and
runs the row's fused epilogue.  Checked against the oracle (iterates, checks,
restart decisions), against the unsplit layout (iterates, sigma_max, the
normalized gap, the adjoint), in FP64 and mixed precision, and between the
GPU-built and host-built layouts (bitwise)."""
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


def dense_lp():
    """3,001 x 9,001 with a 9,001-element row and a 3,001-element column."""
    return lpgen.with_dense_lines(lpgen.large_mixed(7, m=3000, n=9000), seed=1)


ETA = 0.9 / 96.0  # sigma_max of dense_lp() is 94.2 (SciPy's sparse SVD)


def close(got, want, tol, what):
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(np.asarray(got) - np.asarray(want)).max())
    assert err <= tol * scale, f"{what}: {err:.3e} (scale {scale:.3e})"


# split lengths: the default 512 and 2048 (only the dense row and column are
# cut), and a forced one that also cuts every row of A (~35 elements) into
# 32-element chunks
SPLITS = [dict(split_row_len=512), dict(split_row_len=2048),
          dict(split_row_len=32, long_row_threshold=34)]
SPLIT_IDS = ["512", "2048", "forced"]


@pytest.mark.parametrize("opts", SPLITS, ids=SPLIT_IDS)
def test_split_iterates_match_oracle(lpm, oracle_mod, opts):
    data = dense_lp()
    eta = 0.9 / oracle_mod.sigma_max(data)
    K, iters = 16, 160
    with lpm.LP(data, eta=eta, check_every=K, max_iter=iters, autotune=0, **opts) as g:
        assert g.solve(1e-300) == lpm.LP_ITER_LIMIT
        st, info, tr = g.state(), g.info(), g.trace()
    assert info.n_split_slices > 0
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=iters, check_every=K)
    assert info.iters == ref.iters == iters
    for k in ("x", "y", "xbar", "ybar", "x0", "y0"):
        close(st[k], getattr(ref, k), 1e-9, k)
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])
    close(tr[:, 1], ref.trace[:, 1], 1e-8, "rho")
    close(tr[:, 3], ref.trace[:, 3], 1e-8, "kkt avg")


@pytest.mark.parametrize("precision", [0, 1])
def test_split_matches_unsplit(lpm, precision):
    """The same run with and without splitting differs only in the summation
    order of the split rows."""
    data = dense_lp()
    out = {}
    for split in (0, 2048):
        with lpm.LP(data, eta=ETA, check_every=16, max_iter=160, autotune=0,
                    split_row_len=split, precision=precision) as g:
            g.solve(1e-300)
            out[split] = (g.state(), g.info(), g.trace())
    (s0, i0, t0), (s1, i1, t1) = out[0], out[2048]
    assert i0.n_split_slices == 0 and i1.n_split_slices == 5 + 2  # 9,001 and 3,001 elements
    assert all(np.all(np.isfinite(v)) for v in s0.values())
    np.testing.assert_array_equal(t0[:, 2], t1[:, 2])
    tol = 1e-11 if precision == 0 else 1e-5
    for k in s0:
        close(s1[k], s0[k], tol, k)


def test_split_sigma_max_and_gap(lpm):
    data = dense_lp()
    rng = np.random.default_rng(4)
    x = np.clip(rng.standard_normal(data.n), data.lb, data.ub)
    y = rng.standard_normal(data.m)
    y[data.row_type == lpgen.ROW_GE] = np.abs(y[data.row_type == lpgen.ROW_GE])
    res = {}
    for split in (0, 2048):
        with lpm.LP(data, autotune=0, split_row_len=split) as g:
            res[split] = (g.info().sigma_max, g.gap(x, y, 0.7),
                          lpm.lp_normalized_gap_static(g.h, x, y, 0.7))
    assert res[2048][0] == pytest.approx(res[0][0], rel=1e-12)
    assert res[2048][1] == pytest.approx(res[0][1], rel=1e-10)
    assert res[2048][2] == pytest.approx(res[0][2], rel=1e-10)


def test_split_adjoint_matches_unsplit(lpm):
    data = dense_lp()
    rng = np.random.default_rng(5)
    wx, wy = rng.standard_normal(data.n), rng.standard_normal(data.m) * 0.5
    grads = {}
    for split in (0, 2048):
        with lpm.LP(data, eta=ETA, check_every=32, autotune=0, split_row_len=split) as g:
            lpm.lp_solve_recorded(g.h, 256)
            dc, db = np.empty(data.n), np.empty(data.m)
            lpm.lp_backward(g.h, wx, wy, dc, db)
            grads[split] = (dc, db)
    assert np.all(np.isfinite(grads[0][0])) and np.all(np.isfinite(grads[0][1]))
    close(grads[2048][0], grads[0][0], 1e-10, "dc")
    close(grads[2048][1], grads[0][1], 1e-10, "db")


@pytest.mark.parametrize("opts", SPLITS, ids=SPLIT_IDS)
def test_split_layout_device_matches_host(lpm, opts):
    data = dense_lp()
    out = {}
    for dl in (0, 1):
        with lpm.LP(data, eta=ETA, check_every=16, max_iter=96, autotune=0, device_layout=dl,
                    **opts) as g:
            g.solve(1e-300)
            out[dl] = (g.state(), g.info())
    (s0, i0), (s1, i1) = out[0], out[1]
    assert i0.n_split_slices == i1.n_split_slices > 0
    assert all(np.all(np.isfinite(v)) for v in s0.values())
    assert i0.nnz_padded == i1.nnz_padded
    for k in s0:
        np.testing.assert_array_equal(s0[k], s1[k], err_msg=k)


def test_split_row_len_validated(lpm):
    data = lpgen.tiny_standard_form(0, m=10, n=20, per_col=2)
    for bad in (-32, 48):
        with pytest.raises(lpm.LPError) as e:
            lpm.LP(data, eta=0.1, split_row_len=bad)
        assert e.value.status == lpm.LP_ERR_INVALID_ARG
