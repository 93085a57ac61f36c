"""The layout built on the GPU (lp_options.device_layout = 1, the default)
against the one built on the host cores (0): the same arrays give the same
iterates bit for bit, the same padded size and lane-group counts, and the
same sigma_max; invalid inputs are rejected by both."""
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


def _no_rows_lp():
    n = 40
    return lpgen.LPData(0, n, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0),
                        np.linspace(-1.0, 1.0, n), np.zeros(0), np.zeros(n), np.ones(n),
                        np.zeros(0, np.int8), name="no rows")


CASES = [
    ("tiny", lambda: lpgen.tiny_standard_form(0)),
    ("adversarial3", lambda: lpgen.adversarial(3)),
    ("adversarial5", lambda: lpgen.adversarial(5)),
    ("large_mixed", lambda: lpgen.large_mixed(3, m=3000, n=15000)),
    ("multicommodity", lambda: lpgen.multicommodity_grid(2, side=8, commodities=3)),
    ("no_rows", _no_rows_lp),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1])
def test_device_layout_matches_host_layout(lpm, name, make, precision):
    data = make()
    out = {}
    for dl in (0, 1):
        with lpm.LP(data, eta=0.05, check_every=50, max_iter=200, autotune=0, device_layout=dl,
                    precision=precision) as g:
            g.solve(1e-300)
            out[dl] = (g.state(), g.info())
    (s0, i0), (s1, i1) = out[0], out[1]
    assert i0.nnz_padded == i1.nnz_padded
    assert (i0.n_long_rows, i0.n_long_cols) == (i1.n_long_rows, i1.n_long_cols)
    assert i0.iters == i1.iters == 200 and i0.restarts == i1.restarts
    for k in s0:
        np.testing.assert_array_equal(s0[k], s1[k], err_msg=k)


def test_device_layout_sigma_max_and_lane_auto(lpm):
    """The default step size (sigma_max from the same start vector) and the
    lane policy chosen for the SM count agree between the two layouts."""
    data = lpgen.large_mixed(4, m=2000, n=9000)
    info = {}
    for dl in (0, 1):
        with lpm.LP(data, autotune=0, device_layout=dl) as g:
            info[dl] = g.info()
    assert info[0].sigma_max == info[1].sigma_max
    assert info[0].sigma_steps == info[1].sigma_steps
    assert info[0].nnz_padded == info[1].nnz_padded


@pytest.mark.parametrize("dl", [0, 1])
def test_invalid_inputs_rejected_by_both_layouts(lpm, dl):
    data = lpgen.tiny_standard_form(0, m=10, n=20, per_col=2)

    def rejected(d):
        with pytest.raises(lpm.LPError) as e:
            lpm.LP(d, eta=0.1, device_layout=dl)
        return e.value.status == lpm.LP_ERR_INVALID_ARG

    bad = lpgen.LPData(**{**data.__dict__})
    bad.col_idx = data.col_idx.copy()
    bad.col_idx[0] = -1
    assert rejected(bad)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.val = data.val.copy()
    bad.val[5] = np.inf
    assert rejected(bad)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.row_type = data.row_type.copy()
    bad.row_type[2] = 3
    assert rejected(bad)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.b = data.b.copy()
    bad.b[1] = np.nan
    assert rejected(bad)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.row_ptr = data.row_ptr.copy()
    bad.row_ptr[3] = bad.row_ptr[4] + 1  # not monotone (row_ptr[m] = nnz kept)
    assert rejected(bad)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.row_ptr = data.row_ptr.copy()
    bad.row_ptr[0] = 1  # must start at 0
    assert rejected(bad)
    rp = np.array([0, 3], np.int32)
    ci = np.array([2, 0, 2], np.int32)  # column 2 twice in one row
    d2 = lpgen.LPData(1, 3, rp, ci, np.array([1.0, 2.0, 3.0]), np.ones(3), np.ones(1),
                      np.zeros(3), np.full(3, np.inf), np.zeros(1, np.int8))
    assert rejected(d2)
