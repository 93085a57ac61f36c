"""The allocation-free normalized-gap entry point.

lp_normalized_gap_static serves callers that cannot let a library allocate
device memory (cudaFree synchronizes the device; some frameworks reserve
nearly all device memory up front).  It keeps its scratch in a fixed
device array inside liblp.so.  This file checks, through the C ABI, that
it returns what the allocating entry point lp_normalized_gap returns, bit
for bit, and what the oracle's normalized gap returns, on two calls in a row
(the second reuses the array the first one filled), also with split rows
and a histogram wider than 64 blocks, and that it rejects problems larger
than its fixed scratch.  It is collected
last so that a run stopping at its first failure has run every other test.
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


def test_static_scratch_gap_matches_allocating_gap(lpm, oracle_mod):
    """Two calls in a row equal the allocating entry point bit for bit (same
    kernels, same reduction order) and the oracle's normalized gap
    (Algorithm 2) to 1e-9."""
    data = lpgen.large_mixed(5, m=900, n=4000)
    omega = 2.0
    with lpm.LP(data, eta=0.01, omega=omega) as g:
        points = [lpgen.random_state(data, 0) + (0.5,), lpgen.random_state(data, 1) + (7.0,)]
        want = [lpm.lp_normalized_gap(g.h, x, y, r) for x, y, r in points]
        got = [lpm.lp_normalized_gap_static(g.h, x, y, r) for x, y, r in points]
    for (x, y, r), w, v in zip(points, want, got):
        assert np.isfinite(w) and w > 0
        assert v == w
        ref = oracle_mod.normalized_gap(data, x, y, r, omega=omega)
        assert v == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_static_scratch_gap_split_rows_and_wide_histogram(lpm, oracle_mod):
    """n + m near the limit (190,002: 93 histogram blocks, the allocating
    entry point's grid) with a 160,001-element row and a 30,001-element
    column cut into chunk slices whose partial sums and counters come from
    the static array; against the allocating entry point (bit for bit) and
    the oracle (1e-9), on two calls in a row."""
    data = lpgen.with_dense_lines(lpgen.large_mixed(7, m=30_000, n=160_000), seed=1)
    assert (data.n + data.m + 2047) // 2048 > 64
    with lpm.LP(data, eta=0.9 / 400.0) as g:
        assert g.info().n_split_slices > 0
        for seed, r in ((2, 0.3), (3, 5.0)):
            x, y = lpgen.random_state(data, seed)
            want = lpm.lp_normalized_gap(g.h, x, y, r)
            got = lpm.lp_normalized_gap_static(g.h, x, y, r)
            assert got == want
            ref = oracle_mod.normalized_gap(data, x, y, r)
            assert got == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_static_scratch_rejects_oversized_problem(lpm):
    m, n = 1, (1 << 18)  # n + m one past the limit
    d = lpgen.LPData(m, n, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([1.0]),
                     np.ones(n), np.ones(m), np.zeros(n), np.full(n, np.inf), np.zeros(m, np.int8))
    with lpm.LP(d, eta=0.5) as g:
        x, y = np.zeros(n), np.zeros(m)
        with pytest.raises(lpm.LPError) as e:
            lpm.lp_normalized_gap_static(g.h, x, y, 1.0)
        assert e.value.status == lpm.LP_ERR_INVALID_ARG
        assert "static scratch limit" in str(e.value)
