"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerance: FP64 iterates agree to 1e-9 relative (max-abs difference over
max(1, max|oracle|)).  The two sides sum in different orders (FMA chains
per row on the GPU, plain multiply-add loops in the oracle), so
agreement is to rounding, not bitwise.
"""
import numpy as np
import pytest

from paper_2105_12715_gb300 import lpgen

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def lpm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2105_12715_gb300 import lp

    lp.load()
    return lp


def close(gpu, ref, tol=TOL, what=""):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    assert gpu.shape == ref.shape, what
    if ref.size == 0:
        return
    scale = max(1.0, float(np.abs(ref).max()))
    err = float(np.abs(gpu - ref).max())
    assert err <= tol * scale, f"{what}: max abs err {err:.3e} (scale {scale:.3e})"


# Kernel variants of the two passes (lp_options.spmv_unroll): register
# batches of 2, 4, 8 gathers, software-pipelined batches (-2, -4), and the
# same with registers capped for higher occupancy (+-100).
VARIANTS = [2, 4, 8, -2, -4, 102, -104]


def run_both(lpm, oracle_mod, data, iters, eta, K=64, omega=1.0, scheme=2, long_thr=512,
             x_init=None, y_init=None, unroll=4, **opts):
    with lpm.LP(data, eta=eta, omega=omega, check_every=K, restart_scheme=scheme,
                max_iter=iters, long_row_threshold=long_thr, spmv_unroll=unroll,
                spmv_unroll_rows=unroll, autotune=0, **opts) as g:
        if x_init is not None:
            g.set_state(x_init, y_init)
        status = g.solve(1e-300)
        st = g.state()
        info = g.info()
        tr = g.trace()
    ref = oracle_mod.solve(data, eta, omega=omega, tol=1e-300, max_iter=iters, check_every=K,
                           restart_scheme=scheme, x_init=x_init, y_init=y_init)
    return status, st, info, tr, ref


def compare_states(st, ref, tol=TOL):
    for k, rk in [("x", "x"), ("y", "y"), ("xbar", "xbar"), ("ybar", "ybar"), ("x0", "x0"),
                  ("y0", "y0")]:
        close(st[k], getattr(ref, rk), tol, k)


def eta_of(oracle_mod, data):
    return 0.9 / oracle_mod.sigma_max(data)


@pytest.mark.parametrize("seed", [0, 3])
def test_first_100_iterations_tiny(lpm, oracle_mod, seed):
    data = lpgen.tiny_standard_form(seed)
    eta = eta_of(oracle_mod, data)
    status, st, info, tr, ref = run_both(lpm, oracle_mod, data, 100, eta)
    assert status == lpm.LP_ITER_LIMIT
    assert info.iters == ref.iters == 100
    compare_states(st, ref)
    assert info.restarts == ref.restarts


def test_checks_and_restarts_match_oracle(lpm, oracle_mod):
    """Same restart decisions at every check for 40 checks (K = 16)."""
    data = lpgen.tiny_standard_form(1)
    eta = eta_of(oracle_mod, data)
    status, st, info, tr, ref = run_both(lpm, oracle_mod, data, 640, eta, K=16)
    assert tr.shape[0] == ref.trace.shape[0] == 40
    np.testing.assert_array_equal(tr[:, 0], ref.trace[:, 0])
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])
    close(tr[:, 1], ref.trace[:, 1], 1e-8, "rho")
    close(tr[:, 3], ref.trace[:, 3], 1e-8, "kkt avg")
    close(tr[:, 4], ref.trace[:, 4], 1e-8, "kkt cur")
    close(tr[:, 5], ref.trace[:, 5], 1e-8, "radius")
    compare_states(st, ref, 1e-8)


@pytest.mark.parametrize("omega,unroll", [(0.3, 4), (1.0, -4), (4.0, 2), (1.0, -2)])
def test_mixed_bounds_rows_and_long_rows(lpm, oracle_mod, omega, unroll):
    """EQ/GE/LE rows, every bound kind, empty rows/cols, a dense row and a
    dense column on the warp-per-row path (threshold 16)."""
    data = lpgen.adversarial(7)
    eta = eta_of(oracle_mod, data)
    x0, y0 = lpgen.random_state(data, 5)
    status, st, info, tr, ref = run_both(lpm, oracle_mod, data, 200, eta, K=32, omega=omega,
                                         long_thr=16, x_init=x0, y_init=y0, unroll=unroll)
    assert info.n_long_rows >= 1 and info.n_long_cols >= 1
    compare_states(st, ref)
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])


@pytest.mark.parametrize("unroll", VARIANTS)
def test_ragged_multi_slice_power_law(lpm, oracle_mod, unroll):
    """Several hundred slices with a ragged last slice, power-law columns;
    every kernel variant of the two passes."""
    data = lpgen.large_mixed(11, m=3001, n=15007)
    eta = eta_of(oracle_mod, data)
    status, st, info, tr, ref = run_both(lpm, oracle_mod, data, 130, eta, K=64, unroll=unroll)
    assert (info.spmv_unroll, info.spmv_unroll_rows) == (unroll, unroll)
    compare_states(st, ref)
    assert info.restarts == ref.restarts


@pytest.mark.parametrize("tau0_mult", [0, 2.5, 3])
def test_first_restart_length_tau0(lpm, oracle_mod, tau0_mult):
    """Eq. (adaptive-restart-scheme), n = 0: the first restart at the first
    check with t >= tau^0 (tau^0 = 1, 2.5 K, 3 K), then the beta rule; the
    CUDA path's restart flags, gaps and iterates against the oracle's."""
    data = lpgen.tiny_standard_form(6)
    eta = eta_of(oracle_mod, data)
    K = 16
    tau0 = 1 if tau0_mult == 0 else int(tau0_mult * K)
    with lpm.LP(data, eta=eta, check_every=K, max_iter=20 * K, tau0=tau0, autotune=0) as g:
        g.solve(1e-300)
        st, tr = g.state(), g.trace()
    ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=20 * K, check_every=K, tau0=tau0)
    np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])
    first = int(np.flatnonzero(ref.trace[:, 2])[0]) + 1
    assert first == max(1, -(-tau0 // K))  # first check with t >= tau0
    close(tr[:, 1], ref.trace[:, 1], 1e-8, "rho")
    compare_states(st, ref, 1e-8)


def test_flexible_and_fixed_schemes(lpm, oracle_mod):
    data = lpgen.tiny_standard_form(4)
    eta = eta_of(oracle_mod, data)
    for scheme in (3, 1, 0):
        with lpm.LP(data, eta=eta, check_every=32, restart_scheme=scheme, fixed_len=128,
                    max_iter=512) as g:
            g.solve(1e-300)
            st = g.state()
            tr = g.trace()
        ref = oracle_mod.solve(data, eta, tol=1e-300, max_iter=512, check_every=32,
                               restart_scheme=scheme, fixed_len=128)
        compare_states(st, ref, 1e-8)
        np.testing.assert_array_equal(tr[:, 2], ref.trace[:, 2])


def test_power_iteration_sigma_max(lpm, oracle_mod):
    """Section 7's power iteration (sigma_method = LP_SIGMA_POWER) against the oracle's."""
    for data in [lpgen.tiny_standard_form(0), lpgen.adversarial(3)]:
        with lpm.LP(data, sigma_method=lpm.LP_SIGMA_POWER) as g:
            info = g.info()
        want = oracle_mod.sigma_max(data)
        assert info.sigma_max == pytest.approx(want, rel=1e-8)
        assert info.eta == pytest.approx(0.9 / want, rel=1e-8)
        assert info.sigma_steps > 0


def _one_by_one():
    return lpgen.LPData(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32),
                        np.array([-3.0]), np.array([1.0]), np.array([4.0]), np.zeros(1),
                        np.full(1, np.inf), np.zeros(1, np.int8))


def test_lanczos_sigma_max_exact(lpm):
    """The default estimator (Lanczos on A^T A) against the largest singular
    value from a dense SVD; the 1 x 1 problem breaks down at the first step
    (beta_0 = 0), where the Ritz value is exact."""
    cases = [lpgen.tiny_standard_form(0), lpgen.adversarial(3), lpgen.adversarial(5),
             lpgen.large_mixed(3, m=300, n=1200), lpgen.tiny_standard_form(2, m=5, n=9, per_col=2),
             _one_by_one()]
    for data in cases:
        with lpm.LP(data, autotune=0) as g:
            info = g.info()
        want = float(np.linalg.norm(data.dense(), 2))
        assert info.sigma_max == pytest.approx(want, rel=1e-9), data.name
        assert info.eta == pytest.approx(0.9 / info.sigma_max, rel=1e-15)
        assert 0 < info.sigma_steps <= 200
    with lpm.LP(_one_by_one(), autotune=0) as g:
        assert g.info().sigma_steps == 1


def test_lanczos_takes_fewer_steps_than_power_iteration(lpm):
    data = lpgen.large_mixed(4, m=2000, n=9000)
    steps = {}
    for method in (lpm.LP_SIGMA_POWER, lpm.LP_SIGMA_LANCZOS):
        with lpm.LP(data, autotune=0, sigma_method=method) as g:
            steps[method] = (g.info().sigma_steps, g.info().sigma_max)
    assert steps[lpm.LP_SIGMA_LANCZOS][0] < steps[lpm.LP_SIGMA_POWER][0]
    assert steps[lpm.LP_SIGMA_LANCZOS][1] == pytest.approx(steps[lpm.LP_SIGMA_POWER][1], rel=1e-6)


def test_zero_matrix_needs_explicit_eta(lpm):
    """sigma_max(A) = 0 leaves no step size: both estimators refuse."""
    m, n = 3, 4
    d = lpgen.LPData(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0),
                     np.ones(n), np.zeros(m), np.zeros(n), np.full(n, 1.0), np.zeros(m, np.int8))
    for method in (lpm.LP_SIGMA_POWER, lpm.LP_SIGMA_LANCZOS):
        with pytest.raises(lpm.LPError) as e:
            lpm.LP(d, sigma_method=method)
        assert e.value.status == lpm.LP_ERR_NUMERICAL


def test_normalized_gap_vs_algorithm2(lpm, oracle_mod):
    """Device multiplier search vs the oracle's Algorithm 2 at random points."""
    for data in [lpgen.tiny_standard_form(2), lpgen.adversarial(8), lpgen.large_mixed(5, m=900, n=4000)]:
        with lpm.LP(data, eta=0.01) as g:
            for seed in range(4):
                x, y = lpgen.random_state(data, seed)
                for omega_r in [1e-3, 0.5, 7.0, 1e4]:
                    want = oracle_mod.normalized_gap(data, x, y, omega_r)
                    got = g.gap(x, y, omega_r)
                    assert got == pytest.approx(want, rel=1e-9, abs=1e-12)
            assert g.gap(x, y, 0.0) == 0.0


def test_full_solve_to_1e8(lpm, oracle_mod):
    """Planted LP solved to relative KKT 1e-8; objective within 1e-7 of c^T x*;
    the same iteration count as the oracle (within one check interval)."""
    data = lpgen.tiny_standard_form(2)
    eta = eta_of(oracle_mod, data)
    with lpm.LP(data, eta=eta, check_every=64, max_iter=200000) as g:
        status = g.solve(1e-8)
        info = g.info()
        x, y = g.solution()
    ref = oracle_mod.solve(data, eta, tol=1e-8, max_iter=200000, check_every=64)
    assert status == lpm.LP_OK and ref.status == 0
    assert abs(info.iters - ref.iters) <= 64
    k = oracle_mod.kkt(data, x, y)
    assert k["rel"] <= 1e-8
    assert k["pobj"] == pytest.approx(data.obj_star, rel=1e-7)


def test_edge_cases(lpm, oracle_mod):
    # no nonzeros at all: x moves to its bounds, every row empty
    m, n = 5, 7
    d = lpgen.LPData(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0),
                     np.linspace(-1, 1, n), np.zeros(m), np.zeros(n), np.full(n, 2.0),
                     np.zeros(m, np.int8))
    status, st, info, tr, ref = run_both(lpm, oracle_mod, d, 50, 0.5, K=8)
    compare_states(st, ref)
    # one row, one column
    d1 = lpgen.LPData(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0]),
                      np.array([1.0]), np.array([4.0]), np.zeros(1), np.full(1, np.inf),
                      np.zeros(1, np.int8))
    with lpm.LP(d1, eta=0.4, check_every=8) as g:
        assert g.solve(1e-10) == lpm.LP_OK
        x, y = g.solution()
    assert x[0] == pytest.approx(2.0, rel=1e-9) and y[0] == pytest.approx(0.5, rel=1e-8)


def test_invalid_inputs_rejected(lpm):
    data = lpgen.tiny_standard_form(0, m=10, n=20, per_col=2)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.col_idx = data.col_idx.copy()
    bad.col_idx[0] = data.n  # out of range
    with pytest.raises(lpm.LPError) as e:
        lpm.LP(bad, eta=0.1)
    assert e.value.status == lpm.LP_ERR_INVALID_ARG
    bad = lpgen.LPData(**{**data.__dict__})
    bad.c = data.c.copy()
    bad.c[3] = np.nan
    with pytest.raises(lpm.LPError):
        lpm.LP(bad, eta=0.1)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.lb = data.lb.copy()
    bad.lb[0] = 5.0
    bad.ub = data.ub.copy()
    bad.ub[0] = 1.0
    with pytest.raises(lpm.LPError):
        lpm.LP(bad, eta=0.1)
    bad = lpgen.LPData(**{**data.__dict__})
    bad.row_ptr = data.row_ptr.copy()
    bad.row_ptr[3] = bad.row_ptr[4] + 1  # not monotone
    with pytest.raises(lpm.LPError):
        lpm.LP(bad, eta=0.1)
    # duplicate column within a row
    rp = np.array([0, 2], np.int32)
    ci = np.array([1, 1], np.int32)
    d2 = lpgen.LPData(1, 3, rp, ci, np.array([1.0, 2.0]), np.ones(3), np.ones(1), np.zeros(3),
                      np.full(3, np.inf), np.zeros(1, np.int8))
    with pytest.raises(lpm.LPError):
        lpm.LP(d2, eta=0.1)
    # tol <= 0
    with lpm.LP(data, eta=0.1) as g:
        with pytest.raises(lpm.LPError):
            g.solve(0.0)


def test_device_and_host_pointers_agree(lpm):
    import torch

    data = lpgen.tiny_standard_form(6, m=50, n=120)
    dev = lpgen.LPData(data.m, data.n, *[torch.as_tensor(a).cuda() for a in
                                         (data.row_ptr, data.col_idx, data.val, data.c, data.b,
                                          data.lb, data.ub, data.row_type)])
    with lpm.LP(data, eta=0.05, max_iter=256) as g1, lpm.LP(dev, eta=0.05, max_iter=256) as g2:
        g1.solve(1e-300)
        g2.solve(1e-300)
        a, b = g1.state(), g2.state()
        xd = torch.empty(data.n, dtype=torch.float64, device="cuda")
        yd = torch.empty(data.m, dtype=torch.float64, device="cuda")
        lpm.lp_get_solution(g2.h, xd, yd)
        torch.cuda.synchronize()
        xs, ys = g1.solution()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(xd.cpu().numpy(), xs)
    np.testing.assert_array_equal(yd.cpu().numpy(), ys)


def test_reproducible_bitwise(lpm):
    data = lpgen.large_mixed(2, m=2000, n=9000)
    outs = []
    for _ in range(2):
        with lpm.LP(data, eta=0.02, max_iter=320, check_every=32) as g:
            g.solve(1e-300)
            outs.append(g.state())
    for k in outs[0]:
        np.testing.assert_array_equal(outs[0][k], outs[1][k])


def test_select_omega_matches_oracle_runs(lpm, oracle_mod):
    """Section 7's primal-weight grid: per-omega relative KKT after a fixed
    number of non-restarted iterations, against the oracle's runs."""
    data = lpgen.tiny_standard_form(3)
    eta = eta_of(oracle_mod, data)
    omegas = [0.25, 1.0, 4.0]
    with lpm.LP(data, eta=eta, check_every=64) as g:
        best, kkt = g.select_omega(omegas, iters=640)
        info = g.info()
        assert info.iters == 0 and info.omega == best
    want = []
    for om in omegas:
        r = oracle_mod.solve(data, eta, omega=om, tol=1e-300, max_iter=640, check_every=64,
                             restart_scheme=oracle_mod.RESTART_NONE)
        want.append(min(r.kkt_avg[4], r.kkt_cur[4]))
    np.testing.assert_allclose(kkt, want, rtol=1e-7)
    assert best == omegas[int(np.argmin(want))]


def test_variant_tuner_picks_a_variant_and_keeps_results(lpm):
    """lp_options.autotune times the unroll variants at lp_create: the chosen
    variants are valid codes, and the iterates equal those of any fixed
    variant (every variant sums each row in the same order)."""
    data = lpgen.large_mixed(11, m=3001, n=15007)
    states = []
    for opts in ({"autotune": 1}, {"autotune": 0, "spmv_unroll": 2, "spmv_unroll_rows": 2},
                 {"autotune": 0, "spmv_unroll": -4, "spmv_unroll_rows": 4}):
        with lpm.LP(data, eta=0.05, check_every=32, max_iter=160, **opts) as g:
            info = g.info()
            if opts["autotune"]:
                assert info.spmv_unroll in (2, 4, -2, -4) and info.spmv_unroll_rows in (2, 4, -2, -4)
            else:
                assert info.spmv_unroll == opts["spmv_unroll"]
            g.solve(1e-300)
            states.append(g.state())
    for st in states[1:]:
        for k in st:
            np.testing.assert_array_equal(st[k], states[0][k])


def test_graph_kernel_count(lpm):
    """lp_info.graph_kernels: none before the first solve; then the 2K iteration
    kernels and the check's 23 (two pair packs, two check passes, finalize,
    eight search passes of two kernels, decision, restart copy)."""
    data = lpgen.tiny_standard_form(0)
    with lpm.LP(data, eta=0.05, check_every=32, max_iter=64, autotune=0) as g:
        assert g.info().graph_kernels == 0
        g.solve(1e-300)
        assert g.info().graph_kernels == 2 * 32 + 23
