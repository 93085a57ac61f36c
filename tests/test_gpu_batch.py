"""Parity of the batched solver (include/lp_batch.h, through the C ABI)
against the CPU oracle run on each problem alone.

Every problem of a batch must follow the single-problem iteration exactly:
same step sizes, same checks every K_k iterations, same restart decisions,
iterates equal to rounding (1e-9 relative, as for the single-problem
solver).  Batches mix problem sizes so that problems span one to many
slices with ragged last slices, and mix row senses and bound kinds.
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


def mixed_batch():
    """Uneven problems: 1 to ~40 slices per operator, every row sense and
    bound kind, empty rows and columns, a dense row and column."""
    return [lpgen.tiny_standard_form(0, m=37, n=61, per_col=3),
            lpgen.adversarial(7),
            lpgen.tiny_standard_form(1),
            lpgen.large_mixed(11, m=301, n=1507),
            lpgen.tiny_standard_form(2, m=5, n=9, per_col=2),
            lpgen.tiny_standard_form(3, m=700, n=1300, per_col=6)]


def norm_bound(d):
    """sqrt(||A||_1 ||A||_inf) >= sigma_max(A): a step size valid for every problem."""
    a = np.abs(d.val)
    rows = np.add.reduceat(a, d.row_ptr[:-1]) if d.nnz else np.zeros(1)
    rows[np.diff(d.row_ptr) == 0] = 0.0
    cols = np.bincount(d.col_idx, weights=a, minlength=d.n)
    return float(np.sqrt(rows.max() * cols.max()))


def start(d):
    """z^{0,0} = proj_{X x Y}(0), the library's starting point."""
    return np.clip(np.zeros(d.n), d.lb, d.ub), np.zeros(d.m)


def osolve(oracle_mod, d, eta, **kw):
    x0, y0 = start(d)
    return oracle_mod.solve(d, eta, x_init=x0, y_init=y0, **kw)


def common_eta(oracle_mod, probs):
    return 0.9 / max(oracle_mod.sigma_max(d) for d in probs)


def states_of(g, probs):
    st = g.state()
    out = []
    for k, d in enumerate(probs):
        xs, ys = slice(g.col_start[k], g.col_start[k + 1]), slice(g.row_start[k], g.row_start[k + 1])
        out.append({key: st[key][xs if key[0] == "x" else ys] for key in st})
    return out


def compare(stk, ref, tol=TOL, what=""):
    for key in ["x", "y", "xbar", "ybar", "x0", "y0"]:
        close(stk[key], getattr(ref, key), tol, f"{what} {key}")


@pytest.mark.parametrize("K", [50, 16])
def test_batch_iterates_match_oracle_per_problem(lpm, oracle_mod, K):
    """The first 100 (K = 50) or 480 (K = 16, 30 checks) iterations."""
    probs = mixed_batch()
    iters = 100 if K == 50 else 480
    eta = common_eta(oracle_mod, probs)
    with lpm.LPBatch(probs, eta=eta, check_every=K, max_iter=iters) as g:
        status = g.solve(1e-300)
        summary, per = g.info()
        sts = states_of(g, probs)
    assert status == lpm.LP_ITER_LIMIT
    assert summary["running"] == 0
    for k, d in enumerate(probs):
        ref = osolve(oracle_mod, d, eta, tol=1e-300, max_iter=iters, check_every=K)
        assert per[k]["iters"] == ref.iters == iters
        assert per[k]["restarts"] == ref.restarts, k
        assert per[k]["checks"] == iters // K
        compare(sts[k], ref, TOL if K == 50 else 1e-8, f"problem {k}")


def test_batch_per_problem_check_periods(lpm, oracle_mod):
    """K_k = 16, 32 or 64 within one batch (K_base = 16): each problem checks
    and restarts on its own schedule."""
    probs = mixed_batch()
    ks = [16, 32, 64, 16, 48, 32]
    eta = common_eta(oracle_mod, probs)
    with lpm.LPBatch(probs, eta=eta, check_every=16, max_iter=384) as g:
        g.set_check_every(ks)
        g.solve(1e-300)
        summary, per = g.info()
        sts = states_of(g, probs)
    for k, d in enumerate(probs):
        ref = osolve(oracle_mod, d, eta, tol=1e-300, max_iter=384, check_every=ks[k])
        assert per[k]["check_every"] == ks[k]
        assert per[k]["checks"] == 384 // ks[k]
        assert per[k]["restarts"] == ref.restarts, k
        compare(sts[k], ref, 1e-8, f"problem {k}")


def test_batch_flexible_and_fixed_schemes(lpm, oracle_mod):
    probs = mixed_batch()[:4]
    eta = common_eta(oracle_mod, probs)
    for scheme, extra in [(3, {}), (1, {"fixed_len": 96}), (0, {})]:
        with lpm.LPBatch(probs, eta=eta, check_every=32, max_iter=320, restart_scheme=scheme,
                         **extra) as g:
            g.solve(1e-300)
            summary, per = g.info()
            sts = states_of(g, probs)
        for k, d in enumerate(probs):
            ref = osolve(oracle_mod, d, eta, tol=1e-300, max_iter=320, check_every=32,
                         restart_scheme=scheme, fixed_len=extra.get("fixed_len", 0))
            assert per[k]["restarts"] == ref.restarts, (scheme, k)
            compare(sts[k], ref, 1e-8, f"scheme {scheme} problem {k}")


def test_batch_sigma_max_per_problem(lpm):
    """Lanczos per problem (the default estimator of sigma_max for Section 7's
    step size) against each problem's largest singular value (dense SVD)."""
    probs = mixed_batch()
    with lpm.LPBatch(probs) as g:
        summary, per = g.info()
    for k, d in enumerate(probs):
        want = float(np.linalg.norm(d.dense(), 2))
        assert per[k]["sigma_max"] == pytest.approx(want, rel=1e-9), k
        assert per[k]["eta"] == pytest.approx(0.9 / per[k]["sigma_max"], rel=1e-15)
        assert 0 < per[k]["sigma_steps"] <= 200


def test_batch_sigma_max_power_iteration(lpm, oracle_mod):
    """Power iteration per problem (Section 7) against the oracle's."""
    probs = mixed_batch()
    with lpm.LPBatch(probs, sigma_method=lpm.LP_SIGMA_POWER) as g:
        summary, per = g.info()
    for k, d in enumerate(probs):
        s_ref = oracle_mod.sigma_max(d)
        assert per[k]["sigma_max"] == pytest.approx(s_ref, rel=1e-8), k
        assert per[k]["eta"] == pytest.approx(0.9 / s_ref, rel=1e-8)
        assert per[k]["tau"] == pytest.approx(per[k]["eta"], rel=1e-15)


def test_batch_full_solve_to_1e8(lpm, oracle_mod):
    """Every problem reaches relative KKT <= 1e-8 (checked by the oracle on
    the returned solution), objective within 1e-7 of the planted optimum,
    with the oracle's iteration count."""
    probs = [lpgen.tiny_standard_form(s, m=m, n=2 * m, per_col=5)
             for s, m in [(0, 40), (1, 80), (2, 150), (9, 60), (4, 100)]]
    eta = common_eta(oracle_mod, probs)
    with lpm.LPBatch(probs, eta=eta, check_every=64, max_iter=150000) as g:
        status = g.solve(1e-8)
        summary, per = g.info()
        x, y = g.solution()
    assert status == lpm.LP_OK
    xs, ys = g.split(x), g.split(y, rows=True)
    for k, d in enumerate(probs):
        assert per[k]["status"] == lpm.LP_OK
        kk = oracle_mod.kkt(d, xs[k], ys[k])
        assert kk["rel"] <= 1e-8 * (1 + 1e-6), k
        assert kk["pobj"] == pytest.approx(d.obj_star, rel=1e-7, abs=1e-7)
        ref = osolve(oracle_mod, d, eta, tol=1e-8, max_iter=150000, check_every=64)
        assert ref.status == 0
        assert per[k]["iters"] == ref.iters, k
        assert per[k]["returned"] == ref.returned


def test_batch_problem_without_rows_and_single_problem(lpm, oracle_mod):
    """Edge cases: a problem with no rows (min c^T x over a box) inside a
    batch, and a batch of one problem."""
    n = 7
    box = lpgen.LPData(0, n, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0),
                       np.linspace(-1.0, 1.0, n), np.zeros(0), np.full(n, -2.0), np.full(n, 3.0),
                       np.zeros(0, np.int8))
    probs = [lpgen.tiny_standard_form(0, m=37, n=61, per_col=3), box]
    eta = 0.1
    with lpm.LPBatch(probs, eta=eta, check_every=16, max_iter=64) as g:
        g.solve(1e-300)
        sts = states_of(g, probs)
    for k, d in enumerate(probs):
        ref = osolve(oracle_mod, d, eta, tol=1e-300, max_iter=64, check_every=16)
        compare(sts[k], ref, TOL, f"problem {k}")
    one = [lpgen.adversarial(7)]
    with lpm.LPBatch(one, eta=eta, check_every=16, max_iter=64) as g:
        g.solve(1e-300)
        sts = states_of(g, one)
    compare(sts[0], osolve(oracle_mod, one[0], eta, tol=1e-300, max_iter=64, check_every=16))


def test_batch_rejects_cross_problem_columns(lpm):
    a, b = lpgen.tiny_standard_form(0, m=5, n=9, per_col=2), lpgen.tiny_standard_form(1, m=5, n=9, per_col=2)
    bad_col = np.concatenate([a.col_idx, b.col_idx])  # problem 1 indexes problem 0's columns
    rp = np.concatenate([a.row_ptr, b.row_ptr[1:] + a.nnz]).astype(np.int32)
    cat = lambda f: np.concatenate([getattr(a, f), getattr(b, f)])
    with pytest.raises(lpm.LPError) as e:
        lpm.lp_batch_create([0, 5, 10], [0, 9, 18], a.nnz + b.nnz, rp, bad_col, cat("val"),
                            cat("c"), cat("b"), cat("lb"), cat("ub"), cat("row_type"))
    assert e.value.status == lpm.LP_ERR_INVALID_ARG
    assert "outside its problem" in str(e.value)


def test_batch_is_bitwise_reproducible(lpm):
    probs = mixed_batch()
    outs = []
    for _ in range(2):
        with lpm.LPBatch(probs, check_every=32, max_iter=640) as g:
            g.solve(1e-300)
            outs.append(g.state())
    for key in outs[0]:
        np.testing.assert_array_equal(outs[0][key], outs[1][key])


def test_batch_tuner_choices_are_valid_and_consistent(lpm):
    """The tuner's check periods are K_base 2^s (s <= max_k_shift) per size
    class, and a tuned batch computes what an untuned batch given the same
    periods computes (the kernel variants only change the launch shape)."""
    probs = mixed_batch()
    with lpm.LPBatch(probs, eta=0.05, check_every=16, max_iter=256,
                     tuning={"autotune": 1, "max_k_shift": 2, "check_budget": 0.05}) as g:
        summary, per = g.info()
        assert summary["tune_ms"] > 0
        ks = [p["check_every"] for p in per]
        for p in per:
            assert p["check_every"] in (16, 32, 64)
            assert summary["class_k"][p["size_class"]] == p["check_every"]
            assert summary["class_iter_ms"][p["size_class"]] > 0
        assert summary["spmv_unroll"] in (2, 4, -2, -4)
        g.solve(1e-300)
        tuned = g.state()
    with lpm.LPBatch(probs, eta=0.05, check_every=16, max_iter=256) as g:
        g.set_check_every(ks)
        g.solve(1e-300)
        plain = g.state()
    for key in tuned:
        close(tuned[key], plain[key], 1e-12, key)


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


def test_batch_mixed_tracks_fp64_oracle(lpm, oracle_mod):
    """Mixed precision in a batch: every problem's iterates follow the FP64
    oracle to FP32 rounding (1e-5 relative, the single-problem mixed
    path's stated error) with the same restart decisions."""
    probs = mixed_batch()
    eta = common_eta(oracle_mod, probs)
    with lpm.LPBatch(probs, eta=eta, check_every=32, max_iter=192,
                     precision=lpm.LP_PRECISION_MIXED) as g:
        g.solve(1e-300)
        summary, per = g.info()
        sts = states_of(g, probs)
    for k, d in enumerate(probs):
        ref = osolve(oracle_mod, d, eta, tol=1e-300, max_iter=192, check_every=32)
        assert per[k]["restarts"] == ref.restarts, k
        for key in ("x", "y", "xbar", "ybar", "x0", "y0"):
            assert rel_err(sts[k][key], getattr(ref, key)) <= 1e-5, (k, key)


def test_batch_mixed_full_solve_reaches_fp64_tolerance(lpm, oracle_mod):
    probs = [lpgen.tiny_standard_form(s, m=m, n=2 * m, per_col=5)
             for s, m in [(0, 40), (1, 80), (9, 60)]]
    with lpm.LPBatch(probs, check_every=64, max_iter=400000,
                     precision=lpm.LP_PRECISION_MIXED) as g:
        status = g.solve(1e-8)
        summary, per = g.info()
        x, y = g.solution()
    assert status == lpm.LP_OK
    xs, ys = g.split(x), g.split(y, rows=True)
    for k, d in enumerate(probs):
        kk = oracle_mod.kkt(d, xs[k], ys[k])
        assert kk["rel"] <= 1e-8 * (1 + 1e-6), k
        assert kk["pobj"] == pytest.approx(d.obj_star, rel=1e-7, abs=1e-7)
        assert np.all(xs[k] >= d.lb)


def test_batch_of_many_tiny_problems(lpm, oracle_mod):
    """1,500 problems (more than one 1,024-thread block of the work-list scan,
    down to 3 rows): sampled problems against the oracle after 96 iterations."""
    rng = np.random.default_rng(9)
    probs = [lpgen.tiny_standard_form(int(s), m=int(m), n=2 * int(m), per_col=2)
             for s, m in zip(range(1500), rng.integers(3, 25, 1500))]
    eta = 0.1
    with lpm.LPBatch(probs, eta=eta, check_every=32, max_iter=96) as g:
        g.solve(1e-300)
        summary, per = g.info()
        st = g.state()
    assert summary["count"] == 1500 and summary["running"] == 0
    for k in [0, 1, 777, 1023, 1024, 1025, 1499]:
        d = probs[k]
        ref = osolve(oracle_mod, d, eta, tol=1e-300, max_iter=96, check_every=32)
        assert per[k]["iters"] == 96 and per[k]["restarts"] == ref.restarts, k
        xs = slice(int(g.col_start[k]), int(g.col_start[k + 1]))
        ys = slice(int(g.row_start[k]), int(g.row_start[k + 1]))
        close(st["x"][xs], ref.x, TOL, f"{k} x")
        close(st["y"][ys], ref.y, TOL, f"{k} y")
        close(st["xbar"][xs], ref.xbar, TOL, f"{k} xbar")


def test_batch_device_input_arrays(lpm):
    """The batch reads device arrays as well as host arrays (same result)."""
    import torch

    probs = mixed_batch()[:3]
    with lpm.LPBatch(probs, eta=0.05, check_every=32, max_iter=128) as g:
        g.solve(1e-300)
        want = g.state()
        rs, cs = g.row_start, g.col_start
    ms = [d.m for d in probs]
    rp = np.concatenate([[0]] + [np.asarray(d.row_ptr[1:], np.int64) + o for d, o in
                                 zip(probs, np.cumsum([0] + [d.nnz for d in probs])[:-1])])
    ci = np.concatenate([np.asarray(d.col_idx, np.int64) + c0 for d, c0 in zip(probs, cs[:-1])])
    cat = lambda f, dt: torch.as_tensor(np.concatenate([np.asarray(getattr(d, f), dt) for d in probs])).cuda()
    opt = lpm.lp_default_options()
    opt.eta, opt.check_every, opt.max_iter = 0.05, 32, 128
    h = lpm.lp_batch_create(rs, cs, int(rp[-1]), torch.as_tensor(rp.astype(np.int32)).cuda(),
                            torch.as_tensor(ci.astype(np.int32)).cuda(), cat("val", np.float64),
                            cat("c", np.float64), cat("b", np.float64), cat("lb", np.float64),
                            cat("ub", np.float64), cat("row_type", np.int8), opt)
    try:
        lpm.lp_batch_solve(h, 1e-300)
        got = {k: np.empty_like(v) for k, v in want.items()}
        lpm.lp_batch_get_state(h, got["x"], got["y"], got["xbar"], got["ybar"], got["x0"], got["y0"])
    finally:
        lpm.lp_batch_destroy(h)
    for k in want:
        np.testing.assert_array_equal(got[k], want[k])
    assert sum(ms) == int(rs[-1])


def test_batch_warm_start_matches_oracle(lpm, oracle_mod):
    """lp_batch_set_state: every problem restarts from the projection of the
    given point (random, partly outside the bounds) and follows the oracle
    started there."""
    probs = mixed_batch()[:4]
    eta = common_eta(oracle_mod, probs)
    starts = [lpgen.random_state(d, 20 + k) for k, d in enumerate(probs)]
    x0 = np.concatenate([s[0] for s in starts]) * 1.5  # some coordinates leave the box
    y0 = np.concatenate([s[1] for s in starts])
    with lpm.LPBatch(probs, eta=eta, check_every=32, max_iter=160) as g:
        g.set_state(x0, y0)
        g.solve(1e-300)
        sts = states_of(g, probs)
    co, ro = 0, 0
    for k, d in enumerate(probs):
        xs = np.clip(x0[co:co + d.n], d.lb, d.ub)
        ys = y0[ro:ro + d.m].copy()
        ys[d.row_type == 1] = np.maximum(ys[d.row_type == 1], 0.0)
        ys[d.row_type == 2] = np.minimum(ys[d.row_type == 2], 0.0)
        ref = oracle_mod.solve(d, eta, tol=1e-300, max_iter=160, check_every=32, x_init=xs,
                               y_init=ys)
        compare(sts[k], ref, TOL, f"problem {k}")
        co += d.n
        ro += d.m


def test_batch_select_omega_matches_oracle(lpm, oracle_mod):
    """Section 7's primal-weight grid for every problem at once: each problem's
    relative KKT per omega (no restarts, 256 iterations) against the oracle's,
    the same choice per problem, and afterwards each problem iterates with its
    own omega exactly as the oracle does."""
    probs = mixed_batch()[:4]
    eta = common_eta(oracle_mod, probs)
    grid = [0.25, 1.0, 4.0]
    with lpm.LPBatch(probs, eta=eta, check_every=32, max_iter=192) as g:
        best, kkt = g.select_omega(grid, iters=256)
        _, per = g.info()
        g.solve(1e-300)
        sts = states_of(g, probs)
    for k, d in enumerate(probs):
        ref = [osolve(oracle_mod, d, eta, omega=om, tol=1e-300, max_iter=256, check_every=32,
                      restart_scheme=0) for om in grid]
        ref_kkt = [min(r.kkt_avg[4], r.kkt_cur[4]) for r in ref]
        np.testing.assert_allclose(kkt[k], ref_kkt, rtol=1e-7)
        assert best[k] == grid[int(np.argmin(ref_kkt))]
        assert per[k]["omega"] == best[k]
        assert per[k]["tau"] == pytest.approx(eta / best[k], rel=1e-15)
        after = osolve(oracle_mod, d, eta, omega=best[k], tol=1e-300, max_iter=192, check_every=32)
        compare(sts[k], after, 1e-8, f"problem {k} after selection")
