"""Benchmark: restarted-PDHG iterations per second on the large mixed LP.

Workload: m = 200,000 rows (70% EQ, 30% GE), n = 1,000,000 columns (40%
[0,inf), 40% [0,U(1,10)], 20% free), power-law column degree on 2..200
(~10.07M nonzeros), N(0,1) values, planted optimum; seeded (seed 1).
A step is one block of K = 64 PDHG iterations followed by one check (KKT
of average and current iterate, normalized duality gap by the multiplier
search, adaptive restart decision): every row of the hot path.

value = PDHG iterations / second (device-timed, inputs resident in HBM;
the working set, ~330 MB, exceeds the 129 MB L2, so no flush is needed).
e2e   = the same metric through the C ABI from HOST buffers: lp_create
        (host arrays, H2D inside), lp_solve for a fixed iteration budget,
        lp_get_solution into host memory, lp_destroy, per step.

Also reported (outside the timed region): time to relative KKT 1e-8 with the
paper's recipe (primal weight by Section 7's grid search, then adaptive
restarted PDHG), FP64 vs mixed, on the benchmark LP itself (with the reduced
and with the paper's own grid) and on two smaller LPs; mixed-precision
throughput; the multicommodity LP (throughput, a 100 x 100 grid to 1e-8 FP64
vs mixed, a small instance against HiGHS); the adjoint (single LP,
implicit-KKT check, 64-LP batch); the 200 x 400 LP alone and 512 of them as
one batch; the 512-LP batched solver to 1e-8; the column pass's roofline
(traffic from a committed ncu capture keyed by the kernels' source hash) and
its gather ceilings; the oracle on all host cores and on one.

--impl reference times the CPU oracle (plain C, FP64, its OpenMP build on
all host cores) on a bounded sample of the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K_CHECK = 64
OMEGA_GRID = [4.0 ** k for k in range(-3, 4)]  # reduced Section 7 grid, 2048 iterations each
OMEGA_ITERS = 2048  # a multiple of the check period (the batch needs one)
PAPER_OMEGA_GRID = [4.0 ** k for k in range(-5, 6)]  # Section 7: 4^-5 .. 4^5
PAPER_OMEGA_ITERS = 5000  # Section 7: 5,000 iterations without restarts per weight
FALLBACK_HBM_GBS = 6800.0
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one column-pass
# launch on this workload with warm L2, per kernel variant, from one-pass ncu
# captures kept as text under profiles/; each row names the hash of the kernel
# sources it was taken with, so a kernel changed since reports null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "primal_kernel_traffic_large_mixed.md")
KERNEL_SOURCES = ["lp_kernels.cu", "spmv_core.cuh", "lp_internal.h"]
# Random-gather ceilings on GB300 (G gathers/s), measured once by a gather
# microbenchmark with every block resident: 8-byte __ldg gathers from a
# 1.6 MB L2-resident vector alone, and a sliced SpMV (one warp per 32 columns
# of 10 elements, int32 indices and FP64 values streamed from a 126 MB matrix)
# with the column pass's per-column reads and writes.
GATHER_CEILINGS = {"random_gathers_1p6MB": 330.0, "sliced_spmv_with_epilogue_traffic": 224.0}


def kernel_source_hash():
    """SHA-256 (first 16 hex digits) of the iteration kernels' sources."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2105_12715_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(variant):
    """Bytes per launch of the column pass for this variant, read from the
    committed capture table (rows '| variant | source hash | bytes |'), or
    None when no row matches the variant and the current sources."""
    try:
        want = kernel_source_hash()
        for line in open(TRAFFIC_FILE):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 3 and cells[0] == str(variant) and cells[1] == want:
                return float(cells[2])
    except (OSError, ValueError):
        pass
    return None


def host_info():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                             timeout=10).stdout.decode()
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": os.uname().machine}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=200_000)
    p.add_argument("--n", type=int, default=1_000_000)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--e2e-iters", type=int, default=6400)
    p.add_argument("--cpu-iters", type=int, default=64)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--no-ttk", action="store_true")
    p.add_argument("--no-mcf", action="store_true")
    p.add_argument("--no-long-row", action="store_true")
    p.add_argument("--no-schemes", action="store_true")
    p.add_argument("--schemes-cap", type=int, default=400_000)
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--adjoint-lps", type=int, default=4)
    p.add_argument("--no-ttk-large", action="store_true")
    p.add_argument("--ttk-large-cap", type=int, default=1_500_000)
    p.add_argument("--no-paper-grid", action="store_true",
                   help="skip the benchmark LP solved with the paper's full primal-weight grid")
    p.add_argument("--no-mcf-ttk", action="store_true",
                   help="skip the multicommodity LP solved to a relative KKT tolerance")
    p.add_argument("--mcf-full-ttk", action="store_true",
                   help="also run the full-size multicommodity LP to --mcf-tol, FP64 and mixed")
    p.add_argument("--mcf-tol", type=float, default=1e-3,
                   help="tolerance of the full-size multicommodity time-to-tolerance runs")
    p.add_argument("--mcf-cap", type=int, default=1_000_000)
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--batch-cap", type=int, default=1_000_000)
    p.add_argument("--batch-loop-sample", type=int, default=8)
    p.add_argument("--batch-schemes", action="store_true",
                   help="also solve the batch with the flexible and no-restart schemes")
    p.add_argument("--batch-only", action="store_true",
                   help="run only the batched section and print its JSON (profiling)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--kernel-reps", type=int, default=50)  # >= 1
    p.add_argument("--spmv-unroll", type=int, default=None, choices=[-4, -2, 2, 4],
                   help="fix the column-pass variant (no tuner) for the headline solver")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args):
    from paper_2105_12715_gb300 import lpgen

    return lpgen.large_mixed(args.seed, m=args.m, n=args.n)


def config_of(args, data):
    return {"workload": f"large_mixed LP m={data.m} n={data.n} nnz={data.nnz} "
                        f"(70% EQ/30% GE rows; 40% [0,inf), 40% [0,U], 20% free cols; "
                        f"power-law col degree 2..200; seed {args.seed})",
            "m": data.m, "n": data.n, "nnz": data.nnz, "check_every": K_CHECK,
            "restart": "adaptive beta=e^-1", "precision": "fp64",
            "l2": "working set > L2 (129 MB); no flush"}


def algorithmic_bytes(m, n, nnz):
    """Bytes one FP64 PDHG iteration must move (each array once, gathers once)."""
    primal = 12 * nnz + 64 * n + 8 * m  # A^T values+indices; c,l,u,x,xbar in; x,xhat,xbar out; y gathered
    dual = 12 * nnz + 41 * m + 8 * n    # A values+indices; b,y,ybar,rowtype in; y,ybar out; xhat gathered
    return primal, dual


def algorithmic_bytes_mixed(m, n, nnz):
    """The same for the mixed path: FP32 values, iterates and correction data, FP64 averages."""
    primal = 8 * nnz + 40 * n + 4 * m  # cf,lf,uf,dx (f32) + dxbar in; dx,dxhat (f32) + dxbar out; dy gathered
    dual = 8 * nnz + 36 * m + 4 * n    # bf,ylo,yhi,dy (f32) + dybar in; dy (f32) + dybar out; dxhat gathered
    return primal, dual


def time_steps(lp, g, stream, steps):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.iterate(steps, 1e-300)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def time_kernel(lp, g, which, reps, stream):
    import torch

    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    lp.lp_profile_kernel(g.h, which, reps, stream)
    k1.record(stream)
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / reps


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs_sustained", "hbm_gbs"):
                if k in d and d[k]:
                    return float(d[k]), f"measured ({k})"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        """Starts nvidia-smi and waits (up to 5 s) for its first sample, so the
        samples of the region that follows are not lost to its start-up."""
        self.skip = 0
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def mark(self):
        """Start of the timed region: samples written before it are dropped."""
        try:
            with open(self.path) as fh:
                self.skip = sum(1 for _ in fh)
        except OSError:
            self.skip = 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        # the samples of the timed region, and the one taken just before it
        # when the region was shorter than the sampling interval
        lines = lines[max(0, self.skip - 1):] if len(lines) > self.skip else lines[-1:]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_openmp_available():
    import oracle

    try:
        oracle.build(openmp=True)
        return True
    except Exception:  # noqa: BLE001
        return False


def highs_objective(d):
    """Optimal objective of an LP by SciPy's HiGHS (None if unavailable)."""
    try:
        import scipy.sparse as sp
        from scipy.optimize import linprog
    except ImportError:
        return None
    A = sp.csr_matrix((d.val, d.col_idx, d.row_ptr), shape=(d.m, d.n))
    eq, ge, le = d.row_type == 0, d.row_type == 1, d.row_type == 2
    A_ub = sp.vstack([A[le], -A[ge]]).tocsr()
    b_ub = np.concatenate([d.b[le], -d.b[ge]])
    bounds = [(lo if np.isfinite(lo) else None, hi if np.isfinite(hi) else None)
              for lo, hi in zip(d.lb, d.ub)]
    r = linprog(d.c, A_ub=A_ub if A_ub.shape[0] else None, b_ub=b_ub if b_ub.size else None,
                A_eq=A[eq] if eq.any() else None, b_eq=d.b[eq] if eq.any() else None,
                bounds=bounds, method="highs")
    return float(r.fun) if r.status == 0 else None


def cpu_baseline(args, data, eta):
    """The oracle on a bounded sample: cpu_iters iterations with one check
    every 64 (the same workload, the GPU's step size), on all host cores (its
    OpenMP build: the row products and elementwise loops split over the
    cores, A^T y a serial scatter) and on one thread (the default build)."""
    import oracle

    olp = oracle.OracleLP(data)
    host = host_info()
    single = None
    t = time.perf_counter()
    res = oracle.solve(olp, eta, tol=1e-300, max_iter=args.cpu_iters, check_every=K_CHECK)
    dt = time.perf_counter() - t
    single = {"value": res.iters / dt, "cores": 1, "seconds": dt}
    out = {"value": single["value"], "unit": "iters/s", "cores": 1, "kind": "oracle",
           "sample": f"{res.iters} oracle iterations incl. {res.n_checks} check(s) on the full "
                     f"workload, {dt:.1f} s", "host": host, "single_thread": single}
    if oracle_openmp_available():
        t = time.perf_counter()
        res = oracle.solve(olp, eta, tol=1e-300, max_iter=args.cpu_iters, check_every=K_CHECK,
                           openmp=True)
        dt = time.perf_counter() - t
        out.update({"value": res.iters / dt, "cores": host["nproc"],
                    "sample": f"{res.iters} oracle iterations incl. {res.n_checks} check(s) on "
                              f"the full workload, OpenMP build on {host['nproc']} threads, "
                              f"{dt:.1f} s"})
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    data = workload(args)
    import oracle

    oracle.build()
    # a valid step size without a sigma_max estimate on the host: sigma_max(A) is at most
    # sqrt(||A||_1 ||A||_inf) (largest column and row absolute sums)
    a = np.abs(data.val)
    row_sums = np.add.reduceat(a, data.row_ptr[:-1]) if data.nnz else np.zeros(1)
    row_sums[np.diff(data.row_ptr) == 0] = 0.0
    col_sums = np.bincount(data.col_idx, weights=a, minlength=data.n)
    eta = 0.9 / max(float(np.sqrt(row_sums.max() * col_sums.max())), 1e-300)
    per_step = 4  # oracle iterations per step (bounded sample; a check every 64 iterations)
    omp = oracle_openmp_available()
    host = host_info()
    cores = host["nproc"] if omp else 1
    olp = oracle.OracleLP(data)
    oracle.solve(olp, eta, tol=1e-300, max_iter=per_step * args.warmup, check_every=K_CHECK,
                 openmp=omp)
    total = per_step * args.steps
    t = time.perf_counter()
    res = oracle.solve(olp, eta, tol=1e-300, max_iter=total, check_every=K_CHECK, openmp=omp)
    dt = time.perf_counter() - t
    v = res.iters / dt
    line = {"metric": "PDHG iterations/s (fp64 restarted PDHG, large mixed LP)", "value": v,
            "unit": "iters/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(args, data),
            "cpu_baseline": {"value": v, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"{res.iters} oracle iterations ({per_step} per step), "
                                       f"{res.n_checks} check(s)"
                                       + (f", OpenMP build on {cores} threads" if omp else
                                          ", one thread"),
                             "host": host},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args, lp, stream, barrier):
    """Batched solver on 512 uneven standard-form LPs (m log-uniform in
    [50, 20000], n = 2m, 3-12 nonzeros per column): tuned create, aggregate
    throughput (device-timed blocks of 64 iterations), and time to relative
    KKT 1e-8 (per-problem cap batch_cap iterations) against solving the same
    problems one at a time with the plain FP64 path (lp_create + lp_solve on
    a seeded sample, scaled to the whole batch)."""
    import torch

    from paper_2105_12715_gb300 import lpgen

    from paper_2105_12715_gb300 import dist as pdist

    probs = lpgen.batch_standard_form(2, args.batch_count)
    M = sum(d.m for d in probs)
    N = sum(d.n for d in probs)
    Z = sum(d.nnz for d in probs)
    res = {"workload": f"batch_standard_form seed 2: {len(probs)} LPs, m log-uniform [50,20000], "
                       f"n=2m, 3-12 nnz/col, x>=0, EQ rows; total m={M} n={N} nnz={Z}",
           "check_every_base": K_CHECK}
    ws, rank, _ = dist_env()
    if ws > 1:  # shard by problem (balanced by nonzeros); no data-path collective
        mine = pdist.shard_by_weight([d.nnz for d in probs], ws, rank)
        probs = [probs[i] for i in mine]
        M = sum(d.m for d in probs)
        N = sum(d.n for d in probs)
        Z = sum(d.nnz for d in probs)
        res["sharding"] = f"{ws} ranks, problems balanced by nonzeros"
    barrier()
    t0 = time.perf_counter()
    g = lp.LPBatch(probs, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                   tuning={"autotune": 1})
    torch.cuda.synchronize()
    res["create_s"] = time.perf_counter() - t0
    summary, per = g.info()
    res["tuner"] = {"spmv_unroll": summary["spmv_unroll"],
                    "spmv_unroll_rows": summary["spmv_unroll_rows"],
                    "grid_cols": summary["grid_cols"], "grid_rows": summary["grid_rows"],
                    "class_k": summary["class_k"],
                    "class_iter_ms": [round(v, 4) for v in summary["class_iter_ms"]],
                    "class_check_ms": [round(v, 4) for v in summary["class_check_ms"]],
                    "tune_ms": summary["tune_ms"]}
    g.iterate(2, 1e-300)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb = 8
    torch.cuda.nvtx.range_push("batch_blocks")
    e0.record(stream)
    g.iterate(nb, 1e-300)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms_block = e0.elapsed_time(e1) / nb
    pb, db = algorithmic_bytes(M, N, Z)
    rate, slowest = pdist.job_throughput(len(probs) * K_CHECK * nb, ms_block * nb / 1000.0)
    bytes_all = pdist.reduce_scalar(pb + db, "sum")
    res["iter_us"] = 1e6 * slowest / (K_CHECK * nb)
    res["problem_iters_per_s"] = rate
    res["achieved_gbs_per_iter"] = bytes_all / (slowest / (K_CHECK * nb)) / 1e9
    res["bytes_per_iter_algorithmic"] = bytes_all
    g.close()
    # time to 1e-8 (fresh batch; setup = create incl. the sigma_max estimate and tuning; omega = 1:
    # on these problems the grid of Section 7 converges fewer of them within the cap)
    barrier()
    t0 = time.perf_counter()
    g = lp.LPBatch(probs, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                   tuning={"autotune": 1})
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    g.solve(1e-8)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    summary, per = g.info()
    its = np.array([p["iters"] for p in per])
    conv = np.array([p["status"] == lp.LP_OK for p in per])
    g.close()
    t_batch = pdist.reduce_scalar(t_batch, "max")
    t_setup = pdist.reduce_scalar(t_setup, "max")
    kkt_fin = np.array([min(p["kkt_avg"][4], p["kkt_cur"][4]) for p in per])
    unconv = np.flatnonzero(~conv)
    res["solve"] = {"tol": 1e-8, "cap_iters": args.batch_cap, "seconds": t_batch,
                    "seconds_with_setup": t_batch + t_setup,
                    "converged": int(pdist.reduce_scalar(conv.sum(), "sum")),
                    "problems": int(pdist.reduce_scalar(len(probs), "sum")),
                    "iters_median": float(np.median(its)),
                    "iters_sum": int(pdist.reduce_scalar(its.sum(), "sum")), "omega": 1.0,
                    # every problem that did not reach 1e-8 within the cap, with its final
                    # relative KKT error (the smaller of its two candidates) and its rows
                    "unconverged": {
                        "count": int(unconv.size),
                        "final_rel_kkt_quantiles_0_50_90_100": (
                            [float(q) for q in np.quantile(kkt_fin[unconv], [0, 0.5, 0.9, 1])]
                            if unconv.size else None),
                        "below_1e6": int((kkt_fin[unconv] <= 1e-6).sum()),
                        "below_1e7": int((kkt_fin[unconv] <= 1e-7).sum()),
                        "problems": [[int(k), int(probs[k].m), float("%.3g" % kkt_fin[k])]
                                     for k in unconv]}}
    # the plain FP64 path, one problem at a time, on a seeded sample
    rng = np.random.default_rng(0)
    idx = rng.choice(len(probs), size=min(max(args.batch_loop_sample, 1), len(probs)),
                     replace=False)
    t_loop, same, conv_loop = 0.0, 0, 0
    for k in idx:
        barrier()
        t0 = time.perf_counter()
        h = lp.LP(probs[k], stream=stream, check_every=K_CHECK, max_iter=args.batch_cap)
        st = h.solve(1e-8)
        torch.cuda.synchronize()
        t_loop += time.perf_counter() - t0
        conv_loop += int(st == lp.LP_OK)
        same += int(abs(h.info().iters - int(its[k])) <= K_CHECK)
        h.close()
    est = pdist.reduce_scalar(t_loop * len(probs) / len(idx), "max")  # ranks loop in parallel
    res["loop_fp64"] = {"sample": len(idx), "sample_seconds": t_loop,
                        "extrapolated_seconds": est, "converged_in_sample": conv_loop,
                        "same_iteration_count": same,
                        "note": "lp_create + lp_solve per problem (setup included); total = "
                                "sample time x problems / sample size (per rank, max over ranks)"}
    res["speedup_vs_loop"] = est / (t_batch + t_setup)  # both with setup
    # the FP32-mixed batch: same problems, same timing
    barrier()
    t0 = time.perf_counter()
    g = lp.LPBatch(probs, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                   tuning={"autotune": 1}, precision=lp.LP_PRECISION_MIXED)
    torch.cuda.synchronize()
    t_setup_m = time.perf_counter() - t0
    g.iterate(2, 1e-300)
    barrier()
    e0.record(stream)
    g.iterate(nb, 1e-300)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_block_m = e0.elapsed_time(e1) / nb
    g.close()
    barrier()
    t0 = time.perf_counter()
    g = lp.LPBatch(probs, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                   tuning={"autotune": 1}, precision=lp.LP_PRECISION_MIXED)
    torch.cuda.synchronize()
    t_setup_m = time.perf_counter() - t0
    t0 = time.perf_counter()
    g.solve(1e-8)
    torch.cuda.synchronize()
    t_mixed = time.perf_counter() - t0
    summary, per = g.info()
    its_m = np.array([p["iters"] for p in per])
    conv_m = np.array([p["status"] == lp.LP_OK for p in per])
    g.close()
    rate_m, slowest_m = pdist.job_throughput(len(probs) * K_CHECK * nb, ms_block_m * nb / 1000.0)
    t_mixed = pdist.reduce_scalar(t_mixed, "max")
    t_setup_m = pdist.reduce_scalar(t_setup_m, "max")
    res["mixed"] = {"iter_us": 1e6 * slowest_m / (K_CHECK * nb), "problem_iters_per_s": rate_m,
                    "solve_seconds": t_mixed, "solve_seconds_with_setup": t_mixed + t_setup_m,
                    "converged": int(pdist.reduce_scalar(conv_m.sum(), "sum")),
                    "iters_median": float(np.median(its_m)),
                    "converged_both": int(pdist.reduce_scalar((conv & conv_m).sum(), "sum"))}
    if args.batch_schemes:
        # the shape of Table 3 on the batch: problems converged to relative KKT 1e-8 within the
        # iteration cap with the adaptive, flexible and no-restart schemes (FP64, K = 64)
        res["restart_schemes"] = {}
        for name, scheme in (("adaptive", lp.LP_RESTART_ADAPTIVE),
                             ("flexible", lp.LP_RESTART_FLEXIBLE),
                             ("no_restart", lp.LP_RESTART_NONE)):
            t0 = time.perf_counter()
            gb = lp.LPBatch(probs, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                            restart_scheme=scheme)
            gb.solve(1e-8)
            torch.cuda.synchronize()
            _, per_s = gb.info()
            gb.close()
            its_s = [p["iters"] for p in per_s if p["status"] == lp.LP_OK]
            res["restart_schemes"][name] = {
                "converged": int(pdist.reduce_scalar(len(its_s), "sum")),
                "median_iters_converged": float(np.median(its_s)) if its_s else None,
                "seconds_with_setup": pdist.reduce_scalar(time.perf_counter() - t0, "max")}
    return res


def run_batch_only(args):
    import torch

    from paper_2105_12715_gb300 import lp

    torch.cuda.set_device(0)
    lp.load()
    res = run_batched(args, lp, torch.cuda.current_stream(), torch.cuda.synchronize)
    print(json.dumps({"batched": res}))
    return 0


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2105_12715_gb300 import lp

    lp.load()
    data = workload(args)
    stream = torch.cuda.current_stream()
    fixed = ({} if args.spmv_unroll is None
             else {"autotune": 0, "spmv_unroll": args.spmv_unroll})
    g = lp.LP(data, stream=stream, check_every=K_CHECK, **fixed)
    info0 = g.info()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    # warm-up
    g.iterate(args.warmup, 1e-300)
    barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    sampler.mark()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.iterate(args.steps, 1e-300)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    iters = args.steps * K_CHECK
    from paper_2105_12715_gb300 import dist as pdist

    # replicas: iterations of all ranks over the slowest rank's time
    value, slowest = pdist.job_throughput(iters, ms / 1000.0, device="cuda")
    ms = 1000.0 * slowest
    info = g.info()
    # per step: one replay of the graph (2 K iteration kernels and the check's kernels)
    launches_per_step = info.graph_kernels

    # dominant kernel timed alone with CUDA events (same stream, same data)
    primal_b, dual_b = algorithmic_bytes(data.m, data.n, data.nnz)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    lp.lp_profile_kernel(g.h, 0, args.kernel_reps, stream)
    k1.record(stream)
    torch.cuda.synchronize()
    primal_ms = k0.elapsed_time(k1) / args.kernel_reps
    k0.record(stream)
    lp.lp_profile_kernel(g.h, 1, args.kernel_reps, stream)
    k1.record(stream)
    torch.cuda.synchronize()
    dual_ms = k0.elapsed_time(k1) / args.kernel_reps
    peak, peak_kind = peaks()
    achieved = primal_b / (primal_ms / 1000.0) / 1e9
    g.close()
    # the column pass against the random-gather ceilings of this GPU (one
    # 8-byte gather per nonzero from the L2-resident y)
    ach_g = data.nnz / (primal_ms / 1000.0) / 1e9
    gather_bound = {"gathers_per_launch": data.nnz, "achieved_ggathers_per_s": ach_g,
                    "ceilings_ggathers_per_s": GATHER_CEILINGS,
                    "frac_of_random_gathers": ach_g / GATHER_CEILINGS["random_gathers_1p6MB"],
                    "frac_of_sliced_spmv": ach_g / GATHER_CEILINGS["sliced_spmv_with_epilogue_traffic"],
                    "source": "gather microbenchmark on GB300, measured once (not re-run here)"}

    # end to end through the C ABI from host buffers
    e2e_vals, h2d, e2e_setup = [], 0, None
    host = [np.ascontiguousarray(a) for a in (data.row_ptr, data.col_idx, data.val, data.c, data.b,
                                              data.lb, data.ub, data.row_type)]
    pinned = [torch.from_numpy(a).pin_memory() for a in host]
    h2d = sum(a.numel() * a.element_size() for a in pinned)
    xo = torch.empty(data.n, dtype=torch.float64).pin_memory()
    yo = torch.empty(data.m, dtype=torch.float64).pin_memory()
    d2h = (data.n + data.m) * 8
    for _ in range(args.e2e_steps):
        barrier()
        t = time.perf_counter()
        opt = lp.lp_default_options()
        opt.check_every = K_CHECK
        opt.max_iter = args.e2e_iters
        h = lp.lp_create(data.m, data.n, data.nnz, *pinned, opt=opt, stream=stream)
        lp.lp_solve(h, 1e-300, stream)
        lp.lp_get_solution(h, xo, yo, stream)
        e2e_setup = list(lp.lp_get_info(h).setup_ms)
        lp.lp_destroy(h)
        barrier()
        e2e_vals.append(args.e2e_iters / (time.perf_counter() - t))
    e2e = {"value": ws * float(np.median(e2e_vals)) if e2e_vals else None, "unit": "iters/s",
           "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h,
           "what": f"lp_create(host arrays)+lp_solve({args.e2e_iters} iters)+lp_get_solution(host)",
           "lp_create_ms": (dict(zip(["inputs", "layout", "upload", "sigma_max"], e2e_setup))
                            if e2e_setup else None)}

    # mixed precision on the same workload (same step, same timing rules)
    mixed = None
    if not args.no_mixed:
        gm = lp.LP(data, stream=stream, check_every=K_CHECK, eta=info0.eta,
                   precision=lp.LP_PRECISION_MIXED)
        gm.iterate(args.warmup, 1e-300)
        barrier()
        msm = time_steps(lp, gm, stream, args.steps)
        mp, md = algorithmic_bytes_mixed(data.m, data.n, data.nnz)
        mp_ms = time_kernel(lp, gm, 0, args.kernel_reps, stream)
        md_ms = time_kernel(lp, gm, 1, args.kernel_reps, stream)
        gm.close()
        mixed = {"value": ws * args.steps * K_CHECK / (msm / 1000.0), "unit": "iters/s",
                 "ms_per_step": msm / args.steps, "dtype": "f32 iterations, f64 averages/checks",
                 "bytes_per_iter_algorithmic": mp + md,
                 "primal_kernel_ms": mp_ms, "dual_kernel_ms": md_ms,
                 "primal_achieved_gbs": mp / (mp_ms / 1000.0) / 1e9}

    # time to relative KKT 1e-8 (the paper's recipe: primal weight by the grid search of
    # Section 7, then adaptive restarted PDHG), FP64 vs mixed, setup included
    def ttk_run(d, tol, prec, select, cap, grid=None, grid_iters=None):
        barrier()
        t0 = time.perf_counter()
        gt = lp.LP(d, stream=stream, check_every=K_CHECK, max_iter=cap, precision=prec)
        omega, t_sel = 1.0, 0.0
        if select:
            ts = time.perf_counter()
            omega, _ = gt.select_omega(grid or OMEGA_GRID, iters=grid_iters or OMEGA_ITERS)
            t_sel = time.perf_counter() - ts
        st = gt.solve(tol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        it = gt.info()
        gt.close()
        pobj = it.kkt_avg[2] if it.returned == 0 else it.kkt_cur[2]
        out = {"seconds": dt, "omega": omega, "omega_select_seconds": t_sel, "iters": it.iters,
               "eta": it.eta, "omega_grid": [min(grid or OMEGA_GRID), max(grid or OMEGA_GRID),
                                             grid_iters or OMEGA_ITERS] if select else None,
               "restarts": it.restarts, "status": lp.STATUS_NAMES.get(st, st),
               "rel_kkt": min(it.kkt_avg[4], it.kkt_cur[4]), "pobj": pobj}
        if d.obj_star is not None:  # the planted optimum's objective (unique)
            out["obj_rel_err_vs_planted"] = abs(pobj - d.obj_star) / max(1.0, abs(d.obj_star))
        return out

    def mixed_error(res):
        """The mixed-precision result against the FP64 one on the same LP."""
        f, m_ = res["fp64"]["pobj"], res["mixed"]["pobj"]
        res["mixed_vs_fp64_obj_rel"] = abs(m_ - f) / max(1.0, abs(f))

    ttk = ttk8 = ttk_large = None
    if not args.no_ttk:
        from paper_2105_12715_gb300 import lpgen

        med = lpgen.large_mixed(5, m=20_000, n=100_000)
        ttk = {"lp": f"large_mixed m={med.m} n={med.n} nnz={med.nnz} seed 5", "tol": 1e-8,
               "omega": "grid search (Section 7)"}
        for name, prec in (("fp64", lp.LP_PRECISION_FP64), ("mixed", lp.LP_PRECISION_MIXED)):
            ttk[name] = ttk_run(med, 1e-8, prec, True, 3_000_000)
        mixed_error(ttk)
        small = lpgen.large_mixed(5, m=5000, n=25000)
        ttk8 = {"lp": f"large_mixed m={small.m} n={small.n} nnz={small.nnz} seed 5", "tol": 1e-8}
        for name, prec in (("fp64", lp.LP_PRECISION_FP64), ("mixed", lp.LP_PRECISION_MIXED)):
            ttk8[name + "_omega1"] = ttk_run(small, 1e-8, prec, False, 3_000_000)
            ttk8[name] = ttk_run(small, 1e-8, prec, True, 3_000_000)
        mixed_error(ttk8)
    schemes = None
    if not args.no_ttk and not args.no_schemes:
        # the shape of Table 3: restart schemes to relative KKT 1e-8 on the 5k x 25k LP at the
        # primal weight the grid picked for it (FP64, setup included, cap in iterations)
        from paper_2105_12715_gb300 import lpgen

        small = lpgen.large_mixed(5, m=5000, n=25000)
        w = ttk8["fp64"]["omega"] if ttk8 else 1.0
        schemes = {"lp": f"large_mixed m={small.m} n={small.n} nnz={small.nnz} seed 5",
                   "tol": 1e-8, "omega": w, "cap_iters": args.schemes_cap, "runs": {}}
        runs = [("adaptive", dict(restart_scheme=lp.LP_RESTART_ADAPTIVE)),
                ("flexible", dict(restart_scheme=lp.LP_RESTART_FLEXIBLE))]
        runs += [(f"fixed_{L}", dict(restart_scheme=lp.LP_RESTART_FIXED, fixed_len=L))
                 for L in (256, 1024, 4096, 16384)]
        runs += [("no_restart", dict(restart_scheme=lp.LP_RESTART_NONE))]
        for name, kw in runs:
            barrier()
            t0 = time.perf_counter()
            gs = lp.LP(small, stream=stream, check_every=K_CHECK, max_iter=args.schemes_cap,
                       omega=w, **kw)
            st = gs.solve(1e-8)
            torch.cuda.synchronize()
            it = gs.info()
            gs.close()
            schemes["runs"][name] = {"iters": it.iters, "restarts": it.restarts,
                                     "status": lp.STATUS_NAMES.get(st, st),
                                     "returned": "average" if it.returned == 0 else "current",
                                     "rel_kkt": min(it.kkt_avg[4], it.kkt_cur[4]),
                                     "seconds": time.perf_counter() - t0}
    if not args.no_ttk and not args.no_ttk_large and ws == 1:
        # the benchmark LP itself (m = 200k, n = 1M, nnz = 10M)
        ttk_large = {"lp": config_of(args, data)["workload"], "tol": 1e-8,
                     "omega": "grid search (Section 7)"}
        for name, prec in (("fp64", lp.LP_PRECISION_FP64), ("mixed", lp.LP_PRECISION_MIXED)):
            ttk_large[name] = ttk_run(data, 1e-8, prec, True, args.ttk_large_cap)
        ttk_large["mixed_speedup"] = ttk_large["fp64"]["seconds"] / ttk_large["mixed"]["seconds"]
        mixed_error(ttk_large)
        if not args.no_paper_grid:
            # Section 7's own recipe: 4^-5 .. 4^5, 5,000 iterations without restarts each
            ttk_large["fp64_paper_grid"] = ttk_run(data, 1e-8, lp.LP_PRECISION_FP64, True,
                                                   args.ttk_large_cap, PAPER_OMEGA_GRID,
                                                   PAPER_OMEGA_ITERS)

    # an LP with one dense row and one dense column: split rows (lp_options.split_row_len)
    # against one warp per long row
    long_row = None
    if not args.no_long_row:
        from paper_2105_12715_gb300 import lpgen

        dl = lpgen.with_dense_lines(lpgen.large_mixed(7, m=20_000, n=200_000), seed=1)
        long_row = {"lp": f"large_mixed m=20000 n=200000 seed 7 + a dense row ({dl.n} elements) "
                          f"and a dense column ({dl.m} elements): m={dl.m} n={dl.n} nnz={dl.nnz}"}
        for name, split in (("one_warp_per_row", 0), ("split_512", 512)):
            gl = lp.LP(dl, stream=stream, check_every=K_CHECK, split_row_len=split)
            gl.iterate(args.warmup, 1e-300)
            barrier()
            lms = time_steps(lp, gl, stream, 20)
            long_row[name] = {"iters_per_s": 20 * K_CHECK / (lms / 1000.0),
                              "split_slices": gl.info().n_split_slices}
            gl.close()
        long_row["speedup"] = (long_row["split_512"]["iters_per_s"]
                               / long_row["one_warp_per_row"]["iters_per_s"])

    # the 200 x 400 LP (2,000 nonzeros): a step is launch- and latency-bound, not
    # bandwidth-bound; microseconds per iteration, K iterations + check per graph replay
    tiny, tiny_lp = None, None
    if not args.no_mcf:
        from paper_2105_12715_gb300 import lpgen

        tiny_lp = lpgen.tiny_standard_form(0)
        gt0 = lp.LP(tiny_lp, stream=stream, check_every=K_CHECK)
        gt0.iterate(args.warmup, 1e-300)
        barrier()
        tms = time_steps(lp, gt0, stream, args.steps)
        tiny = {"lp": f"tiny_standard_form seed 0: m={tiny_lp.m} n={tiny_lp.n} nnz={tiny_lp.nnz}",
                "us_per_iter": 1000.0 * tms / (args.steps * K_CHECK),
                "iters_per_s": args.steps * K_CHECK / (tms / 1000.0),
                "graph_kernels_per_step": gt0.info().graph_kernels, "eta": gt0.info().eta}
        gt0.close()
        # LPs this small belong in the batched solver: 512 such LPs (seeds 0..511) as one
        # batch, aggregate throughput and all of them to relative KKT 1e-8
        tl = [lpgen.tiny_standard_form(sd) for sd in range(512)]
        gbt = lp.LPBatch(tl, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                         tuning={"autotune": 1})
        gbt.iterate(2, 1e-300)
        barrier()
        e0t, e1t = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0t.record(stream)
        gbt.iterate(8, 1e-300)
        e1t.record(stream)
        torch.cuda.synchronize()
        bms = e0t.elapsed_time(e1t) / 8
        gbt.close()
        barrier()
        t0 = time.perf_counter()
        gbt = lp.LPBatch(tl, stream=stream, check_every=K_CHECK, max_iter=args.batch_cap,
                         tuning={"autotune": 1})
        gbt.solve(1e-8)
        torch.cuda.synchronize()
        tsolve = time.perf_counter() - t0
        _, pert = gbt.info()
        gbt.close()
        conv_t = [p_ for p_ in pert if p_["status"] == lp.LP_OK]
        tiny["batch_512"] = {
            "lp": "512 x tiny_standard_form (seeds 0..511), one batch",
            "us_per_batch_iter": 1000.0 * bms / K_CHECK,
            "problem_iters_per_s": 512 * K_CHECK / (bms / 1000.0),
            "to_1e8_seconds_with_setup": tsolve, "converged": len(conv_t),
            "iters_median": float(np.median([p_["iters"] for p_ in pert]))}

    # multicommodity flow LP (300 x 300 grid, 8 commodities): FP64 vs mixed throughput
    mcf = None
    if not args.no_mcf:
        from paper_2105_12715_gb300 import lpgen

        mc = lpgen.multicommodity_grid(4)
        mcf = {"lp": f"multicommodity grid 300x300, 8 commodities: m={mc.m} n={mc.n} nnz={mc.nnz}"}
        mp, md = algorithmic_bytes(mc.m, mc.n, mc.nnz)
        for name, prec in (("fp64", lp.LP_PRECISION_FP64), ("mixed", lp.LP_PRECISION_MIXED)):
            gmc = lp.LP(mc, stream=stream, check_every=K_CHECK, precision=prec)
            gmc.iterate(args.warmup, 1e-300)
            barrier()
            msm = time_steps(lp, gmc, stream, args.steps)
            mcf[name] = {"iters_per_s": args.steps * K_CHECK / (msm / 1000.0),
                         "ms_per_step": msm / args.steps}
            if prec == lp.LP_PRECISION_FP64:
                mcf[name]["achieved_gbs_per_iter"] = (mp + md) * mcf[name]["iters_per_s"] / 1e9
                mcf["eta"] = gmc.info().eta
            gmc.close()
        if not args.no_mcf_ttk and not args.no_ttk:
            # FP32-mixed (FP64 restarts, checks and refinement) against plain FP64 to a relative
            # KKT tolerance (mcf_tol), omega by Section 7's grid (4^-5 .. 4^5, 5,000 iterations
            # each), setup included; the mixed result's objective against the FP64 one.  On this
            # network LP restarted PDHG needs millions of iterations below 1e-4, so the default
            # tolerance is one both arms reach within the cap.
            t8 = {"tol": args.mcf_tol, "cap_iters": args.mcf_cap}
            if args.mcf_full_ttk:
                for name, prec in (("fp64", lp.LP_PRECISION_FP64),
                                   ("mixed", lp.LP_PRECISION_MIXED)):
                    t8[name] = ttk_run(mc, args.mcf_tol, prec, True, args.mcf_cap,
                                       PAPER_OMEGA_GRID, PAPER_OMEGA_ITERS)
                mixed_error(t8)
                t8["mixed_speedup"] = t8["fp64"]["seconds"] / t8["mixed"]["seconds"]
            # a 30 x 30 grid with 4 commodities: both arms against HiGHS's optimum
            small = lpgen.multicommodity_grid(4, side=30, commodities=4)
            ref = highs_objective(small)
            sm = {"lp": f"multicommodity grid 30x30, 4 commodities: m={small.m} n={small.n} "
                        f"nnz={small.nnz}", "highs_objective": ref}
            for name, prec in (("fp64", lp.LP_PRECISION_FP64), ("mixed", lp.LP_PRECISION_MIXED)):
                r = ttk_run(small, 1e-8, prec, True, 1_000_000, PAPER_OMEGA_GRID,
                            PAPER_OMEGA_ITERS)
                if ref is not None:
                    r["obj_rel_err_vs_highs"] = abs(r["pobj"] - ref) / max(1.0, abs(ref))
                sm[name] = r
            t8["small_vs_highs"] = sm
            mcf["time_to_tolerance"] = t8
            # the same shape at a size it reaches 1e-8 at: a 100 x 100 grid, 8 commodities
            mid = lpgen.multicommodity_grid(4, side=100, commodities=8)
            t8m = {"lp": f"multicommodity grid 100x100, 8 commodities: m={mid.m} n={mid.n} "
                         f"nnz={mid.nnz}", "tol": 1e-8, "cap_iters": 2_000_000}
            for name, prec in (("fp64", lp.LP_PRECISION_FP64), ("mixed", lp.LP_PRECISION_MIXED)):
                t8m[name] = ttk_run(mid, 1e-8, prec, True, 2_000_000, PAPER_OMEGA_GRID,
                                    PAPER_OMEGA_ITERS)
            mixed_error(t8m)
            t8m["mixed_speedup"] = t8m["fp64"]["seconds"] / t8m["mixed"]["seconds"]
            mcf["time_to_kkt_1e8_grid100"] = t8m

    # adjoint of the unrolled map on differentiable-LP-shaped instances
    # (m=2000, n=5000, nnz=50k, box [0,1]; 2000 iterations, checkpoint every 100)
    adjoint = None
    if not args.no_adjoint:
        from paper_2105_12715_gb300 import lpgen

        fw, bw = [], []
        for sd in range(args.adjoint_lps):
            d3 = lpgen.box_standard_form(100 + sd)
            g3 = lp.LP(d3, stream=stream, check_every=100)
            wv = np.random.default_rng(sd).standard_normal(d3.n)
            dc, db = np.empty(d3.n), np.empty(d3.m)
            barrier()
            t0 = time.perf_counter()
            lp.lp_solve_recorded(g3.h, 2000, stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            lp.lp_backward(g3.h, wv, None, dc, db, stream)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            fw.append(t1 - t0)
            bw.append(t2 - t1)
            g3.close()
        adjoint = {"lp": "box_standard_form m=2000 n=5000 nnz=50000 (4 seeds), K=100, 2000 iterations",
                   "forward_recorded_ms": 1000 * float(np.median(fw)),
                   "backward_ms": 1000 * float(np.median(bw)),
                   "backward_over_forward": float(np.median(bw) / np.median(fw))}
        # implicit-KKT active-set gradient (reported, not binding): on the face the
        # solve reaches, w = A_B^T u on the interior set B gives d(w^T x)/db = u
        d3 = lpgen.box_standard_form(100)
        g3 = lp.LP(d3, stream=stream, check_every=100, max_iter=200_000)
        st3 = g3.solve(1e-8)
        xs, _ = g3.solution()
        conv_iters = g3.info().iters
        g3.close()
        Bset = (xs > 1e-7) & (xs < 1 - 1e-7)
        import scipy.sparse as sp

        A3 = sp.csr_matrix((d3.val, d3.col_idx, d3.row_ptr), shape=(d3.m, d3.n))
        u3 = np.random.default_rng(7).standard_normal(d3.m)
        w3 = np.zeros(d3.n)
        w3[Bset] = (A3[:, np.flatnonzero(Bset)].T @ u3)
        imp = {"solve_status": lp.STATUS_NAMES.get(st3, st3), "interior": int(Bset.sum()),
               "rows": d3.m}
        for T in (2000, ((conv_iters + 400) // 100) * 100):
            g3 = lp.LP(d3, stream=stream, check_every=100)
            lp.lp_solve_recorded(g3.h, T, stream)
            dc, db = np.empty(d3.n), np.empty(d3.m)
            lp.lp_backward(g3.h, w3, None, dc, db, stream)
            g3.close()
            imp[f"iters_{T}"] = {
                "cosine": float(db @ u3 / (np.linalg.norm(db) * np.linalg.norm(u3))),
                "rel_err": float(np.linalg.norm(db - u3) / np.linalg.norm(u3))}
        adjoint["implicit_kkt"] = imp
        # the differentiable-LP batch: 64 such LPs through the batched adjoint
        probs3 = [lpgen.box_standard_form(100 + sd) for sd in range(64)]
        gb = lp.LPBatch(probs3, stream=stream, check_every=100)
        wb = np.random.default_rng(11).standard_normal(gb.n)
        barrier()
        t0 = time.perf_counter()
        gb.solve_recorded(2000)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        gb.backward(wb, None)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        gb.close()
        loop_s = 64 * (float(np.median(fw)) + float(np.median(bw)))
        adjoint["batch64"] = {
            "lp": "64 x box_standard_form (m=2000, n=5000, nnz=50k each), K=100, 2000 iterations",
            "forward_recorded_ms": 1000 * (t1 - t0), "backward_ms": 1000 * (t2 - t1),
            "one_lp_at_a_time_ms": 1000 * loop_s,
            "speedup_vs_one_at_a_time": loop_s / (t2 - t0)}

    batched = run_batched(args, lp, stream, barrier) if not args.no_batch else None

    out = None
    if rank == 0:
        out = {"metric": "PDHG iterations/s (fp64 restarted PDHG, large mixed LP)", "value": value,
               "unit": "iters/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": config_of(args, data),
               "parallelism": "replicas" if ws > 1 else "single",
               "gpu_launches": launches_per_step * args.steps,
               "iters_per_step": K_CHECK,
               "bytes_per_iter_algorithmic": primal_b + dual_b,
               "achieved_gbs_per_iter": (primal_b + dual_b) * value / ws / 1e9,
               "roofline": {"bound": "hbm", "kernel": "primal_kernel", "achieved": achieved,
                            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                            "peak_kind": peak_kind,
                            "traffic": measured_traffic(info0.spmv_unroll),
                            "traffic_source": {"file": os.path.relpath(TRAFFIC_FILE, ROOT),
                                               "kernel_source_hash": kernel_source_hash()},
                            "variant": info0.spmv_unroll,
                            "algorithmic_bytes": primal_b, "avg_launch_ms": primal_ms,
                            "dual_kernel_ms": dual_ms, "dual_algorithmic_bytes": dual_b,
                            "gather_bound": gather_bound},
               "clocks": clocks, "e2e": e2e, "mixed": mixed, "time_to_kkt": ttk,
               "time_to_kkt_1e8": ttk8, "time_to_kkt_1e8_large": ttk_large,
               "tiny": tiny, "multicommodity": mcf, "long_row": long_row,
               "restart_schemes": schemes,
               "adjoint": adjoint,
               "batched": batched,
               "solver": {"eta": info0.eta, "sigma_max": info0.sigma_max,
                          "sigma_steps": info0.sigma_steps,
                          "setup_ms": dict(zip(["inputs", "layout", "upload", "sigma_max"],
                                               info0.setup_ms)),
                          "iters_done": info.iters, "restarts": info.restarts,
                          "rel_kkt_avg": info.kkt_avg[4], "rel_kkt_cur": info.kkt_cur[4],
                          "nnz_padded": info.nnz_padded}}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args, data, info0.eta)
            if ttk is not None:
                import oracle

                for key, entry, d_ in (("time_to_kkt", ttk, med), ("time_to_kkt_1e8", ttk8, small)):
                    t0 = time.perf_counter()
                    r = oracle.solve(d_, entry["fp64"]["eta"], tol=1e-300, max_iter=256,
                                     check_every=K_CHECK)
                    rate = r.iters / (time.perf_counter() - t0)
                    entry["oracle_iters_per_s"] = rate
                    entry["oracle_extrapolated_seconds"] = entry["fp64"]["iters"] / rate
                    entry["oracle_note"] = ("oracle time = GPU FP64 iteration count / oracle "
                                            "iterations/s over 256 iterations (extrapolation)")
            if ttk_large is not None:
                rate = out["cpu_baseline"]["value"]
                ttk_large["oracle_extrapolated_seconds"] = ttk_large["fp64"]["iters"] / rate
            # the oracle on the other workloads (bounded samples, 1 thread)
            import oracle

            other = {}
            if tiny is not None:
                t0 = time.perf_counter()
                r = oracle.solve(tiny_lp, tiny["eta"], tol=1e-300, max_iter=1024,
                                 check_every=K_CHECK)
                other["tiny_200x400"] = {"iters_per_s": r.iters / (time.perf_counter() - t0),
                                         "sample": f"{r.iters} iterations"}
            if mcf is not None:
                t0 = time.perf_counter()
                r = oracle.solve(mc, mcf["eta"], tol=1e-300, max_iter=16, check_every=K_CHECK)
                other["multicommodity"] = {"iters_per_s": r.iters / (time.perf_counter() - t0),
                                           "sample": f"{r.iters} iterations"}
            out["cpu_baseline"]["other_workloads"] = other
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    args.kernel_reps = max(1, args.kernel_reps)
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_only:
        return run_batch_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
