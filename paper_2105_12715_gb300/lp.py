"""Thin ctypes binding of liblp.so (include/lp.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Functions keep the C names; arrays may be torch tensors
(CUDA or CPU) or NumPy arrays, passed by pointer.  Streams default to
torch's current CUDA stream.  There is no CPU fallback: if liblp.so is
missing or CUDA is unavailable the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

LP_OK, LP_ERR_INVALID_ARG, LP_ERR_CUDA, LP_ERR_OOM, LP_ITER_LIMIT = 0, 1, 2, 3, 4
LP_ERR_NUMERICAL, LP_ERR_TIMEOUT, LP_ERR_NOT_SOLVED = 5, 6, 7
LP_ROW_EQ, LP_ROW_GE, LP_ROW_LE = 0, 1, 2
LP_RESTART_NONE, LP_RESTART_FIXED, LP_RESTART_ADAPTIVE, LP_RESTART_FLEXIBLE = 0, 1, 2, 3
LP_PRECISION_FP64, LP_PRECISION_MIXED = 0, 1
LP_SIGMA_POWER, LP_SIGMA_LANCZOS = 0, 1

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "ITER_LIMIT",
                5: "NUMERICAL", 6: "TIMEOUT", 7: "NOT_SOLVED"}


class lp_options(C.Structure):
    _fields_ = [("beta", C.c_double), ("check_every", C.c_int32), ("restart_scheme", C.c_int32),
                ("tau0", C.c_int64), ("fixed_len", C.c_int64), ("omega", C.c_double),
                ("eta", C.c_double), ("power_iters", C.c_int32), ("power_tol", C.c_double),
                ("max_iter", C.c_int64), ("long_row_threshold", C.c_int32),
                ("trace_capacity", C.c_int32), ("spmv_unroll", C.c_int32),
                ("spmv_unroll_rows", C.c_int32), ("lane_steps", C.c_int32),
                ("single_lane_max", C.c_int32), ("spmv_mode", C.c_int32),
                ("precision", C.c_int32), ("lane_auto", C.c_int32), ("autotune", C.c_int32),
                ("sigma_method", C.c_int32), ("device_layout", C.c_int32),
                ("split_row_len", C.c_int32)]


class lp_info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("restarts", C.c_int64), ("checks", C.c_int64),
                ("status", C.c_int32), ("returned", C.c_int32),
                ("kkt_avg", C.c_double * 5), ("kkt_cur", C.c_double * 5),
                ("eta", C.c_double), ("sigma_max", C.c_double), ("omega", C.c_double),
                ("tau", C.c_double), ("sigma", C.c_double), ("rho_stored", C.c_double),
                ("last_rho", C.c_double), ("last_radius", C.c_double),
                ("nnz_padded", C.c_int64), ("n_long_rows", C.c_int32), ("n_long_cols", C.c_int32),
                ("setup_ms", C.c_double * 4), ("spmv_unroll", C.c_int32),
                ("spmv_unroll_rows", C.c_int32), ("sigma_steps", C.c_int32),
                ("graph_kernels", C.c_int32), ("n_split_slices", C.c_int32)]


class lp_batch_tuning(C.Structure):
    _fields_ = [("autotune", C.c_int32), ("max_k_shift", C.c_int32), ("check_budget", C.c_double)]


class lp_batch_problem_info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("restarts", C.c_int64), ("checks", C.c_int64),
                ("status", C.c_int32), ("returned", C.c_int32), ("check_every", C.c_int32),
                ("size_class", C.c_int32), ("kkt_avg", C.c_double * 5),
                ("kkt_cur", C.c_double * 5), ("eta", C.c_double), ("sigma_max", C.c_double),
                ("tau", C.c_double), ("sigma", C.c_double), ("rho_stored", C.c_double),
                ("last_rho", C.c_double), ("omega", C.c_double), ("sigma_steps", C.c_int32)]


class lp_batch_info(C.Structure):
    _fields_ = [("count", C.c_int32), ("running", C.c_int32), ("m", C.c_int32), ("n", C.c_int32),
                ("nnz", C.c_int64), ("blocks", C.c_int64), ("k_base", C.c_int32),
                ("spmv_unroll", C.c_int32), ("spmv_unroll_rows", C.c_int32),
                ("grid_cols", C.c_int32), ("grid_rows", C.c_int32), ("n_classes", C.c_int32), ("class_k", C.c_int32 * 8),
                ("class_iter_ms", C.c_double * 8), ("class_check_ms", C.c_double * 8),
                ("tune_ms", C.c_double), ("setup_ms", C.c_double)]


EXPORTED = ["lp_default_options", "lp_create", "lp_solve", "lp_iterate", "lp_get_solution",
            "lp_get_state", "lp_set_state", "lp_get_info", "lp_get_trace", "lp_normalized_gap",
            "lp_normalized_gap_static", "lp_select_omega", "lp_solve_recorded", "lp_backward",
            "lp_profile_kernel", "lp_destroy", "lp_last_error",
            # include/lp_batch.h
            "lp_batch_default_tuning", "lp_batch_create", "lp_batch_set_check_every",
            "lp_batch_solve", "lp_batch_iterate", "lp_batch_get_solution", "lp_batch_get_state",
            "lp_batch_get_info", "lp_batch_solve_recorded", "lp_batch_backward",
            "lp_batch_set_state", "lp_batch_select_omega", "lp_batch_destroy"]

_lib = None


class LPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblp.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"liblp.so not found at {path}; run paper_2105_12715_gb300.build.build()")
    lib = C.CDLL(path)
    P, D, I32, I64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
    lib.lp_default_options.argtypes = [C.POINTER(lp_options)]
    lib.lp_default_options.restype = None
    lib.lp_create.argtypes = [I32, I32, I64, P, P, P, P, P, P, P, P, C.POINTER(lp_options), P,
                              C.POINTER(P)]
    lib.lp_solve.argtypes = [P, D, P]
    lib.lp_iterate.argtypes = [P, I32, D, P]
    lib.lp_get_solution.argtypes = [P, P, P, P]
    lib.lp_get_state.argtypes = [P, P, P, P, P, P, P, P]
    lib.lp_set_state.argtypes = [P, P, P, P]
    lib.lp_get_info.argtypes = [P, C.POINTER(lp_info)]
    lib.lp_get_trace.argtypes = [P, P, I64, C.POINTER(I64)]
    lib.lp_normalized_gap.argtypes = [P, P, P, D, C.POINTER(D), P]
    lib.lp_normalized_gap_static.argtypes = [P, P, P, D, C.POINTER(D), P]
    lib.lp_profile_kernel.argtypes = [P, I32, I32, P]
    lib.lp_select_omega.argtypes = [P, P, I32, I64, P, P, P]
    lib.lp_solve_recorded.argtypes = [P, I64, P]
    lib.lp_backward.argtypes = [P, P, P, P, P, P]
    lib.lp_destroy.argtypes = [P]
    lib.lp_destroy.restype = None
    lib.lp_last_error.argtypes = []
    lib.lp_last_error.restype = C.c_char_p
    lib.lp_batch_default_tuning.argtypes = [C.POINTER(lp_batch_tuning)]
    lib.lp_batch_default_tuning.restype = None
    lib.lp_batch_create.argtypes = [I32, P, P, I64, P, P, P, P, P, P, P, P,
                                    C.POINTER(lp_options), C.POINTER(lp_batch_tuning), P,
                                    C.POINTER(P)]
    lib.lp_batch_set_check_every.argtypes = [P, P, P]
    lib.lp_batch_solve.argtypes = [P, D, P]
    lib.lp_batch_iterate.argtypes = [P, I32, D, P]
    lib.lp_batch_get_solution.argtypes = [P, P, P, P]
    lib.lp_batch_get_state.argtypes = [P, P, P, P, P, P, P, P]
    lib.lp_batch_get_info.argtypes = [P, C.POINTER(lp_batch_info), P, I32]
    lib.lp_batch_solve_recorded.argtypes = [P, I64, P]
    lib.lp_batch_set_state.argtypes = [P, P, P, P]
    lib.lp_batch_select_omega.argtypes = [P, P, I32, I64, P, P, P]
    lib.lp_batch_backward.argtypes = [P, P, P, P, P, P]
    lib.lp_batch_destroy.argtypes = [P]
    lib.lp_batch_destroy.restype = None
    for name in ["lp_create", "lp_solve", "lp_iterate", "lp_get_solution", "lp_get_state",
                 "lp_set_state", "lp_get_info", "lp_get_trace", "lp_normalized_gap",
                 "lp_normalized_gap_static", "lp_profile_kernel", "lp_select_omega",
                 "lp_solve_recorded", "lp_backward", "lp_batch_create",
                 "lp_batch_set_check_every", "lp_batch_solve", "lp_batch_iterate",
                 "lp_batch_get_solution", "lp_batch_get_state", "lp_batch_get_info",
                 "lp_batch_solve_recorded", "lp_batch_backward", "lp_batch_set_state",
                 "lp_batch_select_omega"]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _last_error() -> str:
    return load().lp_last_error().decode(errors="replace")


def _check(status, allow=(LP_OK,)):
    if status not in allow:
        raise LPError(status, _last_error())
    return status


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


def _ptr(a, dtype):
    """Pointer of a contiguous torch tensor or NumPy array of the given dtype."""
    if a is None:
        return None, None
    try:
        import torch

        if isinstance(a, torch.Tensor):
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int8: torch.int8}[dtype]
            if a.dtype != tdt or not a.is_contiguous():
                a = a.to(tdt).contiguous()
            return C.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), arr


def lp_default_options() -> lp_options:
    o = lp_options()
    load().lp_default_options(C.byref(o))
    return o


def lp_create(m, n, nnz, row_ptr, col_idx, val, c, b, lb, ub, row_type, opt=None, stream=None):
    """Returns a handle (C void*).  Arrays: host or device, see include/lp.h."""
    keep = []
    ptrs = []
    for a, dt in [(row_ptr, np.int32), (col_idx, np.int32), (val, np.float64), (c, np.float64),
                  (b, np.float64), (lb, np.float64), (ub, np.float64), (row_type, np.int8)]:
        p, k = _ptr(a, dt)
        ptrs.append(p)
        keep.append(k)
    h = C.c_void_p()
    o = C.byref(opt) if opt is not None else None
    _check(load().lp_create(int(m), int(n), int(nnz), *ptrs, o, _stream(stream), C.byref(h)))
    return h


def lp_solve(h, tol, stream=None) -> int:
    return _check(load().lp_solve(h, float(tol), _stream(stream)),
                  allow=(LP_OK, LP_ITER_LIMIT, LP_ERR_NUMERICAL))


def lp_iterate(h, n_checks, tol, stream=None) -> int:
    return _check(load().lp_iterate(h, int(n_checks), float(tol), _stream(stream)))


def lp_get_solution(h, x, y, stream=None):
    px, _ = _ptr(x, np.float64) if not isinstance(x, np.ndarray) else (C.c_void_p(x.ctypes.data), x)
    py, _ = _ptr(y, np.float64) if not isinstance(y, np.ndarray) else (C.c_void_p(y.ctypes.data), y)
    return _check(load().lp_get_solution(h, px, py, _stream(stream)))


def _out_ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return C.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def lp_get_state(h, x=None, y=None, xbar=None, ybar=None, x0=None, y0=None, stream=None):
    return _check(load().lp_get_state(h, *[_out_ptr(a) for a in (x, y, xbar, ybar, x0, y0)],
                                      _stream(stream)))


def lp_set_state(h, x=None, y=None, stream=None):
    px, kx = _ptr(x, np.float64)
    py, ky = _ptr(y, np.float64)
    return _check(load().lp_set_state(h, px, py, _stream(stream)))


def lp_get_info(h) -> lp_info:
    info = lp_info()
    _check(load().lp_get_info(h, C.byref(info)))
    return info


def lp_get_trace(h, capacity=1 << 20) -> np.ndarray:
    rows = np.empty((capacity, 6))
    cnt = C.c_int64()
    _check(load().lp_get_trace(h, C.c_void_p(rows.ctypes.data), capacity, C.byref(cnt)))
    return rows[:cnt.value].copy()


def lp_normalized_gap(h, x, y, r, stream=None) -> float:
    px, kx = _ptr(x, np.float64)
    py, ky = _ptr(y, np.float64)
    out = C.c_double()
    _check(load().lp_normalized_gap(h, px, py, float(r), C.byref(out), _stream(stream)))
    return out.value


def lp_normalized_gap_static(h, x, y, r, stream=None) -> float:
    """lp_normalized_gap with the library's fixed static scratch (no device
    allocation; n + m <= 262,144; concurrent calls must be serialized)."""
    px, kx = _ptr(x, np.float64)
    py, ky = _ptr(y, np.float64)
    out = C.c_double()
    _check(load().lp_normalized_gap_static(h, px, py, float(r), C.byref(out), _stream(stream)))
    return out.value


def lp_select_omega(h, omegas, iters=5000, stream=None):
    """Section 7's primal-weight search; returns (best omega, relative KKT per omega)."""
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    kkt = np.empty(om.shape[0])
    best = C.c_double()
    _check(load().lp_select_omega(h, C.c_void_p(om.ctypes.data), om.shape[0], int(iters),
                                  C.c_void_p(kkt.ctypes.data), C.byref(best), _stream(stream)))
    return best.value, kkt


def lp_solve_recorded(h, iters, stream=None):
    return _check(load().lp_solve_recorded(h, int(iters), _stream(stream)))


def lp_backward(h, dl_dx, dl_dy, dl_dc, dl_db, stream=None):
    px, kx = _ptr(dl_dx, np.float64)
    py, ky = _ptr(dl_dy, np.float64)
    return _check(load().lp_backward(h, px, py, _out_ptr(dl_dc), _out_ptr(dl_db), _stream(stream)))


def lp_profile_kernel(h, which, reps, stream=None):
    return _check(load().lp_profile_kernel(h, int(which), int(reps), _stream(stream)))


def lp_destroy(h):
    if h is not None and h.value:
        load().lp_destroy(h)


# ------------------------------------------------------------ convenience

@dataclass
class Info:
    iters: int
    restarts: int
    checks: int
    status: int
    returned: int
    kkt_avg: tuple
    kkt_cur: tuple
    eta: float
    sigma_max: float
    omega: float
    tau: float
    sigma: float
    rho_stored: float
    last_rho: float
    last_radius: float
    nnz_padded: int
    n_long_rows: int
    n_long_cols: int
    setup_ms: tuple = ()
    spmv_unroll: int = 0
    spmv_unroll_rows: int = 0
    sigma_steps: int = 0
    graph_kernels: int = 0
    n_split_slices: int = 0

    @property
    def rel_kkt(self) -> float:
        return self.kkt_avg[4] if self.returned == 0 else self.kkt_cur[4]


class LP:
    """Owning wrapper of an lp_handle built from an lpgen.LPData-like object."""

    def __init__(self, data, stream=None, **options):
        opt = lp_default_options()
        for k, v in options.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, v)
        self.m, self.n = int(data.m), int(data.n)
        self.stream = stream
        self.h = lp_create(data.m, data.n, int(data.row_ptr[-1]), data.row_ptr, data.col_idx,
                           data.val, data.c, data.b, data.lb, data.ub, data.row_type, opt, stream)

    def close(self):
        if getattr(self, "h", None) is not None:
            lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, tol=1e-8):
        return lp_solve(self.h, tol, self.stream)

    def iterate(self, n_checks, tol=1e-8):
        return lp_iterate(self.h, n_checks, tol, self.stream)

    def solution(self):
        x, y = np.empty(self.n), np.empty(self.m)
        lp_get_solution(self.h, x, y, self.stream)
        return x, y

    def state(self):
        arrs = [np.empty(self.n), np.empty(self.m), np.empty(self.n), np.empty(self.m),
                np.empty(self.n), np.empty(self.m)]
        lp_get_state(self.h, *arrs, stream=self.stream)
        return dict(zip(["x", "y", "xbar", "ybar", "x0", "y0"], arrs))

    def set_state(self, x=None, y=None):
        lp_set_state(self.h, x, y, self.stream)

    def info(self) -> Info:
        i = lp_get_info(self.h)
        return Info(i.iters, i.restarts, i.checks, i.status, i.returned, tuple(i.kkt_avg),
                    tuple(i.kkt_cur), i.eta, i.sigma_max, i.omega, i.tau, i.sigma, i.rho_stored,
                    i.last_rho, i.last_radius, i.nnz_padded, i.n_long_rows, i.n_long_cols,
                    tuple(i.setup_ms), i.spmv_unroll, i.spmv_unroll_rows, i.sigma_steps,
                    i.graph_kernels, i.n_split_slices)

    def trace(self, capacity=1 << 20):
        return lp_get_trace(self.h, capacity)

    def gap(self, x, y, r):
        return lp_normalized_gap(self.h, x, y, r, self.stream)

    def select_omega(self, omegas=None, iters=5000):
        """Primal weight by the grid of Section 7 (4^-5 .. 4^5 by default)."""
        if omegas is None:
            omegas = 4.0 ** np.arange(-5, 6)
        return lp_select_omega(self.h, omegas, iters, self.stream)


def default_beta() -> float:
    return math.exp(-1.0)


# ------------------------------------------------------------ batched solver

def lp_batch_default_tuning() -> lp_batch_tuning:
    t = lp_batch_tuning()
    load().lp_batch_default_tuning(C.byref(t))
    return t


def lp_batch_create(row_start, col_start, nnz, row_ptr, col_idx, val, c, b, lb, ub, row_type,
                    opt=None, tuning=None, stream=None):
    """Returns a batch handle (C void*); see include/lp_batch.h.  row_start and
    col_start are host arrays of count + 1 problem boundaries."""
    rs = np.ascontiguousarray(row_start, dtype=np.int32)
    cs = np.ascontiguousarray(col_start, dtype=np.int32)
    keep, ptrs = [rs, cs], []
    for a, dt in [(row_ptr, np.int32), (col_idx, np.int32), (val, np.float64), (c, np.float64),
                  (b, np.float64), (lb, np.float64), (ub, np.float64), (row_type, np.int8)]:
        p, k = _ptr(a, dt)
        ptrs.append(p)
        keep.append(k)
    h = C.c_void_p()
    o = C.byref(opt) if opt is not None else None
    t = C.byref(tuning) if tuning is not None else None
    _check(load().lp_batch_create(rs.shape[0] - 1, C.c_void_p(rs.ctypes.data),
                                  C.c_void_p(cs.ctypes.data), int(nnz), *ptrs, o, t,
                                  _stream(stream), C.byref(h)))
    return h


def lp_batch_set_check_every(h, ks, stream=None):
    k = np.ascontiguousarray(ks, dtype=np.int32)
    return _check(load().lp_batch_set_check_every(h, C.c_void_p(k.ctypes.data), _stream(stream)))


def lp_batch_solve(h, tol, stream=None) -> int:
    return _check(load().lp_batch_solve(h, float(tol), _stream(stream)),
                  allow=(LP_OK, LP_ITER_LIMIT, LP_ERR_NUMERICAL))


def lp_batch_iterate(h, n_blocks, tol, stream=None) -> int:
    return _check(load().lp_batch_iterate(h, int(n_blocks), float(tol), _stream(stream)))


def lp_batch_get_solution(h, x, y, stream=None):
    return _check(load().lp_batch_get_solution(h, _out_ptr(x), _out_ptr(y), _stream(stream)))


def lp_batch_get_state(h, x=None, y=None, xbar=None, ybar=None, x0=None, y0=None, stream=None):
    return _check(load().lp_batch_get_state(h, *[_out_ptr(a) for a in (x, y, xbar, ybar, x0, y0)],
                                            _stream(stream)))


def lp_batch_get_info(h, count):
    info = lp_batch_info()
    probs = (lp_batch_problem_info * max(1, count))()
    _check(load().lp_batch_get_info(h, C.byref(info), C.cast(probs, C.c_void_p), int(count)))
    return info, probs


def lp_batch_solve_recorded(h, iters, stream=None):
    return _check(load().lp_batch_solve_recorded(h, int(iters), _stream(stream)))


def lp_batch_backward(h, dl_dx, dl_dy, dl_dc, dl_db, stream=None):
    px, kx = _ptr(dl_dx, np.float64)
    py, ky = _ptr(dl_dy, np.float64)
    return _check(load().lp_batch_backward(h, px, py, _out_ptr(dl_dc), _out_ptr(dl_db),
                                           _stream(stream)))


def lp_batch_set_state(h, x=None, y=None, stream=None):
    px, kx = _ptr(x, np.float64)
    py, ky = _ptr(y, np.float64)
    return _check(load().lp_batch_set_state(h, px, py, _stream(stream)))


def lp_batch_select_omega(h, count, omegas, iters=2000, stream=None):
    """Section 7's primal-weight grid for every problem of a batch: returns
    (best omega per problem [count], relative KKT per problem and omega [count, len])."""
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    kkt = np.empty((count, om.shape[0]))
    best = np.empty(count)
    _check(load().lp_batch_select_omega(h, C.c_void_p(om.ctypes.data), om.shape[0], int(iters),
                                        C.c_void_p(kkt.ctypes.data), C.c_void_p(best.ctypes.data),
                                        _stream(stream)))
    return best, kkt


def lp_batch_destroy(h):
    if h is not None and h.value:
        load().lp_batch_destroy(h)


class LPBatch:
    """Owning wrapper of an lp_batch_handle built from a list of lpgen.LPData-like
    problems (concatenated into the block-diagonal batch here, on the host)."""

    def __init__(self, problems, stream=None, tuning=None, c=None, b=None, **options):
        """c, b (optional): the concatenated objective and right-hand side, host or
        device arrays, in place of the problems' own."""
        opt = lp_default_options()
        for k, v in options.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, v)
        self.stream = stream
        self.count = len(problems)
        ms = [int(p.m) for p in problems]
        ns = [int(p.n) for p in problems]
        self.row_start = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
        self.col_start = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        self.m, self.n = int(self.row_start[-1]), int(self.col_start[-1])
        rp = [np.zeros(1, np.int64)]
        off = 0
        for p in problems:
            rp.append(np.asarray(p.row_ptr[1:], np.int64) + off)
            off += int(p.row_ptr[-1])
        row_ptr = np.concatenate(rp)
        col_idx = np.concatenate([np.asarray(p.col_idx, np.int64) + int(cs)
                                  for p, cs in zip(problems, self.col_start[:-1])])
        cat = lambda f, dt: np.concatenate([np.asarray(getattr(p, f), dt) for p in problems])
        if isinstance(tuning, dict):
            t = lp_batch_default_tuning()
            for k, v in tuning.items():
                setattr(t, k, v)
            tuning = t
        self.h = lp_batch_create(self.row_start, self.col_start, int(row_ptr[-1]), row_ptr,
                                 col_idx, cat("val", np.float64),
                                 cat("c", np.float64) if c is None else c,
                                 cat("b", np.float64) if b is None else b, cat("lb", np.float64),
                                 cat("ub", np.float64), cat("row_type", np.int8), opt, tuning,
                                 stream)

    def close(self):
        if getattr(self, "h", None) is not None:
            lp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, tol=1e-8):
        return lp_batch_solve(self.h, tol, self.stream)

    def iterate(self, n_blocks, tol=1e-8):
        return lp_batch_iterate(self.h, n_blocks, tol, self.stream)

    def set_state(self, x=None, y=None):
        """Warm start of every problem from proj(x, y) (concatenated vectors)."""
        lp_batch_set_state(self.h, x, y, self.stream)

    def select_omega(self, omegas=None, iters=2000):
        """Primal weight per problem by the grid of Section 7 (4^-3 .. 4^3 by default)."""
        if omegas is None:
            omegas = 4.0 ** np.arange(-3, 4)
        return lp_batch_select_omega(self.h, self.count, omegas, iters, self.stream)

    def set_check_every(self, ks):
        lp_batch_set_check_every(self.h, ks, self.stream)

    def split(self, vec, rows=False):
        st = self.row_start if rows else self.col_start
        return [vec[st[k]:st[k + 1]] for k in range(self.count)]

    def solution(self):
        x, y = np.empty(self.n), np.empty(self.m)
        lp_batch_get_solution(self.h, x, y, self.stream)
        return x, y

    def state(self):
        arrs = [np.empty(self.n), np.empty(self.m), np.empty(self.n), np.empty(self.m),
                np.empty(self.n), np.empty(self.m)]
        lp_batch_get_state(self.h, *arrs, stream=self.stream)
        return dict(zip(["x", "y", "xbar", "ybar", "x0", "y0"], arrs))

    def solve_recorded(self, iters):
        """Unrolled forward of exactly `iters` iterations, recorded for backward()."""
        lp_batch_solve_recorded(self.h, iters, self.stream)

    def backward(self, dl_dx=None, dl_dy=None):
        """Gradients (dL/dc [n], dL/db [m]) of the recorded unrolled maps."""
        dc, db = np.empty(self.n), np.empty(self.m)
        lp_batch_backward(self.h, dl_dx, dl_dy, dc, db, self.stream)
        return dc, db

    def info(self):
        """(batch summary, list of per-problem dicts)."""
        info, probs = lp_batch_get_info(self.h, self.count)
        per = []
        for k in range(self.count):
            p = probs[k]
            per.append(dict(iters=p.iters, restarts=p.restarts, checks=p.checks, status=p.status,
                            returned=p.returned, check_every=p.check_every,
                            size_class=p.size_class, kkt_avg=tuple(p.kkt_avg),
                            kkt_cur=tuple(p.kkt_cur), eta=p.eta, sigma_max=p.sigma_max,
                            tau=p.tau, sigma=p.sigma, rho_stored=p.rho_stored,
                            last_rho=p.last_rho, omega=p.omega, sigma_steps=p.sigma_steps))
        summary = {f: getattr(info, f) for f, _ in lp_batch_info._fields_}
        for f in ("class_k", "class_iter_ms", "class_check_ms"):
            summary[f] = list(getattr(info, f))
        return summary, per
