"""CPU FP64 oracle for restarted PDHG (test infrastructure).

This package is TEST INFRASTRUCTURE: only the test suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
It is a plain C restatement of the method (``rpdhg_oracle.c``) loaded with
ctypes, plus NumPy marshalling.  It shares no code with the CUDA library.

Functions follow the paper's sections:
  * ``pdhg_step``       Eq. (PDHG-update) with tau = eta/omega, sigma = eta*omega
  * ``sigma_max``       power iteration for sigma_max(A) (Section 7)
  * ``trust_region``    Algorithm 2 (Appendix F), two-sided bounds (Section 6.3)
  * ``normalized_gap``  Eq. (rhorz) via Sections 6.1-6.3
  * ``kkt``             relative KKT error from Eq. (define:K-and-h-for-lp)
  * ``solve``           Algorithm 1 with the restart schemes of Section 4
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpdhg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")  # OpenMP build, for timing only

RESTART_NONE, RESTART_FIXED, RESTART_ADAPTIVE, RESTART_FLEXIBLE, RESTART_SCHEDULE = 0, 1, 2, 3, 4
STATUS_OK, STATUS_ITER_LIMIT, STATUS_NUMERICAL = 0, 4, 5


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so (the build
    the tests use, one thread), or with openmp=True into liboracle_omp.so
    (the same source with its OpenMP pragmas honored; used to time the
    oracle on all host cores)."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC",
                           *(["-fopenmp"] if openmp else []),
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, lib)
    return lib


class _LP(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("c", C.c_void_p), ("b", C.c_void_p), ("lb", C.c_void_p), ("ub", C.c_void_p),
                ("row_type", C.c_void_p)]


class _Options(C.Structure):
    _fields_ = [("eta", C.c_double), ("omega", C.c_double), ("beta", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int64), ("check_every", C.c_int32),
                ("restart_scheme", C.c_int32), ("tau0", C.c_int64), ("fixed_len", C.c_int64),
                ("schedule", C.c_void_p), ("nschedule", C.c_int64)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("restarts", C.c_int64), ("inner_t", C.c_int64),
                ("status", C.c_int32), ("returned", C.c_int32), ("rho_stored", C.c_double),
                ("kkt_avg", C.c_double * 5), ("kkt_cur", C.c_double * 5),
                ("n_checks", C.c_int64)]


_lib = None
_lib_omp = None


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = _declare(C.CDLL(build(openmp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(lib):
    """Argument and result types of the oracle's C functions."""
    P = C.c_void_p
    lib.orc_matvec.argtypes = [P, P, P]
    lib.orc_matvec_t.argtypes = [P, P, P]
    lib.orc_pdhg_step.argtypes = [P, C.c_double, C.c_double, P, P, P, P, P]
    lib.orc_sigma_max.argtypes = [P, C.c_int32, C.c_double]
    lib.orc_sigma_max.restype = C.c_double
    lib.orc_trust_region_lower.argtypes = [C.c_int64, P, P, P, C.c_double, P, P]
    lib.orc_trust_region.argtypes = [C.c_int64, P, P, P, P, C.c_double, P]
    lib.orc_trust_region.restype = C.c_double
    lib.orc_normalized_gap.argtypes = [P, C.c_double, P, P, C.c_double]
    lib.orc_normalized_gap.restype = C.c_double
    lib.orc_weighted_dist.argtypes = [C.c_int32, C.c_int32, C.c_double, P, P, P, P]
    lib.orc_weighted_dist.restype = C.c_double
    lib.orc_kkt.argtypes = [P, P, P, P]
    lib.orc_solve.argtypes = [P, P, P, P, P, P, P, P, P, P, C.c_int64]
    lib.orc_solve.restype = C.c_int32
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleLP:
    """Holds contiguous copies of an LP's arrays and the ctypes struct."""

    def __init__(self, lp):
        self.m, self.n = int(lp.m), int(lp.n)
        self.row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
        self.val = _f64(lp.val)
        self.c, self.b = _f64(lp.c), _f64(lp.b)
        self.lb, self.ub = _f64(lp.lb), _f64(lp.ub)
        self.row_type = np.ascontiguousarray(lp.row_type, dtype=np.int8)
        self.s = _LP(self.m, self.n, _ptr(self.row_ptr).value, _ptr(self.col_idx).value,
                     _ptr(self.val).value, _ptr(self.c).value, _ptr(self.b).value,
                     _ptr(self.lb).value, _ptr(self.ub).value, _ptr(self.row_type).value)

    @property
    def ref(self):
        return C.byref(self.s)


def _olp(lp):
    return lp if isinstance(lp, OracleLP) else OracleLP(lp)


def matvec(lp, x):
    lp = _olp(lp)
    x = _f64(x)
    out = np.empty(lp.m)
    _load().orc_matvec(lp.ref, _ptr(x), _ptr(out))
    return out


def matvec_t(lp, y):
    lp = _olp(lp)
    y = _f64(y)
    out = np.empty(lp.n)
    _load().orc_matvec_t(lp.ref, _ptr(y), _ptr(out))
    return out


def pdhg_step(lp, tau, sigma, x, y):
    lp = _olp(lp)
    x, y = _f64(x), _f64(y)
    xn, yn = np.empty(lp.n), np.empty(lp.m)
    work = np.empty(lp.n + lp.m + 1)
    _load().orc_pdhg_step(lp.ref, tau, sigma, _ptr(x), _ptr(y), _ptr(xn), _ptr(yn), _ptr(work))
    return xn, yn


def sigma_max(lp, max_iter=5000, tol=1e-10):
    lp = _olp(lp)
    return float(_load().orc_sigma_max(lp.ref, max_iter, tol))


def trust_region_lower(z, l, g, r):
    z, l, g = _f64(z), _f64(l), _f64(g)
    zt = np.empty_like(z)
    lam = C.c_double()
    _load().orc_trust_region_lower(z.shape[0], _ptr(z), _ptr(l), _ptr(g), float(r), _ptr(zt),
                                   C.byref(lam))
    return zt, lam.value


def trust_region(z, lo, hi, g, r):
    z, lo, hi, g = _f64(z), _f64(lo), _f64(hi), _f64(g)
    zt = np.empty_like(z)
    lam = _load().orc_trust_region(z.shape[0], _ptr(z), _ptr(lo), _ptr(hi), _ptr(g), float(r),
                                   _ptr(zt))
    return zt, float(lam)


def normalized_gap(lp, x, y, r, omega=1.0):
    lp = _olp(lp)
    x, y = _f64(x), _f64(y)
    return float(_load().orc_normalized_gap(lp.ref, omega, _ptr(x), _ptr(y), float(r)))


def weighted_dist(x, y, x0, y0, omega=1.0):
    x, y, x0, y0 = _f64(x), _f64(y), _f64(x0), _f64(y0)
    return float(_load().orc_weighted_dist(x.shape[0], y.shape[0], omega, _ptr(x), _ptr(y),
                                           _ptr(x0), _ptr(y0)))


def kkt(lp, x, y):
    """Returns dict(rp, rd, pobj, dobj, rel)."""
    lp = _olp(lp)
    x, y = _f64(x), _f64(y)
    out = np.empty(5)
    _load().orc_kkt(lp.ref, _ptr(x), _ptr(y), _ptr(out))
    return dict(rp=out[0], rd=out[1], pobj=out[2], dobj=out[3], rel=out[4])


@dataclass
class SolveResult:
    status: int
    iters: int
    restarts: int
    inner_t: int
    returned: int
    rho_stored: float
    n_checks: int
    kkt_avg: np.ndarray
    kkt_cur: np.ndarray
    x: np.ndarray
    y: np.ndarray
    xbar: np.ndarray
    ybar: np.ndarray
    x0: np.ndarray
    y0: np.ndarray
    trace: np.ndarray

    @property
    def x_sol(self):
        return self.xbar if self.returned == 0 else self.x

    @property
    def y_sol(self):
        return self.ybar if self.returned == 0 else self.y


def solve(lp, eta, omega=1.0, beta=float(np.exp(-1.0)), tol=1e-8, max_iter=100000,
          check_every=64, restart_scheme=RESTART_ADAPTIVE, tau0=None, fixed_len=0,
          x_init=None, y_init=None, trace_cap=100000, schedule=None,
          openmp=False) -> SolveResult:
    """Algorithm 1 (restarted PDHG) from z^{0,0} = (x_init, y_init) (zeros by default).

    schedule (RESTART_SCHEDULE): one flag per check, restart where nonzero.
    openmp: run the OpenMP build (all host cores; same results) -- for timing."""
    lp = _olp(lp)
    x = np.zeros(lp.n) if x_init is None else _f64(x_init).copy()
    y = np.zeros(lp.m) if y_init is None else _f64(y_init).copy()
    xbar, ybar = np.empty(lp.n), np.empty(lp.m)
    x0, y0 = np.empty(lp.n), np.empty(lp.m)
    sched = np.ascontiguousarray([] if schedule is None else schedule, dtype=np.int8)
    opt = _Options(eta, omega, beta, tol, int(max_iter), int(check_every), int(restart_scheme),
                   int(check_every if tau0 is None else tau0), int(fixed_len),
                   sched.ctypes.data if sched.size else None, int(sched.size))
    info = _Info()
    cap = max(1, min(trace_cap, max_iter // max(1, check_every) + 1))
    trace = np.full((cap, 6), np.nan)
    _load(openmp).orc_solve(lp.ref, C.byref(opt), _ptr(x), _ptr(y), _ptr(xbar), _ptr(ybar),
                            _ptr(x0), _ptr(y0), C.byref(info), _ptr(trace), cap)
    nck = int(info.n_checks)
    return SolveResult(int(info.status), int(info.iters), int(info.restarts), int(info.inner_t),
                       int(info.returned), float(info.rho_stored), nck,
                       np.array(info.kkt_avg[:]), np.array(info.kkt_cur[:]),
                       x, y, xbar, ybar, x0, y0, trace[:min(nck, cap)])
