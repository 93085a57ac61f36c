"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point include/lp.h declares, and rejects bad
arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:lp_status|void|const char \*)\s*(lp_\w+)\s*\(", src,
                            flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_12715_gb300 import lp

    return lp.load()


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for required in ["lp_create", "lp_solve", "lp_get_solution", "lp_get_info", "lp_destroy",
                     "lp_last_error", "lp_default_options", "lp_batch_create", "lp_batch_solve",
                     "lp_batch_get_solution", "lp_batch_get_info", "lp_batch_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2105_12715_gb300 import lp

    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in lp.EXPORTED, name


def test_default_options(lib):
    from paper_2105_12715_gb300 import lp

    o = lp.lp_default_options()
    assert o.beta == pytest.approx(np.exp(-1))
    assert o.check_every == 64
    assert o.restart_scheme == lp.LP_RESTART_ADAPTIVE
    assert o.omega == 1.0 and o.eta == 0.0


def test_create_rejects_bad_sizes_and_options_on_host(lib):
    from paper_2105_12715_gb300 import lp

    rp = np.array([0, 1], dtype=np.int32)
    ci = np.array([0], dtype=np.int32)
    v = np.array([1.0])
    c = np.array([1.0])
    b = np.array([1.0])
    lb, ub = np.array([0.0]), np.array([np.inf])
    rt = np.zeros(1, dtype=np.int8)
    with pytest.raises(lp.LPError) as e:
        lp.lp_create(1, 0, 1, rp, ci, v, c, b, lb, ub, rt, stream=0)
    assert e.value.status == lp.LP_ERR_INVALID_ARG
    opt = lp.lp_default_options()
    opt.beta = 1.5
    with pytest.raises(lp.LPError) as e:
        lp.lp_create(1, 1, 1, rp, ci, v, c, b, lb, ub, rt, opt, stream=0)
    assert e.value.status == lp.LP_ERR_INVALID_ARG
    assert "beta" in lp._last_error()
    opt = lp.lp_default_options()
    opt.check_every = 0
    with pytest.raises(lp.LPError):
        lp.lp_create(1, 1, 1, rp, ci, v, c, b, lb, ub, rt, opt, stream=0)
    h = C.c_void_p()
    st = lib.lp_create(1, 1, 1, None, None, None, None, None, None, None, None, None, None,
                       C.byref(h))
    assert st == lp.LP_ERR_INVALID_ARG


def test_batch_create_rejects_bad_boundaries_on_host(lib):
    from paper_2105_12715_gb300 import lp

    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    v = np.array([1.0, 1.0])
    ones, zeros = np.ones(2), np.zeros(2)
    rt = np.zeros(2, dtype=np.int8)
    cases = [([0], [0], "count"),                      # no problems
             ([1, 2], [0, 1, 2], "start at 0"),         # row boundaries not from 0
             ([0, 2, 1], [0, 1, 2], "nondecreasing"),   # decreasing row boundaries
             ([0, 1, 2], [0, 0, 2], "column")]          # a problem without columns
    for rs, cs, what in cases:
        rs_a, cs_a = np.array(rs, np.int32), np.array(cs, np.int32)
        h = C.c_void_p()
        st = lib.lp_batch_create(max(0, len(rs) - 1), C.c_void_p(rs_a.ctypes.data),
                                 C.c_void_p(cs_a.ctypes.data), 2, C.c_void_p(rp.ctypes.data),
                                 C.c_void_p(ci.ctypes.data), C.c_void_p(v.ctypes.data),
                                 C.c_void_p(ones.ctypes.data), C.c_void_p(ones.ctypes.data),
                                 C.c_void_p(zeros.ctypes.data), C.c_void_p(ones.ctypes.data),
                                 C.c_void_p(rt.ctypes.data), None, None, None, C.byref(h))
        assert st == lp.LP_ERR_INVALID_ARG, what
        assert what in lp._last_error(), (what, lp._last_error())
    t = lp.lp_batch_default_tuning()
    assert t.autotune == 1 and t.max_k_shift == 2 and t.check_budget == pytest.approx(0.05)
