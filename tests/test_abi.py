"""The C-ABI library builds, loads and exports every symbol include/gwl.h declares (CPU only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1909_11873_gb300 import build as B
from paper_1909_11873_gb300 import gwl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return gwl.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gwl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "gwl_create" in names and "ns_replace" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(gwl.EXPORTS)


def test_argument_errors_are_synchronous(L):
    """Invalid arguments fail with GWL_ERR_ARG before any device work."""
    out = C.c_void_p()
    f = np.arange(16, dtype=np.float64) + 20.0
    s = np.zeros((1, 16, 2))
    p = np.ones((1, 16))
    dets = gwl.detectors(np.zeros(9))
    opt = gwl.GwlOptions()
    opt.n_dim = 1
    assert L.gwl_create(None, 16, s.ctypes.data, p.ctypes.data, dets, 1, C.byref(opt), C.byref(out)) == -1
    assert L.gwl_create(f.ctypes.data, 16, s.ctypes.data, p.ctypes.data, dets, 0, C.byref(opt), C.byref(out)) == -1
    assert b"n_det" in L.gwl_last_error()
    bad = f.copy()
    bad[5] += 0.01
    assert L.gwl_create(bad.ctypes.data, 16, s.ctypes.data, p.ctypes.data, dets, 1, C.byref(opt), C.byref(out)) == -1
    assert b"uniformly" in L.gwl_last_error()
    neg = -p
    assert L.gwl_create(f.ctypes.data, 16, s.ctypes.data, neg.ctypes.data, dets, 1, C.byref(opt), C.byref(out)) == -1
    opt.precision = 7
    assert L.gwl_create(f.ctypes.data, 16, s.ctypes.data, p.ctypes.data, dets, 1, C.byref(opt), C.byref(out)) == -1
    assert L.gwl_loglike(None, None, 1, None, None) == -1
    assert L.gwl_autotune(None, None, 1, 1, None, None) == -1
    assert L.gwl_set_tuning(None, None) == -1
    assert L.gwl_get_tuning(None, None) == -1
    assert L.gwl_set_calibration(None, 10, f.ctypes.data, 0.1, 0.1) == -1
    assert L.gwl_get_calibration(None, None, None) == -1
    assert L.gwl_test_wait_timeout(None, 0.05, None) == -1
    assert L.gwl_ff_eval(None, 4, gwl.GWL_FF_EXP, None, None) == -1
    assert L.gwl_ff_eval(f.ctypes.data, 4, 7, f.ctypes.data, None) == -1
    assert L.gwl_ff_eval(f.ctypes.data, -1, gwl.GWL_FF_EXP, f.ctypes.data, None) == -1
    assert L.gwl_ff_eval(None, 0, gwl.GWL_FF_EXP, None, None) == 0
    assert out.value is None


def test_grid_tolerance_is_1e9_of_the_spacing(L):
    """Frequencies are accepted within 1e-9 of the spacing of f0 + j df and refused beyond it: the
    bin count at the ISCO cut is taken from the grid away from grid points on that bound.  After an
    accepted grid a non-positive PSD stops the call, which shows which check refused it (no device
    work happens before either check)."""
    out = C.c_void_p()
    f = np.arange(16, dtype=np.float64) + 20.0
    s = np.zeros((1, 16, 2))
    bad_psd = -np.ones((1, 16))
    dets = gwl.detectors(np.zeros(9))
    opt = gwl.GwlOptions()
    opt.n_dim = 1
    near = f.copy()
    near[7] += 5e-10
    assert L.gwl_create(near.ctypes.data, 16, s.ctypes.data, bad_psd.ctypes.data, dets, 1, C.byref(opt),
                        C.byref(out)) == -1
    assert b"psd" in L.gwl_last_error()
    far = f.copy()
    far[7] += 2e-9
    assert L.gwl_create(far.ctypes.data, 16, s.ctypes.data, bad_psd.ctypes.data, dets, 1, C.byref(opt),
                        C.byref(out)) == -1
    assert b"uniformly" in L.gwl_last_error()
    assert out.value is None


def test_checkpoint_size_and_argument_errors(L):
    """ns_state_doubles: a header of 26 doubles, the live set (K (D + 1)) and up to max_dead dead points
    (D + 2 each); invalid sizes give -1; ns_run_resumable and the multi-event entry points refuse a null
    context or batch synchronously."""
    assert L.ns_state_doubles(250, 4, 1000) == 26 + 250 * 5 + 1000 * 6
    assert L.ns_state_doubles(2, 1, 0) == 26 + 2 * 2
    assert L.ns_state_doubles(1, 4, 0) == -1
    assert L.ns_state_doubles(10, 0, 0) == -1
    assert L.ns_state_doubles(10, 4, -1) == -1
    res = gwl.GwlNsResult()
    assert L.ns_run_resumable(None, 10, 10, 1, 0, 0.1, 1, 1.0, 0, None, None, None, C.byref(res), None, None,
                              None) == -1
    # the multi-event counterparts: a null batch is refused synchronously
    assert L.gwl_multi_ns_state_doubles(None, 250) == -1
    assert L.gwl_multi_ns_run_resumable(None, 10, 10, 1, 0, 0.1, 1, 1.0, C.byref(res), None, None, None) == -1


def test_binding_buffer_addresses():
    """The binding's host-buffer addresses (taken without numpy's ctypes helper where the buffer is
    writable) equal numpy's own for whole arrays, row views, read-only and empty arrays; a
    non-contiguous array is refused."""
    import numpy as np
    from paper_1909_11873_gb300 import gwl
    a = np.zeros((10, 11))
    ro = np.zeros(5)
    ro.flags.writeable = False
    for t in (a, a[3:], a[3:4], ro, np.zeros(0), np.zeros((0, 11))):
        assert gwl._ptr(t) == t.ctypes.data
    with pytest.raises(ValueError):
        gwl._ptr(a[:, 1:])
