"""C ABI checks that need no GPU: the library loads, exports every function
include/*.h declares, rejects bad arguments on the host before touching the
device, and its host-side shower tables agree with the oracle's independent
ones."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_5341_gb300 as m
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b((?:fdtd|sur|cyl)_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(fd):
    names = _declared()
    assert len(names) >= 40
    lib = C.CDLL(fd.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror(fd):
    for code, name in fd.STATUS.items():
        s = fd.fdtd_strerror(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert fd.fdtd_strerror(-99) == b"unknown status"


def _create(fd, *a):
    h = C.c_void_p()
    rc = fd.fdtd_create(C.byref(h), *a)
    return rc, h


def test_create_rejects_bad_arguments_on_host(fd):
    dx = 0.02
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    assert fd.fdtd_create(None, 8, 8, 8, dx, dt, 3.17, 1, 0, None) == -1
    cases = [
        (3, 8, 8, dx, dt, 3.17, 1, 0),        # too small
        (8, 8, 8, -dx, dt, 3.17, 1, 0),       # negative dx
        (8, 8, 8, dx, 0.0, 3.17, 1, 0),       # zero dt
        (8, 8, 8, dx, dt, 0.5, 1, 0),         # eps_r < 1
        (8, 8, 8, dx, dt, 3.17, 7, 0),        # unknown boundary
        (20, 20, 20, dx, dt, 3.17, 2, 0),     # CPML without layer
        (20, 20, 20, dx, dt, 3.17, 2, 9),     # layer too deep for the grid
    ]
    for a in cases:
        rc, h = _create(fd, *a, None)
        assert rc == -1, a
        assert not h.value


def test_create_rejects_courant_violation(fd):
    dx = 0.02
    dt_max = dx * math.sqrt(W.EPS_R_ICE) / (W.C0 * math.sqrt(3.0))
    rc, h = _create(fd, 8, 8, 8, dx, dt_max * 1.001, W.EPS_R_ICE, 1, 0, None)
    assert rc == -2 and not h.value


def test_create_without_device_reports_cuda_error(fd):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    rc, h = _create(fd, 8, 8, 8, 0.02, W.courant_dt(0.02, W.EPS_R_ICE), W.EPS_R_ICE, 1, 0, None)
    assert rc == -5 and not h.value


def test_null_handle_calls_are_argument_errors(fd):
    assert fd.fdtd_step(None, 1) == -1
    assert fd.fdtd_sync(None) == -1
    assert fd.fdtd_reset(None) == -1
    fd.fdtd_destroy(None)


def test_cyl_create_rejects_bad_arguments_on_host(fd):
    d = 0.01
    dt = W.courant_dt_2d(d, W.EPS_R_ICE)
    assert fd.cyl_create(None, 8, 8, d, dt, 3.17, 1, None) == -1
    cases = [
        (3, 8, d, dt, 3.17, 1),        # too few rows
        (8, 3, d, dt, 3.17, 1),        # too few columns
        (8, 8, -d, dt, 3.17, 1),       # negative cell
        (8, 8, d, 0.0, 3.17, 1),       # zero dt
        (8, 8, d, dt, 0.5, 1),         # eps_r < 1
        (8, 8, d, dt, 3.17, 2),        # no CPML on the 2D grid
    ]
    for a in cases:
        h = C.c_void_p()
        assert fd.cyl_create(C.byref(h), *a, None) == -1, a
        assert not h.value
    h = C.c_void_p()
    dt_max = d * math.sqrt(W.EPS_R_ICE) / (W.C0 * math.sqrt(2.0))
    assert fd.cyl_create(C.byref(h), 8, 8, d, dt_max * 1.001, W.EPS_R_ICE, 1, None) == -2
    assert fd.cyl_step(None, 1) == -1 and fd.cyl_sync(None) == -1 and fd.cyl_set_kernel(None, 1, 0) == -1
    fd.cyl_destroy(None)


# ---- the library's host tables against the oracle's -------------------------

def test_profile_tables_agree_with_oracle(fd):
    for w in (W.parity96(), W.greisen384(), W.gh640(), W.greisen_small(), W.gh_small()):
        qa, wa = fd.tables(w)
        qb, wb = oracle.tables(w)
        assert qa.shape == qb.shape and wa.shape == wb.shape
        assert np.allclose(qa, qb, rtol=1e-12, atol=1e-15 * np.abs(qb).max()), w.name
        assert np.allclose(wa, wb, rtol=1e-12, atol=1e-15), w.name
        assert wa.sum() == pytest.approx(1.0)


def test_greisen_table_rejects_bad_energy(fd):
    out = np.zeros(4)
    assert fd.fdtd_profile_greisen(0.01, 4, 1e6, 78.6e6, 0.39, 0.2,
                                   out.ctypes.data_as(C.POINTER(C.c_double))) == -1


def test_trace_spectrum_rejects_bad_arguments_on_host(fd):
    f = np.array([1e8, 2e8])
    fp = f.ctypes.data_as(C.POINTER(C.c_double))
    out = np.zeros(8, dtype=np.float32)
    op = C.c_void_p(out.ctypes.data)
    # null traces, no traces, five components, taper > 1, dt <= 0, no frequencies: refused before any device call
    assert fd.fdtd_trace_spectrum(None, 2, 10, 2, None, None, 0.0, 1e-11, 0.0, fp, 2, op, 0, None) == -1
    assert fd.fdtd_trace_spectrum(op, 0, 10, 2, None, None, 0.0, 1e-11, 0.0, fp, 2, op, 0, None) == -1
    assert fd.fdtd_trace_spectrum(op, 2, 10, 5, None, None, 0.0, 1e-11, 0.0, fp, 2, op, 0, None) == -1
    assert fd.fdtd_trace_spectrum(op, 2, 10, 2, None, None, 1.5, 1e-11, 0.0, fp, 2, op, 0, None) == -1
    assert fd.fdtd_trace_spectrum(op, 2, 10, 2, None, None, 0.0, 0.0, 0.0, fp, 2, op, 0, None) == -1
    assert fd.fdtd_trace_spectrum(op, 2, 10, 2, None, None, 0.0, 1e-11, 0.0, fp, 0, op, 0, None) == -1
