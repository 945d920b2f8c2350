"""Spectra of detector traces (spectra.h, Sec. V) on the GPU.

* Parity: fdtd_trace_spectrum against the oracle (oracle/spectra.py) on the
  same float32 traces -- ragged gates (empty, one sample, whole trace),
  tapers, component weights, negative and zero frequencies, t0 != 0, and a
  200 000-sample trace whose phases wrap many times.  The bound is
  2e-6 x dt x sum |x| per value (float32 partial sums, 2^-24 turns of phase).
* Argument checks, including a host pointer for the traces.
"""
import math

import numpy as np
import pytest

from oracle import spectra as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _check(E, X, dt, freqs, t0, coef, gate, taper):
    ref = S.spectrum(X, dt, freqs, t0=t0, coef=coef, gate=gate, taper=taper)
    n_tr = X.shape[0]
    Xc = X if X.ndim == 3 else X[:, :, None]
    co = coef if coef is not None else np.eye(Xc.shape[2])[:1].repeat(n_tr, 0)
    g = gate if gate is not None else np.tile([0, Xc.shape[1]], (n_tr, 1))
    for p in range(n_tr):
        a, b = g[p]
        l1 = dt * (np.abs(Xc[p, a:a + b].astype(np.float64)) @ np.abs(co[p])).sum()
        err = np.abs(E[p] - ref[p]).max() if b else np.abs(E[p]).max()
        assert err <= 2e-6 * l1 + 1e-30, (p, a, b, err, l1)
    return ref


@pytest.mark.parametrize("n_comp", [1, 2, 3])
@pytest.mark.parametrize("taper", [0.0, 0.3, 1.0])
def test_matches_oracle_ragged(fd, n_comp, taper):
    import torch
    rng = np.random.default_rng(100 + n_comp)
    n_tr, n_t = 37, 5003
    X = rng.standard_normal((n_tr, n_t, n_comp)).astype(np.float32)
    coef = rng.standard_normal((n_tr, n_comp))
    first = rng.integers(0, n_t, n_tr)
    count = np.array([rng.integers(0, n_t - f + 1) for f in first])
    count[0], count[1], count[2] = 0, 1, 2
    first[3], count[3] = 0, n_t
    gate = np.stack([first, count], 1)
    dt, t0 = 2.1e-11, -3.3e-10
    freqs = np.concatenate([[0.0, -4e8], np.linspace(1e7, 1 / dt, 29)])   # up to the sampling rate
    E = fd.trace_spectrum(torch.from_numpy(X).cuda(), dt, freqs, t0=t0, coef=coef, gate=gate, taper=taper)
    _check(E.cpu().numpy().astype(np.complex128), X, dt, freqs, t0, coef, gate, taper)


def test_default_component_and_whole_trace(fd):
    import torch
    rng = np.random.default_rng(7)
    X = rng.standard_normal((5, 777, 2)).astype(np.float32)
    f = np.linspace(-1e9, 1e9, 17)
    E = fd.trace_spectrum(torch.from_numpy(X).cuda(), 1e-11, f).cpu().numpy()
    _check(E.astype(np.complex128), X, 1e-11, f, 0.0, None, None, 0.0)
    E2 = fd.trace_spectrum(torch.from_numpy(np.ascontiguousarray(X[:, :, 0])).cuda(), 1e-11, f).cpu().numpy()
    assert np.array_equal(E, E2)


def test_long_trace_phase(fd):
    """A sinusoid over 200 000 samples: the phase runs through ~10^4 turns."""
    import torch
    dt, n_t = 1.7e-11, 200000
    f0 = 2.9e9
    t = dt * (1 + np.arange(n_t))
    X = np.stack([np.cos(2 * math.pi * f0 * t), np.sin(2 * math.pi * 0.37 * f0 * t)], 0).astype(np.float32)
    freqs = np.array([-f0, f0, 0.37 * f0, -0.37 * f0, 1e9])
    E = fd.trace_spectrum(torch.from_numpy(X).cuda(), dt, freqs, t0=dt, taper=0.1).cpu().numpy()
    ref = _check(E.astype(np.complex128), X, dt, freqs, dt, None, None, 0.1)
    assert abs(abs(ref[0, 0]) - 0.5 * dt * n_t * (1 - 0.05)) < 1e-3 * dt * n_t   # the line itself


def test_simulation_and_cylinder_spectrum(fd):
    """The solvers' spectrum() = trace_spectrum of their own traces at t_s = (s + 1) dt."""
    from oracle import cyl_oracle as CO
    d = 0.01
    dt = CO.courant_dt(d, 3.17)
    q = -1e-12 * np.exp(-0.5 * ((np.arange(60) - 20) / 6.0) ** 2)
    c = fd.Cylinder(50, 130, d, dt, 3.17)
    c.set_shower(q, 0.05, 0.01, CO.C0, [1.0])
    rz = np.array([[0.1, 0.3], [0.2, 0.5]])
    c.set_probes(rz, 120)
    c.step(120)
    th = np.array([0.5, 1.0])
    f = np.linspace(1e8, 2e9, 9)
    E = c.spectrum(f, theta=th, gate=[[10, 100], [0, 120]], taper=0.2).cpu().numpy()
    tr = c.probes()
    _check(E.astype(np.complex128), tr, dt, f, dt, S.theta_coef(th), np.array([[10, 100], [0, 120]]), 0.2)


def test_arguments(fd):
    import ctypes as C
    import torch
    X = torch.zeros((2, 10, 2), device="cuda")
    out = torch.zeros((2, 3, 2), device="cuda")
    f = np.array([1e8, 2e8, 3e8])
    fp = f.ctypes.data_as(C.POINTER(C.c_double))
    call = lambda tr, n_tr, n_t, n_c, gate, taper, dt, o, on_dev: fd.fdtd_trace_spectrum(
        tr, n_tr, n_t, n_c, None, gate, taper, dt, 0.0, fp, 3, o, on_dev, None)
    ok = (C.c_void_p(X.data_ptr()), 2, 10, 2, None, 0.0, 1e-11, C.c_void_p(out.data_ptr()), 1)
    assert call(*ok) == 0
    torch.cuda.synchronize()
    host = np.zeros((2, 10, 2), dtype=np.float32)
    bad_gate = np.array([[0, 10], [5, 6]], dtype=np.int32)
    for args in [(None,) + ok[1:], ok[:1] + (0,) + ok[2:], ok[:3] + (5,) + ok[4:],
                 ok[:5] + (1.5,) + ok[6:], ok[:6] + (0.0,) + ok[7:], ok[:6] + (float("nan"),) + ok[7:],
                 ok[:4] + (bad_gate.ctypes.data_as(C.POINTER(C.c_int)),) + ok[5:],
                 (C.c_void_p(host.ctypes.data),) + ok[1:]]:
        assert call(*args) == -1, args
    with pytest.raises(ValueError):
        fd.trace_spectrum(torch.zeros(3, 4), 1e-11, f)
