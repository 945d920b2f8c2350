"""FP64 CPU oracle of the detector-trace spectra (Sec. V) -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's reference legs may use this
module.  It shares no code with the CUDA library (csrc/spectra.cu); the two
meet only through the traces they are given.

Sec. V reads the detector fields as spectra E_omega.  The Fourier convention
is that of eq. GreenMethod, whose time factor is exp(+i omega t'):
    E(t) = 1/(2 pi) int E_omega exp(-i omega t) d omega,
    E_omega = int E(t) exp(+i omega t) dt,
and for a trace sampled at t_n = t0 + n dt the integral becomes the sum
    E_omega(f) = dt * sum_{m=0}^{count-1} g_m x_{first+m} exp(i 2 pi f t_{first+m}),
over a gate of `count` samples starting at `first`, with g the Tukey window
of taper fraction alpha (alpha = 0: rectangular; alpha = 1: Hann):
    u = m / (count - 1),
    g = (1 - cos(2 pi u / alpha)) / 2          for u < alpha / 2,
    g = 1                                      for alpha / 2 <= u <= 1 - alpha / 2,
    g = (1 - cos(2 pi (1 - u) / alpha)) / 2    for u > 1 - alpha / 2
(g = 1 for count = 1).  A trace of several components (the detectors record
(E_z, E_r)) enters as the combination x_n = sum_c a_c X_n[c]; the field along
the direction theta-hat of a spherical frame about the shower maximum is
a = (-sin theta, cos theta).
"""
from __future__ import annotations

import math

import numpy as np


def tukey(count: int, taper: float) -> np.ndarray:
    """The window g_m, m = 0 .. count-1 (definition in the module docstring)."""
    if count < 1:
        return np.zeros(0)
    if count == 1 or taper <= 0.0:
        return np.ones(count)
    u = np.arange(count) / (count - 1)
    g = np.ones(count)
    lo = u < taper / 2
    hi = u > 1 - taper / 2
    g[lo] = 0.5 * (1 - np.cos(2 * math.pi * u[lo] / taper))
    g[hi] = 0.5 * (1 - np.cos(2 * math.pi * (1 - u[hi]) / taper))
    return g


def spectrum(x, dt, freqs, t0=0.0, coef=None, gate=None, taper=0.0):
    """E_omega at the frequencies `freqs` (Hz) of every trace.

    x: [n_traces, n_t] or [n_traces, n_t, n_comp] samples at t0 + n dt;
    coef: [n_traces, n_comp] combination of the components (default: the
    first component alone); gate: [n_traces, 2] (first, count) (default: the
    whole trace); taper: Tukey fraction.  Returns complex128 [n_traces, n_f]."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 2:
        x = x[:, :, None]
    n_tr, n_t, n_c = x.shape
    if coef is None:
        coef = np.zeros((n_tr, n_c))
        coef[:, 0] = 1.0
    coef = np.asarray(coef, dtype=np.float64).reshape(n_tr, n_c)
    if gate is None:
        gate = np.tile([0, n_t], (n_tr, 1))
    gate = np.asarray(gate, dtype=np.int64).reshape(n_tr, 2)
    f = np.asarray(freqs, dtype=np.float64).ravel()
    out = np.zeros((n_tr, f.size), dtype=np.complex128)
    for p in range(n_tr):
        first, count = int(gate[p, 0]), int(gate[p, 1])
        if first < 0 or count < 0 or first + count > n_t:
            raise ValueError("gate outside the trace")
        if count == 0:
            continue
        s = x[p, first:first + count, :] @ coef[p]
        g = tukey(count, taper)
        t = t0 + dt * (first + np.arange(count))
        out[p] = dt * ((g * s) @ np.exp(2j * math.pi * np.outer(t, f)))
    return out


def theta_coef(theta):
    """(E_z, E_r) coefficients of the theta-hat component in a spherical frame
    whose polar axis is the shower axis: E_theta = E_r cos(theta) - E_z sin(theta)."""
    th = np.asarray(theta, dtype=np.float64).ravel()
    return np.stack([-np.sin(th), np.cos(th)], axis=1)
