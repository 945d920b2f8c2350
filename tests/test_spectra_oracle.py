"""Pins of the spectrum oracle (oracle/spectra.py, the E_omega of Sec. V)
against closed forms and a library routine:

* a sampled Gaussian pulse has the continuous transform
  s sqrt(2 pi) exp(-w^2 s^2 / 2) exp(+i w tau) (sign of the exponent, dt scale,
  the time origin t0 and the absolute sample times under a gate);
* Parseval's identity on the DFT frequency grid f_k = k / (N dt);
* the taper is scipy's Tukey window;
* a gate that holds the whole pulse leaves the spectrum unchanged;
* the theta-hat combination of (E_z, E_r).
"""
import math

import numpy as np
import pytest

from oracle import spectra as S


def _gauss(n_t, dt, t0, tau, s):
    t = t0 + dt * np.arange(n_t)
    return np.exp(-0.5 * ((t - tau) / s) ** 2)


@pytest.mark.parametrize("t0", [0.0, 3.7e-11])
def test_gaussian_pulse_transform(t0):
    dt, s, tau = 1e-11, 1.2e-10, 2.0e-9
    x = _gauss(400, dt, t0, tau, s)
    f = np.linspace(-3e9, 3e9, 41)
    E = S.spectrum(x[None], dt, f, t0=t0)[0]
    w = 2 * math.pi * f
    ref = s * math.sqrt(2 * math.pi) * np.exp(-0.5 * (w * s) ** 2) * np.exp(1j * w * tau)
    assert np.max(np.abs(E - ref)) <= 1e-12 * s


def test_parseval_on_dft_grid():
    rng = np.random.default_rng(5)
    N, dt = 128, 2.5e-11
    x = rng.standard_normal(N)
    f = np.arange(N) / (N * dt)
    E = S.spectrum(x[None], dt, f)[0]
    assert abs(dt * np.sum(x * x) - np.sum(np.abs(E) ** 2) / (N * dt)) <= 1e-12 * dt * np.sum(x * x)


@pytest.mark.parametrize("N", [1, 2, 7, 64, 301])
@pytest.mark.parametrize("alpha", [0.0, 0.1, 0.25, 0.5, 1.0])
def test_taper_is_tukey(N, alpha):
    sig = pytest.importorskip("scipy.signal")
    assert np.allclose(S.tukey(N, alpha), sig.windows.tukey(N, alpha, sym=True), atol=1e-14)


def test_gate_holding_the_pulse_changes_nothing():
    dt, s, tau = 1e-11, 1e-10, 3e-9
    x = _gauss(1000, dt, 0.0, tau, s)
    f = np.linspace(5e7, 2e9, 30)
    full = S.spectrum(x[None], dt, f)[0]
    k = int(tau / dt)
    gated = S.spectrum(x[None], dt, f, gate=[[k - 150, 300]])[0]
    tap = S.spectrum(x[None], dt, f, gate=[[k - 200, 400]], taper=0.3)[0]   # taper only where x ~ 0
    assert np.max(np.abs(gated - full)) <= 1e-12 * np.max(np.abs(full))
    assert np.max(np.abs(tap - full)) <= 1e-12 * np.max(np.abs(full))
    with pytest.raises(ValueError):
        S.spectrum(x[None], dt, f, gate=[[900, 200]])


def test_theta_component():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((3, 50, 2))
    th = np.array([0.3, 1.0, 2.0])
    f = np.array([1e8, 7e8])
    E = S.spectrum(X, 1e-11, f, coef=S.theta_coef(th))
    for p in range(3):
        x = X[p, :, 1] * math.cos(th[p]) - X[p, :, 0] * math.sin(th[p])
        assert np.allclose(E[p], S.spectrum(x[None], 1e-11, f)[0], rtol=1e-13, atol=0)
    # real traces: E(-f) = conj E(f)
    Em = S.spectrum(X, 1e-11, -f, coef=S.theta_coef(th))
    assert np.allclose(Em, np.conj(E), rtol=1e-13, atol=0)
