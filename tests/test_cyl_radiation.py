"""Radiation pins of the 2D axisymmetric oracle (oracle/cyl_oracle.py) and the
spectrum oracle together (Sec. II and V).

A Gaussian charge profile (eq. showerModel, l = 10 cm, on the axis) moves at
v = c through ice; four detectors sit R = 2 m from the profile's maximum at
theta_c -25, -15, +15, +25 degrees.  The theta-hat spectrum of each detector's
trace, gated around the direct pulse so that the Mur walls' reflections stay
out, must match
* the exact solution of eq. GreenMethod for the same line current
  (superposed Hertzian elements, tests/physics.py) to 1.5 % in magnitude from
  150 to 800 MHz (the grid has 21 cells per wavelength at 800 MHz);
* the far-field formula eq. 1d_appro (Fraunhofer, eq. fraun_appr) to 2 % from
  200 to 800 MHz, where l^2 sin^2(theta) / (lambda R) < 0.03 and kR > 15.
"""
import math

import numpy as np
import pytest

from oracle import cyl_oracle as CO
from oracle import spectra as S
from physics import far_field_1d, far_field_1d_gauss, line_current_field_w

D = 0.01
EPS_R = 3.17
N_IDX = math.sqrt(EPS_R)
L_PROF = 0.10
ZM = 1.5
Q_MAX = -1e-9
R_DET = 2.0


@pytest.fixture(scope="module")
def run():
    dt = CO.courant_dt(D, EPS_R)
    z0 = ZM - 5 * L_PROF
    bdz = D / 2
    zb = z0 + bdz * np.arange(int(10 * L_PROF / bdz) + 1)
    q = Q_MAX * np.exp(-0.5 * ((zb - ZM) / L_PROF) ** 2)
    thc = math.acos(1 / N_IDX)
    ths = thc + np.radians([-25.0, -15.0, 15.0, 25.0])
    rz = np.stack([R_DET * np.sin(ths), ZM + R_DET * np.cos(ths)], 1)
    steps = 860
    o = CO.CylOracle(320, 440, D, dt, EPS_R)      # walls >= 1.2 m beyond the detectors
    o.set_shower(q, z0, bdz, CO.C0, [1.0])
    o.set_probes(rz)
    o.step(steps)
    return dict(dt=dt, z0=z0, zb=zb, q=q, nodes=o.probes * D, tr=o.traces(), steps=steps)


def _gated_theta_spectrum(run, p, freqs):
    dt, tr = run["dt"], run["tr"]
    rr, zz = run["nodes"][p]
    R, th = math.hypot(rr, zz - ZM), math.atan2(rr, zz - ZM)
    a = S.theta_coef([th])
    k0 = int(np.argmax(np.abs(tr[p] @ a[0])))
    W = int(4e-9 / dt)                            # reflections arrive >= 10 ns later
    first = k0 - W
    assert first > 0 and first + 2 * W <= run["steps"]
    E = S.spectrum(tr[p][None], dt, freqs, t0=dt, coef=a, gate=[[first, 2 * W]], taper=0.25)[0]
    return E, R, th


def test_matches_exact_line_current_solution(run):
    freqs = np.arange(150e6, 801e6, 50e6)
    hq = D / 40
    zq = np.arange(run["z0"], run["zb"][-1], hq) + hq / 2
    qq = np.interp(zq, run["zb"], run["q"]) * hq
    tq = (zq - run["z0"]) / CO.C0
    for p in range(4):
        E, R, th = _gated_theta_spectrum(run, p, freqs)
        rr, zz = run["nodes"][p]
        Ez, Er = line_current_field_w(freqs, rr, zz, zq, qq, tq, EPS_R * CO.EPS0)
        Eg = Er * math.cos(th) - Ez * math.sin(th)
        err = np.abs(np.abs(E) / np.abs(Eg) - 1)
        assert err.max() <= 0.015, (math.degrees(th), err)


def test_far_field_formula(run):
    freqs = np.arange(200e6, 801e6, 50e6)
    t_ref = (ZM - run["z0"]) / CO.C0
    for p in range(4):
        E, R, th = _gated_theta_spectrum(run, p, freqs)
        Ef = far_field_1d_gauss(freqs, th, R, N_IDX, Q_MAX, L_PROF, t_ref=t_ref)
        err = np.abs(np.abs(E) / np.abs(Ef) - 1)
        assert err.max() <= 0.02, (math.degrees(th), err)
        # the form factor exp(-l^2 p^2 / 2) is part of what is checked: it is far from 1 here
        pw = 2 * math.pi * freqs[-1] * (1 - N_IDX * math.cos(th)) / CO.C0
        assert p not in (0, 3) or math.exp(-0.5 * (L_PROF * pw) ** 2) < 0.8


def test_far_field_closed_form_is_its_integral():
    """Eq. 1d_appro's Gaussian closed form against quadrature of its integral form."""
    l, th, R = 0.3, 1.2, 40.0
    z = np.arange(-8 * l, 8 * l, l / 200)
    qdz = -2e-9 * np.exp(-0.5 * (z / l) ** 2) * (l / 200)
    f = np.linspace(1e7, 2e9, 25)
    a = far_field_1d(f, th, R, N_IDX, z, qdz, t_ref=3e-9)
    b = far_field_1d_gauss(f, th, R, N_IDX, -2e-9, l, t_ref=3e-9)
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))
