"""Fraunhofer pin of the 3D oracle (oracle/fdtd_oracle.c) in the frequency domain.

A Gaussian charge profile (eq. showerModel, l = 12 cm, -1 nC) moves at v = c
along the axis node line of a 200 x 200 x 400 grid (dx = 2 cm, 10-cell CPML);
four detectors sit 1.5 m from the profile's maximum at theta_c -25, -15, +15
and +25 degrees.  Their theta-hat spectra (oracle/spectra.py, gated +-5 ns
around the arrival of the maximum's radiation) from 150 to 500 MHz must match
* the exact line-current solution of eq. GreenMethod (tests/physics.py) to
  1.5 % (17 or more cells per wavelength);
* the far-field formula eq. 1d_appro to 4 % -- here l^2 sin^2(theta) /
  (lambda R) < 0.03 and kR > 9, and the formula itself is within 2.3 % of the
  exact solution.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import spectra as S
from physics import EPS0, far_field_1d_gauss, line_current_field_w

DX = 0.02
NPML = 10
NX, NZ = 200, 400
L_PROF = 0.12
Q_MAX = -1e-9
R_DET = 1.5
STEPS = 480
FREQS = np.arange(150e6, 501e6, 50e6)
N_IDX = math.sqrt(W.EPS_R_ICE)


@pytest.fixture(scope="module")
def run():
    dt = W.courant_dt(DX, W.EPS_R_ICE)
    z0 = (NPML + 4) * DX
    zm = z0 + 5 * L_PROF
    bdz = DX / 4
    zb = z0 + bdz * np.arange(int(10 * L_PROF / bdz) + 1)
    q = Q_MAX * np.exp(-0.5 * ((zb - zm) / L_PROF) ** 2)
    ax = NX // 2 * DX
    thc = math.acos(1 / N_IDX)
    ths = thc + np.radians([-25.0, -15.0, 15.0, 25.0])
    xyz = np.stack([ax + R_DET * np.sin(ths), np.full(4, ax), zm + R_DET * np.cos(ths)], 1)
    o = oracle.Oracle(NX, NX, NZ, DX, dt, W.EPS_R_ICE, oracle.CPML, NPML)
    o.set_shower(q, z0, bdz, W.C0, np.array([1.0]), 0)
    o.set_probes(xyz, STEPS)
    o.step(STEPS)
    nodes = np.asarray(o.probe_nodes())
    r = (nodes[:, 0] - NX // 2) * DX
    z = nodes[:, 2] * DX
    Rn, th = np.hypot(r, z - zm), np.arctan2(r, z - zm)
    W5 = int(5e-9 / dt)
    first = np.round(((zm - z0) / W.C0 + Rn * N_IDX / W.C0) / dt).astype(np.int64) - 1 - W5
    assert first.min() >= 0 and (first + 2 * W5).max() <= STEPS
    E = np.abs(S.spectrum(o.probes(), dt, FREQS, t0=dt, coef=S.theta_coef(th),
                          gate=np.stack([first, np.full(4, 2 * W5)], 1), taper=0.25))
    return dict(E=E, r=r, z=z, Rn=Rn, th=th, z0=z0, zb=zb, q=q)


def test_matches_exact_line_current_solution(run):
    hq = DX / 40
    zq = np.arange(run["z0"], run["zb"][-1], hq) + hq / 2
    qq = np.interp(zq, run["zb"], run["q"]) * hq
    tq = (zq - run["z0"]) / W.C0
    for p in range(4):
        Ez, Er = line_current_field_w(FREQS, run["r"][p], run["z"][p], zq, qq, tq, W.EPS_R_ICE * EPS0)
        G = np.abs(Er * math.cos(run["th"][p]) - Ez * math.sin(run["th"][p]))
        dev = np.abs(run["E"][p] / G - 1)
        assert dev.max() <= 0.015, (math.degrees(run["th"][p]), dev)


def test_far_field_formula(run):
    for p in range(4):
        F = np.abs(far_field_1d_gauss(FREQS, run["th"][p], run["Rn"][p], N_IDX, Q_MAX, L_PROF))
        dev = np.abs(run["E"][p] / F - 1)
        assert dev.max() <= 0.04, (math.degrees(run["th"][p]), dev)
