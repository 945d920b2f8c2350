"""The 3D hot path (default tile kernel, CPML) against the exact solution of
eq. GreenMethod in the frequency domain, on the GPU.

A Gaussian charge profile (eq. showerModel, l = 12 cm) moves at v = c along
the axis node line of a dx = 2 cm grid with a 10-cell CPML; detectors sit at
theta_c -25, -15, +15, +25 degrees about the profile's maximum.  Their
theta-hat spectra (fdtd_trace_spectrum, gated around the direct pulse) from
150 to 500 MHz (17 or more cells per wavelength) must match
* the exact line-current solution (superposed Hertzian elements,
  tests/physics.py) to 2 % -- the FP64 oracle on the smaller grid reaches
  1.2 %, and the GPU path equals the oracle to 1e-4;
* at R = 4 m, where l^2 sin^2(theta) / (lambda R) < 0.01, also the far-field
  formula eq. 1d_appro to 3 %.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import spectra as S
from physics import EPS0, far_field_1d_gauss, line_current_field_w

pytestmark = pytest.mark.gpu

DX = 0.02
NPML = 10
L_PROF = 0.12
Q_MAX = -1e-9
FREQS = np.arange(150e6, 501e6, 50e6)
N_IDX = math.sqrt(W.EPS_R_ICE)


@pytest.mark.parametrize("nx,nz,R,steps", [(200, 400, 1.5, 480), (480, 800, 4.0, 900)])
def test_spectra_match_exact_solution(nx, nz, R, steps):
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as fd
    dt = W.courant_dt(DX, W.EPS_R_ICE)
    z0 = (NPML + 4) * DX
    zm = z0 + 5 * L_PROF
    bdz = DX / 4
    zb = z0 + bdz * np.arange(int(10 * L_PROF / bdz) + 1)
    q = Q_MAX * np.exp(-0.5 * ((zb - zm) / L_PROF) ** 2)
    ax = nx // 2 * DX
    thc = math.acos(1 / N_IDX)
    ths = thc + np.radians([-25.0, -15.0, 15.0, 25.0])
    xyz = np.stack([ax + R * np.sin(ths), np.full(4, ax), zm + R * np.cos(ths)], 1)
    sim = fd.Simulation(nx, nx, nz, DX, dt, W.EPS_R_ICE, boundary=fd.FDTD_CPML, npml=NPML)
    # the default path of a CPML grid: two steps per pass from FDTD_TWO_STEP_MIN_CELLS (3 * 2^22) cells
    assert sim.kernel_name == ("tblock2-120x8" if nx * nx * nz >= 3 << 22 else "fused-vtile-128x8")
    sim.set_shower(q, z0, bdz, W.C0, np.array([1.0]), 0)
    sim.set_probes(xyz, steps)
    sim.step(steps)
    nodes = np.asarray(sim.probe_nodes())
    r = (nodes[:, 0] - nx // 2) * DX
    z = nodes[:, 2] * DX
    Rn, th = np.hypot(r, z - zm), np.arctan2(r, z - zm)
    # gate: +-5 ns around the arrival of the maximum's radiation (sample s at (s + 1) dt)
    W5 = int(5e-9 / dt)
    first = np.round(((zm - z0) / W.C0 + Rn * N_IDX / W.C0) / dt).astype(np.int64) - 1 - W5
    assert first.min() >= 0 and (first + 2 * W5).max() <= steps
    E = np.abs(sim.spectrum(FREQS, theta=th, gate=np.stack([first, np.full(4, 2 * W5)], 1), taper=0.25)
               .cpu().numpy())
    sim.close()
    hq = DX / 40
    zq = np.arange(z0, zb[-1], hq) + hq / 2
    qq = np.interp(zq, zb, q) * hq
    tq = (zq - z0) / W.C0
    worst = 0.0
    for p in range(4):
        Ez, Er = line_current_field_w(FREQS, r[p], z[p], zq, qq, tq, W.EPS_R_ICE * EPS0)
        G = np.abs(Er * math.cos(th[p]) - Ez * math.sin(th[p]))
        dev = np.abs(E[p] / G - 1)
        worst = max(worst, dev.max())
        assert dev.max() <= 0.02, (math.degrees(th[p]), dev)
        if R >= 4.0:
            F = np.abs(far_field_1d_gauss(FREQS, th[p], Rn[p], N_IDX, Q_MAX, L_PROF))
            assert np.abs(E[p] / F - 1).max() <= 0.03, (math.degrees(th[p]), E[p] / F)
    print(f"R = {R} m: worst deviation from the exact solution {worst:.4f}")
