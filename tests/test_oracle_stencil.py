"""Pins of the oracle's Yee stencil (Sec. III.A: Maxwell curl equations,
central differences, staggered leapfrog) against closed forms.

* discrete eigenmodes of a PEC cavity oscillate exactly at the Yee dispersion
  relation's frequency, and that frequency tends to the continuum cavity mode
  frequency as O(dx^2);
* the discrete energy 1/2 eps |E^n|^2 + 1/2 mu H^{n-1/2}.H^{n+1/2} of a
  lossless PEC cavity is conserved to rounding;
* with the moving source switched on, the energy changes by exactly the work
  -dt/2 <J^{n+1/2}, E^n + E^{n+1}> of the current.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from physics import EPS0, MU0, discrete_omega, live_masks


def _cavity_mode(nx, ny, nz, dx, m, n, p, A):
    """E of the (m,n,p) PEC cavity mode sampled at the Yee positions."""
    Lx, Ly, Lz = nx * dx, ny * dx, nz * dx
    kx, ky, kz = m * math.pi / Lx, n * math.pi / Ly, p * math.pi / Lz
    z, y, x = np.meshgrid(np.arange(nz + 1) * dx, np.arange(ny + 1) * dx,
                          np.arange(nx + 1) * dx, indexing="ij")
    h = dx / 2
    Ex = A[0] * np.cos(kx * (x + h)) * np.sin(ky * y) * np.sin(kz * z)
    Ey = A[1] * np.sin(kx * x) * np.cos(ky * (y + h)) * np.sin(kz * z)
    Ez = A[2] * np.sin(kx * x) * np.sin(ky * y) * np.cos(kz * (z + h))
    masks = live_masks(nx, ny, nz)
    return [np.where(masks[c], F, 0.0) for c, F in enumerate((Ex, Ey, Ez))], (kx, ky, kz)


@pytest.mark.parametrize("mnp", [(1, 1, 1), (2, 1, 3), (1, 3, 2)])
def test_cavity_eigenmode_follows_yee_dispersion(mnp):
    nx, ny, nz = 14, 12, 10
    dx = 0.02
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    o = oracle.Oracle(nx, ny, nz, dx, dt, W.EPS_R_ICE, oracle.PEC)
    Lk = [math.pi * q / (N * dx) for q, N in zip(mnp, (nx, ny, nz))]
    kt = [2.0 / dx * math.sin(k * dx / 2) for k in Lk]
    # divergence-free amplitude: A orthogonal to the discrete wave vector
    a = np.cross(kt, [0.3, -0.7, 0.5])
    E0, kv = _cavity_mode(nx, ny, nz, dx, *mnp, a)
    for c in range(3):
        o.set_field(c, E0[c])
    cp = W.C0 / math.sqrt(W.EPS_R_ICE)
    w = discrete_omega(kv, dx, dt, cp)
    nrm = sum((e * e).sum() for e in E0)
    th = w * dt
    for n in range(1, 121):
        o.step(1)
        En = [o.field(c) for c in range(3)]
        amp = sum((en * e).sum() for en, e in zip(En, E0)) / nrm
        # leapfrog oscillator started from H^{-1/2} = 0:
        # E^n / E^0 = cos((n + 1/2) w dt) / cos(w dt / 2)
        expect = math.cos((n + 0.5) * th) / math.cos(0.5 * th)
        assert abs(amp - expect) < 1e-10, (n, amp, expect)
        # the field stays proportional to the mode shape (no index mixing)
        resid = sum(((en - amp * e) ** 2).sum() for en, e in zip(En, E0))
        assert resid < 1e-20 * nrm


def test_cavity_frequency_converges_to_continuum():
    """Analytic TM_110 frequency w = c' pi sqrt(1/Lx^2 + 1/Ly^2); the discrete
    one approaches it as O(dx^2)."""
    cp = W.C0 / math.sqrt(W.EPS_R_ICE)
    Lx, Ly, Lz = 0.24, 0.20, 0.16
    w_exact = cp * math.pi * math.sqrt(1 / Lx ** 2 + 1 / Ly ** 2)
    errs = []
    for N in (1, 2, 4):
        dx = 0.02 / N
        nx, ny, nz = round(Lx / dx), round(Ly / dx), round(Lz / dx)
        dt = W.courant_dt(dx, W.EPS_R_ICE)
        o = oracle.Oracle(nx, ny, nz, dx, dt, W.EPS_R_ICE, oracle.PEC)
        E0, kv = _cavity_mode(nx, ny, nz, dx, 1, 1, 0, [0.0, 0.0, 1.0])
        o.set_field(2, E0[2])
        o.step(1)
        # E^1 = (2 cos(w dt) - 1) E^0 for H^{-1/2} = 0
        c1 = (o.field(2) * E0[2]).sum() / (E0[2] ** 2).sum()
        w = math.acos(0.5 * (c1 + 1.0)) / dt
        errs.append(abs(w - w_exact) / w_exact)
    assert errs[0] < 5e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def _energy(E, Hm, Hp, eps, dx):
    we = 0.5 * eps * sum((e * e).sum() for e in E)
    wh = 0.5 * MU0 * sum((a * b).sum() for a, b in zip(Hm, Hp))
    return (we + wh) * dx ** 3


def test_energy_conserved_in_pec_cavity():
    nx, ny, nz = 13, 11, 9
    dx = 0.02
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    o = oracle.Oracle(nx, ny, nz, dx, dt, W.EPS_R_ICE, oracle.PEC)
    rng = np.random.default_rng(5)
    masks = live_masks(nx, ny, nz)
    for c in range(6):
        scale = 1.0 if c < 3 else 1.0 / 377.0
        o.set_field(c, np.where(masks[c], rng.standard_normal(o.shape) * scale, 0.0))
    eps = W.EPS_R_ICE * EPS0
    Ws = []
    for n in range(2000):
        E = [o.field(c) for c in range(3)]
        Hm = [o.field(c) for c in range(3, 6)]
        o.step(1)
        Hp = [o.field(c) for c in range(3, 6)]
        if n % 100 == 0 or n == 1999:
            Ws.append(_energy(E, Hm, Hp, eps, dx))
    Ws = np.array(Ws)
    assert np.abs(Ws / Ws[0] - 1.0).max() < 1e-12


def test_energy_changes_by_source_work():
    """W^{n+1} - W^n = -dt/2 dx^3 sum J^{n+1/2} (E^n + E^{n+1}) in a PEC box."""
    w = W.parity96(n=32, steps=90, n_probes=2)
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.eps_r, oracle.PEC)
    q, lw = oracle.tables(w)
    o.set_shower(q, w.z0, w.bin_dz, w.v, lw, w.lateral["L"])
    eps = w.eps_r * EPS0
    E = [o.field(c) for c in range(3)]
    Hm = [o.field(c) for c in range(3, 6)]
    prev = None
    worst = scale = 0.0
    for n in range(w.steps):
        o.step(1)
        Hp = [o.field(c) for c in range(3, 6)]
        En1 = [o.field(c) for c in range(3)]
        idx, J = o.source()
        Wn = _energy(E, Hm, Hp, eps, w.dx)
        if prev is not None:
            W_prev, work_prev = prev
            worst = max(worst, abs((Wn - W_prev) - work_prev))
            scale = max(scale, abs(work_prev))
        work = -0.5 * w.dt * w.dx ** 3 * float((J * (E[2] + En1[2]).ravel()[idx]).sum())
        prev = (Wn, work)
        E, Hm = En1, Hp
    assert scale > 0.0
    assert worst < 1e-9 * scale
