"""Pins of the oracle's whole path against the physics of Sec. II.

* Green's-function solution: the field of a charge moving along the axis is
  the superposition of retarded Hertzian dipoles (the time-domain form of
  eq. GreenMethod).  After the same Gaussian low-pass on both sides, the
  oracle's detector traces match it to a few per cent at dx = 2 cm, and the
  error falls about four-fold when dx halves (second-order scheme).
* Cherenkov angle: behind a long uniformly charged shower moving at v = c, the
  shock reaches radius rho at t = (z + rho tan(theta_c))/v with
  cos(theta_c) = 1/(n beta) = 55.83 deg in ice.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from physics import EPS0, gauss_filter_trace, moving_charge_field


def _green_case(N, P, dx, steps, sig_steps, l=0.1):
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    o = oracle.Oracle(N, N, N, dx, dt, W.EPS_R_ICE, oracle.CPML, P)
    z0 = (P + 4) * dx
    zc = 0.80
    bin_dz = dx / 8
    nb = int(((N - P) * dx - z0) / bin_dz) + 1
    q = oracle.profile_gaussian(z0, bin_dz, nb, zc, l, -1e-9)
    o.set_shower(q, z0, bin_dz, W.C0, np.array([1.0]), 0)
    ax = (N // 2) * dx
    probes = [(ax + rho, ax, zc + dz) for rho in (0.16, 0.24, 0.32) for dz in (-0.2, 0.0, 0.2)]
    probes.append((ax + 0.12, ax + 0.16, zc + 0.1))
    o.set_probes(np.array(probes), steps)
    o.step(steps)
    tr = o.probes()
    nodes = o.probe_nodes()
    sigma = sig_steps * dt
    ts = np.arange(0, (steps + 1) * dt, dt / 2)
    ts = ts[(ts > 40 * dt / 2) & (ts < (steps - 3 * sig_steps) * dt)]
    hq = dx / 16
    zq = np.arange(z0, (N - P) * dx, hq) + hq / 2
    qq = np.interp(zq, z0 + bin_dz * np.arange(nb), q) * hq
    tq = (zq - z0) / W.C0
    eps = W.EPS_R_ICE * EPS0
    errs = []
    for p in range(len(probes)):
        i, j, k = nodes[p]
        obs = np.array([(i - N // 2) * dx, (j - N // 2) * dx, k * dx])
        Ec = moving_charge_field(obs, zq, qq, tq, ts, eps, sigma)
        rr = math.hypot(obs[0], obs[1])
        er_c = (obs[0] * Ec[:, 0] + obs[1] * Ec[:, 1]) / rr
        ez_f = gauss_filter_trace(tr[p, :, 0], dt, sigma, ts, t0=dt)
        er_f = gauss_filter_trace(tr[p, :, 1], dt, sigma, ts, t0=dt)
        errs.append((np.linalg.norm(ez_f - Ec[:, 2]) / np.linalg.norm(Ec[:, 2]),
                     np.linalg.norm(er_f - er_c) / np.linalg.norm(er_c)))
    return np.array(errs)


def test_green_function_superposition_dx2cm():
    e = _green_case(80, 10, 0.02, 300, 12)
    assert e.max() < 0.05
    assert e.mean() < 0.025


def test_green_function_error_is_second_order():
    """Same physical box, filter and detectors at dx = 2 cm and 1 cm."""
    e1 = _green_case(80, 10, 0.02, 300, 12)
    e2 = _green_case(160, 20, 0.01, 600, 24)
    ratio = e1.mean() / e2.mean()
    assert 3.0 < ratio < 5.5, ratio
    assert e2.max() < 0.015


def test_cherenkov_angle():
    NX, NZ, P, dx, steps = 72, 170, 10, 0.02, 320
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    o = oracle.Oracle(NX, NX, NZ, dx, dt, W.EPS_R_ICE, oracle.CPML, P)
    z0 = (P + 4) * dx
    bin_dz = dx / 4
    nb = int(((NZ - P) * dx - z0) / bin_dz) + 1
    zt = z0 + bin_dz * np.arange(nb)
    q = -1e-9 * np.clip((zt - z0) / 0.2, 0, 1)   # 20 cm ramp, then uniform charge
    o.set_shower(q, z0, bin_dz, W.C0, oracle.lateral_gaussian(1, 0.7), 1)
    ax = (NX // 2) * dx
    zp = 130 * dx
    rhos = np.arange(4, 24, 2) * dx
    o.set_probes(np.array([(ax + r, ax, zp) for r in rhos]), steps)
    o.step(steps)
    tr = o.probes()[:, :, 0]
    sigma = 8 * dt
    ts = np.arange(0, steps * dt, dt / 8)
    arrival = np.array([ts[np.argmax(np.abs(gauss_filter_trace(tr[p], dt, sigma, ts, t0=dt)))]
                        for p in range(len(rhos))])
    slope, icpt = np.polyfit(rhos, arrival, 1)
    theta = math.degrees(math.atan(slope * W.C0))
    theta_c = math.degrees(math.acos(1.0 / math.sqrt(W.EPS_R_ICE)))
    assert abs(theta_c - 55.83) < 0.01
    assert abs(theta - theta_c) < 1.0, theta
    # the front is a cone: arrival times are linear in rho
    assert np.abs(arrival - (slope * rhos + icpt)).max() < 1.5 * dt
