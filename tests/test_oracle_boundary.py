"""Pins of the oracle's absorbing boundaries (the paper is silent on them; the
readings are first-order Mur and a Roden-Gedney CPML).

A small box with the boundary under test is compared with a large PEC box
holding the same source and detectors, over a window in which no reflection
from the large box's walls can arrive.  The difference is what the boundary
reflects: large for PEC (the check is sensitive), about 1-2 % for first-order
Mur, about 1e-3 for an 8-cell CPML.  The CPML coefficients obey their closed
forms at the interface and the outer wall, and a CPML box stays stable over
thousands of steps.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _box(n, bc, P, off, dx=0.02):
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    o = oracle.Oracle(n, n, n, dx, dt, W.EPS_R_ICE, bc, P)
    z0 = (off + 12) * dx
    bin_dz = dx / 4
    q = oracle.profile_gaussian(z0, bin_dz, 97, z0 + 0.14, 0.04, -1e-9)
    o.set_shower(q, z0, bin_dz, W.C0, oracle.lateral_gaussian(1, 0.8), 1)
    return o


@pytest.fixture(scope="module")
def reflections():
    ns, P, M, steps, dx = 40, 8, 44, 140, 0.02
    pn = np.array([(20, 20, 3 + P), (20, 20, ns - 3 - P), (3 + P, 20, 20), (ns - 3 - P, 15, 25),
                   (20, 3 + P, 12), (12, 27, 30), (28, 12, 9)], float)
    big = _box(ns + 2 * M, oracle.PEC, 0, M)
    big.set_probes((pn + M) * dx, steps)
    big.step(steps)
    tb = big.probes()
    out = {}
    for name, bc, p in (("pec", oracle.PEC, 0), ("mur", oracle.MUR1, 0), ("cpml", oracle.CPML, P)):
        s = _box(ns, bc, p, 0)
        s.set_probes(pn * dx, steps)
        s.step(steps)
        out[name] = np.abs(s.probes() - tb).max() / np.abs(tb).max()
    return out


def test_pec_box_reflects(reflections):
    assert reflections["pec"] > 0.1


def test_mur_absorbs(reflections):
    assert reflections["mur"] < 0.04
    assert reflections["mur"] < 0.2 * reflections["pec"]


def test_cpml_absorbs(reflections):
    assert reflections["cpml"] < 3e-3
    assert reflections["cpml"] < 0.1 * reflections["mur"]


def test_cpml_coefficients_closed_form():
    n, P, dx = 40, 10, 0.02
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    o = oracle.Oracle(n, n, n, dx, dt, W.EPS_R_ICE, oracle.CPML, P)
    aE, bE, aH, bH = o.cpml_coefs(0)
    eps = o.eps
    alpha_max = 2 * math.pi * 50e6 * eps
    eta = oracle.mu0() * oracle.c0() / math.sqrt(W.EPS_R_ICE)
    smax = -4.0 * math.log(1e-6) / (2 * eta * P * dx)
    # interface (depth 0): sigma = 0, alpha = alpha_max
    for i in (P, n - P):
        assert aE[i] == 0.0
        assert bE[i] == pytest.approx(math.exp(-alpha_max * dt / eps), rel=1e-14)
    # first E-type node next to the outer wall, depth P-1
    d = P - 1
    s = smax * (d / P) ** 3
    al = alpha_max * (1 - d / P)
    b = math.exp(-(s + al) * dt / eps)
    for i in (1, n - 1):
        assert bE[i] == pytest.approx(b, rel=1e-14)
        assert aE[i] == pytest.approx(s * (b - 1) / (s + al), rel=1e-13)
    # H-type half-integer depths are symmetric about the domain centre
    assert np.allclose(bH[:P], bH[n - P:n][::-1], rtol=1e-15)
    assert np.all(aE[P + 1:n - P] == 0.0) and np.all(aH[P:n - P] == 0.0)
    # the cubic conductivity dominates deep in the layer: loss grows towards the wall
    assert np.all(np.diff(bE[1:P - 1]) > 0)


def test_cpml_long_run_stable():
    s = _box(36, oracle.CPML, 8, 0)
    energies = []
    for _ in range(12):
        s.step(250)
        energies.append(sum((s.field(c) ** 2).sum() for c in range(3)))
    e = np.array(energies)
    # after the transient only the static field of the charge left behind remains
    assert np.abs(e[4:] / e[4] - 1.0).max() < 1e-3
