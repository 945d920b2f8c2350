"""Pins of the 2D axisymmetric oracle (oracle/cyl_oracle.py) against facts it
does not compute itself: the TM_010 frequency of a PEC cylinder from the
first zero of J_0 (scipy), second-order convergence to it, exact
conservation of the discrete energy, the discrete Gauss law under the moving
deposit, linearity and the zero source."""
import math

import numpy as np
import pytest

from oracle import cyl_oracle as O

scipy_special = pytest.importorskip("scipy.special")


def _tm010_period_error(nr):
    R, L = 0.3, 0.2
    d = R / nr
    nz = int(round(L / d))
    o = O.CylOracle(nr, nz, d, O.courant_dt(d, 3.17), 3.17, boundary=O.PEC)
    j01 = scipy_special.jn_zeros(0, 1)[0]
    r = np.arange(nr + 1) * d
    o.Ez[:] = scipy_special.j0(j01 * r / R)[:, None]
    o.Ez[nr, :] = 0.0
    series = []
    for _ in range(int(6 * 2 * math.pi / (j01 / R * O.C0 / math.sqrt(3.17)) / o.dt)):
        o.step()
        series.append(o.Ez[0, nz // 2])
    s = np.array(series)
    # zero crossings -> period (linear interpolation between samples)
    idx = np.where(np.sign(s[:-1]) != np.sign(s[1:]))[0]
    t = (idx + s[idx] / (s[idx] - s[idx + 1])) * o.dt
    period = 2.0 * np.mean(np.diff(t))
    w_num = 2 * math.pi / period
    w_exact = j01 / R * O.C0 / math.sqrt(3.17)
    return abs(w_num - w_exact) / w_exact


def test_tm010_frequency_converges_to_bessel_zero():
    e1 = _tm010_period_error(15)
    e2 = _tm010_period_error(30)
    assert e2 < 2e-3
    assert 2.8 < e1 / e2 < 5.5, (e1, e2)   # second order: ratio ~ 4


def test_energy_is_conserved_in_a_pec_cylinder():
    rng = np.random.default_rng(3)
    nr, nz, d = 24, 20, 0.01
    o = O.CylOracle(nr, nz, d, O.courant_dt(d, 3.17), 3.17, boundary=O.PEC)
    o.Er[:] = rng.normal(size=o.Er.shape)
    o.Ez[:] = rng.normal(size=o.Ez.shape)
    o.Er[:, 0] = o.Er[:, nz] = 0.0
    o.Ez[nr, :] = 0.0
    Vr = 2 * math.pi * (np.arange(nr) + 0.5) * d ** 3
    Vz = O.ring_area(nr, d) * d

    def W(hprev):
        we = 0.5 * o.eps * ((Vr[:, None] * o.Er ** 2).sum() + (Vz[:, None] * o.Ez ** 2).sum())
        return we + 0.5 * O.MU0 * (Vr[:, None] * hprev * o.Hp).sum()

    vals = []
    for n in range(400):
        hprev = o.Hp.copy()
        o.step()
        # W^n pairs E^n with H^{n-1/2} H^{n+1/2}: evaluate before the E update of the next step
        if n > 0:
            vals.append(W_keep)
        E_r, E_z = o.Er.copy(), o.Ez.copy()
        W_keep = None
        # energy at the new E with H^{n+1/2} and the H of the next half step
        o2 = O.CylOracle(nr, nz, d, o.dt, 3.17, boundary=O.PEC)
        o2.Er, o2.Ez, o2.Hp = E_r.copy(), E_z.copy(), o.Hp.copy()
        h_half = o2.Hp.copy()
        o2.Hp -= o.dt / (O.MU0 * d) * ((o2.Er[:, 1:] - o2.Er[:, :-1]) - (o2.Ez[1:, :] - o2.Ez[:-1, :]))
        we = 0.5 * o.eps * ((Vr[:, None] * E_r ** 2).sum() + (Vz[:, None] * E_z ** 2).sum())
        W_keep = we + 0.5 * O.MU0 * (Vr[:, None] * h_half * o2.Hp).sum()
    vals = np.array(vals)
    assert np.abs(vals - vals[0]).max() <= 1e-11 * abs(vals[0])


def test_gauss_law_under_the_moving_deposit():
    nr, nz, d = 20, 80, 0.01
    o = O.CylOracle(nr, nz, d, O.courant_dt(d, 3.17), 3.17, boundary=O.PEC)
    q = -1e-9 * np.exp(-0.5 * ((np.arange(60) - 25) / 6.0) ** 2)
    w = np.array([0.5, 0.3, 0.2])
    o.set_shower(q, 0.1, 0.01, O.C0, w)
    o.step(90)
    div = o.divergence()
    # charge deposited by the moving cloud so far: at the nodes the CIC
    # weights of the current position carry qbar(n-1/2) w_i; what changed of
    # qbar on the way stays where it was created (charge at rest); so
    # eps div E equals the sum of the per-step CIC deposits
    rho = np.zeros((nr, nz + 1))
    A = O.ring_area(nr, d)
    for n in range(90):
        za, zb = 0.1 + O.C0 * n * o.dt, 0.1 + O.C0 * (n + 1) * o.dt
        qb = o._q(0.1 + O.C0 * (n + 0.5) * o.dt)
        for zz, sgn in ((zb, 1.0), (za, -1.0)):
            x = zz / d
            j = math.floor(x)
            f = x - j
            for i in range(3):
                rho[i, j] += sgn * qb * w[i] * (1 - f) / (A[i] * d)
                rho[i, j + 1] += sgn * qb * w[i] * f / (A[i] * d)
    inner = (slice(0, nr - 2), slice(2, nz - 1))
    scale = np.abs(rho).max()
    assert np.abs(div[inner] - rho[inner]).max() <= 1e-9 * scale


def test_zero_source_and_linearity():
    nr, nz, d = 16, 40, 0.01
    dt = O.courant_dt(d, 3.17)
    q = -1e-9 * np.exp(-0.5 * ((np.arange(30) - 10) / 4.0) ** 2)
    outs = []
    for scale in (1.0, 2.5):
        o = O.CylOracle(nr, nz, d, dt, 3.17)
        o.set_shower(scale * q, 0.05, 0.01, O.C0, [0.6, 0.4])
        o.set_probes([[0.05, 0.2], [0.1, 0.25]])
        o.step(60)
        outs.append(o.traces())
    assert np.abs(outs[1] - 2.5 * outs[0]).max() <= 1e-12 * np.abs(outs[1]).max()
    z = O.CylOracle(nr, nz, d, dt, 3.17)
    z.set_probes([[0.05, 0.2]])
    z.step(30)
    assert np.all(z.traces() == 0)


def test_patch_matches_full_grid_inside_its_dependency_cone():
    """A patch (rows i0.., columns j0..) advanced n steps reproduces the full
    grid wherever the cells are more than n + 1 cells from an edge of the patch
    that is not an edge of the full grid (each step reaches one cell)."""
    rng = np.random.default_rng(11)
    nr, nz, d, n = 40, 60, 0.01, 9
    dt = O.courant_dt(d, 3.17)
    q = -1e-12 * np.exp(-0.5 * ((np.arange(40) - 12) / 5.0) ** 2)
    w = np.array([0.3, 0.25, 0.2, 0.15, 0.1])
    for boundary in (O.PEC, O.MUR1):
        full = O.CylOracle(nr, nz, d, dt, 3.17, boundary=boundary)
        full.Er[:] = rng.normal(size=full.Er.shape)
        full.Ez[:] = rng.normal(size=full.Ez.shape)
        full.Hp[:] = rng.normal(size=full.Hp.shape) / 212.0
        E0 = (full.Er.copy(), full.Ez.copy(), full.Hp.copy())
        full.set_shower(q, 0.123, 0.01, O.C0, w)
        full.step(n)
        for i0, j0 in ((0, 0), (3, 17), (18, 25), (14, 0)):
            pr, pz = nr - i0, nz - j0
            p = O.CylOracle(pr, pz, d, dt, 3.17, boundary=boundary, i0=i0)
            p.Er[:] = E0[0][i0:, j0:]
            p.Ez[:] = E0[1][i0:, j0:]
            p.Hp[:] = E0[2][i0:, j0:]
            p.set_shower(q, 0.123 - j0 * d, 0.01, O.C0, w)
            p.step(n)
            lo_i = 0 if i0 == 0 else n + 2
            lo_j = 0 if j0 == 0 else n + 2
            for a, b in ((p.Er, full.Er[i0:, j0:]), (p.Ez, full.Ez[i0:, j0:]), (p.Hp, full.Hp[i0:, j0:])):
                sl = (slice(lo_i, None), slice(lo_j, None))
                scale = np.abs(b).max()
                assert np.abs(a[sl] - b[sl]).max() <= 1e-12 * scale, (boundary, i0, j0)
            # the cone is tight: one cell closer to the cut, the patch differs
            if i0 > 0:
                assert np.abs(p.Ez[n - 1] - full.Ez[i0 + n - 1, j0:]).max() > 1e-9 * np.abs(full.Ez).max()


def test_ring_weights_integrate_the_radial_gaussian():
    """The ring weights of the paper's radial Gaussian (Sec. III.B) against a
    numerical quadrature of 2 pi r rho(r) over each ring, rho the
    normalised 2D Gaussian density; and the library's generator agrees."""
    integrate = pytest.importorskip("scipy.integrate")
    d, sigma = 0.005, 0.05
    n = 31
    w = O.ring_weights_gaussian(n, d, sigma)
    rho = lambda r: math.exp(-0.5 * (r / sigma) ** 2) / (2.0 * math.pi * sigma ** 2)
    edges = [0.0] + [(i + 0.5) * d for i in range(n)]
    ref = np.array([integrate.quad(lambda r: 2.0 * math.pi * r * rho(r), a, b, epsabs=0, epsrel=1e-13)[0]
                    for a, b in zip(edges[:-1], edges[1:])])
    assert abs(ref.sum() - (1.0 - math.exp(-0.5 * (edges[-1] / sigma) ** 2))) < 1e-12
    np.testing.assert_allclose(w, ref / ref.sum(), rtol=1e-11, atol=0)
    assert abs(w.sum() - 1.0) < 1e-14
    # one ring: all the charge on the axis disc
    assert np.array_equal(O.ring_weights_gaussian(1, d, sigma), [1.0])


def test_library_and_oracle_build_the_same_2d_tables():
    import workloads as W
    try:
        import paper_1001_5341_gb300 as fd
    except ImportError:
        pytest.skip("library not built")
    for n in (256, 8192):
        w = W.cyl_table1(n)
        q_lib, w_lib = fd.cyl_tables(w)
        q_orc, w_orc = O.tables(w)
        np.testing.assert_allclose(q_lib, q_orc, rtol=1e-13, atol=0)
        np.testing.assert_allclose(w_lib, w_orc, rtol=1e-12, atol=0)
        assert abs(q_orc).max() == pytest.approx(abs(w.shower["q_max"]), rel=1e-3)
