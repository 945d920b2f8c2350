"""The seeded input generators: deterministic, inside the grid interior, and
every shape the GPU tests use can be built (checked here, without a GPU)."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("make", [W.parity96, W.greisen384, W.gh640, W.greisen_small, W.gh_small])
def test_workloads_deterministic_and_inside(make):
    a, b = make(), make()
    assert np.array_equal(a.probes_xyz, b.probes_xyz) and a.profile == b.profile
    lo = a.npml + 1 if a.boundary == W.CPML else 1
    ijk = np.floor(a.probes_xyz / a.dx + 0.5).astype(int)
    for ax, n in enumerate((a.nx, a.ny, a.nz)):
        assert ijk[:, ax].min() >= lo and ijk[:, ax].max() <= n - lo
    L = a.lateral["L"]
    assert a.nx // 2 - L >= lo and a.nx // 2 + L <= a.nx - lo
    dt_max = a.dx * math.sqrt(a.eps_r) / (W.C0 * math.sqrt(3))
    assert a.dt == pytest.approx(0.5 * dt_max)


def test_benchmark_workload_matches_the_stated_configuration():
    w = W.greisen384()
    assert (w.nx, w.ny, w.nz, w.npml, w.steps) == (384, 384, 1536, 10, 4000)
    assert w.dx == 0.02 and w.eps_r == 3.17 and w.probes_xyz.shape == (64, 3)
    assert 1e16 <= w.profile["E0_eV"] <= 1e18 and w.profile["frac"] == 0.2
    r = np.hypot(w.probes_xyz[:, 0] - 192 * w.dx, w.probes_xyz[:, 1] - 192 * w.dx)
    assert r.min() >= 1.0 and r.max() <= 5.0
    assert w.dt == pytest.approx(34.2885e-12, rel=1e-5)


def test_gpu_test_shapes_build():
    # shapes used by tests/test_gpu_*.py
    W.greisen_small(nx=40, ny=36, nz=90, steps=120, n_probes=4)
    W.parity96(n=24, steps=10, n_probes=2)
    W.parity96(n=32, steps=60, n_probes=2)
    W.parity96(n=40, steps=120, n_probes=4)
    W.greisen384(steps=120)
