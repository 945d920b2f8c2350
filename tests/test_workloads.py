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


GPU_TEST_SHAPES = [
    # workloads built by tests/test_gpu_*.py and smoke(); each must be a valid
    # simulation (the oracle rejects footprints or detectors outside the interior)
    lambda: W.greisen_small(nx=64, ny=60, nz=80, steps=120, n_probes=4),
    lambda: W.greisen_small(nx=72, ny=70, nz=140, steps=160, n_probes=6),
    lambda: W.parity96(n=24, steps=10, n_probes=2),
    lambda: W.parity96(n=24, steps=30, n_probes=3),
    lambda: W.parity96(n=32, steps=60, n_probes=2),
    lambda: W.parity96(n=32, steps=20, n_probes=2),
    lambda: W.parity96(n=40, steps=120, n_probes=4),
    W.greisen_small, W.gh_small, W.parity96,
]


@pytest.mark.parametrize("make", GPU_TEST_SHAPES)
def test_gpu_test_shapes_are_valid(make):
    import oracle
    w = make()
    oracle.from_workload(w)   # raises on an invalid footprint or detector


def test_fullsize_test_workload_is_valid():
    w = W.greisen384(steps=120)
    ax = (w.nx // 2) * w.dx
    lo = w.npml + 1
    near = np.array([[ax + 0.24, ax, 0.46], [ax, ax - 0.32, 0.62], [ax + 0.2, ax + 0.2, 0.90],
                     [ax - 0.5, ax + 0.1, 0.70]])
    ijk = np.floor(near / w.dx + 0.5).astype(int)
    assert ijk.min() >= lo and ijk[:, 0].max() <= w.nx - lo
