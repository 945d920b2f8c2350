"""Parity at the benchmarked step counts.

The two benchmarked 3D workloads run 4000 steps (384 x 384 x 1536, dx = 2 cm,
10-cell CPML, Greisen shower) and 6000 steps (640 x 640 x 2048, dx = 3 cm,
12-cell CPML, Gaisser-Hillas subshowers over 40 m).  The oracle cannot follow
the full cross-sections for that long, so these tests keep everything about
the physics -- dx, dt, CPML depth, profile family and its seed, NKG lateral
spread, the whole length of the grid and the whole step count -- and shrink
only the cross-section:

* 128 x 128 x 1536 cells, dx = 2 cm, CPML 10, Greisen shower (seed 2002),
  4000 steps, 64 detectors at r in [0.8, 1.0] m along the whole shower;
* 112 x 112 x 2048 cells, dx = 3 cm, CPML 12, the seed-3003 Gaisser-Hillas
  subshowers over their full 40 m, 6000 steps, 64 detectors at r in
  [0.8, 1.2] m.

The GPU runs the selected field-update path (the benchmark's default, and the
two-step temporal-blocking path) through the C ABI; the FP64 oracle runs the
same workload.  Compared (Sec. III.A, III.B; relative L2, the parity metric):
every detector trace at 1/8, 1/4, 1/2 and all of the run (overall and per
detector), and all six field components at N/2 and N (each normalised by its
vector field, as in the other parity tests).  The growth of the error with the
step count is printed (pytest -s) for the design notes.
"""
import math
import time

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _greisen_long():
    return W.greisen384(nx=128, ny=128, nz=1536, steps=4000, n_probes=64, r_lo=0.8, r_hi=1.0)


def _gh_long():
    return W.gh640(nx=112, ny=112, nz=2048, steps=6000, n_probes=64, r_lo=0.8, r_hi=1.2)


def _fields_err(sim, ref, torch, w):
    got, want = [], []
    dev = torch.empty((w.nz + 1, w.ny + 1, w.nx + 1), dtype=torch.float32, device="cuda")
    for c in range(6):
        sim.field(c, out=dev)
        got.append(dev.cpu().numpy().astype(np.float64).ravel())
        want.append(ref.field(c).ravel())
    errs = {}
    for base in (0, 3):
        nrm = math.sqrt(sum(np.dot(want[c], want[c]) for c in range(base, base + 3)))
        assert nrm > 0
        for c in range(base, base + 3):
            errs[oracle.COMPONENTS[c]] = float(np.linalg.norm(got[c] - want[c]) / nrm)
    return errs


_RUNS = {}


def _run(make, kernel):
    """GPU and oracle runs of a workload, with snapshots at N/2 and N; the
    oracle run is shared by the kernels."""
    import torch
    import paper_1001_5341_gb300 as fd
    torch.cuda.set_device(0)
    w = make()
    key = w.name
    if key not in _RUNS:
        ref = oracle.from_workload(w)
        t0 = time.time()
        ref.step(w.steps // 2)
        half = {c: ref.field(c) for c in range(6)}
        ref.step(w.steps - w.steps // 2)
        _RUNS[key] = (ref, half, time.time() - t0)
    ref, half, t_ref = _RUNS[key]

    class _Half:   # the oracle's snapshot at N/2, read like the live oracle
        def field(self, c):
            return half[c]

    sim = fd.Simulation.from_workload(w, kernel=kernel)
    sim.step(w.steps // 2)
    e_half = _fields_err(sim, _Half(), torch, w)
    sim.step(w.steps - w.steps // 2)
    e_end = _fields_err(sim, ref, torch, w)
    tg = sim.probes().astype(np.float64)
    name = sim.kernel_name
    sim.close()
    torch.cuda.empty_cache()
    return w, tg, ref.probes(), e_half, e_end, name, t_ref


@pytest.mark.parametrize("kernel", [None, 1], ids=["default", "onestep"])
@pytest.mark.parametrize("make", [_greisen_long, _gh_long], ids=["greisen128x128x1536", "gh112x112x2048"])
def test_parity_at_benchmarked_step_count(make, kernel):
    w, tg, to, e_half, e_end, name, t_ref = _run(make, kernel)
    n = w.steps
    assert np.abs(to).max() > 0
    # every detector has seen the shower's field by the end of the run
    assert np.all(np.abs(to).max(axis=(1, 2)) > 0)
    growth = []
    for m in (n // 8, n // 4, n // 2, n):
        ref_norm = np.linalg.norm(to[:, :m])
        if ref_norm > 0:   # the shower's field may not have reached any detector yet
            growth.append((m, float(np.linalg.norm(tg[:, :m] - to[:, :m]) / ref_norm)))
    per = np.linalg.norm(tg - to, axis=(1, 2)) / np.linalg.norm(to, axis=(1, 2))
    print(f"\n{w.name} kernel={name} oracle {t_ref:.0f} s; trace relL2 by steps "
          + ", ".join(f"{m}: {e:.2e}" for m, e in growth)
          + f"; worst detector {per.max():.2e}; fields N/2 max {max(e_half.values()):.2e}, "
          f"N max {max(e_end.values()):.2e}")
    for m, e in growth:
        assert e <= TOL, (m, e)
    assert per.max() <= TOL, per.max()
    for c, e in e_half.items():
        assert e <= TOL, ("N/2", c, e)
    for c, e in e_end.items():
        assert e <= TOL, ("N", c, e)
