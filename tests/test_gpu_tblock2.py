"""The two-step path (fdtd_set_kernel 2, temporal blocking of the leapfrog of
Sec. III.A) against the one-step tile path on the same inputs: every field and
every detector trace, with detectors placed on the seams between tiles (narrow
tiles of 24 columns over the x layers of a CPML grid, wide ones of 120
between), tile rows (every 8 rows) and z chunks, step counts that leave a
single step over, and calls of one step at a time; the FP64 oracle judges
both in tests/test_gpu_parity.py.  The two paths evaluate the same update
expressions, so they agree to FP32 rounding (the compiler may contract them
differently)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _seams(nx, npml):
    """First columns of the two-step path's tiles: narrow tiles of 24 columns
    over [0, a) and [b, nx), wide ones of 120 over [a, b), where a and b are
    multiples of four clear of the x layers by two cells (all narrow when the
    wide part would be shorter than 24 columns; all wide on a PEC grid); the
    columns of a short last wide tile move to the narrow tiles where those
    have room."""
    if npml == 0:
        return list(range(0, nx, 120))
    a, b = (npml + 6) // 4 * 4, (nx - npml - 2) // 4 * 4
    if b - a < 24:
        return list(range(0, nx, 24))
    r = (b - a) % 120   # a short last wide tile goes to room in the narrow tiles
    room_l, room_r = -a % 24, (-(nx - b) % 24) // 4 * 4
    if 0 < r <= room_l + room_r and b - a > 120:
        dl = min(r, room_l)
        a, b = a + dl, b - (r - dl)
    return list(range(0, a, 24)) + list(range(a, b, 120)) + list(range(b, nx, 24))


def _seam_workload(nx, ny, nz, npml, steps, seed=5):
    """A Greisen/NKG shower on a CPML (npml > 0) or PEC grid with detectors on
    the seams of the two-step path's tiles."""
    w = W.greisen384(seed=seed, nx=nx, ny=ny, nz=nz, npml=max(npml, 1), steps=steps, n_probes=4,
                     r_lo=0.1, r_hi=0.2)
    if npml == 0:
        w.boundary, w.npml = W.PEC, 0
        w.z0 = 3 * w.dx
    lo = npml + 1
    pts = []
    cols = sorted({c + d for c in _seams(nx, npml)[1:] for d in (-1, 0, 1)})
    for i in cols:
        for j in (lo + 3, 16, 24, ny - lo - 1):
            if lo <= i <= nx - lo and lo <= j <= ny - lo:
                pts.append((i, j, lo + 2 + (len(pts) * 7) % (nz - 2 * lo - 4)))
    for k in range(lo, nz - lo, 9):   # a column of detectors through every chunk seam nearby
        pts.append((nx // 2 + 5, ny // 2 - 3, k))
    w.probes_xyz = np.array(pts, dtype=np.float64) * w.dx
    return w


def _run(fd, w, kernel, pieces):
    sim = fd.Simulation.from_workload(w, kernel=kernel)
    for n in pieces:
        sim.step(n)
    f = [sim.field(c).astype(np.float64) for c in range(6)]
    t = sim.probes().astype(np.float64)
    name = sim.kernel_name
    sim.close()
    return f, t, name


def _agree(fa, fb, ta, tb, tol=TOL):
    for base in (0, 3):
        nrm = math.sqrt(sum((x * x).sum() for x in fb[base:base + 3]))
        assert nrm > 0
        for c in range(base, base + 3):
            e = np.linalg.norm(fa[c] - fb[c]) / nrm
            assert e <= tol, (oracle.COMPONENTS[c], e)
    assert np.abs(tb).max() > 0
    e = np.linalg.norm(ta - tb) / np.linalg.norm(tb)
    assert e <= tol, e
    per = np.linalg.norm(ta - tb, axis=1) / np.maximum(np.linalg.norm(tb, axis=1), 1e-30)
    live = np.abs(tb).max(axis=(1, 2)) > 0
    assert per[live].max() <= 10 * tol, per[live].max()


@pytest.mark.parametrize("dims,npml", [((250, 60, 180), 10), ((130, 48, 96), 6), ((245, 35, 60), 0)],
                         ids=["cpml10-3tiles", "cpml6-2tiles", "pec-3tiles"])
def test_two_step_path_equals_one_step_path(fd, dims, npml):
    steps = 150
    w = _seam_workload(*dims, npml, steps)
    fa, ta, name = _run(fd, w, 2, [steps])
    assert name.startswith("tblock2")
    fb, tb, _ = _run(fd, w, 1, [steps])
    _agree(fa, fb, ta, tb)


def test_odd_counts_and_single_steps(fd):
    """Calls of odd lengths leave one step to the one-step path; one step at a
    time never uses the two-step kernel.  All give the same fields."""
    steps = 61
    w = _seam_workload(130, 48, 96, 6, steps)
    fa, ta, _ = _run(fd, w, 2, [7, 1, 20, 3, 30])
    fb, tb, _ = _run(fd, w, 1, [steps])
    _agree(fa, fb, ta, tb)
    fc, tc, _ = _run(fd, w, 2, [1] * steps)
    fd_, td, _ = _run(fd, w, 1, [1] * steps)
    for c in range(6):
        assert np.array_equal(fc[c], fd_[c])
    assert np.array_equal(tc, td)


def test_kernel_switch_mid_run(fd):
    steps = 60
    w = _seam_workload(130, 48, 96, 6, steps)
    sim = fd.Simulation.from_workload(w, kernel=2)
    sim.step(22)
    sim.set_kernel(1)
    sim.step(9)
    sim.set_kernel(0)
    sim.step(3)
    sim.set_kernel(2)
    sim.step(26)
    fa = [sim.field(c).astype(np.float64) for c in range(6)]
    ta = sim.probes().astype(np.float64)
    sim.close()
    fb, tb, _ = _run(fd, w, 1, [steps])
    _agree(fa, fb, ta, tb)


def test_mur_grid_and_argument_errors(fd):
    w = W.parity96(n=32, steps=10, n_probes=2)
    sim = fd.Simulation.from_workload(w)
    with pytest.raises(fd.FdtdError) as e:
        sim.set_kernel(2)
    assert e.value.code == -1
    assert sim.kernel_name.startswith("fused-vtile")
    with pytest.raises(fd.FdtdError):
        sim.set_kernel(3)
    sim.close()


def test_detectors_moved_between_calls(fd):
    """The two-step kernel's detector records follow fdtd_set_probes."""
    steps = 40
    w = _seam_workload(130, 48, 96, 6, steps)
    sim = fd.Simulation.from_workload(w, kernel=2)
    sim.step(10)
    ref = fd.Simulation.from_workload(w, kernel=1)
    ref.step(10)
    moved = w.probes_xyz[::-1] + np.array([w.dx, -w.dx, 0.0])
    for s in (sim, ref):
        s.set_probes(moved, 10 + steps)
        s.step(steps)
    a, b = sim.probes().astype(np.float64), ref.probes().astype(np.float64)
    assert np.abs(b).max() > 0
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
    sim.close()
    ref.close()


def test_many_detectors_in_one_tile(fd):
    """Detectors on every node of a row segment inside one tile: more records
    on one plane of one block than the block has threads (5 per detector on
    plane k, 1 on plane k-1), so the record service takes several rounds."""
    steps = 30
    w = _seam_workload(250, 60, 80, 10, steps)
    j, k = 26, 36
    pts = [(i, j, k) for i in range(20, 116)] + [(i, j + 1, k) for i in range(20, 116)]
    w.probes_xyz = np.array(pts, dtype=np.float64) * w.dx
    fa, ta, name = _run(fd, w, 2, [steps])
    assert name.startswith("tblock2")
    fb, tb, _ = _run(fd, w, 1, [steps])
    assert len(pts) * 5 > 352
    _agree(fa, fb, ta, tb)

