"""GPU parity of the 2D axisymmetric solver (cyl.h) with the FP64 oracle
(oracle/cyl_oracle.py): every kernel (two-kernel path and the three
wavefront variants) with PEC and Mur boundaries, random initial fields, a
moving shower and detectors on the axis, the wall, the caps and the segment
and band seams; step counts that leave remainders; degenerate grids; and the
8192 x 8192 benchmark grid in its benchmark launch configuration, checked on
patches the oracle advances inside their dependency cones."""
import numpy as np
import pytest

import workloads as W
from oracle import cyl_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-4   # relative L2 and max-abs / max, FP32 against FP64


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _fields(seed, nr, nz, i0=0, j0=0):
    out = []
    for c, (rows, cols) in enumerate(((nr, nz + 1), (nr + 1, nz), (nr, nz))):
        i = np.arange(i0, i0 + rows, dtype=np.int64)[:, None]
        j = np.arange(j0, j0 + cols, dtype=np.int64)[None, :]
        out.append(W.cyl_field(seed, c, i, j))
    return out


def _close(a, b, tol=TOL, what=""):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    assert nb > 0, what
    rel = np.linalg.norm(a - b) / nb
    mx = np.abs(a - b).max() / np.abs(b).max()
    assert rel <= tol and mx <= 10 * tol, (what, rel, mx)


def _shower(nz, d, q_max=-1e-14):
    n_bins = 60
    q = q_max * np.exp(-0.5 * ((np.arange(n_bins) - 20) / 7.0) ** 2)
    w = np.array([0.35, 0.3, 0.2, 0.1, 0.05])
    return q, 0.37 * d, 0.9 * d, O.C0, w


def _run_pair(fd, nr, nz, steps, kernel, boundary, seg=0, probes=None, seed=5, shower=True, chunks=None):
    d = 0.01
    dt = O.courant_dt(d, 3.17)
    o = O.CylOracle(nr, nz, d, dt, 3.17, boundary=boundary)
    g = fd.Cylinder(nr, nz, d, dt, 3.17, boundary=boundary)
    g.set_kernel(kernel, seg)
    F = _fields(seed, nr, nz)
    o.Er[:], o.Ez[:], o.Hp[:] = F
    for c in range(3):
        g.set_field(c, F[c])
    if shower:
        q, z0, bdz, v, w = _shower(nz, d)
        o.set_shower(q, z0, bdz, v, w)
        g.set_shower(q, z0, bdz, v, w)
    if probes is not None:
        rz = np.asarray(probes, np.float64) * d
        o.set_probes(rz)
        g.set_probes(rz, steps + 3)
    for n in (chunks or [steps]):
        g.step(n)
    o.step(steps)
    g.sync()
    return o, g


def _compare(o, g, steps, what):
    for c, ref in enumerate((o.Er, o.Ez, o.Hp)):
        _close(g.field(c), ref, what=f"{what} comp {c}")
    if len(o.probes):
        tr = g.probes()[:, :steps]
        ref = o.traces()
        _close(tr[..., 0], ref[..., 0], what=f"{what} E_z traces")
        nz_r = np.abs(ref[..., 1]).max() > 0
        if nz_r:
            _close(tr[..., 1], ref[..., 1], what=f"{what} E_r traces")
        assert np.all(tr[o.probes[:, 0] == 0, :, 1] == 0)     # E_r = 0 on the axis


PROBES = [(0, 1), (0, 75), (1, 40), (15, 47), (16, 48), (17, 49), (31, 96), (32, 97), (33, 55),
          (69, 149), (69, 1), (40, 120), (40, 120), (5, 56), (5, 57)]


@pytest.mark.parametrize("boundary", [O.PEC, O.MUR1])
@pytest.mark.parametrize("kernel,seg", [(0, 0), (1, 16), (2, 16), (3, 16), (4, 16), (5, 16), (2, 0), (2, 33),
                                        (4, 0), (3, 35), (1, 14)])   # 71 rows: 35 and 14 leave one row over
def test_kernel_matches_oracle(fd, kernel, seg, boundary):
    o, g = _run_pair(fd, 70, 150, 37, kernel, boundary, seg, PROBES)
    _compare(o, g, 37, f"kernel {kernel} seg {seg} boundary {boundary}")
    info = g.kernel_info
    assert info["kernel"] == kernel and g.steps_done == 37


@pytest.mark.parametrize("kernel", [0, 2])
def test_shower_crosses_the_grid_mur(fd, kernel):
    nr, nz, steps = 64, 300, 640
    d = 0.01
    dt = O.courant_dt(d, 3.17)
    o = O.CylOracle(nr, nz, d, dt, 3.17)
    g = fd.Cylinder(nr, nz, d, dt, 3.17)
    g.set_kernel(kernel)
    q = -1e-12 * np.exp(-0.5 * ((np.arange(200) - 60) / 18.0) ** 2)
    w = [0.5, 0.3, 0.2]
    for s in (o, g):
        s.set_shower(q, 0.2, 0.01, O.C0, w)
    rz = np.array([[r, z] for r in (0.0, 0.1, 0.3, 0.6) for z in (0.5, 1.5, 2.5)])
    o.set_probes(rz)
    g.set_probes(rz, steps)
    g.step(steps)
    o.step(steps)
    _compare(o, g, steps, f"long run kernel {kernel}")


@pytest.mark.parametrize("nr,nz", [(4, 4), (5, 300), (300, 5), (4, 130), (129, 4)])
@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5])
def test_degenerate_grids(fd, nr, nz, kernel):
    probes = [(0, 1), (nr - 1, nz - 1)]
    o, g = _run_pair(fd, nr, nz, 19, kernel, O.MUR1, 0, probes)
    _compare(o, g, 19, f"{nr}x{nz} kernel {kernel}")


def test_step_splitting_and_kernel_switching(fd):
    """1 + 3 + 8 + 9 + 16 steps with switches between kernels equal one call
    of the two-kernel path (same FP32 arithmetic, up to contraction)."""
    a = _run_pair(fd, 70, 150, 37, 0, O.MUR1, 0, PROBES)[1]
    d = 0.01
    b = fd.Cylinder(70, 150, d, O.courant_dt(d, 3.17), 3.17)
    F = _fields(5, 70, 150)
    for c in range(3):
        b.set_field(c, F[c])
    q, z0, bdz, v, w = _shower(150, d)
    b.set_shower(q, z0, bdz, v, w)
    b.set_probes(np.asarray(PROBES, np.float64) * d, 40)
    for kern, n in ((2, 1), (1, 3), (2, 8), (3, 9), (2, 16)):
        b.set_kernel(kern)
        b.step(n)
    b.sync()
    for c in range(3):
        _close(b.field(c), a.field(c), tol=2e-6, what=f"comp {c}")
    _close(b.probes()[:, :37], a.probes()[:, :37], tol=2e-6, what="traces")


def test_reset_and_errors(fd):
    d = 0.01
    g = fd.Cylinder(40, 60, d, O.courant_dt(d, 3.17), 3.17)
    g.set_probes([[0.1, 0.2]], 16)
    g.step(16)
    with pytest.raises(fd.FdtdError):
        g.step(1)                       # trace capacity
    g.reset()
    assert g.steps_done == 0 and np.all(g.probes() == 0)
    with pytest.raises(fd.FdtdError):
        g.set_kernel(7)
    with pytest.raises(ValueError):
        g.set_field(0, np.zeros((3, 3), np.float32))
    with pytest.raises(fd.FdtdError):
        g.set_probes([[0.1, 0.6]], 4)   # z = nz d is not inside
    g.step(8)
    g.sync()
    assert all(np.all(g.field(c) == 0) for c in range(3))


def test_full_size_grid_on_patches(fd):
    """8192 x 8192 (the benchmark grid) in its benchmark launch configuration,
    64 steps from counter-based random fields with the shower of the benchmark
    (its tail deposits about 1 V/m per step near the axis, the order of the
    random fields) and two detectors; the oracle
    advances patches of radius n + 10 around sample cells (axis, wall, caps,
    corners, the source, segment and band seams) and the cores of radius 8
    must agree, as must two detectors' traces."""
    import torch
    n = 64
    wl = W.cyl_table1(8192)
    nr = nz = 8192
    g = fd.Cylinder(nr, nz, wl.d, wl.dt, wl.eps_r, boundary=wl.boundary)
    info = g.kernel_info
    assert info["kernel"] == 3
    for c, (rows, cols) in enumerate(((nr, nz + 1), (nr + 1, nz), (nr, nz))):
        i = torch.arange(rows, dtype=torch.int64, device="cuda")[:, None]
        j = torch.arange(cols, dtype=torch.int64, device="cuda")[None, :]
        g.set_field(c, W.cyl_field(17, c, i, j, xp=torch).contiguous())
        del i, j
    q, rings = fd.cyl_tables(wl)
    qo, rings_o = O.tables(wl)
    g.set_shower(q, wl.z0, wl.bin_dz, wl.v, rings)
    L, U = info["seg_rows"], 128 - 2 * info["steps_per_launch"]
    zs = wl.z0 + wl.v * n * wl.dt
    js = int(zs / wl.d)
    # detectors: one at the source's path, one at a seam
    det = np.array([[3, js - 20], [L, U * 40]], dtype=np.int64)
    g.set_probes(det * wl.d, n)
    g.step(n)
    g.sync()
    full = [g.field(c, out=torch.empty(g.shape(c), dtype=torch.float32, device="cuda")) for c in range(3)]
    tr = g.probes()
    M = n + 10
    centres = [(0, nz // 2), (0, js), (2, js - 20), (nr, 7), (nr, nz - 1), (nr // 2, 0), (nr // 2, nz),
               (L - 1, U * 40), (L, U * 40 + 1), (2 * L + 1, U * 3 - 1), (4000, 4111), (nr - 3, nz // 3)]
    checked = n_det = 0
    for (ci, cj) in centres:
        i0, i1 = max(0, ci - M), min(nr, ci + M)
        j0, j1 = max(0, cj - M), min(nz, cj + M)
        pr, pz = i1 - i0, j1 - j0
        o = O.CylOracle(pr, pz, wl.d, wl.dt, wl.eps_r, boundary=wl.boundary, i0=i0)
        o.Er[:], o.Ez[:], o.Hp[:] = _fields(17, pr, pz, i0, j0)
        o.set_shower(qo, wl.z0 - j0 * wl.d, wl.bin_dz, wl.v, rings_o)
        lo_i = 0 if i0 == 0 else n + 2
        lo_j = 0 if j0 == 0 else n + 2
        hi_i = pr if i1 == nr else pr - n - 2
        hi_j = pz if j1 == nz else pz - n - 2
        # detectors whose cells (and the cells below and left of them) lie in the core
        loc = [(a - i0, b - j0) for a, b in det]
        loc = [(a, b) for a, b in loc if (a >= lo_i + 1 or (i0 == 0 and a >= 0)) and a < min(hi_i, pr)
               and b >= lo_j + 1 and b < min(hi_j, pz)]
        if loc:
            o.set_probes(np.asarray(loc, np.float64) * wl.d)
        o.step(n)
        for c, ref in enumerate((o.Er, o.Ez, o.Hp)):
            rows, cols = ref.shape
            a_i, b_i = lo_i, min(hi_i + 1, rows)
            a_j, b_j = lo_j, min(hi_j + 1, cols)
            got = full[c][i0 + a_i:i0 + b_i, j0 + a_j:j0 + b_j].double().cpu().numpy()
            _close(got, ref[a_i:b_i, a_j:b_j], what=f"centre {(ci, cj)} comp {c}")
            checked += got.size
        for k, (a, b) in enumerate(loc):
            p = [m for m, (x, y) in enumerate(det) if (x - i0, y - j0) == (a, b)][0]
            _close(tr[p, :, 0], o.traces()[k, :, 0], what=f"detector {p} E_z")
            _close(tr[p, :, 1], o.traces()[k, :, 1], what=f"detector {p} E_r")
            n_det += 1
    assert checked > 5000 and n_det >= 2


def test_tune_segment_length(fd):
    """cyl_tune on the 2048 x 2048 grid of Table I: it tries segment lengths
    from 12 rows until the tiles fit one wave of the resident blocks, keeps
    one of them, and its steps are real steps: after them and 32 more, the
    fields and traces agree with an untuned run of the same steps (2e-6: the
    same arithmetic, up to contraction)."""
    w = W.cyl_table1(2048, seed=4004)
    q_tab, ring_w = fd.cyl_tables(w)
    F = _fields(11, w.nr, w.nz)
    runs = []
    for tune in (True, False):
        g = fd.Cylinder(w.nr, w.nz, w.d, w.dt, w.eps_r, w.boundary)
        assert g.kernel_info["kernel"] == 3
        for c in range(3):
            g.set_field(c, F[c])
        g.set_shower(q_tab, w.z0, w.bin_dz, w.v, ring_w)
        g.set_probes(w.probes_rz, 512)
        if tune:
            used = g.tune(2)
            info = g.kernel_info
            assert used % 8 == 0 and used >= 16 and g.steps_done == used
            assert info["seg_rows"] >= 12 and info["seg_rows"] % 4 == 0
        else:
            g.step(used)
        g.step(32)
        g.sync()
        runs.append(([g.field(c) for c in range(3)], g.probes()[:, :used + 32]))
        g.close()
    (fa, ta), (fb, tb) = runs
    for c in range(3):
        _close(fa[c], fb[c], tol=2e-6, what=f"comp {c}")
    _close(ta, tb, tol=2e-6, what="traces")


def test_tune_capacity_and_two_kernel_path(fd):
    d = 0.01
    g = fd.Cylinder(1024, 1024, d, O.courant_dt(d, 3.17), 3.17)
    g.set_kernel(3)
    g.set_probes([[0.1, 0.2]], 7)
    with pytest.raises(fd.FdtdError):
        g.tune(2)                       # the trace has no room for the tuning steps (at least 2 x 4)
    assert g.steps_done == 0
    with pytest.raises(fd.FdtdError):
        g.tune(0)
    g.set_kernel(0)
    assert g.tune(2) == 0 and g.steps_done == 0
