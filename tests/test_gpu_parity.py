"""GPU (FP32, sm_103a kernels through the C ABI) against the FP64 oracle on the
same seeded inputs: detector traces and all six field components, relative L2
<= 1e-4 (the spec bar for the whole path), on the 96^3 Mur workload, on
small versions of the two CPML workloads, and on ragged grids that leave
partial tiles in every direction."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


# the field-update paths: 1 = vector-tile z-march (default), 2 = two steps per
# pass (PEC and CPML grids), 0 = unfused sweeps
@pytest.fixture(params=[1, 2, 0], ids=["vtile", "tblock2", "unfused"])
def kernel(request):
    return request.param


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def face_normal_h_mask(nx, ny, nz):
    """Entries of H normal to an outer face on that face: they drive no updated
    E, the library does not maintain them (zero) while the oracle updates them."""
    sh = (nz + 1, ny + 1, nx + 1)
    m = [np.ones(sh, bool) for _ in range(6)]
    m[3][:, :, [0, nx]] = False
    m[4][:, [0, ny], :] = False
    m[5][[0, nz], :, :] = False
    return m


def compare_fields(sim, ref, tol=TOL):
    """Per-component L2 error relative to the norm of its vector field (E or
    H): on an axisymmetric shower Hz and the azimuthal E vanish by symmetry, so
    a component's own norm is round-off and no scale for an error."""
    mask = face_normal_h_mask(sim.nx, sim.ny, sim.nz)
    g = [sim.field(c).astype(np.float64)[mask[c]] for c in range(6)]
    o = [ref.field(c)[mask[c]] for c in range(6)]
    for c in range(6):
        assert np.all(sim.field(c)[~mask[c]] == 0.0), oracle.COMPONENTS[c]
    errs = {}
    for base in (0, 3):
        nrm = math.sqrt(sum(np.dot(o[c], o[c]) for c in range(base, base + 3)))
        assert nrm > 0
        for c in range(base, base + 3):
            errs[oracle.COMPONENTS[c]] = np.linalg.norm(g[c] - o[c]) / nrm
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, errs
    return errs


NAMES = {0: "unfused", 1: "fused-vtile", 2: "tblock2-120"}


def run_pair(fd, w, snaps, kernel=1):
    if kernel == 2 and w.boundary == oracle.MUR1:
        pytest.skip("the two-step path runs PEC and CPML grids")
    sim = fd.Simulation.from_workload(w, kernel=kernel)
    assert sim.kernel_name.startswith(NAMES[kernel])
    ref = oracle.from_workload(w)
    done = 0
    out = []
    for s in snaps:
        sim.step(s - done)
        ref.step(s - done)
        done = s
        out.append(compare_fields(sim, ref))
    tg, to = sim.probes().astype(np.float64), ref.probes()
    e_all = rel_l2(tg, to)
    per = [rel_l2(tg[p], to[p]) for p in range(tg.shape[0]) if np.abs(to[p]).max() > 0]
    assert np.abs(to).max() > 0
    assert e_all <= TOL, (e_all, per)
    return sim, ref, e_all, per, out


def test_parity96_mur_full(fd, kernel):
    w = W.parity96()
    sim, ref, e, per, snaps = run_pair(fd, w, [w.steps // 2, w.steps], kernel)
    assert max(per) <= 3 * TOL
    assert np.array_equal(sim.probe_nodes(), ref.probe_nodes())


def test_greisen_small_cpml(fd, kernel):
    w = W.greisen_small()
    run_pair(fd, w, [150, w.steps], kernel)


def test_gh_small_cpml(fd, kernel):
    w = W.gh_small()
    run_pair(fd, w, [w.steps], kernel)


@pytest.mark.parametrize("fused", [1, 2])
def test_fused_and_unfused_agree(fd, fused):
    """The paths compute the same update; they may differ only by FP32
    rounding (FMA contraction)."""
    w = W.greisen_small(nx=72, ny=70, nz=140, steps=160, n_probes=6)
    a = fd.Simulation.from_workload(w, kernel=fused)
    b = fd.Simulation.from_workload(w, kernel=0)
    a.step(w.steps)
    b.step(w.steps)
    for base in (0, 3):   # each component against its vector field's norm
        fa = [a.field(c).astype(np.float64) for c in range(base, base + 3)]
        fb = [b.field(c).astype(np.float64) for c in range(base, base + 3)]
        nrm = math.sqrt(sum((x * x).sum() for x in fb))
        for x, y in zip(fa, fb):
            assert np.linalg.norm(x - y) / nrm < 1e-5
    assert rel_l2(a.probes(), b.probes()) < 1e-5


def _custom(nx, ny, nz, boundary, npml, v_frac=1.0, L=2, steps=80, seed=0):
    dx = 0.02
    rng = np.random.default_rng(seed)
    z0 = (npml + 2) * dx + 0.3 * dx
    nb = 4 * nz
    lo = npml + 1 if boundary == oracle.CPML else 1
    probes = []
    while len(probes) < 6:
        p = rng.uniform([lo, lo, lo], [nx - lo, ny - lo, nz - lo]) * dx
        probes.append(p)
    wl = rng.uniform(0.2, 1.0, size=(2 * L + 1) ** 2)
    return W.Workload(
        name=f"ragged{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=W.courant_dt(dx, W.EPS_R_ICE),
        eps_r=W.EPS_R_ICE, boundary=boundary, npml=npml, steps=steps,
        profile={"kind": "table", "q": (-1e-9 * rng.uniform(0.3, 1.0, size=nb)).tolist()},
        lateral={"kind": "table", "L": L, "w": (wl / wl.sum()).tolist()},
        z0=z0, bin_dz=dx / 4, n_bins=nb, v=v_frac * W.C0, probes_xyz=np.array(probes))


@pytest.mark.parametrize("dims,boundary,npml,v_frac", [
    ((12, 16, 20), oracle.PEC, 0, 1.0),
    ((13, 17, 23), oracle.MUR1, 0, 0.7),
    ((33, 9, 41), oracle.MUR1, 0, 1.0),
    ((29, 31, 37), oracle.CPML, 5, 1.0),
    ((70, 66, 45), oracle.CPML, 8, 2.2),
    # several 128-column tiles: a tile edge inside the x+ layer, a partial
    # group of four columns at x+
    ((136, 30, 30), oracle.CPML, 10, 1.0),
    ((262, 26, 28), oracle.CPML, 6, 1.0),
    # two-step path: narrow x-layer tiles and one wide tile, 8-row tile
    # rows, many z chunks; a PEC grid with several wide tiles; two narrow
    # tiles at each x layer and a short wide tile; two wide tiles, the
    # second owning 24 columns
    ((124, 40, 200), oracle.CPML, 8, 1.0),
    ((245, 19, 33), oracle.PEC, 0, 1.0),
    ((120, 70, 76), oracle.CPML, 30, 1.0),
    ((175, 24, 40), oracle.CPML, 10, 1.0),
])
def test_ragged_grids(fd, kernel, dims, boundary, npml, v_frac):
    w = _custom(*dims, boundary, npml, v_frac, L=2 if min(dims[:2]) > 2 * npml + 7 else 1)
    run_pair(fd, w, [w.steps // 3, w.steps], kernel)


def test_zero_source_and_no_probes(fd):
    w = W.parity96(n=24, steps=30, n_probes=3)
    sim = fd.Simulation(w.nx, w.ny, w.nz, w.dx, w.dt, w.eps_r, w.boundary)
    sim.set_probes(np.zeros((0, 3)), 0)
    sim.step(0)
    sim.step(w.steps)
    for c in range(6):
        assert np.all(sim.field(c) == 0.0)
    assert sim.steps_done == w.steps


def test_errors_are_reported(fd):
    w = W.parity96(n=24, steps=10, n_probes=2)
    sim = fd.Simulation.from_workload(w)
    sim.step(10)
    with pytest.raises(fd.FdtdError) as e:
        sim.step(1)
    assert e.value.code == -7  # trace capacity
    with pytest.raises(fd.FdtdError) as e:
        sim.set_probes([[0.0, 0.0, 0.0]], 5)
    assert e.value.code == -1
    q, lw = fd.tables(w)
    with pytest.raises(fd.FdtdError):
        sim.set_shower(q, w.z0, w.bin_dz, w.v, lw, w.lateral["L"], axis=0)
    with pytest.raises(fd.FdtdError):
        sim.set_shower(q, w.z0, w.bin_dz, w.v, np.ones(25 * 25) / 625, 12)
    # the handle stays usable after rejected calls
    sim.set_probes(w.probes_xyz, 40)
    sim.step(5)
    sim.sync()


def test_steps_are_deterministic_and_resumable(fd, kernel):
    w = W.greisen_small(nx=64, ny=60, nz=80, steps=120, n_probes=4)
    a = fd.Simulation.from_workload(w, kernel=kernel)
    a.step(w.steps)
    ta = a.probes()
    fa = [a.field(c) for c in range(6)]
    b = fd.Simulation.from_workload(w, kernel=kernel)
    b.step(46)                # the two-step path: an odd number of passes
    b.step(4)
    blob = b.save_state()
    b.step(20)                # diverge, then restore
    c = fd.Simulation.from_workload(w, kernel=kernel)
    c.load_state(blob)
    assert c.steps_done == 50
    c.step(w.steps - 50)
    assert np.array_equal(c.probes(), ta)
    for k in range(6):
        assert np.array_equal(c.field(k), fa[k])
    a.reset()
    assert a.steps_done == 0 and np.all(a.probes() == 0)
    a.step(w.steps)
    assert np.array_equal(a.probes(), ta)


def test_energy_and_instability_flag(fd):
    from physics import EPS0, MU0
    w = W.parity96(n=32, steps=60, n_probes=2)
    sim = fd.Simulation.from_workload(w)
    sim.step(w.steps)
    e = sim.energy()
    E = [sim.field(c).astype(np.float64) for c in range(6)]
    ref = 0.5 * w.eps_r * EPS0 * sum((x * x).sum() for x in E[:3]) + 0.5 * MU0 * sum((x * x).sum() for x in E[3:])
    assert e == pytest.approx(ref * w.dx ** 3, rel=1e-9)
    # a non-finite value planted on the host is reported, not trapped
    bad = E[2].astype(np.float32)
    bad[10, 10, 10] = np.nan
    sim.set_field(2, bad)
    with pytest.raises(fd.FdtdError) as ex:
        sim.energy()
    assert ex.value.code == -4


def test_timing_and_launch_counter(fd):
    w = W.parity96(n=32, steps=20, n_probes=2)
    sim = fd.Simulation.from_workload(w)
    n0 = sim.launches
    sim.timing_begin(100)
    sim.step(w.steps)
    ms, nl = sim.timing_end()
    assert nl >= w.steps and ms > 0.0
    assert sim.launches - n0 >= w.steps
