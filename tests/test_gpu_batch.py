"""GPU batched persistent stepping (batch.h): uneven grids with PEC, Mur and
CPML boundaries, showers and detectors, advanced together, must equal the
same simulations stepped one by one on the one-pass tile path (path 1) bit
for bit (the persistent kernel runs that path's tile body, Mur and readout
code for the PEC and Mur grids; the CPML grids step alone on their handle's
path), and the FP64 oracle within 1e-4; grids that step alone (solo
threshold) equal their handle stepped by itself; the autotuner's trial
steps are real steps; capacity and argument checks."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

DX = 0.02
DT = W.courant_dt(DX, W.EPS_R_ICE)

SPECS = [  # nx, ny, nz, boundary, npml, seed
    (40, 36, 64, 1, 0, 1),
    (24, 24, 24, 0, 0, 2),
    (48, 44, 90, 2, 8, 3),
    (33, 29, 41, 1, 0, 4),
    (64, 64, 128, 1, 0, 5),
    (30, 30, 70, 2, 6, 6),
]


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _setup(nx, ny, nz, boundary, npml, seed):
    rng = np.random.default_rng(seed)
    nb = 40
    z0, bdz = 0.03, 0.03
    zb = z0 + bdz * np.arange(nb)
    q = -1e-9 * np.exp(-0.5 * ((zb - rng.uniform(0.2, 0.6)) / 0.2) ** 2)
    L = 2
    w = np.exp(-0.5 * (np.arange(-L, L + 1)[:, None] ** 2 + np.arange(-L, L + 1)[None, :] ** 2) / 1.2)
    w = (w / w.sum()).ravel()
    m = (npml if boundary == 2 else 0) + 2
    xyz = np.stack([rng.uniform(m, nx - m, 3) * DX, rng.uniform(m, ny - m, 3) * DX, rng.uniform(m, nz - m, 3) * DX], 1)
    return dict(q=q, z0=z0, bdz=bdz, w=w, L=L, xyz=xyz)


def _make(fd, spec, steps, kernel=None):
    nx, ny, nz, b, p, seed = spec
    s = fd.Simulation(nx, ny, nz, DX, DT, W.EPS_R_ICE, boundary=b, npml=p)
    if kernel is not None:
        s.set_kernel(kernel)
    u = _setup(*spec)
    s.set_shower(u["q"], u["z0"], u["bdz"], W.C0, u["w"], u["L"])
    s.set_probes(u["xyz"], steps)
    return s


def _state(s):
    return [s.field(c) for c in range(6)], s.probes()


@pytest.mark.parametrize("cfg", [(64, 8), (5, 5), (256, 64), (1, 3)])
def test_batch_equals_one_by_one(fd, cfg):
    steps = 37
    ref = [_make(fd, sp, steps, kernel=1) for sp in SPECS]
    for s in ref:
        s.step(steps)
    sims = [_make(fd, sp, steps, kernel=1) for sp in SPECS]
    b = fd.Batch(sims)
    b.set_config(*cfg)
    b.step(10)
    b.step(27)
    b.sync()
    assert b.graph_mode in (0, 1)
    for s, r in zip(sims, ref):
        (fa, ta), (fb, tb) = _state(s), _state(r)
        for c in range(6):
            assert np.array_equal(fa[c], fb[c]), c
        assert np.array_equal(ta, tb)
        assert s.steps_done == steps


def test_batch_matches_oracle(fd):
    steps = 60
    spec = SPECS[0]
    sims = [_make(fd, sp, steps) for sp in SPECS[:3]]
    b = fd.Batch(sims)
    b.step(steps)
    b.sync()
    nx, ny, nz, bd, p, seed = spec
    u = _setup(*spec)
    o = oracle.Oracle(nx, ny, nz, DX, DT, W.EPS_R_ICE, boundary=bd, npml=p)
    o.set_shower(u["q"], u["z0"], u["bdz"], W.C0, u["w"], u["L"])
    o.set_probes(u["xyz"], steps)
    o.step(steps)
    # H normal to an outer face, on that face, drives no updated E: the library
    # keeps it at zero, the oracle updates it
    keep = [np.ones((nz + 1, ny + 1, nx + 1), bool) for _ in range(6)]
    keep[3][:, :, [0, nx]] = False
    keep[4][:, [0, ny], :] = False
    keep[5][[0, nz], :, :] = False
    # errors relative to the norm of the vector field (E or H): on an
    # axisymmetric shower Hz vanishes by symmetry
    ref = [o.field(c)[keep[c]] for c in range(6)]
    got = [sims[0].field(c).astype(np.float64)[keep[c]] for c in range(6)]
    for base in (0, 3):
        nrm = np.sqrt(sum(float(np.dot(ref[c], ref[c])) for c in range(base, base + 3)))
        for c in range(base, base + 3):
            assert np.linalg.norm(got[c] - ref[c]) <= 1e-4 * nrm, c
    tr, ref = sims[0].probes().astype(np.float64), o.probes()
    assert np.linalg.norm(tr - ref) <= 1e-4 * np.linalg.norm(ref)


def test_solo_grids_equal_their_own_path(fd):
    """Grids of at least the threshold step with their handle's own kernel on
    the batch's stream; the rest share the persistent kernel."""
    steps = 41
    thr = 150000                          # (48, 44, 90) and (64, 64, 128) step alone,
    big = [sp[0] * sp[1] * sp[2] >= thr or sp[3] == 2 for sp in SPECS]   # as do the CPML grids
    sims = [_make(fd, sp, steps) for sp in SPECS]
    ref = [_make(fd, sp, steps, kernel=None if bg else 1) for sp, bg in zip(SPECS, big)]
    for r in ref:   # in the batch's calls: an odd call ends on one step of path 1 on the two-step path
        r.step(13)
        r.step(28)
    b = fd.Batch(sims)
    b.set_config(32, 5)
    b.set_solo(thr)
    assert b.solo == {"min_cells": thr, "n_solo": 3}
    b.step(13)
    b.step(28)
    b.sync()
    for s, r in zip(sims, ref):
        (fa, ta), (fb, tb) = _state(s), _state(r)
        for c in range(6):
            assert np.array_equal(fa[c], fb[c]), c
        assert np.array_equal(ta, tb)
        assert s.steps_done == steps
    # every grid alone, and back to none
    b.set_solo(1)
    assert b.solo["n_solo"] == len(SPECS)
    b.set_solo(-1)
    assert b.solo["n_solo"] == 2         # the CPML grids
    with pytest.raises(fd.FdtdError):
        b.set_solo(-2)


def test_tuner_steps_are_real_steps(fd):
    steps = 200
    # path 1 on every handle: a grid that the tuner makes step alone then
    # runs the same tile code as inside the persistent kernel
    sims = [_make(fd, sp, steps, kernel=1) for sp in SPECS]
    b = fd.Batch(sims)
    used = b.tune(trial_steps=2)
    assert used > 0 and all(s.steps_done == used for s in sims)
    b.step(steps - used)
    b.sync()
    ref = [_make(fd, sp, steps, kernel=1) for sp in SPECS]
    for r in ref:
        r.step(steps)
    for s, r in zip(sims, ref):
        for c in range(6):
            assert np.array_equal(s.field(c), r.field(c))
    cfg = b.config
    assert cfg["chunk_planes"] in (64, 128, 256, 512) and cfg["steps_per_launch"] == 8
    assert b.solo["min_cells"] >= -1


def test_mixing_batch_and_single_steps(fd):
    steps = 30
    sims = [_make(fd, sp, steps, kernel=1) for sp in SPECS[:4]]
    ref = [_make(fd, sp, steps, kernel=1) for sp in SPECS[:4]]
    b = fd.Batch(sims)
    b.step(7)
    sims[1].set_kernel(1)
    sims[1].step(3)          # one simulation ahead of the others
    b.step(11)
    for r, n in zip(ref, (18, 21, 18, 18)):
        r.step(n)
    for s, r in zip(sims, ref):
        assert s.steps_done == r.steps_done
        for c in range(6):
            assert np.array_equal(s.field(c), r.field(c))


def test_batch_errors(fd):
    sims = [_make(fd, sp, 10) for sp in SPECS[:2]]
    b = fd.Batch(sims)
    with pytest.raises(fd.FdtdError):
        b.step(11)            # trace capacity
    with pytest.raises(fd.FdtdError):
        b.set_config(0, 8)
    with pytest.raises(fd.FdtdError):
        b.set_config(64, 0)
    with pytest.raises(fd.FdtdError):
        b.set_config(64, 65)
    with pytest.raises(fd.FdtdError):
        fd.Batch([sims[0], sims[0]])
    with pytest.raises(fd.FdtdError):
        fd.Batch([])
