"""The batched and adjoint workload at its full size, in the configurations
bench.py times:

* batch: 64 showers on 64^3 .. 256 x 256 x 512 (dx = 2 cm, Mur).  With the solo
  threshold at the median grid, the two smallest grids (persistent kernel,
  the one-pass tile body) and the two largest (stepping alone, their default
  path, on the solo streams) equal their handles stepped by themselves, bit
  for bit; with no threshold the whole batch (one persistent kernel) equals
  path 1 stepped handle by handle on a sample of grids;
* adjoint: the gradient of a quadratic detector misfit with respect to the
  256-bin charge table on the 256 x 256 x 512 PEC grid over 2000 steps,
  against central differences of the GPU forward at h = 1e-3 of the table's
  largest entry (exact for a quadratic loss up to float32 rounding), for the
  three largest components, to 2 %.
"""
import numpy as np
import pytest

import bench

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def test_batch_full_size(fd):
    steps = 24
    dims, make = bench.batch_workload(fd, "config4", 0, steps)
    sims = [make(d, 7000 + i) for i, d in enumerate(dims)]
    cells = np.array([a * b * c for a, b, c in dims])
    thr = int(np.median(cells))
    b = fd.Batch(sims)
    b.set_config(64, 8)
    b.set_solo(thr)
    assert 0 < b.solo["n_solo"] < len(sims)
    b.step(10)
    b.step(14)
    b.sync()
    order = np.argsort(cells)
    for i in (order[0], order[1], order[-2], order[-1]):
        r = make(dims[i], 7000 + int(i))
        if cells[i] < thr:
            r.set_kernel(1)
        r.step(steps)
        for c in range(6):
            assert np.array_equal(sims[i].field(c), r.field(c)), (dims[i], c)
        assert np.array_equal(sims[i].probes(), r.probes())
        assert sims[i].steps_done == steps
        r.close()
    b.close()
    for s in sims:
        s.close()


def test_batch_full_size_persistent(fd):
    """Every grid in the persistent kernel (no solo threshold): the smallest
    and largest grids equal path 1 on their own handles, bit for bit."""
    steps = 17
    dims, make = bench.batch_workload(fd, "config4", 0, steps)
    sims = [make(d, 7100 + i) for i, d in enumerate(dims)]
    cells = np.array([a * b * c for a, b, c in dims])
    b = fd.Batch(sims)
    b.set_config(48, 8)
    assert b.solo["n_solo"] == 0
    b.step(9)
    b.step(8)
    b.sync()
    order = np.argsort(cells)
    for i in (order[0], order[1], order[-2], order[-1]):
        r = make(dims[i], 7100 + int(i))
        r.set_kernel(1)
        r.step(steps)
        for c in range(6):
            assert np.array_equal(sims[i].field(c), r.field(c)), (dims[i], c)
        assert np.array_equal(sims[i].probes(), r.probes())
        r.close()
    b.close()
    for s in sims:
        s.close()


def test_adjoint_full_size_central_differences(fd):
    import torch
    from paper_1001_5341_gb300.adjoint import TraceModel
    steps = 2000
    sim, model, q = bench.adjoint_problem(fd, TraceModel, 0, steps)
    with torch.no_grad():
        target = model(torch.tensor(q * 0.9)).double()
    qg = torch.tensor(q, requires_grad=True)
    loss = 0.5 * ((model(qg).double() - target) ** 2).sum()
    loss.backward()
    g = qg.grad.numpy()
    assert np.abs(g).max() > 0

    def L(qq):
        with torch.no_grad():
            return float(0.5 * ((model(torch.tensor(qq)).double() - target) ** 2).sum())

    h = 1e-3 * np.abs(q).max()
    for b in np.argsort(-np.abs(g))[:3]:
        e = np.zeros_like(q)
        e[b] = h
        fdg = (L(q + e) - L(q - e)) / (2 * h)
        assert abs(fdg - g[b]) <= 2e-2 * abs(g[b]), (int(b), fdg, g[b])
    sim.close()
