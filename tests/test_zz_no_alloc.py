"""fdtd_energy_noalloc: the energy check of caller-owned device field arrays
with the library's fixed scratch area, against fdtd_energy of a handle.

Collected last on purpose: it must pass on a fresh process and after every
other GPU test (the scratch area is shared and never cleared between calls).
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _export(fd, sim, w):
    """The six components of the handle, node layout, into one device buffer."""
    import torch
    nodes = (w.nx + 1) * (w.ny + 1) * (w.nz + 1)
    buf = torch.zeros(6 * nodes, dtype=torch.float32, device="cuda")
    for c in range(6):
        fd.check(fd.fdtd_fields(sim.h, c, C.c_void_p(buf.data_ptr() + 4 * c * nodes), 1), "fdtd_fields")
    torch.cuda.synchronize()
    return buf


def _noalloc(fd, buf, w, nblocks=0, stream=None):
    e = C.c_double(-1.0)
    rc = fd.fdtd_energy_noalloc(C.c_void_p(buf.data_ptr()), w.nx, w.ny, w.nz, w.dx, w.eps_r, nblocks,
                                stream, C.byref(e))
    return rc, e.value


def test_noalloc_energy_matches_handle_energy(fd):
    import torch
    w = W.greisen_small(nx=64, ny=60, nz=80, steps=120, n_probes=4)
    sim = fd.Simulation.from_workload(w)
    sim.step(w.steps)
    ref = sim.energy()
    assert ref > 0.0
    buf = _export(fd, sim, w)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row: the second reuses the scratch the first left behind
    for _ in range(2):
        rc, e = _noalloc(fd, buf, w, 0, stream)
        assert rc == fd.FDTD_OK
        assert abs(e - ref) <= 1e-12 * ref, (e, ref)
    # an explicit number of partial sums, and the largest allowed
    for nb in (7, 1024):
        rc, e = _noalloc(fd, buf, w, nb, stream)
        assert rc == fd.FDTD_OK
        assert abs(e - ref) <= 1e-12 * ref, (nb, e, ref)
    sim.close()


def test_noalloc_energy_errors(fd):
    import torch
    w = W.parity96(n=24, steps=10, n_probes=2)
    sim = fd.Simulation.from_workload(w)
    sim.step(w.steps)
    buf = _export(fd, sim, w)
    # beyond the scratch area
    rc, _ = _noalloc(fd, buf, w, 1025)
    assert rc == -7   # FDTD_ERR_CAPACITY
    rc, _ = _noalloc(fd, buf, w, -1)
    assert rc == -1   # FDTD_ERR_ARG
    e = C.c_double()
    assert fd.fdtd_energy_noalloc(None, w.nx, w.ny, w.nz, w.dx, w.eps_r, 0, None, C.byref(e)) == -1
    # a non-finite value is reported, the energy still written
    nodes = (w.nx + 1) * (w.ny + 1) * (w.nz + 1)
    buf[2 * nodes + 5] = float("nan")
    torch.cuda.synchronize()
    rc, e = _noalloc(fd, buf, w)
    assert rc == -4   # FDTD_ERR_UNSTABLE
    assert not np.isfinite(e) or e >= 0.0
    sim.close()
