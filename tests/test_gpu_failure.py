"""Failure detection on the stepping path, made to happen without a GPU fault.

* The watchdog (fdtd_set_watchdog): a non-finite value planted on the host
  with fdtd_set_field spreads through the grid and is reported as
  FDTD_ERR_UNSTABLE by the next synchronising call; the status is sticky until
  fdtd_reset; with the watchdog off nothing is reported.
* The bounded waits of the batched persistent kernel (an item waiting for the
  items of its simulation it depends on, the grid barrier that ends a
  launch): with a wait limit of one clock cycle a wait gives up while the
  other blocks still work; the kernel returns, and the batch and every
  simulation that shared the kernel report FDTD_ERR_TIMEOUT.  The context
  stays usable.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

UNSTABLE, TIMEOUT = -4, -6


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _plant(sim, comp, ijk):
    f = sim.field(comp)
    i, j, k = ijk
    f[k, j, i] = np.nan
    sim.set_field(comp, f)


@pytest.mark.parametrize("kernel", [None, 1, 0])
@pytest.mark.parametrize("boundary", ["cpml", "mur"])
def test_watchdog_reports_planted_nan(fd, boundary, kernel):
    if boundary == "cpml":
        w = W.greisen_small(nx=64, ny=60, nz=96, steps=200, n_probes=2)
    else:
        w = W.parity96(n=40, steps=200, n_probes=2)
    sim = fd.Simulation.from_workload(w, kernel=kernel)
    fd.check(fd.fdtd_set_watchdog(sim.h, 16), "fdtd_set_watchdog")
    sim.step(20)
    sim.sync()
    # between two sampled planes (every eighth), away from the detectors
    _plant(sim, 2, (w.nx // 2 + 3, w.ny // 2 - 2, (w.nz // 16) * 8 + 4))
    sim.step(12)     # steps 21..32: the check after step 32 sees it
    with pytest.raises(fd.FdtdError) as ex:
        sim.sync()
    assert ex.value.code == UNSTABLE
    # sticky: stepping and reading are refused
    assert fd.fdtd_step(sim.h, 1) == UNSTABLE
    with pytest.raises(fd.FdtdError):
        sim.probes()
    # a reset clears it: the same handle runs clean again
    sim.reset()
    sim.step(40)
    sim.sync()
    assert all(np.isfinite(sim.field(c)).all() for c in range(6))
    sim.close()


def test_watchdog_off_and_default_interval(fd):
    w = W.parity96(n=32, steps=200, n_probes=2)
    sim = fd.Simulation.from_workload(w)
    assert fd.fdtd_set_watchdog(sim.h, -1) == -1
    fd.check(fd.fdtd_set_watchdog(sim.h, 0), "fdtd_set_watchdog")
    _plant(sim, 3, (10, 11, 12))
    sim.step(70)
    sim.sync()          # off: nothing reported
    assert not np.isfinite(sim.field(2)).all()
    sim.close()
    # the default interval (64 steps) after fdtd_create
    sim = fd.Simulation.from_workload(w)
    _plant(sim, 3, (10, 11, 12))
    sim.step(63)
    sim.sync()          # no check yet
    sim.step(1)
    with pytest.raises(fd.FdtdError) as ex:
        sim.sync()
    assert ex.value.code == UNSTABLE
    sim.close()


def test_batch_barrier_wait_runs_out(fd):
    import torch
    dx = 0.02
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    sims = [fd.Simulation(n, n, 2 * n, dx, dt, W.EPS_R_ICE, boundary=fd.FDTD_PEC) for n in (24, 32, 40)]
    b = fd.Batch(sims)
    assert fd.fdtd_batch_set_wait_limit(b.h, -1) == -1
    b.set_wait_limit(1)           # one clock cycle: a wait gives up at once
    b.step(3)
    with pytest.raises(fd.FdtdError) as ex:
        b.sync()
    assert ex.value.code == TIMEOUT
    for s in sims:                # every simulation of the persistent kernel
        assert fd.fdtd_sync(s.h) == TIMEOUT
        assert fd.fdtd_step(s.h, 1) == TIMEOUT
    assert fd.fdtd_batch_step(b.h, 1) == TIMEOUT
    b.close()
    for s in sims:
        s.close()
    # the context is still usable
    s = fd.Simulation(24, 24, 24, dx, dt, W.EPS_R_ICE, boundary=fd.FDTD_PEC)
    f = np.zeros((25, 25, 25), np.float32)
    f[12, 12, 12] = 1.0
    s.set_field(2, f)
    s.step(5)
    s.sync()
    assert np.isfinite(s.field(2)).all() and np.abs(s.field(3)).max() > 0
    s.close()
    torch.cuda.synchronize()
