"""bench.py host logic that needs no GPU: the oracle samples of the reference
arm and of the CPU baseline are valid workloads at every size the bench asks
for (the lateral footprint stays clear of the CPML)."""
import pytest

import bench
import oracle
import workloads as W


@pytest.mark.parametrize("target", [5e4, 2e5, 1e6])
def test_oracle_sample_accepts_the_shower(target):
    w = W.greisen384()
    sw = bench._oracle_sample(w, target)
    L = sw.lateral["L"]
    assert min(sw.nx, sw.ny) // 2 - L >= sw.npml + 1
    o = oracle.from_workload(sw, max_steps=2)
    o.step(2)
    assert o.probes().shape == (sw.probes_xyz.shape[0], 2, 2)
