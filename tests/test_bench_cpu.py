"""bench.py host logic that needs no GPU: the oracle samples of the reference
arm and of the CPU baseline are valid workloads at every size the bench asks
for (the lateral footprint stays clear of the CPML)."""
import pytest

import bench
import oracle
import workloads as W


@pytest.mark.parametrize("workload", ["greisen384", "gh640"])
@pytest.mark.parametrize("target", [5e4, 2e5, 1e6])
def test_oracle_sample_accepts_the_shower(workload, target):
    w = bench.replica_workload(0, workload)
    sw = bench._oracle_sample(w, target)
    L = sw.lateral["L"]
    assert min(sw.nx, sw.ny) // 2 - L >= sw.npml + 1
    o = oracle.from_workload(sw, max_steps=2)
    o.step(2)
    assert o.probes().shape == (sw.probes_xyz.shape[0], 2, 2)


def test_traffic_record_lookup(tmp_path, monkeypatch):
    """Records are found by '<kernel>@<workload>' or by the kernel's name, only
    for their own workload and while the listed sources are unchanged."""
    import json
    h = bench.kernel_source_hash(["cyl.cu"])
    recs = {"k@w1": {"workload": "w1", "sources": ["cyl.cu"], "source_hash": h, "dram_bytes_per_cell": 1.0},
            "k": {"workload": "w2", "sources": ["cyl.cu"], "source_hash": h, "dram_bytes_per_cell": 2.0},
            "old": {"workload": "w1", "sources": ["cyl.cu"], "source_hash": "0", "dram_bytes_per_cell": 3.0}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(recs))
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    assert bench.ncu_traffic("k", "w1") == 1.0
    assert bench.ncu_traffic("k", "w2") == 2.0
    assert bench.ncu_traffic("k", "w3") is None
    assert bench.ncu_traffic("old", "w1") is None


@pytest.mark.parametrize("workload", ["greisen384", "gh640"])
def test_oracle_sample_never_exceeds_the_workload(workload):
    """A fast host asks for more cells per step than the grid has: the sample
    is then the workload's own grid, not a larger one."""
    w = bench.replica_workload(0, workload)
    sw = bench._oracle_sample(w, 1e12)
    assert (sw.nx, sw.ny, sw.nz) == (w.nx, w.ny, w.nz)
