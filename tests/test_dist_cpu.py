"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): the
slowest rank sets the time, each replica draws its own shower, and only rank 0
runs the reference arm.  No GPU: the ranks are host processes."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.5], ws)
    w = bench.replica_workload(rank)
    env = bench.dist_env()

    class A:
        steps, warmup, n = 2, 3, 64
    ref = bench.run_cyl_reference(A)   # the reference arm: rank 0 only
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, w.profile["E0_eV"], env, ref is None))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, got0, e0, env0, none0), (r1, got1, e1, env1, none1) = res
    assert got0 == got1 == [2.0, 10.0, 3.5]          # element-wise max over ranks
    assert e0 != e1                                  # replicas draw their own showers
    assert env0 == (2, 0, 0) and env1 == (2, 1, 1)
    assert not none0 and none1                       # reference arm: rank 0 only


def test_one_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([4.0, 2.0], 1) == [4.0, 2.0]
