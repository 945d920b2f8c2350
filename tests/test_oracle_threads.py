"""The oracle's OpenMP loops run over independent cells with no reductions,
so its results do not depend on the thread count: one thread and all threads
give the same fields and traces, bit for bit (CPML and Mur grids, with a
shower and detectors)."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("make", [lambda: W.greisen_small(steps=30), lambda: W.parity96(n=32, steps=30, n_probes=4)])
def test_results_independent_of_thread_count(make):
    n0 = oracle.set_threads(0)
    out = []
    try:
        for threads in (1, max(2, n0)):
            oracle.set_threads(threads)
            w = make()
            o = oracle.from_workload(w)
            o.step(w.steps)
            out.append(([o.field(c) for c in range(6)], o.probes()))
    finally:
        oracle.set_threads(n0)
    (fa, ta), (fb, tb) = out
    for c in range(6):
        assert np.array_equal(fa[c], fb[c]), oracle.COMPONENTS[c]
    assert np.array_equal(ta, tb)
    assert np.abs(ta).max() > 0
