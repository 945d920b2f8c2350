"""The warp synchronisation of the kernels without block barriers in their z
march, modelled on the CPU: the two-step kernel (csrc/kernels_tb2.cu) and
the one-step kernel's form used by k_vtile (csrc/vtile_tile.cuh).

The warps (row warps, the one-step kernel's halo warp, the refill warp) run
the kernel's order of signals and waits over model mbarriers with the
semantics of
`mbarrier.try_wait.parity`: a wait for the completion of phase k passes when
the number of completed phases differs from k in parity, so it is only
right while the barrier is neither behind the waiter nor two phases ahead of
it.  Random and skewed interleavings (some warps far slower than others,
copies landing late) check that
- no interleaving deadlocks;
- every wait passes only after the completion it stands for (no parity alias);
- every read of an exchange row or a stage finds the plane it expects, and
  nothing rewrites it between the wait and the end of the read.
Forms that were rejected are shown to hang: in the two-step kernel, the
wait for the B row above inside C, after the A row was signalled (the warp
above can then finish a whole iteration, and that barrier runs two phases
ahead of the wait); in the one-step kernel, a single halo barrier, or the
wait for the warp above's E phase two planes back instead of one.
"""
import random

import pytest

NWR = 11   # row warps of a block


class Barrier:
    """An mbarrier: expected arrivals per phase, completed phases."""

    def __init__(self, count, log):
        self.count, self.pending, self.done, self.log = count, count, 0, log

    def arrive(self):
        self.log.append(1)
        self.pending -= 1
        if self.pending == 0:
            self.done += 1
            self.pending = self.count

    def try_wait(self, parity):
        return parity != (self.done & 1)


class Hang(Exception):
    pass


def simulate(nplanes, ns, stage_in_b, seed, b_wait_in_c=False, skew=True):
    rng = random.Random(seed)
    log = []
    full = [Barrier(1, log) for _ in range(ns)]
    empty = [Barrier(NWR, log) for _ in range(ns)]
    xa = [[Barrier(1, log) for _ in range(NWR)] for _ in range(2)]
    xb = [Barrier(1, log) for _ in range(NWR)]
    xc = [Barrier(1, log) for _ in range(NWR)]
    stage = [None] * ns                      # plane held by each stage
    XA = [[None] * NWR for _ in range(2)]    # iteration whose rows each buffer holds
    XB, XC = [None] * NWR, [None] * NWR
    inflight = []

    def wait(bar, k, what):
        while not bar.try_wait(k & 1):
            yield "wait"
        assert bar.done > k, ("parity alias", what, k, bar.done)

    def row_warp(w):
        for rel in range(nplanes - 1):
            s0, s1 = rel % ns, (rel + 1) % ns
            if rel == 0:
                yield from wait(full[0], 0, "full")
            yield from wait(full[s1], (rel + 1) // ns, "full")
            assert stage[s0] == rel and stage[s1] == rel + 1, ("stage", w, rel)
            yield "A"
            assert stage[s0] == rel and stage[s1] == rel + 1, ("stage rewritten", w, rel)
            XA[rel & 1][w] = rel
            yield "store"
            if not b_wait_in_c and w + 1 < NWR and rel >= 1:
                yield from wait(xb[w + 1], rel - 1, "xb")
            xa[rel & 1][w].arrive()
            if not stage_in_b:
                empty[s0].arrive()
            if w >= 1:
                yield from wait(xa[rel & 1][w - 1], rel >> 1, "xa")
                assert XA[rel & 1][w - 1] == rel, ("A row", w, rel)
                yield "B"
                assert XA[rel & 1][w - 1] == rel, ("A row rewritten", w, rel)
                if stage_in_b:
                    assert stage[s0] == rel, ("stage rewritten before B", w, rel)
            if stage_in_b:
                empty[s0].arrive()
            if b_wait_in_c and w + 1 < NWR and rel >= 1:
                yield from wait(xb[w + 1], rel - 1, "xb")
            if rel >= 2 and 1 <= w <= NWR - 2:    # C reads the B row above
                assert XB[w + 1] == rel - 1, ("B row", w, rel)
                yield "C"
                assert XB[w + 1] == rel - 1, ("B row rewritten", w, rel)
                XC[w] = rel
                yield "store"
            xc[w].arrive()
            if w >= 2:
                yield from wait(xc[w - 1], rel, "xc")
            if rel >= 3 and 2 <= w <= NWR - 2:    # D reads the C row below
                assert XC[w - 1] == rel, ("C row", w, rel)
                yield "D"
                assert XC[w - 1] == rel, ("C row rewritten", w, rel)
            if w >= 1:
                XB[w] = rel
                yield "store"
            xb[w].arrive()

    def refill_warp():
        for r in range(min(ns, nplanes)):
            inflight.append((r % ns, r))
            yield "issue"
        for r in range(ns, nplanes):
            yield from wait(empty[r % ns], (r - ns) // ns, "empty")
            inflight.append((r % ns, r))
            yield "issue"

    warps = [row_warp(w) for w in range(NWR)] + [refill_warp()]
    speed = [rng.choice((0.1, 1.0, 10.0)) if skew else 1.0 for _ in warps]
    alive = list(range(len(warps)))
    waiting, seen = set(), 0
    while alive or inflight:
        if inflight and (not alive or rng.random() < 0.3):
            s, r = inflight.pop(rng.randrange(len(inflight)))
            stage[s] = r
            full[s].arrive()
            continue
        g = rng.choices(alive, weights=[speed[i] for i in alive])[0]
        try:
            ev = next(warps[g])
        except StopIteration:
            alive.remove(g)
            waiting.clear()
            continue
        if len(log) != seen:
            seen = len(log)
            waiting.clear()
        if ev == "wait":
            waiting.add(g)
            if waiting >= set(alive) and not inflight:
                raise Hang((nplanes, ns, stage_in_b, seed))
        else:
            waiting.clear()


@pytest.mark.parametrize("ns", [2, 3, 5, 8])
@pytest.mark.parametrize("stage_in_b", [False, True], ids=["release-after-A", "release-after-B"])
def test_protocol_never_hangs_or_aliases(ns, stage_in_b):
    for seed in range(12):
        for nplanes in (4, 9, 21):
            simulate(nplanes, ns, stage_in_b, seed * 101 + nplanes, skew=seed % 3 != 0)


def test_first_form_hangs():
    """With the B-row wait inside C the warp above can run a whole iteration
    ahead; the model finds the hang the GPU showed."""
    hung = 0
    for seed in range(40):
        try:
            simulate(21, 5, False, seed, b_wait_in_c=True, skew=False)
        except (Hang, AssertionError):
            hung += 1
    assert hung > 0


# ---- the one-step kernel's form without block barriers (csrc/vtile_tile.cuh) ----
BY = 8   # row warps of a block; one halo warp besides


def simulate_vtile(nplanes, ns, stage_in_e, seed, skew=True, single_halo=False, edone_back=1):
    """Row warps 0..BY-1, the halo warp (row jb-1 and column i0-1 of the H
    plane) and the refill warp.  A row warp writes its H row (read by the
    warp above), waits until the warp above is done with its E phase
    `edone_back` planes back, signals the row; its E phase waits for the row
    below (or the halo warp's) and the halo; it then signals its E phase.
    The halo warp rewrites its row and column after every row warp's E phase
    two planes back.  H rows and halo live in two buffers by plane parity."""
    rng = random.Random(seed)
    log = []
    full = [Barrier(1, log) for _ in range(ns)]
    empty = [Barrier(BY + 1, log) for _ in range(ns)]
    hrow = [Barrier(1, log) for _ in range(BY - 1)]
    halo = [Barrier(1, log) for _ in range(1 if single_halo else 2)]
    edone = [Barrier(1, log) for _ in range(BY)]
    eall = [Barrier(BY, log) for _ in range(2)]
    stage = [None] * ns
    HR = [[None] * (BY - 1) for _ in range(2)]
    HH = [None, None]
    inflight = []

    def wait(bar, k, what):
        while not bar.try_wait(k & 1):
            yield "wait"
        assert bar.done > k, ("parity alias", what, k, bar.done)

    def halo_bar(rel):
        return (halo[0], rel) if single_halo else (halo[rel & 1], rel >> 1)

    def row_warp(w):
        for rel in range(nplanes - 1):
            s0, s1 = rel % ns, (rel + 1) % ns
            if rel == 0:
                yield from wait(full[0], 0, "full")
            yield from wait(full[s1], (rel + 1) // ns, "full")
            yield "H"
            assert stage[s0] == rel and stage[s1] == rel + 1, ("stage", w, rel)
            if w < BY - 1:
                HR[rel & 1][w] = rel
                yield "store"
                if rel >= edone_back:
                    yield from wait(edone[w + 1], rel - edone_back, "edone")
                hrow[w].arrive()
            if not stage_in_e:
                empty[s0].arrive()
            if w >= 1:
                yield from wait(hrow[w - 1], rel, "hrow")
            bar, k = halo_bar(rel)
            yield from wait(bar, k, "halo")
            assert (w == 0 or HR[rel & 1][w - 1] == rel) and HH[rel & 1] == rel, ("H rows", w, rel)
            yield "E"
            assert (w == 0 or HR[rel & 1][w - 1] == rel) and HH[rel & 1] == rel, ("H rows rewritten", w, rel)
            if stage_in_e:
                assert stage[s0] == rel, ("stage rewritten before E", w, rel)
                empty[s0].arrive()
            edone[w].arrive()
            eall[rel & 1].arrive()

    def halo_warp():
        for rel in range(nplanes - 1):
            s0, s1 = rel % ns, (rel + 1) % ns
            if rel == 0:
                yield from wait(full[0], 0, "full")
            yield from wait(full[s1], (rel + 1) // ns, "full")
            if rel >= 2:
                yield from wait(eall[rel & 1], (rel >> 1) - 1, "eall")
            yield "H"
            assert stage[s0] == rel and stage[s1] == rel + 1, ("stage", "halo", rel)
            HH[rel & 1] = rel
            yield "store"
            halo_bar(rel)[0].arrive()
            empty[s0].arrive()

    def refill_warp():
        for r in range(min(ns, nplanes)):
            inflight.append((r % ns, r))
            yield "issue"
        for r in range(ns, nplanes):
            yield from wait(empty[r % ns], (r - ns) // ns, "empty")
            inflight.append((r % ns, r))
            yield "issue"

    run([row_warp(w) for w in range(BY)] + [halo_warp(), refill_warp()], full, stage, inflight, log, rng, skew,
        (nplanes, ns, stage_in_e, seed))


def run(warps, full, stage, inflight, log, rng, skew, tag):
    speed = [rng.choice((0.1, 1.0, 10.0)) if skew else 1.0 for _ in warps]
    alive = list(range(len(warps)))
    waiting, seen = set(), 0
    while alive or inflight:
        if inflight and (not alive or rng.random() < 0.3):
            s, r = inflight.pop(rng.randrange(len(inflight)))
            stage[s] = r
            full[s].arrive()
            continue
        g = rng.choices(alive, weights=[speed[i] for i in alive])[0]
        try:
            ev = next(warps[g])
        except StopIteration:
            alive.remove(g)
            waiting.clear()
            continue
        if len(log) != seen:
            seen = len(log)
            waiting.clear()
        if ev == "wait":
            waiting.add(g)
            if waiting >= set(alive) and not inflight:
                raise Hang(tag)
        else:
            waiting.clear()


@pytest.mark.parametrize("ns", [2, 3, 7])
@pytest.mark.parametrize("stage_in_e", [False, True], ids=["release-after-H", "release-after-E"])
def test_one_step_protocol_never_hangs_or_aliases(ns, stage_in_e):
    for seed in range(10):
        for nplanes in (4, 9, 21):
            simulate_vtile(nplanes, ns, stage_in_e, seed * 131 + nplanes, skew=seed % 3 != 0)


@pytest.mark.parametrize("form", ["single-halo-barrier", "E-wait-two-back"])
def test_one_step_rejected_forms_hang(form):
    """One halo barrier (the halo warp runs two phases ahead of a row warp),
    or the wait for the E phase of the warp above two planes back instead of
    one (the warp above finishes two E phases before the wait)."""
    hung = 0
    for seed in range(30):
        try:
            simulate_vtile(9, 2, False, seed, skew=False, single_halo=form == "single-halo-barrier",
                           edone_back=2 if form == "E-wait-two-back" else 1)
        except (Hang, AssertionError):
            hung += 1
    assert hung > 0
