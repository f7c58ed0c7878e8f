"""Model check of the stage protocol of the TMA-fed step kernel (no GPU).

The kernel's producer warp fills stage `it % ns` with this CTA's tile `it` and
completes phase `it // ns` of that stage's "full" mbarrier; the consumer warps
of group g take tiles g, g + G, ... and, for each, wait on "full" with parity
`(it // ns) & 1`, read the stage and arrive on its "empty" mbarrier (one
arrival per warp of the group); before refilling a stage for tile `it` the
producer waits on "empty" with parity `((it // ns) & 1) ^ 1`.

An mbarrier parity wait only tells whether the phase *before* the current one
has the given parity, so a waiter that runs two phases ahead passes on a stale
phase.  This model runs the same index arithmetic under many random
interleavings of the producer, the landing of its copies and every consumer
warp, with mbarriers that keep a phase counter, and checks that no wait ever
passes on a stale phase, that every warp reads the tile it expects, that no
stage is refilled before all its readers arrived, and that nothing deadlocks.
The planner makes the stage count a multiple of the group count, and the
launcher rejects any other plan: with two groups and an odd count a group can
reach a stage whose previous tile, the other group's, has not landed yet.
The model must find that hazard (and the one of more groups than stages),
which shows it can see a stale phase.  With bounded waits that give up, the
producer stops issuing and, before the CTA exits, waits for the last fill of
every stage -- the last `ns` tiles it issued; counting the tile it gave up on
as issued would let that drain pass on a stale phase while the stage's
previous copy is still in flight, which the model also finds.
"""
import random

import pytest


class MBarrier:
    """Phase counter and pending arrivals (expected-transaction bytes folded
    into one 'copy landed' arrival)."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0           # index of the current (incomplete) phase

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def try_wait_parity(self, parity):
        # true once the phase preceding the current one has this parity
        return (self.phase & 1) != parity


class Hazard(AssertionError):
    pass


def run_cta(ntiles, ns, groups, consumers, seed, check_stale=True, timeouts=0.0,
            drain_counts_unissued=False):
    """One CTA: `ntiles` tiles, `ns` stages, `groups` x `consumers` consumer
    warps.  With `timeouts`, any blocked wait may give up (the kernel's bounded
    waits): the warp sets the abort flag and leaves, the others leave at their
    next wait, the producer stops issuing and drains the copies it issued
    (`timeouts` is the chance per scheduling step that blocked waits may give up).
    `drain_counts_unissued` counts the tile the producer gave up on as issued.
    Returns the number of scheduling steps taken."""
    rng = random.Random(seed)
    full = [MBarrier(1) for _ in range(ns)]                 # producer's copy lands
    empty = [MBarrier(consumers) for _ in range(ns)]        # one group consumes a tile
    stage_tile = [None] * ns                                # which tile a stage holds
    readers_left = [0] * ns                                 # warps still to read it
    prod = {"it": 0, "issued": 0, "inflight": [], "drain": None, "done": False}
    warps = [{"g": g, "it": g, "out": False} for g in range(groups) for _ in range(consumers)]
    consumed = {}
    state = {"abort": False}
    steps = 0

    def producer_enabled():
        it = prod["it"]
        if prod["drain"] is not None or it >= ntiles or state["abort"]:
            return False
        st, k = it % ns, it // ns
        return empty[st].try_wait_parity((k & 1) ^ 1)

    def producer_step():
        it = prod["it"]
        st, k = it % ns, it // ns
        # the parity wait passed: the stage's previous use must be fully released
        if check_stale and empty[st].phase < k:
            raise Hazard(f"producer passed empty[{st}] for tile {it} on a stale phase")
        if readers_left[st] != 0:
            raise Hazard(f"stage {st} refilled for tile {it} while {readers_left[st]} warps read it")
        stage_tile[st] = None                               # copy in flight
        prod["inflight"].append(it)
        prod["it"] += 1
        prod["issued"] += 1

    def producer_stops():
        # loop left (all issued, or abort seen / own wait gave up): drain the
        # last fill of every stage, i.e. the last ns issued tiles
        if prod["it"] < ntiles and drain_counts_unissued:
            prod["it"] += 1                                 # the tile it gave up on
            last = prod["it"]
        else:
            last = prod["issued"]
        prod["drain"] = list(range(max(0, last - ns), last))

    def drain_enabled():
        q = prod["drain"][0]
        return full[q % ns].try_wait_parity((q // ns) & 1)

    def land_step():
        it = prod["inflight"].pop(rng.randrange(len(prod["inflight"])))
        # copies complete in any order; each completes its own stage's phase
        st = it % ns
        stage_tile[st] = it
        readers_left[st] = consumers
        full[st].arrive()

    def warp_live(w):
        return not w["out"] and w["it"] < ntiles

    def warp_enabled(w):
        it = w["it"]
        st, k = it % ns, it // ns
        return full[st].try_wait_parity(k & 1)

    def warp_step(w):
        it = w["it"]
        st, k = it % ns, it // ns
        if check_stale and full[st].phase <= k:
            raise Hazard(f"warp of group {w['g']} passed full[{st}] for tile {it} on a stale phase")
        if stage_tile[st] != it:
            raise Hazard(f"warp of group {w['g']} read tile {stage_tile[st]} expecting {it}")
        readers_left[st] -= 1
        consumed[it] = consumed.get(it, 0) + 1
        empty[st].arrive()
        w["it"] += groups

    while True:
        moves = []
        giveup = timeouts > 0 and rng.random() < timeouts
        if not prod["done"]:
            if prod["drain"] is None:
                if producer_enabled():
                    moves.append(("p", None))
                elif prod["it"] >= ntiles or state["abort"]:
                    moves.append(("stop", None))
                elif giveup:
                    moves.append(("ptimeout", None))
            elif not prod["drain"]:
                moves.append(("exit", None))
            elif drain_enabled():
                moves.append(("drain", None))
            elif prod["drain"][0] >= prod["issued"]:
                # waiting for a copy that was never issued: the bounded wait
                # gives up (copies that were issued always land in this model)
                moves.append(("drain", None))
        if prod["inflight"]:
            moves.append(("l", None))
        for w in warps:
            if warp_live(w):
                if state["abort"]:
                    moves.append(("leave", w))
                elif warp_enabled(w):
                    moves.append(("w", w))
                elif giveup:
                    moves.append(("wtimeout", w))
        if not moves:
            break
        kind, w = rng.choice(moves)
        if kind == "p":
            producer_step()
        elif kind == "stop":
            producer_stops()
        elif kind == "ptimeout":
            state["abort"] = True
            producer_stops()
        elif kind == "drain":
            prod["drain"].pop(0)
        elif kind == "exit":
            prod["done"] = True
            if prod["inflight"]:
                raise Hazard(f"producer left with copies of tiles {prod['inflight']} in flight")
        elif kind == "l":
            land_step()
        elif kind == "w":
            warp_step(w)
        elif kind == "wtimeout":
            state["abort"] = True
            w["out"] = True
        else:                                               # leave after an abort
            w["out"] = True
        steps += 1
    # no deadlock: the producer drained and left, every warp finished or left
    assert prod["done"] and not prod["inflight"], "producer stalled"
    assert all(not warp_live(w) for w in warps), "a consumer warp stalled"
    if not state["abort"]:
        assert prod["issued"] == ntiles
        assert consumed == {t: consumers for t in range(ntiles)}
    return steps


@pytest.mark.parametrize("ns,groups", [(2, 1), (3, 1), (4, 1), (5, 1), (6, 1), (8, 1),
                                       (2, 2), (4, 2), (6, 2), (8, 2)])
def test_protocol_is_safe(ns, groups):
    # the plans the launcher accepts: nstages >= 2 and a multiple of the groups
    for ntiles in (0, 1, 2, ns - 1, ns, ns + 1, 2 * ns + 1, 23):
        for seed in range(60):
            run_cta(ntiles, ns, groups, consumers=3, seed=seed)


def test_kernel_shapes():
    # FP64: two groups of 8 warps and four stages; FP32 vectors: one group of
    # 16 warps, two stages; BF16 levels plan five or six
    for ns, groups, consumers in ((4, 2, 8), (2, 1, 16), (5, 1, 16), (6, 1, 16)):
        for seed in range(10):
            run_cta(3 * ns + 2, ns, groups, consumers, seed)


@pytest.mark.parametrize("ns,groups", [(3, 2), (5, 2), (7, 2), (2, 3)])
def test_stage_count_not_a_multiple_of_groups_is_unsafe(ns, groups):
    # e.g. two groups on three stages: group 1 finishes tile 1 and waits for
    # tile 3 on stage 0 while tile 0 (group 0's) has not landed, and the
    # parity wait passes on the stale phase
    seen = False
    for seed in range(400):
        try:
            run_cta(4 * ns + 3, ns, groups, consumers=2, seed=seed)
        except Hazard:
            seen = True
            break
    assert seen


@pytest.mark.parametrize("ns,groups", [(2, 1), (3, 1), (5, 1), (2, 2), (4, 2)])
def test_abort_path_drains_every_copy(ns, groups):
    # any wait may give up; the producer still leaves only after every copy it
    # issued has landed, and no warp waits forever
    for ntiles in (1, ns, 2 * ns + 1, 17):
        for seed in range(150):
            run_cta(ntiles, ns, groups, consumers=2, seed=seed, timeouts=0.3)


def test_counting_the_unissued_tile_in_the_drain_is_unsafe():
    # if the tile the producer gave up on were counted as issued, the drain
    # would wait on that stage's phase, see the stale phase of the stage's
    # previous tile as complete and leave while that copy is still in flight
    seen = False
    for seed in range(5000):
        try:
            run_cta(9, 2, 1, consumers=2, seed=seed, timeouts=0.05,
                    drain_counts_unissued=True)
        except Hazard:
            seen = True
            break
    assert seen
