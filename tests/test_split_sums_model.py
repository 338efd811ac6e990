"""Host model of the deterministic iteration kernel's split sums.

On a cluster of K blocks that shares one chunk, each block holds the
fixed-point sums of the rows it updates; a block's adds for another block's
rows go to that block's shared memory (cluster-scope reductions, landing at
arbitrary later times but before the adding block passes its next cluster
barrier).  Per chunk: every block clears its sums, a cluster barrier, then
per pass: adds, a cluster barrier, each block reads and clears its own
rows' sums (the update) and the rest of its slots, a cluster barrier (the
map broadcast), the next pass.

The model replays the blocks with random interleavings and random landing
times of the adds and checks that every pass's sums, as the update reads
them, are exactly the pass's contributions (integer adds: no add lost or
counted twice, in any order).  Two weaker orders must be caught: no barrier
between the initial clearing and the first pass's adds (a fast block's add
lands before a slow block clears), and clearing after the post-update
barrier instead of before it (the next pass's adds land before the clear).
"""
import random

import pytest

CAP = 50000


def replay(seed, K, rows, passes, rules="kernel"):
    rng = random.Random(seed)
    slice_ = -(-rows // K)
    acc = [[rng.randint(-9, 9) for _ in range(slice_)] for _ in range(K)]   # stale values from the last chunk
    pending = []                    # adds in flight: [block, slot, value]
    expect = [[{} for _ in range(K)] for _ in range(passes)]
    seen = [[None] * K for _ in range(passes)]
    arrived = {}                    # barrier id -> blocks arrived

    def land_some(p=0.5):
        keep = []
        for a in pending:
            if rng.random() < p:
                acc[a[0]][a[1]] += a[2]
            else:
                keep.append(a)
        pending[:] = keep

    def barrier(bid, b):
        # a block's own adds land before it passes the barrier (release)
        mine = [a for a in pending if a[3] == b]
        for a in mine:
            acc[a[0]][a[1]] += a[2]
            pending.remove(a)
        arrived.setdefault(bid, set()).add(b)
        while len(arrived[bid]) < K:
            yield

    def block(b):
        # clear this block's sums at the chunk's start
        for l in range(slice_):
            acc[b][l] = 0
            yield
        if rules != "no_initial_barrier":
            yield from barrier(("start",), b)
        for p in range(passes):
            # contributions of this block's tiles: random rows, random values
            for _ in range(rng.randint(5, 25)):
                row = rng.randrange(rows)
                owner, l = row // slice_, row % slice_
                v = rng.randint(1, 1000)
                expect[p][owner][l] = expect[p][owner].get(l, 0) + v
                pending.append([owner, l, v, b])
                if rng.random() < 0.3:
                    yield
            yield from barrier(("adds", p), b)
            # the update: read and clear this block's rows (and the rest)
            got = {}
            for l in range(slice_):
                if acc[b][l]:
                    got[l] = acc[b][l]
                if rules != "clear_after_barrier":
                    acc[b][l] = 0
                if rng.random() < 0.3:
                    yield
            seen[p][b] = got
            yield from barrier(("map", p), b)
            if rules == "clear_after_barrier":
                for l in range(slice_):
                    acc[b][l] = 0
                    if rng.random() < 0.3:
                        yield

    gens = [block(b) for b in range(K)]
    active = list(gens)
    steps = 0
    while active:
        land_some(0.3)
        g = rng.choice(active)
        try:
            next(g)
        except StopIteration:
            active.remove(g)
        steps += 1
        assert steps < CAP, "no progress"
    for p in range(passes):
        for b in range(K):
            want = {l: v for l, v in expect[p][b].items() if v}
            if seen[p][b] != want:
                return f"pass {p}, block {b}: read {seen[p][b]} instead of {want}"
    return "ok"


@pytest.mark.parametrize("K,rows", [(2, 64), (2, 70), (4, 64), (4, 40)])
def test_split_sums_are_exact_in_any_order(K, rows):
    for seed in range(60):
        assert replay(seed, K, rows, 4) == "ok", seed


@pytest.mark.parametrize("rules", ["no_initial_barrier", "clear_after_barrier"])
def test_weaker_orders_lose_adds(rules):
    results = {replay(seed, 2, 48, 3, rules) for seed in range(200)}
    assert results != {"ok"}, rules
