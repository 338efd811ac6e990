"""Host model of the tile pipeline of the batched iteration kernel.

The kernel streams P tiles through a ring of shared-memory buffers: one
producer issues tile q into buffer q % ring after the buffer's `empty` barrier
completes, and the consumer warp of slot q % slots (the kernel evaluates a
tile with one warp; the model also covers groups of G warps per slot) waits on
the buffer's `full` barrier with phase parity (q / ring) & 1.  An mbarrier parity wait only
distinguishes the current phase from the previous one, so a consumer must never
wait two phases ahead.  The kernel guarantees this by sizing the ring as a whole
number of slots.  This test replays the protocol under random interleavings and
out-of-order copy completion: every consumer must read exactly the tile it
expects and the pipeline must never stall, and the ring/slot mismatch that the
sizing rule excludes must be caught by the model.
"""
import random

import pytest


class MBarrier:
    """Arrival count + transaction bytes; parity wait as in PTX try_wait.parity."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0
        self.tx = 0

    def _check(self):
        if self.pending <= 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self):
        self.pending -= 1
        self._check()

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._check()

    def try_wait(self, parity):
        # true once the phase with this parity has completed
        return (self.phase & 1) != parity


def replay(slots, group, ring, ntiles, seed, batch=1):
    """The producer issues tiles in batches of `batch` consecutive stream
    indices (one per producer lane), in any order within a batch; batch k + 1
    starts after every tile of batch k is issued."""
    rng = random.Random(seed)
    full = [MBarrier(1) for _ in range(ring)]
    empty = [MBarrier(group) for _ in range(ring)]
    content = [None] * ring
    inflight = []
    pending = []          # tiles of the current producer batch not yet issued
    next_batch = 0
    next_tile = [[s, s] for s in range(slots) for _ in range(group)]
    for _ in range(10 ** 6):
        if not pending and next_batch < ntiles:
            pending = list(range(next_batch, min(ntiles, next_batch + batch)))
            next_batch += batch
        moves = []
        for q in pending:
            if empty[q % ring].try_wait(((q // ring) & 1) ^ 1):
                moves.append(("issue", q))
        if inflight:
            moves.append("land")
        for w, (_, q) in enumerate(next_tile):
            if q < ntiles and full[q % ring].try_wait((q // ring) & 1):
                moves.append(w)
        if not moves:
            done = not pending and next_batch >= ntiles and all(q >= ntiles for _, q in next_tile)
            return "ok" if done else "stall"
        m = rng.choice(moves)
        if isinstance(m, tuple):
            q = m[1]
            pending.remove(q)
            full[q % ring].arrive_expect_tx(1)
            inflight.append((q % ring, q))
        elif m == "land":
            b, t = inflight.pop(rng.randrange(len(inflight)))
            content[b] = t
            full[b].complete_tx(1)
        else:
            q = next_tile[m][1]
            if content[q % ring] != q:
                return "wrong tile"
            empty[q % ring].arrive()
            next_tile[m][1] = q + slots
    return "stall"


@pytest.mark.parametrize("slots,group", [(24, 1), (12, 2), (6, 4), (8, 1), (4, 4), (1, 4)])
@pytest.mark.parametrize("per_slot", [1, 2, 4])
def test_ring_of_whole_slots_is_safe(slots, group, per_slot):
    for seed in range(20):
        assert replay(slots, group, slots * per_slot, 150, seed) == "ok"


def test_ring_smaller_than_the_slots_is_caught():
    results = {replay(24, 1, 16, 150, seed) for seed in range(10)}
    assert results != {"ok"}


@pytest.mark.parametrize("slots,group,per_slot", [(8, 2, 3), (4, 4, 4), (6, 2, 4), (12, 2, 2), (16, 1, 3),
                                                   (19, 1, 1), (12, 1, 2), (20, 1, 1), (5, 1, 1)])
@pytest.mark.parametrize("max_batch", [8, 32])
def test_warp_parallel_producer_batches_of_at_most_ring(slots, group, per_slot, max_batch):
    """Batches of min(8, ring) (the kernel's) or min(32, ring) tiles."""
    ring = slots * per_slot
    for seed in range(15):
        assert replay(slots, group, ring, 200, seed, batch=min(max_batch, ring)) == "ok"


def test_producer_batch_larger_than_ring_is_caught():
    results = {replay(4, 2, 8, 200, seed, batch=32) for seed in range(10)}
    assert results != {"ok"}
