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

The second half models the bounded waits running out.  Any wait that is not
yet satisfied may run out at any moment, and another block's failure may
freeze the block at any moment.  The kernel's rules: the first failed wait
sets the block's freeze flag, after which every wait that is not yet
satisfied fails at once; a consumer whose wait failed skips that tile and
every later one (no read, no release); the producer issues a copy only after
a successful wait on the buffer's `empty` barrier; before exiting, the
producer waits for the phase of the last copy it issued into each buffer.  The model checks that no copy is ever issued into a
buffer that still has one in flight or whose content was not released, that
every read sees the tile it expects with no copy in flight into it, that the
block exits with no copy in flight, and that the run always ends.  A wait
whose barrier is ready still succeeds after a freeze (the kernel reads the
freeze flag only while a wait is not yet satisfied), which is safe because a
ring buffer belongs to one consumer warp: a phase of it can be left
incomplete only by that warp's own failure (after which it skips its tiles)
or by a copy the producer skipped (after which the producer issues nothing
more, so the warp's next wait simply fails).  Weaker rules must be caught:
the earlier kernel's (a failed consumer wait still released the buffer, a
failed producer wait still issued the copy, the exit drain followed stream
positions), and a consumer or a producer that forgets its own failure.
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


# ---------------------------------------------------------------- waits that run out

def replay_with_timeouts(slots, ring, ntiles, seed, batch, p_out=0.02, p_freeze=0.002, rules="kernel"):
    """One block, one consumer warp per slot.  rules: "kernel" (the kernel's:
    a wait whose barrier is ready succeeds; a wait that is not ready fails at
    once when the block is frozen, else may run out; a consumer that failed a
    wait skips every later tile; the producer issues only after a successful
    wait, and after a batch with a failed wait it issues nothing more),
    "no_consumer_memory" (a consumer goes on waiting normally after its own
    failure), "no_producer_memory" (the producer goes on issuing after its own
    failure), "old" (a failed consumer wait still released its buffer, a
    failed producer wait still issued, the exit drain followed stream
    positions).  Returns "ok", or the first violation."""
    rng = random.Random(seed)
    full = [MBarrier(1) for _ in range(ring)]
    empty = [MBarrier(1) for _ in range(ring)]
    content = [None] * ring
    released = [True] * ring      # the buffer's last copy was read and released (or none yet)
    inflight = {}                 # buffer -> tile of the copy in flight
    issued_ph = {}                # buffer -> full-barrier parity of the last copy issued
    fail = False                  # the block's freeze flag
    failed = [False] * slots      # consumer warp's own failure (kept in a register)
    prod_failed = False           # the producer warp's own failure (noted after each batch)
    prod_failed_now = False
    batch_base, fail_base, fail_issued, batch_issued = 0, None, set(), set()
    old = rules == "old"
    pending, next_batch = [], 0
    next_tile = list(range(slots))   # consumer warp w: its next tile
    for _ in range(10 ** 6):
        if not pending and next_batch < ntiles:
            prod_failed = prod_failed or prod_failed_now
            pending = list(range(next_batch, min(ntiles, next_batch + batch)))
            batch_base = next_batch
            batch_issued = set()
            next_batch += batch
            if prod_failed and rules != "old" and rules != "no_producer_memory":
                pending = []              # after its own failure the producer issues nothing more
                continue
        moves = []
        for q in pending:
            b, ph = q % ring, (q // ring) & 1
            if empty[b].try_wait(ph ^ 1):
                moves.append(("issue", q))
            elif fail or rng.random() < p_out:
                moves.append(("issue_out", q))
        if inflight:
            moves.append(("land", None))
        for w in range(slots):
            q = next_tile[w]
            if q >= ntiles:
                continue
            b, ph = q % ring, (q // ring) & 1
            if failed[w] and rules == "kernel":
                moves.append(("skip_read", w))
            elif full[b].try_wait(ph):
                moves.append(("read", w))
            elif fail or rng.random() < p_out:
                moves.append(("read_out", w))
        if not fail and rng.random() < p_freeze:
            moves.append(("freeze", None))
        if not moves:
            if pending or next_batch < ntiles or any(q < ntiles for q in next_tile):
                return "stall"
            break
        kind, arg = rng.choice(moves)
        if kind == "freeze":
            fail = True
        elif kind in ("issue", "issue_out"):
            q = arg
            b, ph = q % ring, (q // ring) & 1
            if kind == "issue_out":
                fail = True
                if not prod_failed_now:
                    fail_base = batch_base
                    fail_issued = set(batch_issued)   # lanes of this batch that issued before the failure
                prod_failed_now = True
                if not old:
                    pending.remove(q)       # skipped: no copy
                    continue
            if b in inflight:
                return "copy issued into a buffer with a copy in flight"
            if not released[b]:
                return "copy issued into a buffer that was not released"
            pending.remove(q)
            batch_issued.add(q)
            if fail_base is not None and q >= fail_base:
                fail_issued.add(q)
            full[b].arrive_expect_tx(1)
            inflight[b] = q
            released[b] = False
            issued_ph[b] = ph
        elif kind == "land":
            b = rng.choice(sorted(inflight))
            content[b] = inflight.pop(b)
            full[b].complete_tx(1)
        else:
            w = arg
            q = next_tile[w]
            b = q % ring
            next_tile[w] = q + slots
            if kind == "skip_read":
                continue
            if kind == "read_out":
                fail = True
                failed[w] = True
                if old:                   # the earlier kernel still read the header and released
                    if b in inflight:
                        return "read of a buffer with a copy in flight"
                    released[b] = True
                    empty[b].arrive()
                continue
            if b in inflight or content[b] != q:
                return "read of the wrong tile"
            released[b] = True
            empty[b].arrive()
    # exit drain
    if old:
        # the earlier drain: the phases of the last `ring` stream positions
        for q in range(max(0, ntiles - ring), ntiles):
            b, ph = q % ring, (q // ring) & 1
            while not full[b].try_wait(ph) and b in inflight:
                content[b] = inflight.pop(b)
                full[b].complete_tx(1)
        return "ok" if not inflight else "exit with a copy in flight"
    # the kernel keeps no per-buffer record: it rebuilds the last copy issued
    # into each buffer from where its stream stopped and the lanes of its
    # failed batch that did issue
    end = ntiles if fail_base is None else fail_base
    rebuilt = {}
    for b in range(ring):
        cands = [g for g in fail_issued if g % ring == b]
        if end > b:
            cands.append(end - 1 - ((end - 1 - b) % ring))
        if cands:
            rebuilt[b] = (max(cands) // ring) & 1
    if rebuilt != issued_ph:
        return "rebuilt drain differs from the copies issued"
    for b, ph in issued_ph.items():
        while not full[b].try_wait(ph):
            if not inflight:
                return "drain waits on a phase no copy will complete"
            c = rng.choice(sorted(inflight))          # copies land in any order
            content[c] = inflight.pop(c)
            full[c].complete_tx(1)
    return "ok" if not inflight else "exit with a copy in flight"


@pytest.mark.parametrize("slots,per_slot", [(20, 1), (19, 2), (12, 4), (16, 3), (5, 1), (1, 4)])
def test_waits_that_run_out_never_corrupt_the_ring(slots, per_slot):
    ring = slots * per_slot
    batch = min(8, ring)
    outcomes = set()
    for seed in range(60):
        p_out = (0.0, 0.005, 0.05)[seed % 3]
        r = replay_with_timeouts(slots, ring, 150, seed, batch, p_out=p_out, p_freeze=0.001 * (seed % 4))
        assert r == "ok", (seed, r)
        outcomes.add(r)


def test_no_timeouts_consumes_every_tile():
    for seed in range(10):
        assert replay_with_timeouts(12, 24, 200, seed, 8, p_out=0.0, p_freeze=0.0) == "ok"


@pytest.mark.parametrize("rules", ["old", "no_consumer_memory", "no_producer_memory"])
def test_weaker_timeout_rules_are_caught(rules):
    bad = {replay_with_timeouts(12, 24, 150, seed, 8, p_out=0.05, rules=rules) for seed in range(60)}
    assert bad - {"ok"}, bad
