"""Host model of the tile feed of the batched iteration kernel.

Each warp of a block takes a contiguous piece of the block's share of a
chunk's stored tiles, the same piece in every pass, and owns one shared
buffer (4 KB of P plus a 16-byte trailer).  Lane l copies its own eight
16-byte pieces of a tile into the buffer with cp.async (lane 0 also the
trailer), so every lane later reads back exactly what it copied, except the
trailer, which all lanes read.  For each tile the warp:

  1. waits for its own copies (cp.async.wait_group 0, per lane),
  2. __syncwarp (lane 0's trailer becomes visible to the other lanes),
  3. reads its pieces and the trailer into registers,
  4. uses those registers (an empty asm that takes them as inputs, so the
     reads have returned) and __syncwarp,
  5. issues the copy of its next tile into the same buffer (the next tile
     of the piece; after the last, the first again if another pass follows;
     nothing after the chunk's last pass),
  6. evaluates the tile from registers.

Copies complete at arbitrary later times and in any order, and a shared
load returns its value at an arbitrary later time (its value is the
buffer's content when the load is performed, which may be any time before
it returns).  The model replays the protocol with random timings and checks
that every read sees exactly the tile it expects, that no copy is in flight
into a buffer while a read of it is pending, that the warps together read
every tile of the share once per pass, and that nothing is in flight when
the chunk ends.  Weaker rules must be caught: no wait_group, no __syncwarp
before the trailer read, the next copy issued before the reads have
returned, and a copy issued after the chunk's last pass.
"""
import random

import pytest

LANES = 32
PIECES = 8     # 16-byte pieces of P per lane
TRAILER = -1   # piece index of the trailer (copied by lane 0)


def pieces_of(lane):
    out = [(lane, k) for k in range(PIECES)]
    if lane == 0:
        out.append((0, TRAILER))
    return out


class Warp:
    def __init__(self, rng, tiles, npass, rules):
        self.rng = rng
        self.tiles = tiles            # its stored tiles (ids) of the chunk, per pass
        self.npass = npass
        self.rules = rules
        self.buf = {}                 # (lane, piece) -> tile id currently in the buffer
        self.inflight = []            # [lane, piece, tile id, remaining steps]
        self.read = []                # tiles the warp evaluated, in order

    def tick(self):
        """Advance every copy in flight by one step; land those that complete."""
        keep = []
        for c in self.inflight:
            c[3] -= 1
            if c[3] <= 0:
                self.buf[(c[0], c[1])] = c[2]
            else:
                keep.append(c)
        self.inflight = keep

    def issue(self, tile):
        for lane in range(LANES):
            for lane_, piece in pieces_of(lane):
                self.inflight.append([lane_, piece, tile, self.rng.randint(1, 6)])

    def lane_pending(self, lane):
        return any(c[0] == lane for c in self.inflight)

    def wait_lane(self, lane):
        while self.lane_pending(lane):
            self.tick()

    def run(self):
        seq = [(p, j) for p in range(self.npass) for j in range(len(self.tiles))]
        if seq:
            self.issue(self.tiles[0])
        for idx, (p, j) in enumerate(seq):
            # 1. wait_group per lane (lanes in a random order; copies keep landing)
            lanes = list(range(LANES))
            self.rng.shuffle(lanes)
            trailer_seen = None
            if self.rules != "no_wait":
                for lane in lanes:
                    self.wait_lane(lane)
                    if self.rules == "no_syncwarp" and lane != 0 and trailer_seen is None:
                        # without __syncwarp, a lane may read the trailer before lane 0 waited
                        trailer_seen = self.buf.get((0, TRAILER))
            # 2.-3. reads: each value is taken when the load is performed, at a
            # random moment up to the time the registers are used
            expected = self.tiles[j]
            pending_reads = [(lane, k) for lane in range(LANES) for k in range(PIECES)] + [(0, TRAILER)]
            got = {}
            nxt = None
            if idx + 1 < len(seq):
                nxt = self.tiles[seq[idx + 1][1]]
            elif self.rules == "copy_after_last":
                nxt = self.tiles[0]
            if self.rules == "early_issue" and nxt is not None:
                self.issue(nxt)            # next copy issued while the reads are still pending
            for r in pending_reads:
                if self.rng.random() < 0.5:
                    self.tick()
                got[r] = self.buf.get(r)
            # 4. registers used: every read has returned; 5. issue the next copy
            if self.rules != "early_issue" and nxt is not None:
                self.issue(nxt)
            if trailer_seen is not None:
                got[("trailer seen early",)] = trailer_seen
            bad = [k for k, v in got.items() if v != expected]
            if bad:
                return f"read {bad[0]} saw {got[bad[0]]} instead of tile {expected} (pass {p})"
            self.read.append(expected)
            # 6. evaluation takes a while; copies keep landing
            for _ in range(self.rng.randint(0, 4)):
                self.tick()
        if self.inflight:
            return "copies in flight at the chunk's end"
        return "ok"


def replay(nq, W, npass, seed, rules="kernel"):
    rng = random.Random(seed)
    share = list(range(100, 100 + nq))          # the block's stored tiles (ids)
    pieces = [share[(nq * w) // W:(nq * (w + 1)) // W] for w in range(W)]
    reads = []
    for w in range(W):
        r = Warp(rng, pieces[w], npass, rules).run()
        if r != "ok":
            return r
        reads.extend(pieces[w] * npass)
    if sorted(reads) != sorted(share * npass):
        return "the warps did not read every tile once per pass"
    return "ok"


@pytest.mark.parametrize("nq,W", [(1, 16), (7, 16), (16, 16), (45, 16), (300, 12), (1225, 16), (31, 21)])
def test_feed_reads_every_tile_it_expects(nq, W):
    for seed in range(6):
        assert replay(nq, W, 3, seed) == "ok"


def test_pieces_cover_the_share_contiguously():
    for nq in (1, 5, 16, 17, 4465, 2232):
        for W in (1, 7, 12, 16, 21):
            bounds = [(nq * w) // W for w in range(W + 1)]
            assert bounds[0] == 0 and bounds[-1] == nq
            assert all(0 <= b - a <= (nq + W - 1) // W for a, b in zip(bounds, bounds[1:]))


@pytest.mark.parametrize("rules", ["no_wait", "no_syncwarp", "early_issue", "copy_after_last"])
def test_weaker_rules_are_caught(rules):
    results = {replay(45, 16, 2, seed, rules) for seed in range(40)}
    assert results != {"ok"}, rules
