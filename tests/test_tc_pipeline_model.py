"""Host models of the tcgen05 kernels' pipelines, with and without bounded
waits running out.

Two protocols are replayed with random timings: the K-block ring of the
tensor-core GEMMs (the BF16 Gram kernel of the distances, the mapper's
training GEMMs: one thread issues TMA loads into a ring of stages and the
MMAs that read them) and the fused mapper inference kernel (one thread
issuing the weights' TMA loads and the MMAs, two loader warps writing X into
shared memory, epilogue warps reading the tensor-memory accumulators and
writing the layer-2 operand H1).  Asynchronous work is modelled as in the
hardware: TMA loads land in any order and complete their mbarrier's
transaction count; MMAs and commits run in issue order on the tensor pipe,
a commit arriving once every MMA before it is done.  Mbarrier waits follow
the parity rule (a wait for parity P succeeds once the phase of that parity
has completed).

Without a timeout the model checks that every MMA and every epilogue read
sees the data of its own tile and K block, that no buffer is overwritten
before its readers are done, and that every tile's output is written.  With
timeouts injected at random waits (each wait of the main loops may give up
after a few retries; a wait that gave up sets the kernel's failure flag, and
every later wait of every role then gives up unless its barrier is already
complete) the model checks what keeps a timeout harmless: every role ends,
the timeout is counted, and no TMA load or MMA is in flight when the CTA
frees its tensor memory and exits.  Weaker rules must be caught: the former
drains, no drain, issuing on after a timeout, and waits left out of the
normal protocol.
"""
import random
from collections import deque

import pytest

STEP_CAP = 200000


class Hazard(Exception):
    pass


class Bar:
    """An mbarrier: `count` arrivals and a transaction count per phase."""

    def __init__(self, count):
        self.count, self.left, self.tx, self.phase = count, count, 0, 0

    def _check(self):
        if self.left == 0 and self.tx == 0:
            self.phase += 1
            self.left = self.count

    def arrive(self):
        self.left -= 1
        if self.left < 0:   # undefined on the hardware, with or without a timeout
            raise Hazard("more arrivals in a phase than the barrier's count")
        self._check()

    def expect_tx(self, nbytes):          # mbarrier.arrive.expect_tx
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._check()

    def try_wait(self, parity):
        return (self.phase & 1) != parity


class Sim:
    def __init__(self, rng, p_timeout):
        self.rng = rng
        self.p_timeout = p_timeout
        self.fail = False
        self.timed_out = False
        self.tma = []                     # [bar, nbytes, land]
        self.tp = deque()                 # ("mma", execute) | ("commit", bar)
        self.named = {}                   # named barrier: generation bookkeeping

    def hazard(self, msg):
        """A protocol violation of the normal run.  After a wait has run out
        the kernel's results are discarded (the host reports the timeout), so
        stale data is harmless there; what matters is that nothing stays in
        flight."""
        if not (self.fail or self.timed_out):
            raise Hazard(msg)

    # ---- asynchronous units
    def issue_tma(self, bar, nbytes, land):
        self.tma.append([bar, nbytes, land])

    def issue_mma(self, execute):
        self.tp.append(("mma", execute))

    def commit(self, bar):
        self.tp.append(("commit", bar))

    def step_units(self):
        if self.tma and self.rng.random() < 0.5:
            bar, nbytes, land = self.tma.pop(self.rng.randrange(len(self.tma)))
            land()
            bar.complete_tx(nbytes)
        if self.tp and self.rng.random() < 0.5:
            kind, x = self.tp.popleft()
            if kind == "mma":
                x()
            else:
                x.arrive()

    # ---- waits
    def wait(self, bar, parity):
        """A bounded wait of a main loop (iwait): the fast path first; then,
        while the barrier is not complete, give up if the failure flag is set
        or the wait's own budget is spent (injected timeout)."""
        if bar.try_wait(parity):
            return True
        budget = self.rng.randint(0, 3) if self.rng.random() < self.p_timeout else None
        while True:
            if self.fail or (budget is not None and budget <= 0):
                self.fail = True
                if budget is not None and budget <= 0:
                    self.timed_out = True
                return False
            yield
            if budget is not None:
                budget -= 1
            if bar.try_wait(parity):
                return True

    def wait_alone(self, bar, parity):
        """A bounded wait that does not look at the failure flag (the plain
        mbar_wait of the GEMM ring); it may run out like the others."""
        if bar.try_wait(parity):
            return True
        budget = self.rng.randint(0, 3) if self.rng.random() < self.p_timeout else None
        while True:
            if budget is not None and budget <= 0:
                self.timed_out = True
                return False
            yield
            if budget is not None:
                budget -= 1
            if bar.try_wait(parity):
                return True

    def drain_wait(self, bar, parity):
        """The exit drain's wait: for work already issued, which completes."""
        while not bar.try_wait(parity):
            yield

    def named_barrier(self, name, nthreads):
        g = self.named.setdefault(name, [0, 0])
        gen = g[0]
        g[1] += 1
        if g[1] == nthreads:
            g[0] += 1
            g[1] = 0
        while self.named[name][0] == gen:
            yield

    def run(self, roles):
        active = list(roles)
        steps = 0
        while active:
            if self.rng.random() < 0.5:
                self.step_units()
            g = self.rng.choice(active)
            try:
                next(g)
            except StopIteration:
                active.remove(g)
            steps += 1
            if steps > STEP_CAP:
                return "deadlock"
        # every role has passed the final __syncthreads: tensor memory is freed
        if self.tma or self.tp:
            return f"in flight at exit: {len(self.tma)} loads, {len(self.tp)} tensor-pipe ops"
        return "ok"


# ----------------------------------------------------------------- K-block ring

def gemm_ring(seed, nkb, nst, p_timeout, rules="kernel", style="ring"):
    """The issuing thread of the tensor-core GEMMs.  style "ring" (the
    mapper's GEMM): loads of the first nst K blocks, then for each K block:
    wait for its stage, MMAs, commit onto the stage's done barrier, and (the
    stage free again) the load of K block i + nst.  style "lockstep" (the
    BF16 Gram kernel, two stages): for each K block, wait until its stage is
    free, load it, wait for it, MMAs, commit.  Then the wait for the last
    commit."""
    rng = random.Random(seed)
    S = Sim(rng, p_timeout)
    full = [Bar(1) for _ in range(nst)]
    done = [Bar(1) for _ in range(nst)]
    drain = Bar(1)
    stage = [None] * nst                      # K block held by each stage
    readers = [0] * nst                       # MMAs queued on each stage
    acc = []                                  # K blocks accumulated, in order
    counted = [False]

    def load(i):
        s = i % nst
        if readers[s]:
            S.hazard(f"load of K block {i} into stage {s} while an MMA still reads it")
        full[s].expect_tx(1)

        def land(s=s, i=i):
            stage[s] = i
        S.issue_tma(full[s], 1, land)

    def mma(i):
        s = i % nst
        readers[s] += 1

        def execute(s=s, i=i):
            readers[s] -= 1
            if stage[s] != i:
                S.hazard(f"MMA of K block {i} read stage {s} holding {stage[s]}")
            acc.append(i)
        S.issue_mma(execute)

    def thread_lockstep():
        ok, issued = True, 0
        for i in range(nkb):
            s = i % nst
            if i >= nst:
                ok_i = yield from S.wait_alone(done[s], ((i - nst) // nst) & 1)
                if not ok_i:
                    ok = False
                    if rules != "continue":
                        break
            load(i)
            issued = i + 1
            ok_i = yield from S.wait_alone(full[s], (i // nst) & 1)
            if not ok_i:
                ok = False
                if rules != "continue":
                    break
            mma(i)
            S.commit(done[s])
        yield from finish(ok, issued)

    def finish(ok, issued):
        last = nkb - 1
        if ok or rules == "continue":
            ok = (yield from S.wait_alone(done[last % nst], (last // nst) & 1)) and ok
        if not ok:
            counted[0] = True
            if rules in ("kernel", "drain_loads_only"):
                for i in range(max(0, issued - nst), issued):
                    yield from S.drain_wait(full[i % nst], (i // nst) & 1)
            if rules == "kernel":
                S.commit(drain)
                yield from S.drain_wait(drain, 0)

    def thread():
        ok, issued = True, 0
        for i in range(min(nst, nkb)):
            load(i)
            issued = i + 1
        for i in range(nkb):
            s, par = i % nst, (i // nst) & 1
            ok_i = yield from S.wait_alone(full[s], par)
            if not ok_i:
                ok = False
                if rules != "continue":
                    break
            mma(i)
            S.commit(done[s])
            if i + nst < nkb:
                ok_i = yield from S.wait_alone(done[s], par)
                if not ok_i:
                    ok = False
                    if rules != "continue":
                        break
                load(i + nst)
                issued = i + nst + 1
        yield from finish(ok, issued)

    try:
        r = S.run([thread() if style == "ring" else thread_lockstep()])
    except Hazard as h:
        return f"hazard: {h}"
    if r != "ok":
        return r
    if counted[0] != S.timed_out:
        return "timeout not counted"
    if S.timed_out:
        return "ok (timed out)"
    if acc != list(range(nkb)):
        return f"accumulated {acc}"
    return "ok"


@pytest.mark.parametrize("style", ["ring", "lockstep"])
@pytest.mark.parametrize("nkb,nst", [(1, 1), (2, 2), (5, 2), (13, 2), (4, 3), (16, 3), (64, 2)])
def test_gemm_ring_without_timeouts(nkb, nst, style):
    for seed in range(20):
        assert gemm_ring(seed, nkb, nst, 0.0, style=style) == "ok"


@pytest.mark.parametrize("style", ["ring", "lockstep"])
@pytest.mark.parametrize("nkb,nst", [(1, 1), (2, 2), (5, 2), (13, 2), (16, 3)])
def test_gemm_ring_timeouts_leave_nothing_in_flight(nkb, nst, style):
    results = [gemm_ring(seed, nkb, nst, 0.3, style=style) for seed in range(300)]
    assert set(results) <= {"ok", "ok (timed out)"}, set(results)
    assert "ok (timed out)" in results


@pytest.mark.parametrize("style", ["ring", "lockstep"])
@pytest.mark.parametrize("rules", ["continue", "drain_loads_only", "no_drain"])
def test_gemm_ring_weaker_timeout_handling_is_caught(rules, style):
    # "continue": the former form (a wait that ran out was counted and the
    # loop went on issuing loads and MMAs); "drain_loads_only": waits for the
    # loads but not for the MMAs; "no_drain": exits at once
    results = {gemm_ring(seed, 13, 2, 0.3, rules, style) for seed in range(400)}
    assert results != {"ok"}, rules


# ---------------------------------------------------------- fused inference

E = 4          # epilogue warps in the model: warp e takes accumulator column group e
LOADERS = 2
W2ST = 4


def infer(seed, ntl, p_timeout, rules="kernel"):
    rng = random.Random(seed)
    S = Sim(rng, p_timeout)
    W1b = Bar(1)
    XF = [Bar(LOADERS), Bar(LOADERS)]
    WF = [Bar(1) for _ in range(W2ST)]
    WE = [Bar(1) for _ in range(W2ST)]
    M1 = [Bar(1), Bar(1)]
    M2 = [Bar(1), Bar(1)]
    H1R = Bar(E)
    AF = [Bar(E), Bar(E)]
    DR = Bar(1)
    nuse = 8 * ntl

    st = {"w1": False, "y": set()}
    # content and outstanding readers of each buffer
    X = [[None] * LOADERS for _ in range(2)]          # tile written by each loader
    X_writing = [[False] * LOADERS for _ in range(2)]
    X_readers = [0, 0]                                # queued layer-1 MMAs
    X_used = {}                                       # tile -> read by its MMA
    H1 = [None] * E                                   # tile of each K block (column group)
    H1_writing = [False] * E
    H1_readers = [0] * E
    W2 = [None] * W2ST
    W2_readers = [0] * W2ST
    # accumulator b, column group e: (tag, consumed)
    ACC = [[[None, True] for _ in range(E)] for _ in range(2)]
    L2k = [[0, 0], [0, 0]]                            # K blocks of layer 2 done per half

    def load_w1():
        W1b.expect_tx(1)
        S.issue_tma(W1b, 1, lambda: st.__setitem__("w1", True))

    def load_w2(u):
        s = u % W2ST
        if W2_readers[s]:
            S.hazard(f"W2 box {u} loaded into stage {s} while an MMA reads it")
        WF[s].expect_tx(1)

        def land(s=s, u=u):
            W2[s] = u
        S.issue_tma(WF[s], 1, land)

    def overwrite_acc(b, groups, tag):
        for e in groups:
            if not ACC[b][e][1]:
                S.hazard(f"{tag} overwrote accumulator {b} group {e} holding unread {ACC[b][e][0]}")

    def mma1(j, b):
        X_readers[b] += 1

        def execute():
            X_readers[b] -= 1
            X_used[j] = True
            if not st["w1"]:
                S.hazard("layer 1 ran before W1 landed")
            if any(X[b][w] != j for w in range(LOADERS)) or any(X_writing[b]):
                S.hazard(f"layer 1 of tile {j} read X stage {b} holding {X[b]}")
            overwrite_acc(b, range(E), f"layer 1 of tile {j}")
            for e in range(E):
                ACC[b][e] = [("L1", j), False]
            L2k[b] = [0, 0]
        S.issue_mma(execute)

    def mma2(j, b, h, kb, u):
        s = u % W2ST
        W2_readers[s] += 1
        H1_readers[kb] += 1

        def execute():
            W2_readers[s] -= 1
            H1_readers[kb] -= 1
            if W2[s] != u:
                S.hazard(f"layer 2 box {u} read W2 stage {s} holding {W2[s]}")
            if H1[kb] != j or H1_writing[kb]:
                S.hazard(f"layer 2 of tile {j} read H1 block {kb} holding {H1[kb]}")
            groups = (2 * h, 2 * h + 1)
            if kb == 0:
                overwrite_acc(b, groups, f"layer 2 of tile {j}")
                for e in groups:
                    ACC[b][e] = [("L2p", j), True]
            L2k[b][h] += 1
            if L2k[b][h] == 4:
                for e in groups:
                    ACC[b][e] = [("L2", j), False]
        S.issue_mma(execute)

    def mma_thread():
        if ntl == 0:
            return
        w2_issued = 0
        load_w1()
        for u in range(min(W2ST, nuse)):
            load_w2(u)
            w2_issued = u + 1
        mma1_tiles = mma2_tiles = 0
        for j in range(ntl):
            b = j & 1
            if not (yield from S.wait(XF[b], (j >> 1) & 1)):
                break
            if rules != "mma_no_acc_wait" and not (yield from S.wait(AF[b], ((j >> 1) & 1) ^ 1)):
                break
            if j == 0 and not (yield from S.wait(W1b, 0)):
                break
            mma1(j, b)
            S.commit(M1[b])
            mma1_tiles = j + 1
            if not (yield from S.wait(H1R, j & 1)):
                break
            ok = True
            for h in range(2):
                for kb in range(4):
                    u = 8 * j + 4 * h + kb
                    s = u % W2ST
                    if not (yield from S.wait(WF[s], (u // W2ST) & 1)):
                        ok = False
                        break
                    mma2(j, b, h, kb, u)
                    S.commit(WE[s])
                    if u >= 1 and u + W2ST - 1 < nuse:
                        v = u - 1
                        if not (yield from S.wait(WE[v % W2ST], (v // W2ST) & 1)):
                            ok = False
                            break
                        load_w2(u + W2ST - 1)
                        w2_issued = u + W2ST
                if not ok:
                    break
            if not ok:
                break
            S.commit(M2[b])
            mma2_tiles = j + 1
        if rules in ("kernel", "loader_no_wait", "epi_no_h1_wait", "epi_early_h1_arrive", "mma_no_acc_wait"):
            yield from S.drain_wait(W1b, 0)
            for u in range(max(0, w2_issued - W2ST), w2_issued):
                yield from S.drain_wait(WF[u % W2ST], (u // W2ST) & 1)
            S.commit(DR)
            yield from S.drain_wait(DR, 0)
        elif rules == "former_drain" and S.fail:
            # waited for the loads and the last complete tile's commits only,
            # and only when this thread saw the failure
            yield from S.drain_wait(W1b, 0)
            for u in range(max(0, w2_issued - W2ST), w2_issued):
                yield from S.drain_wait(WF[u % W2ST], (u // W2ST) & 1)
            if mma1_tiles:
                t = mma1_tiles - 1
                yield from S.drain_wait(M1[t & 1], (t >> 1) & 1)
            if mma2_tiles:
                t = mma2_tiles - 1
                yield from S.drain_wait(M2[t & 1], (t >> 1) & 1)

    def loader(lw):
        for j in range(ntl):
            b = j & 1
            if j >= 2 and rules != "loader_no_wait":
                if not (yield from S.wait(M1[b], ((j >> 1) & 1) ^ 1)):
                    break
            if X_readers[b] or (X[b][lw] is not None and not X_used.get(X[b][lw], False)):
                S.hazard(f"loader {lw} overwrote X stage {b} (tile {X[b][lw]}) before layer 1 read it")
            X_writing[b][lw] = True
            for _ in range(rng.randint(0, 3)):
                yield
            X[b][lw] = j
            X_writing[b][lw] = False
            XF[b].arrive()

    def read_acc(b, e, tag):
        if ACC[b][e][0] != tag:
            S.hazard(f"epilogue read accumulator {b} group {e} holding {ACC[b][e][0]}, not {tag}")
        ACC[b][e][1] = True

    def epilogue(e):
        for j in range(ntl + 1):
            if j < ntl:
                b = j & 1
                ok = yield from S.wait(M1[b], (j >> 1) & 1)
                if ok and j >= 1 and rules != "epi_no_h1_wait":
                    ok = yield from S.wait(M2[(j - 1) & 1], ((j - 1) >> 1) & 1)
                if rules == "epi_early_h1_arrive":
                    H1R.arrive()
                for _ in range(rng.randint(0, 8)):   # the epilogue's arithmetic takes a while
                    yield
                if ok:
                    read_acc(b, e, ("L1", j))
                    if H1_readers[e]:
                        S.hazard(f"H1 block {e} written for tile {j} while layer 2 reads it")
                    H1_writing[e] = True
                    for _ in range(rng.randint(0, 3)):
                        yield
                    H1[e] = j
                    H1_writing[e] = False
                if rules != "epi_early_h1_arrive":
                    H1R.arrive()
            if j >= 1:
                t = j - 1
                b = t & 1
                ok = yield from S.wait(M2[b], (t >> 1) & 1)
                for _ in range(rng.randint(0, 8)):
                    yield
                if ok:
                    read_acc(b, e, ("L2", t))
                AF[b].arrive()
                yield from S.named_barrier("epi", E)
                if ok and e == 0:
                    st["y"].add(t)

    roles = [mma_thread()] + [loader(w) for w in range(LOADERS)] + [epilogue(e) for e in range(E)]
    try:
        r = S.run(roles)
    except Hazard as h:
        return f"hazard: {h}"
    if r != "ok":
        return r
    if S.timed_out != S.fail:
        return "failure flag without a timeout"
    if S.fail:
        return "ok (timed out)"   # counted: the kernel's thread 0 adds the flag to the timeout count
    if st["y"] != set(range(ntl)):
        return f"outputs of tiles {sorted(st['y'])} of {ntl}"
    return "ok"


@pytest.mark.parametrize("ntl", [0, 1, 2, 3, 7])
def test_inference_pipeline_without_timeouts(ntl):
    for seed in range(40):
        assert infer(seed, ntl, 0.0) == "ok", seed


@pytest.mark.parametrize("ntl,p", [(1, 0.15), (2, 0.15), (3, 0.03), (3, 0.15), (6, 0.02)])
def test_inference_timeouts_leave_nothing_in_flight(ntl, p):
    results = [infer(seed, ntl, p) for seed in range(600)]
    assert set(results) <= {"ok", "ok (timed out)"}, set(results)
    assert "ok (timed out)" in results


@pytest.mark.parametrize("rules", ["former_drain", "no_drain"])
def test_inference_weaker_drains_are_caught(rules):
    # rare timeouts: the failure comes late, with layer-2 MMAs queued
    results = {infer(seed, 3, 0.03, rules) for seed in range(1500)}
    assert any(r.startswith("in flight at exit") for r in results), (rules, results)


@pytest.mark.parametrize("rules", ["loader_no_wait", "epi_early_h1_arrive", "mma_no_acc_wait"])
def test_inference_missing_waits_are_caught(rules):
    results = {infer(seed, 5, 0.0, rules) for seed in range(200)}
    assert results != {"ok"}, rules


def test_layer1_commit_covers_the_previous_layer2():
    """The layer-1 epilogue of tile j also waits for layer 2 of tile j - 1
    (whose MMAs read H1) before writing H1.  The wait is implied: a commit
    tracks every MMA the thread issued before it, and layer 1 of tile j is
    issued after layer 2 of tile j - 1, so its commit arrives only after
    those MMAs are done.  Without that wait the model stays clean."""
    for seed in range(200):
        assert infer(seed, 5, 0.0, "epi_no_h1_wait") == "ok", seed
