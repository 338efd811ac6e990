"""The graph-captured epoch of ptsne_run against plain launches: same maps,
same costs, same kernel count, and a new capture whenever an input that the
graph holds (X, Y, tuning, cost request) changes."""
import numpy as np
import pytest

from paper_1812_09869_gb300 import synth

from parity import rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _setup(n=12000, d=24, chunks=7, epochs=2):
    X, _ = synth.gaussian_mixture(n, d, 9, seed=95, anisotropic=True)
    off = synth.uniform_chunk_offsets(n, 1000, 2500, seed=96)
    perms = synth.permutations(n, epochs, seed=97)
    Y0 = synth.init_gaussian(n, 2, 1e-4, seed=98)
    return X, off, perms, Y0


def _run(dev, X, off, perms, Y0, use_graph, schedule="batched", precision="fp32", Yd=None, tuning=None):
    from paper_1812_09869_gb300 import ptsne
    cfg = ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, perplexity=30.0, iters=5, schedule=schedule,
                       precision=precision, use_graph=use_graph)
    with ptsne.Context(cfg) as ctx:
        if tuning:
            ctx.set_tuning(*tuning)
        Yd = torch.from_numpy(Y0.copy()).to(dev) if Yd is None else Yd
        cost = np.zeros((perms.shape[0], 3))
        ctx.run(torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev), perms.shape[0], Yd, cost_out=cost)
        torch.cuda.synchronize()
        return Yd.cpu().numpy(), cost, ctx.stats().kernel_launches


@pytest.mark.parametrize("schedule,precision", [("batched", "fp32"), ("batched", "bf16_window"),
                                                ("per_chunk", "fp32")])
def test_graph_epochs_match_plain_launches(dev, schedule, precision):
    X, off, perms, Y0 = _setup()
    Yg, cg, lg = _run(dev, X, off, perms, Y0, 1, schedule, precision)
    Ye, ce, le = _run(dev, X, off, perms, Y0, 0, schedule, precision)
    assert rel_max(Yg - Y0, Ye - Y0) <= 1e-4
    assert np.abs(cg - ce).max() <= 1e-5 * np.abs(ce).max()
    assert lg == le > 0


def test_graph_is_recaptured_when_its_inputs_change(dev):
    from paper_1812_09869_gb300 import ptsne
    X, off, perms, Y0 = _setup(epochs=1)
    cfg = ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, perplexity=30.0, iters=5, use_graph=1)
    Xd, Pd = torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev)
    with ptsne.Context(cfg) as ctx:
        outs = []
        for k, tun in enumerate([None, None, (1, 1, 16)]):
            if tun:
                ctx.set_tuning(*tun)
            Yd = torch.from_numpy(Y0.copy()).to(dev)      # a new Y buffer each time
            cost = np.zeros((1, 3)) if k != 1 else None    # cost request toggles too
            ctx.run(Xd, Pd, 1, Yd, cost_out=cost)
            torch.cuda.synchronize()
            outs.append(Yd.cpu().numpy())
    Ye, _, _ = _run(dev, X, off, perms, Y0, 0)
    for Y in outs:
        assert rel_max(Y - Y0, Ye - Y0) <= 1e-4


def test_profiled_graph_records_stage_times(dev):
    from paper_1812_09869_gb300 import ptsne
    X, off, perms, Y0 = _setup(epochs=2)
    cfg = ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, perplexity=30.0, iters=5, use_graph=1)
    with ptsne.Context(cfg) as ctx:
        ctx.set_profiling(True)
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        cost = np.zeros((2, 3))
        ctx.run(torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev), 2, Yd, cost_out=cost)
        torch.cuda.synchronize()
        st = ctx.stats()
    ms = dict(zip(ptsne.STAGES, st.stage_ms))
    calls = dict(zip(ptsne.STAGES, st.stage_calls))
    assert calls["iterate"] == 2 and ms["iterate"] > 0 and ms["distances"] > 0 and ms["perplexity"] > 0
    Ye, ce, _ = _run(dev, X, off, perms, Y0, 0)
    assert rel_max(Yd.cpu().numpy() - Y0, Ye - Y0) <= 1e-4
    assert np.abs(cost - ce).max() <= 1e-5 * np.abs(ce).max()


def test_identical_runs_give_identical_maps(dev):
    """Each epoch's perplexity search starts from the previous epoch's
    precisions, but every ptsne_run call starts cold: two identical
    multi-epoch calls on one context produce the same map, up to the
    floating-point order of the shared-memory accumulation."""
    from paper_1812_09869_gb300 import ptsne
    X, off, perms, Y0 = _setup(epochs=3)
    cfg = ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, perplexity=30.0, iters=5,
                       precision="bf16_window")
    Xd, Pd = torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev)
    with ptsne.Context(cfg) as ctx:
        outs = []
        for _ in range(2):
            Yd = torch.from_numpy(Y0.copy()).to(dev)
            cost = np.zeros((3, 3))
            ctx.run(Xd, Pd, 3, Yd, cost_out=cost)
            torch.cuda.synchronize()
            outs.append((Yd.cpu().numpy(), cost.copy()))
            st = ctx.stats()
            assert st.bisect_failed_rows == 0
    assert rel_max(outs[0][0] - Y0, outs[1][0] - Y0) <= 1e-5
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-6 * np.abs(outs[0][1]).max()


@pytest.mark.parametrize("tuning", [(2, 1, 16), (1, 1, 12), (4, 1, 16)])
def test_deterministic_runs_are_bitwise_identical(dev, tuning):
    """With fixed-point accumulation (ptsne_set_deterministic) two identical
    multi-epoch runs give the same map and costs bit for bit, in either
    launch shape, and agree with the FP32-atomic kernel to its tolerance."""
    from paper_1812_09869_gb300 import ptsne
    X, off, perms, Y0 = _setup(epochs=3)
    cfg = ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, perplexity=30.0, iters=5,
                       precision="bf16_window")
    Xd, Pd = torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev)
    outs = []
    with ptsne.Context(cfg) as ctx:
        ctx.set_tuning(*tuning)
        for det in (True, True, False):
            ctx.set_deterministic(det)
            Yd = torch.from_numpy(Y0.copy()).to(dev)
            cost = np.zeros((3, 3))
            ctx.run(Xd, Pd, 3, Yd, cost_out=cost)
            torch.cuda.synchronize()
            outs.append((Yd.cpu().numpy(), cost.copy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert rel_max(outs[0][0] - Y0, outs[2][0] - Y0) <= 1e-4
    assert np.abs(outs[0][1] - outs[2][1]).max() <= 1e-5 * np.abs(outs[2][1]).max()


def test_deterministic_mode_limits():
    """ptsne_set_deterministic refuses a chunk too large for the fixed-point
    accumulators of the batched kernel: on one block per chunk a 6000-point
    chunk does not fit; on a cluster of 2 or 4 blocks each block holds only
    its own rows' sums, and it does.  A tuning change that would no longer
    fit is refused while the mode is on; the per-chunk schedule takes any
    chunk.  (No GPU work is done.)"""
    from paper_1812_09869_gb300 import ptsne
    cfg = ptsne.Config(n=6000, d=4, offsets=np.array([0, 6000]), perplexity=30.0, iters=1, schedule="batched")
    with ptsne.Context(cfg) as ctx:
        for cluster, ok in ((1, False), (2, True), (4, True)):
            ctx.set_deterministic(False)
            ctx.set_tuning(cluster, 1, 16)
            if ok:
                ctx.set_deterministic(True)
            else:
                with pytest.raises(ptsne.PtsneError):
                    ctx.set_deterministic(True)
        ctx.set_deterministic(False)
        ctx.set_tuning(2, 1, 16)
        ctx.set_deterministic(True)
        with pytest.raises(ptsne.PtsneError):
            ctx.set_tuning(1, 1, 16)
        assert ctx.tuning()[0] == 2
        ctx.set_deterministic(False)
    cfg = ptsne.Config(n=6000, d=4, offsets=np.array([0, 6000]), perplexity=30.0, iters=1, schedule="per_chunk")
    with ptsne.Context(cfg) as ctx:
        ctx.set_deterministic(True)
        ctx.set_deterministic(False)