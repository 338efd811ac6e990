"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Sizes are small enough for the oracle to finish in seconds while spanning
several 64 x 64 tiles and ragged tails (chunk sizes and dimensions that are
not multiples of the tile or of 4), plus degenerate small chunks.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth

from parity import GRAD_TOL, KL_TOL, P_TOL, chunk_blocks, p_error, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _ctx(X, off, **kw):
    from paper_1812_09869_gb300 import ptsne
    cfg = ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, **kw)
    return ptsne.Context(cfg)


def _gpu_affinities(dev, X, perm, off, **kw):
    ctx = _ctx(X, off, **kw)
    z2 = int((np.diff(off) ** 2).sum())
    Xd = torch.from_numpy(X).to(dev)
    pd = torch.from_numpy(perm).to(dev)
    Pd = torch.zeros(z2, dtype=torch.float32, device=dev)
    bd = torch.zeros(X.shape[0], dtype=torch.float32, device=dev)
    ctx.affinities(Xd, pd, P_out=Pd, beta_out=bd)
    torch.cuda.synchronize()
    return ctx, Xd, pd, chunk_blocks(Pd.cpu().numpy(), off), bd.cpu().numpy().astype(np.float64)


def _check_affinities(dev, X, perm, off, perp, **kw):
    ctx, _, _, blocks, beta = _gpu_affinities(dev, X, perm, off, perplexity=perp, **kw)
    st = ctx.stats()
    assert st.bisect_failed_rows == 0
    worst = 0.0
    for c in range(len(off) - 1):
        idx = perm[off[c]:off[c + 1]]
        Pr, br, bad = O.affinities(X[idx], perp)
        assert bad == 0
        Pg = blocks[c]
        assert np.array_equal(Pg, Pg.T), "GPU P must be exactly symmetric"
        assert np.all(np.diag(Pg) == 0)
        worst = max(worst, p_error(Pg, Pr))
        assert np.abs(beta[idx] - br).max() <= 1e-4 * br.max()
        assert abs(Pg.sum() - 1.0) < 1e-4
    assert worst <= P_TOL, worst
    ctx.close()
    return worst


def test_affinities_single_chunk_2000x10(dev):
    w = synth.workload("plain-2000x10")
    _check_affinities(dev, w.X, w.perms[0], w.offsets, 30.0)


@pytest.mark.parametrize("schedule", ["batched", "per_chunk"])
def test_affinities_ragged_chunks(dev, schedule):
    X, _ = synth.gaussian_mixture(3000, 37, 6, seed=31, anisotropic=True)
    off = np.array([0, 700, 1777, 3000])
    perm = synth.permutations(3000, 1, seed=32)[0]
    _check_affinities(dev, X, perm, off, 25.0, schedule=schedule)


def test_affinities_tiny_and_degenerate_chunks(dev):
    X, _ = synth.gaussian_mixture(314, 3, 3, seed=33)
    off = np.array([0, 5, 22, 55, 119, 184, 314])   # z = 5, 17, 33, 64, 65, 130
    perm = synth.permutations(314, 1, seed=34)[0]
    _check_affinities(dev, X, perm, off, 3.0)


def test_affinities_with_duplicate_points(dev):
    """Exact duplicates give zero distances; the search must still converge."""
    X, _ = synth.gaussian_mixture(400, 6, 2, seed=35)
    X[100:110] = X[0]
    perm = np.arange(400, dtype=np.int32)
    _check_affinities(dev, X, perm, np.array([0, 400]), 20.0)


def _step(dev, X, perm, off, Y0, **kw):
    ctx, Xd, pd, blocks, _ = _gpu_affinities(dev, X, perm, off, **kw)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    gd = torch.zeros_like(Yd)
    Zd = torch.zeros(len(off) - 1, dtype=torch.float64, device=dev)
    ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
    torch.cuda.synchronize()
    ctx.close()
    return Yd.cpu().numpy(), gd.cpu().numpy(), Zd.cpu().numpy()


def test_gradient_after_one_step_2000x10(dev):
    w = synth.workload("plain-2000x10")
    perm, off = w.perms[0], w.offsets
    Y1, g, Z = _step(dev, w.X, perm, off, w.Y0, perplexity=30.0)
    idx = perm
    Pr, _, _ = O.affinities(w.X[idx], 30.0)
    gr, Zr = O.gradient(Pr, w.Y0[idx])
    assert rel_max(g[idx], gr) <= GRAD_TOL
    assert abs(Z[0] - Zr) <= 1e-6 * Zr
    Yr = w.Y0[idx].astype(np.float64).copy()
    vel, gains = np.zeros_like(Yr), np.ones_like(Yr)
    O.update(Yr, vel, gains, gr, lr=200.0, momentum=0.5)
    assert rel_max(Y1[idx] - w.Y0[idx], Yr - w.Y0[idx]) <= GRAD_TOL


@pytest.mark.parametrize("schedule", ["batched", "per_chunk"])
def test_step_three_dims_paper_lr_no_gains(dev, schedule):
    X, _ = synth.gaussian_mixture(900, 12, 5, seed=36)
    off = np.array([0, 333, 900])
    perm = synth.permutations(900, 1, seed=37)[0]
    Y0 = synth.init_gaussian(900, 3, 1.0, seed=38)
    Y1, g, Z = _step(dev, X, perm, off, Y0, perplexity=15.0, out_dim=3, lr_mode=1, use_gains=0,
                     schedule=schedule)
    for c in range(2):
        idx = perm[off[c]:off[c + 1]]
        Pr, _, _ = O.affinities(X[idx], 15.0)
        gr, Zr = O.gradient(Pr, Y0[idx])
        assert rel_max(g[idx], gr) <= GRAD_TOL
        assert abs(Z[c] - Zr) <= 1e-6 * Zr
        Yr = Y0[idx].astype(np.float64).copy()
        O.update(Yr, np.zeros_like(Yr), np.ones_like(Yr), gr, momentum=0.5, lr_mode=1, use_gains=0)
        assert rel_max(Y1[idx] - Y0[idx], Yr - Y0[idx]) <= GRAD_TOL


@pytest.mark.parametrize("tuning,det", [((2, 1, 20), False), ((1, 1, 12), False), ((2, 1, 20), True),
                                        ((4, 1, 20), True), ((1, 1, 12), True)])
def test_three_dims_every_build_gradient_and_cost(dev, tuning, det):
    """3-D maps through both builds of the batched kernel for 3-D (more and
    fewer than 18 warps): one step's gradient and Z, and the cost
    (Eq. 5, Eq. 9), against the oracle; two chunks with ragged last blocks."""
    X, _ = synth.gaussian_mixture(1300, 10, 4, seed=60)
    off = np.array([0, 610, 1300])     # 20 and 22 row blocks, both ragged
    perm = synth.permutations(1300, 1, seed=61)[0]
    Y0 = synth.init_gaussian(1300, 3, 2.0, seed=62)
    ctx, Xd, pd, _, _ = _gpu_affinities(dev, X, perm, off, perplexity=12.0, out_dim=3)
    ctx.set_tuning(*tuning)
    ctx.set_deterministic(det)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    cost = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.cost(pd, Yd, cost)
    gd = torch.zeros_like(Yd)
    Zd = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
    torch.cuda.synchronize()
    assert ctx.stats().wait_timeouts == 0
    ctx.close()
    g, Z = gd.cpu().numpy(), Zd.cpu().numpy()
    kl, nc = cost.cpu().numpy()
    kl_r = nc_r = 0.0
    for c in range(2):
        idx = perm[off[c]:off[c + 1]]
        Pr, _, _ = O.affinities(X[idx], 12.0)
        gr, Zr = O.gradient(Pr, Y0[idx])
        assert rel_max(g[idx], gr) <= GRAD_TOL, (c, rel_max(g[idx], gr))
        assert abs(Z[c] - Zr) <= 1e-6 * Zr
        kl_r += O.kl(Pr, Y0[idx]) / 2
        nc_r += O.normalized_cost(Pr, Y0[idx]) / 2
    assert abs(kl - kl_r) <= 1e-4 * abs(kl_r) and abs(nc - nc_r) <= 1e-4 * nc_r, (kl, kl_r, nc, nc_r)


def test_cost_matches_oracle(dev):
    X, _ = synth.gaussian_mixture(1500, 16, 5, seed=39)
    off = np.array([0, 640, 1500])
    perm = synth.permutations(1500, 1, seed=40)[0]
    ctx, Xd, pd, blocks, _ = _gpu_affinities(dev, X, perm, off, perplexity=20.0)
    Y = synth.init_gaussian(1500, 2, 3.0, seed=41)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.cost(pd, torch.from_numpy(Y).to(dev), out)
    kl, nc = out.cpu().numpy()
    ctx.close()
    kl_g = nc_g = kl_r = nc_r = 0.0
    for c in range(2):
        idx = perm[off[c]:off[c + 1]]
        kl_g += O.kl(blocks[c], Y[idx]) / 2
        nc_g += O.normalized_cost(blocks[c], Y[idx]) / 2
        Pr, _, _ = O.affinities(X[idx], 20.0)
        kl_r += O.kl(Pr, Y[idx]) / 2
        nc_r += O.normalized_cost(Pr, Y[idx]) / 2
    # the cost kernels on the GPU's own P: FP32 logs, FP64 sums
    assert abs(kl - kl_g) <= 1e-5 * abs(kl_g) and abs(nc - nc_g) <= 1e-5 * nc_g
    assert abs(kl - kl_r) <= 1e-4 * abs(kl_r) and abs(nc - nc_r) <= 1e-4 * nc_r


@pytest.mark.parametrize("schedule", ["batched", "per_chunk"])
def test_final_kl_within_one_percent_2000x10(dev, schedule):
    w = synth.workload("plain-2000x10")
    ctx = _ctx(w.X, w.offsets, perplexity=30.0, iters=100, schedule=schedule)
    Xd = torch.from_numpy(w.X).to(dev)
    pd = torch.from_numpy(w.perms).to(dev)
    Yd = torch.from_numpy(w.Y0.copy()).to(dev)
    cost = np.zeros((1, 3))
    rc = ctx.run(Xd, pd, 1, Yd, cost_out=cost)
    assert rc == 0
    ctx.close()
    _, cref = O.ptsne_run(w.X, w.Y0, w.perms, w.offsets, O.params(perplexity=30.0, iters=100, epochs=1))
    assert abs(cost[0, 0] - cref[0, 0]) <= KL_TOL * cref[0, 0], (cost, cref)
    assert abs(cost[0, 1] - cref[0, 1]) <= KL_TOL * cref[0, 1]


def test_multi_epoch_run_matches_oracle_cost(dev):
    X, _ = synth.gaussian_mixture(4000, 20, 8, seed=42, anisotropic=True)
    off = synth.equal_chunk_offsets(4000, 4)
    perms = synth.permutations(4000, 3, seed=43)
    Y0 = synth.init_gaussian(4000, 2, 1e-4, seed=44)
    ctx = _ctx(X, off, perplexity=30.0, iters=60)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    cost = np.zeros((3, 3))
    ctx.run(torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev), 3, Yd, cost_out=cost)
    ctx.close()
    prm = O.params(perplexity=30.0, iters=60, epochs=3)
    _, cref = O.ptsne_run(X, Y0, perms, off, prm)
    # epoch 0 is one partial t-SNE per chunk from the same start: tight match
    assert abs(cost[0, 0] - cref[0, 0]) <= 1e-3 * cref[0, 0], (cost, cref)
    # later epochs start from pooled maps; the trajectory is chaotic (a 1e-6
    # relative change of the oracle's own start map moves its epoch-2 KL by
    # ~0.5%), so the GPU must fall within the spread of an oracle ensemble over
    # such perturbed starts, widened by the 1% tolerance
    rng = np.random.default_rng(7)
    ens = [cref]
    for _ in range(3):
        _, ck = O.ptsne_run(X, Y0 * (1 + 1e-6 * rng.standard_normal(Y0.shape)), perms, off, prm)
        ens.append(ck)
    ens = np.stack(ens)
    lo, hi = ens.min(0), ens.max(0)
    kl2 = cost[:, :2]   # the third column is the embedding size (tests/test_gpu_eval.py)
    assert np.all(kl2 >= lo * (1 - KL_TOL)) and np.all(kl2 <= hi * (1 + KL_TOL)), (cost, ens)


def test_run_resumes_from_a_saved_map(dev):
    """Checkpoint and resume: the state a run carries between epochs is the
    map (and, within a context, each point's last beta as the next search's
    start).  A call's first epoch equals the first epoch of a longer call,
    and the epoch after a checkpoint is the same whether the run continues in
    its context or resumes in a fresh one from the saved map (whose searches
    start cold).  Only FP32 rounding differs (the iteration kernel's atomic
    order, the searches' starting points); the chaotic trajectory amplifies
    it to ~1% within two epochs here, so each comparison spans one epoch
    from the same map."""
    X, _ = synth.gaussian_mixture(4000, 20, 8, seed=45, anisotropic=True)
    off = synth.equal_chunk_offsets(4000, 4)
    perms = synth.permutations(4000, 4, seed=46)
    Y0 = synth.init_gaussian(4000, 2, 1e-4, seed=47)
    Xd, Pd = torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev)
    ctx = _ctx(X, off, perplexity=30.0, iters=60)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    c4 = np.zeros((4, 3))
    ctx.run(Xd, Pd, 4, Yd, cost_out=c4)
    ctx.close()
    ctx = _ctx(X, off, perplexity=30.0, iters=60)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    a, b = np.zeros((2, 3)), np.zeros((1, 3))
    ctx.run(Xd, Pd[0:2], 2, Yd, cost_out=a)
    saved = Yd.cpu().numpy().copy()                      # the checkpoint
    ctx.run(Xd, Pd[2:3], 1, Yd, cost_out=b)             # continued in its context
    ctx.close()
    ctx = _ctx(X, off, perplexity=30.0, iters=60)
    Yr = torch.from_numpy(saved).to(dev)
    r = np.zeros((1, 3))
    ctx.run(Xd, Pd[2:3], 1, Yr, cost_out=r)             # resumed in a fresh context
    ctx.close()
    assert np.allclose(a[0], c4[0], rtol=1e-3, atol=0), (a, c4)   # the map's extent moves ~1e-4
    assert np.allclose(r, b, rtol=1e-3, atol=0), (r, b)


def test_batched_iterations_equal_plain_per_chunk_form(dev):
    """The batched kernel (packed symmetric P, one launch for all iterations)
    and the plain per-chunk kernels (dense P, three launches per iteration)
    compute the same iterations, to FP32 summation-order differences."""
    X, _ = synth.gaussian_mixture(2500, 10, 4, seed=45)
    off = np.array([0, 1200, 2500])
    perm = synth.permutations(2500, 1, seed=46)
    Y0 = synth.init_gaussian(2500, 2, 1.0, seed=47)
    Xd, pd = torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev)
    out = []
    for schedule in ("batched", "per_chunk"):
        ctx = _ctx(X, off, perplexity=30.0, iters=5, schedule=schedule)
        Y = torch.from_numpy(Y0.copy()).to(dev)
        ctx.run(Xd, pd, 1, Y)
        torch.cuda.synchronize()
        ctx.close()
        out.append(Y.cpu().numpy())
    assert rel_max(out[0] - Y0, out[1] - Y0) <= 1e-4


# launch shapes of the batched kernel: blocks per chunk (cluster) x warps per block,
# both 2-D builds (at most 12 and 16 warps; more are run as 16), a single warp, and odd counts
TUNINGS = [(1, 1, 16), (2, 1, 16), (4, 1, 12), (4, 1, 8), (1, 1, 4), (1, 1, 1), (2, 1, 17), (1, 1, 19), (2, 1, 20),
           (1, 1, 20), (4, 1, 20)]


def test_invalid_launch_shapes_are_rejected(dev):
    """ptsne_set_tuning refuses shapes the kernel has no build for (a cluster
    of 3, more than one warp per tile, 0 or 22 warps) and keeps the
    previous shape."""
    from paper_1812_09869_gb300 import ptsne
    X, _ = synth.gaussian_mixture(300, 6, 3, seed=57)
    ctx = _ctx(X, np.array([0, 150, 300]), perplexity=5.0)
    ctx.set_tuning(1, 1, 12)
    for bad in [(3, 1, 16), (2, 2, 16), (2, 4, 16), (2, 1, 0), (2, 1, 22), (0, 1, 8)]:
        with pytest.raises(ptsne.PtsneError):
            ctx.set_tuning(*bad)
        assert ctx.tuning() == (1, 1, 12), bad
    ctx.close()


@pytest.mark.parametrize("tuning,det", [(t, False) for t in TUNINGS] + [((2, 1, 16), True), ((1, 1, 5), True),
                                                                   ((4, 1, 12), True)])
def test_gradient_for_every_launch_shape(dev, tuning, det):
    """Gradient, Z, updated map and cost of one step for each launch shape
    (and, det, with the fixed-point accumulators of ptsne_set_deterministic),
    on uneven chunks (an odd and an even number of 32-row blocks, a ragged
    tail, and a chunk smaller than one block) against the oracle."""
    X, _ = synth.gaussian_mixture(2100, 9, 5, seed=50, anisotropic=True)
    off = np.array([0, 1000, 1017, 2100])     # z = 1000 (32 blocks), 17 (1), 1083 (34)
    perm = synth.permutations(2100, 1, seed=51)[0]
    Y0 = synth.init_gaussian(2100, 2, 2.0, seed=52)
    ctx = _ctx(X, off, perplexity=5.0)
    ctx.set_tuning(*tuning)
    ctx.set_deterministic(det)
    assert ctx.tuning() == tuning
    Xd, pd = torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev)
    ctx.affinities(Xd, pd)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    gd = torch.zeros_like(Yd)
    Zd = torch.zeros(3, dtype=torch.float64, device=dev)
    cost = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.cost(pd, Yd, cost)
    ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
    torch.cuda.synchronize()
    assert ctx.stats().wait_timeouts == 0
    ctx.close()
    g, Z, Y1, (kl, nc) = gd.cpu().numpy(), Zd.cpu().numpy(), Yd.cpu().numpy(), cost.cpu().numpy()
    kl_r = nc_r = 0.0
    for c in range(3):
        idx = perm[off[c]:off[c + 1]]
        Pr, _, _ = O.affinities(X[idx], 5.0)
        gr, Zr = O.gradient(Pr, Y0[idx])
        assert rel_max(g[idx], gr) <= GRAD_TOL, (c, rel_max(g[idx], gr))
        assert abs(Z[c] - Zr) <= 1e-6 * Zr
        Yr = Y0[idx].astype(np.float64).copy()
        O.update(Yr, np.zeros_like(Yr), np.ones_like(Yr), gr)
        assert rel_max(Y1[idx] - Y0[idx], Yr - Y0[idx]) <= GRAD_TOL
        kl_r += O.kl(Pr, Y0[idx]) / 3
        nc_r += O.normalized_cost(Pr, Y0[idx]) / 3
    assert abs(kl - kl_r) <= 1e-4 * abs(kl_r) and abs(nc - nc_r) <= 1e-4 * nc_r


def test_run_host_equals_run_device(dev):
    w = synth.workload("plain-2000x10")
    ctx = _ctx(w.X, w.offsets, perplexity=30.0, iters=5)
    Yd = torch.from_numpy(w.Y0.copy()).to(dev)
    ctx.run(torch.from_numpy(w.X).to(dev), torch.from_numpy(w.perms).to(dev), 1, Yd)
    Yh = torch.from_numpy(w.Y0.copy()).pin_memory()
    ctx.run_host(torch.from_numpy(w.X).pin_memory(), torch.from_numpy(w.perms).pin_memory(), 1, Yh)
    ctx.close()
    # same computation on host buffers; the batched kernel merges row sums with
    # shared-memory atomics, so the two runs agree up to FP32 summation order
    assert rel_max(Yh.numpy() - w.Y0, Yd.cpu().numpy() - w.Y0) <= 1e-4


def test_errors_nonfinite_input_and_call_order(dev):
    from paper_1812_09869_gb300 import ptsne
    X, _ = synth.gaussian_mixture(300, 5, 2, seed=48)
    X[7, 2] = np.nan
    perm = synth.permutations(300, 1, seed=49)
    ctx = _ctx(X, np.array([0, 300]), perplexity=10.0, iters=2)
    with pytest.raises(ptsne.PtsneError) as e:
        ctx.step(torch.from_numpy(perm[0]).to(dev), torch.zeros(300, 2, device=dev))
    assert e.value.code == ptsne.ESTATE
    with pytest.raises(ptsne.PtsneError) as e:
        ctx.run(torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev), 1, torch.zeros(300, 2, device=dev))
    assert e.value.code == ptsne.ENONFINITE
    ctx.close()


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp32", "bf16_window"])
def test_maximum_chunk_size(dev, precision):
    """z = 8192, the largest chunk: the batched kernel's map and accumulators
    take 196 KB of shared memory, so it runs with fewer warps; P, β,
    the gradient and Z after one step still match the oracle."""
    z = 8192
    X, _ = synth.gaussian_mixture(z + 700, 16, 12, seed=80, anisotropic=True)
    off = np.array([0, 700, z + 700])                  # a small chunk and a maximal one
    perm = synth.permutations(z + 700, 1, seed=81)[0]
    Y0 = synth.init_disk(z + 700, seed=82)
    ctx, _, pd, blocks, beta = _gpu_affinities(dev, X, perm, off, perplexity=30.0, precision=precision)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    gd = torch.zeros_like(Yd)
    Zd = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.close()
    assert st.bisect_failed_rows == 0 and st.wait_timeouts == 0
    g, Z = gd.cpu().numpy(), Zd.cpu().numpy()
    for c in range(2):
        idx = perm[off[c]:off[c + 1]]
        Pr, br, bad = O.affinities(X[idx], 30.0)
        assert bad == 0
        assert p_error(blocks[c], Pr) <= P_TOL, (c, p_error(blocks[c], Pr))
        assert np.abs(beta[idx] - br).max() <= 1e-4 * br.max()
        gr, Zr = O.gradient(Pr, Y0[idx])
        assert rel_max(g[idx], gr) <= GRAD_TOL
        assert abs(Z[c] - Zr) <= 1e-6 * Zr


@pytest.mark.parametrize("precision", ["fp32", "bf16_window"])
def test_locality_order_changes_no_result(dev, precision):
    """The locality order of the rows within each chunk moves only the FP32
    summation order: P (exported in the caller's order), beta, the gradient
    and Z after one step agree with the plain order, and on clustered data it
    leaves many stored P tiles exactly zero."""
    from paper_1812_09869_gb300 import ptsne
    n, d = 6000, 20
    X, _ = synth.gaussian_mixture(n, d, 12, seed=61, anisotropic=True)
    off = synth.uniform_chunk_offsets(n, 1000, 2500, seed=62)
    perm = torch.from_numpy(synth.permutations(n, 1, seed=63)[0]).to(dev)
    Y0 = synth.init_gaussian(n, 2, 1.0, seed=64)
    Xd = torch.from_numpy(X).to(dev)
    sizes = np.diff(off)
    out = {}
    for loc in (0, 1):
        cfg = ptsne.Config(n=n, d=d, offsets=off, perplexity=30.0, iters=1, precision=precision)
        with ptsne.Context(cfg) as c:
            c.set_locality_order(bool(loc))
            Pd = torch.zeros(int((sizes ** 2).sum()), dtype=torch.float32, device=dev)
            bd = torch.zeros(n, dtype=torch.float32, device=dev)
            c.affinities(Xd, perm, P_out=Pd, beta_out=bd)
            st = c.stats()
            Yd = torch.from_numpy(Y0.copy()).to(dev)
            gd = torch.zeros_like(Yd)
            Zd = torch.zeros(len(sizes), dtype=torch.float64, device=dev)
            c.step(perm, Yd, grad_out=gd, Z_out=Zd)
            torch.cuda.synchronize()
            out[loc] = (Pd.cpu().numpy(), bd.cpu().numpy(), gd.cpu().numpy(), Zd.cpu().numpy(), Yd.cpu().numpy(),
                        st.ptiles_nonzero, st.ptiles_total)
    P0, b0, g0, Z0, Y0s, nz0, tot = out[0]
    P1, b1, g1, Z1, Y1s, nz1, tot1 = out[1]
    for a, b in zip(chunk_blocks(P1, off), chunk_blocks(P0, off)):
        assert p_error(a, b) <= P_TOL
    assert np.abs(b1 - b0).max() <= 1e-4 * b0.max()
    assert rel_max(g1, g0) <= GRAD_TOL
    assert np.abs(Z1 - Z0).max() <= 1e-6 * Z0.max()
    assert rel_max(Y1s - Y0, Y0s - Y0) <= 1e-3
    assert tot1 == tot and nz0 <= tot and nz1 < 0.8 * tot, (nz0, nz1, tot)
    # without the locality order the stored tiles are the 32 x 32 blocks on and
    # above the diagonal of each exported chunk block: the nonzero count is exact
    want_tot = want_nz = 0
    for blk in chunk_blocks(P0, off):
        z = blk.shape[0]
        t = (z + 31) // 32
        for a in range(t):
            for b in range(a, t):
                want_tot += 1
                want_nz += bool(np.any(blk[32 * a:32 * a + 32, 32 * b:32 * b + 32] != 0))
    assert (tot, nz0) == (want_tot, want_nz)
