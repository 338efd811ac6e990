"""Mixed-precision distances (BF16 tensor-core Gram matrix + FP32 window
recompute) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth

from parity import KL_TOL, P_TOL, chunk_blocks, p_error

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
    return ptsne.Context(ptsne.Config(n=X.shape[0], d=X.shape[1], offsets=off, **kw))


def _distances(dev, X, perm, off, precision):
    ctx = _ctx(X, off, perplexity=5.0, precision=precision)
    Dd = torch.zeros(int((np.diff(off) ** 2).sum()), dtype=torch.float32, device=dev)
    ctx.distances(torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev), Dd)
    torch.cuda.synchronize()
    ctx.close()
    return chunk_blocks(Dd.cpu().numpy(), off)


def test_fp32_distances_match_oracle(dev):
    X, _ = synth.gaussian_mixture(1700, 37, 5, seed=60, anisotropic=True)
    off = np.array([0, 300, 429, 1700])
    perm = synth.permutations(1700, 1, seed=61)[0]
    for c, Dg in enumerate(_distances(dev, X, perm, off, "fp32")):
        idx = perm[off[c]:off[c + 1]]
        Dr = O.sqdist(X[idx])
        mask = ~np.eye(len(idx), dtype=bool)
        assert np.abs(Dg - Dr)[mask].max() <= 1e-5 * Dr.max()
        assert np.array_equal(Dg[mask], Dg.T[mask]), "direct differences are symmetric"


@pytest.mark.parametrize("d", [50, 200, 784])   # 1, 4 and 13 blocks of 64 along K
def test_bf16_gram_distances_on_rounded_inputs(dev, d):
    """d~ equals the squared distance of the BF16-rounded rows up to the FP32
    accumulation of the tensor-core dot products."""
    if d == 784:
        X, _ = synth.sparse_images(1100, seed=62)
    else:
        X, _ = synth.gaussian_mixture(1100, d, 4, seed=62)
    off = np.array([0, 300, 429, 1100])        # 128-row tiles with ragged tails
    perm = synth.permutations(1100, 1, seed=63)[0]
    Xr = torch.from_numpy(X).bfloat16().double().numpy()
    nrm = (Xr ** 2).sum(1)
    for c, Dg in enumerate(_distances(dev, X, perm, off, "bf16_window")):
        idx = perm[off[c]:off[c + 1]]
        Dr = O.sqdist(Xr[idx])
        tol = 2e-6 * d * (nrm[idx][:, None] + nrm[idx][None, :]) + 1e-6
        mask = ~np.eye(len(idx), dtype=bool)
        assert np.all((np.abs(Dg - Dr) <= tol)[mask]), np.abs(Dg - Dr)[mask].max()


def _mixed_affinities(dev, X, perm, off, perp):
    ctx = _ctx(X, off, perplexity=perp, precision="bf16_window")
    Pd = torch.zeros(int((np.diff(off) ** 2).sum()), dtype=torch.float32, device=dev)
    bd = torch.zeros(X.shape[0], dtype=torch.float32, device=dev)
    ctx.affinities(torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev), P_out=Pd, beta_out=bd)
    st = ctx.stats()
    ctx.close()
    return chunk_blocks(Pd.cpu().numpy(), off), bd.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("schedule", ["batched", "per_chunk"])
def test_bf16_window_affinities_match_oracle(dev, schedule):
    n = 4000
    X, _ = synth.gaussian_mixture(n, 64, 12, seed=64, sizes=synth.zipf_sizes(n, 12, 1.2), anisotropic=True)
    off = np.array([0, 1000, 2437, 4000])
    perm = synth.permutations(n, 1, seed=65)[0]
    ctx_kw = dict(schedule=schedule)
    ctx = _ctx(X, off, perplexity=30.0, precision="bf16_window", **ctx_kw)
    Pd = torch.zeros(int((np.diff(off) ** 2).sum()), dtype=torch.float32, device=dev)
    bd = torch.zeros(n, dtype=torch.float32, device=dev)
    ctx.affinities(torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev), P_out=Pd, beta_out=bd)
    st = ctx.stats()
    ctx.close()
    blocks, beta = chunk_blocks(Pd.cpu().numpy(), off), bd.cpu().numpy().astype(np.float64)
    assert st.bisect_failed_rows == 0 and st.wait_timeouts == 0
    # sparse rows' candidates plus whole 64 x 64 tiles of the dense rows
    assert 0 < st.window_pairs <= 2 * int((np.diff(off) ** 2).sum())
    for c in range(3):
        idx = perm[off[c]:off[c + 1]]
        Pr, br, _ = O.affinities(X[idx], 30.0)
        assert p_error(blocks[c], Pr) <= P_TOL
        assert np.abs(beta[idx] - br).max() <= 1e-4 * br.max()


def test_bf16_window_sparse_images(dev):
    X, _ = synth.sparse_images(2000, seed=66)
    off = np.array([0, 900, 2000])
    perm = synth.permutations(2000, 1, seed=67)[0]
    blocks, beta, st = _mixed_affinities(dev, X, perm, off, 30.0)
    assert st.bisect_failed_rows == 0 and st.window_pairs > 0
    for c in range(2):
        idx = perm[off[c]:off[c + 1]]
        Pr, br, _ = O.affinities(X[idx], 30.0)
        assert p_error(blocks[c], Pr) <= P_TOL


def test_bf16_window_final_kl_2000x10(dev):
    w = synth.workload("plain-2000x10")
    ctx = _ctx(w.X, w.offsets, perplexity=30.0, iters=100, precision="bf16_window")
    Yd = torch.from_numpy(w.Y0.copy()).to(dev)
    cost = np.zeros((1, 3))
    ctx.run(torch.from_numpy(w.X).to(dev), torch.from_numpy(w.perms).to(dev), 1, Yd, cost_out=cost)
    ctx.close()
    _, cref = O.ptsne_run(w.X, w.Y0, w.perms, w.offsets, O.params(perplexity=30.0, iters=100, epochs=1))
    assert abs(cost[0, 0] - cref[0, 0]) <= KL_TOL * cref[0, 0], (cost, cref)


def _form_bins(sizes):
    zmin, zmax = int(sizes.min()), int(sizes.max())
    return np.minimum(7, (sizes - zmin) * 8 // (zmax - zmin + 1))


def test_form_choice_fp32_chunks_equal_the_fp32_context(dev):
    """Threshold < 0 puts every chunk in FP32 whole: the same distance kernel
    and the same search from the same start as a PTSNE_PREC_FP32 context, so
    P and beta are bitwise those of the FP32 context."""
    n = 3000
    X, _ = synth.gaussian_mixture(n, 50, 8, seed=90, anisotropic=True)
    off = np.array([0, 700, 1333, 3000])
    perm = synth.permutations(n, 1, seed=91)[0]
    Xd, pd = torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev)
    out = {}
    for prec, thr in (("fp32", None), ("bf16_window", -1.0)):
        ctx = _ctx(X, off, perplexity=30.0, precision=prec)
        if thr is not None:
            ctx.set_form_threshold(thr)
        Pd = torch.zeros(int((np.diff(off) ** 2).sum()), dtype=torch.float32, device=dev)
        bd = torch.zeros(n, dtype=torch.float32, device=dev)
        ctx.affinities(Xd, pd, P_out=Pd, beta_out=bd)
        out[prec] = (Pd.cpu().numpy(), bd.cpu().numpy(), ctx.stats())
        ctx.close()
    P32, b32, _ = out["fp32"]
    Pm, bm, st = out["bf16_window"]
    assert st.fp32_chunks == 3 and st.window_pairs == 0 and st.form_threshold == -1.0
    assert np.array_equal(P32, Pm) and np.array_equal(b32, bm)


@pytest.mark.parametrize("schedule", ["batched", "per_chunk"])
def test_form_choice_split_matches_oracle(dev, schedule):
    """Uneven chunks fall in different size bins with different window
    fractions; a threshold between them runs some chunks in FP32 whole and
    the others mixed.  The count of FP32 chunks follows the bins, and every
    chunk's P and beta match the FP64 oracle."""
    n = 4200
    X, _ = synth.gaussian_mixture(n, 64, 12, seed=92, sizes=synth.zipf_sizes(n, 12, 1.2), anisotropic=True)
    off = np.array([0, 200, 450, 1300, 2600, 4200])
    sizes = np.diff(off)
    perm = synth.permutations(n, 1, seed=93)[0]
    Xd, pd = torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev)
    ctx = _ctx(X, off, perplexity=30.0, precision="bf16_window", schedule=schedule)
    ctx.affinities(Xd, pd)                      # measures the bins' window fractions
    frac = np.array(ctx.stats().window_fraction)
    bins = _form_bins(sizes)
    fc = frac[bins]
    assert np.all(fc > 0) and np.all(fc <= 1.0)
    thr = float(np.sort(np.unique(fc))[len(np.unique(fc)) // 2])
    want = int((fc >= thr).sum())
    assert 0 < want < len(sizes), (fc, thr)
    ctx.set_form_threshold(thr)
    Pd = torch.zeros(int((sizes ** 2).sum()), dtype=torch.float32, device=dev)
    bd = torch.zeros(n, dtype=torch.float32, device=dev)
    ctx.affinities(Xd, pd, P_out=Pd, beta_out=bd)
    st = ctx.stats()
    ctx.close()
    assert st.fp32_chunks == want and st.bisect_failed_rows == 0
    blocks, beta = chunk_blocks(Pd.cpu().numpy(), off), bd.cpu().numpy().astype(np.float64)
    for c in range(len(sizes)):
        idx = perm[off[c]:off[c + 1]]
        Pr, br, _ = O.affinities(X[idx], 30.0)
        assert p_error(blocks[c], Pr) <= P_TOL, c
        assert np.abs(beta[idx] - br).max() <= 1e-4 * br.max(), c


def test_dense_window_tiles_in_locality_order(dev):
    """Sparse image-like rows: windows cover ~10% of a chunk, so every row is a
    dense window row and its window pairs are recomputed by whole 64 x 64
    tiles.  In locality order those pairs gather on few tiles: fewer pairs
    are recomputed than in the caller's order, and P still matches the
    oracle."""
    X, _ = synth.sparse_images(4000, seed=94)
    off = np.array([0, 1900, 4000])
    sizes = np.diff(off)
    perm = synth.permutations(4000, 1, seed=95)[0]
    Xd, pd = torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev)
    pairs = {}
    for loc in (False, True):
        ctx = _ctx(X, off, perplexity=30.0, precision="bf16_window")
        ctx.set_locality_order(loc)
        Pd = torch.zeros(int((sizes ** 2).sum()), dtype=torch.float32, device=dev)
        ctx.affinities(Xd, pd, P_out=Pd)
        st = ctx.stats()
        ctx.close()
        assert st.bisect_failed_rows == 0 and st.fp32_chunks == 0
        pairs[loc] = st.window_pairs
        blocks = chunk_blocks(Pd.cpu().numpy(), off)
        for c in range(2):
            idx = perm[off[c]:off[c + 1]]
            Pr, _, _ = O.affinities(X[idx], 30.0)
            assert p_error(blocks[c], Pr) <= P_TOL, (loc, c)
    assert pairs[True] < 0.6 * pairs[False], pairs


def test_autotune_chooses_the_form(dev):
    """ptsne_autotune on BF16_WINDOW times both forms and sets the threshold
    from them; the affinities it leaves match the oracle."""
    n = 3000
    X, _ = synth.gaussian_mixture(n, 64, 10, seed=96, anisotropic=True)
    off = np.array([0, 1000, 3000])
    perm = synth.permutations(n, 1, seed=97)[0]
    Y0 = synth.init_gaussian(n, 2, 1e-2, seed=98)
    Xd, pd = torch.from_numpy(X).to(dev), torch.from_numpy(perm).to(dev)
    ctx = _ctx(X, off, perplexity=30.0, precision="bf16_window", iters=3)
    ctx.autotune(Xd, pd, torch.from_numpy(Y0).to(dev), iters=2)
    st = ctx.stats()
    assert st.form_ms_mixed > 0 and st.form_ms_fp32 > 0 and st.form_ms_window > 0
    thr = st.form_threshold
    assert thr in (-1.0, 2.0) or 0.0 < thr <= 1.0, thr
    Pd = torch.zeros(int((np.diff(off) ** 2).sum()), dtype=torch.float32, device=dev)
    ctx.affinities(Xd, pd, P_out=Pd)
    ctx.close()
    for c, blk in enumerate(chunk_blocks(Pd.cpu().numpy(), off)):
        idx = perm[off[c]:off[c + 1]]
        Pr, _, _ = O.affinities(X[idx], 30.0)
        assert p_error(blk, Pr) <= P_TOL


def test_form_choice_inside_the_captured_epoch(dev):
    """ptsne_run replays a captured epoch graph that reads the threshold from
    device memory: with every chunk in FP32 whole, two epochs cost what the
    FP32 context's two epochs cost (the same distances and warm-started
    searches; only the iteration kernel's atomic order differs, which 100
    iterations amplify to ~1e-4 in the second epoch's map)."""
    n = 3000
    X, _ = synth.gaussian_mixture(n, 40, 6, seed=99, anisotropic=True)
    off = np.array([0, 1100, 3000])
    perms = synth.permutations(n, 2, seed=100)
    Y0 = synth.init_gaussian(n, 2, 1e-4, seed=101)
    Xd, Pd = torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev)
    out = {}
    for prec in ("fp32", "bf16_window"):
        ctx = _ctx(X, off, perplexity=30.0, iters=50, precision=prec)
        if prec == "bf16_window":
            ctx.set_form_threshold(-1.0)
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        cost = np.zeros((2, 3))
        ctx.run(Xd, Pd, 2, Yd, cost_out=cost)
        out[prec] = (cost, ctx.stats())
        ctx.close()
    c32, _ = out["fp32"]
    cm, st = out["bf16_window"]
    assert st.fp32_chunks == 2 * 2 and st.window_pairs == 0
    assert np.allclose(cm[0], c32[0], rtol=1e-4, atol=0), (cm, c32)
    assert np.allclose(cm[1], c32[1], rtol=2e-3, atol=0), (cm, c32)
