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
    assert 0 < st.window_pairs < int((np.diff(off) ** 2).sum())
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
