"""Affinities from precomputed dissimilarities (graph shortest-path lengths,
unsquared Euclidean distances) against the FP64 oracle, and one gradient
step on the resulting P."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth

from parity import GRAD_TOL, P_TOL, chunk_blocks, p_error, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _graph_distances(n, seed):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    rng = np.random.default_rng(seed)
    W = np.zeros((n, n))
    for i in range(n):
        W[i, (i + 1) % n] = rng.uniform(0.5, 2.0)
    for _ in range(4 * n):
        i, j = rng.integers(0, n, 2)
        if i != j:
            W[i, j] = rng.uniform(0.5, 4.0)
    return shortest_path(csr_matrix(W), directed=False).astype(np.float32)


@pytest.mark.parametrize("kind,schedule", [("graph", "batched"), ("graph", "per_chunk"), ("euclid", "batched")])
def test_affinities_from_distances_match_oracle(dev, kind, schedule):
    from paper_1812_09869_gb300 import ptsne
    if kind == "graph":
        n = 900
        D = _graph_distances(n, 50)
        off = np.array([0, 300, 577, 900])
    else:
        n = 3000
        X, _ = synth.gaussian_mixture(n, 20, 6, seed=51, anisotropic=True)
        D = np.sqrt(np.maximum(O.sqdist(X), 0.0)).astype(np.float32)
        off = np.array([0, 1000, 2131, 3000])
    perm = synth.permutations(n, 1, seed=52)[0]
    Y0 = synth.init_disk(n, seed=53)
    cfg = ptsne.Config(n=n, d=1, offsets=off, perplexity=20.0, iters=1, schedule=schedule)
    with ptsne.Context(cfg) as ctx:
        Dd = torch.from_numpy(D).to(dev)
        pd = torch.from_numpy(perm).to(dev)
        Pd = torch.zeros(int((np.diff(off) ** 2).sum()), dtype=torch.float32, device=dev)
        bd = torch.zeros(n, dtype=torch.float32, device=dev)
        ctx.affinities_from_distances(Dd, pd, P_out=Pd, beta_out=bd)
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        gd = torch.zeros_like(Yd)
        ctx.step(pd, Yd, grad_out=gd)
        torch.cuda.synchronize()
        st = ctx.stats()
        blocks = chunk_blocks(Pd.cpu().numpy(), off)
        beta = bd.cpu().numpy().astype(np.float64)
        g = gd.cpu().numpy()
    assert st.bisect_failed_rows == 0 and st.nonfinite_inputs == 0
    for c in range(len(off) - 1):
        idx = perm[off[c]:off[c + 1]]
        Pr, br, bad = O.affinities_from_distances(D[np.ix_(idx, idx)], 20.0)
        assert bad == 0
        assert p_error(blocks[c], Pr) <= P_TOL, (c, p_error(blocks[c], Pr))
        assert np.abs(beta[idx] - br).max() <= 1e-4 * br.max()
        gr, _ = O.gradient(Pr, Y0[idx])
        assert rel_max(g[idx], gr) <= GRAD_TOL


def test_nonfinite_dissimilarities_are_counted(dev):
    from paper_1812_09869_gb300 import ptsne
    n = 400
    D = _graph_distances(n, 54)
    D[3, 7] = np.inf
    D[10, 11] = np.nan
    off = np.array([0, 200, 400])
    perm = synth.permutations(n, 1, seed=55)[0]
    with ptsne.Context(ptsne.Config(n=n, d=1, offsets=off, perplexity=10.0, iters=1)) as ctx:
        ctx.affinities_from_distances(torch.from_numpy(D).to(dev), torch.from_numpy(perm).to(dev))
        st = ctx.stats()
    pos = np.argsort(perm)                   # position of each point in the partition
    same = lambda a, b: np.searchsorted(off, pos[a], side="right") == np.searchsorted(off, pos[b], side="right")
    expect = int(same(3, 7)) + int(same(10, 11))
    assert st.nonfinite_inputs == expect
