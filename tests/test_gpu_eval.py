"""Evaluation on the GPU: the embedding size that the paper monitors beside
the cost (the length of the diagonal of the map's bounding box), through
ptsne_embedding_size and through the third column of ptsne_run's per-epoch
record, against the FP64 oracle on the same maps."""
import numpy as np
import pytest

from paper_1812_09869_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# Minimum and maximum are exact, the sum of squares and the square root run
# in FP64 on both sides on the same float values: only the order of the FP64
# additions could differ (it does not), so the bar is a few ulps.
SIZE_TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _ctx(n, out_dim=2, chunk=1000, **kw):
    from paper_1812_09869_gb300 import ptsne
    nc = max(1, n // chunk)
    off = synth.equal_chunk_offsets(n, nc)
    perp = min(30.0, (n // nc) - 1.5)
    return ptsne.Context(ptsne.Config(n=n, d=4, offsets=off, perplexity=perp, out_dim=out_dim, **kw))


@pytest.mark.parametrize("rows,out_dim", [(3, 2), (257, 2), (100003, 2), (3, 3), (4099, 3), (100003, 3)])
def test_embedding_size_matches_oracle(dev, rows, out_dim):
    """Ragged row counts below, at and far above one block's 256 rows, and
    above the 608 x 256 rows one grid covers (grid-stride); two calls in a
    row reuse the context's per-block extremes and completion counter."""
    from oracle import oracle as O
    rng = np.random.default_rng(rows * 7 + out_dim)
    with _ctx(rows, out_dim, chunk=min(1000, rows)) as c:
        for call in range(2):
            Y = rng.normal(0.0, 10.0 ** (call + 1), size=(rows, out_dim)).astype(np.float32)
            Y[rng.integers(rows), rng.integers(out_dim)] = -3.0e4 * (call + 1)   # a lone extreme
            out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            c.embedding_size(torch.from_numpy(Y).to(dev), out)
            torch.cuda.synchronize()
            ref = O.embedding_size(Y.astype(np.float64))
            assert abs(out.item() - ref) <= SIZE_TOL * ref, (call, out.item(), ref)


def test_embedding_size_of_a_collapsed_map_is_zero(dev):
    with _ctx(3000, 2) as c:
        Y = torch.full((3000, 2), 0.25, dtype=torch.float32, device=dev)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        c.embedding_size(Y, out)
        torch.cuda.synchronize()
        assert out.item() == 0.0


@pytest.mark.parametrize("use_graph", [1, 0])
def test_run_records_the_embedding_size_of_each_epoch(dev, use_graph):
    """ptsne_run's third cost column is the size of the pooled map after each
    epoch: run epoch by epoch and compare with the oracle on the map the GPU
    returned.  The size grows as the map unfolds (the paper's monitor)."""
    from oracle import oracle as O
    n, d = 3000, 10
    X, _ = synth.gaussian_mixture(n, d, 5, seed=31)
    off = synth.equal_chunk_offsets(n, 3)
    perms = synth.permutations(n, 3, seed=32)
    Y0 = synth.init_gaussian(n, 2, 1e-4, seed=33)
    from paper_1812_09869_gb300 import ptsne
    cfg = ptsne.Config(n=n, d=d, offsets=off, perplexity=30.0, iters=30, use_graph=use_graph)
    sizes = []
    with ptsne.Context(cfg) as c:
        Xd = torch.from_numpy(X).to(dev)
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        for e in range(3):
            cost = np.zeros((1, 3))
            c.run(Xd, torch.from_numpy(perms[e:e + 1].copy()).to(dev), 1, Yd, cost_out=cost)
            torch.cuda.synchronize()
            ref = O.embedding_size(Yd.cpu().numpy().astype(np.float64))
            assert abs(cost[0, 2] - ref) <= SIZE_TOL * ref, (e, cost[0, 2], ref)
            sizes.append(cost[0, 2])
        # several epochs in one call: the last row is the returned map's size
        cost = np.zeros((2, 3))
        c.run(Xd, torch.from_numpy(perms[:2].copy()).to(dev), 2, Yd, cost_out=cost)
        torch.cuda.synchronize()
        ref = O.embedding_size(Yd.cpu().numpy().astype(np.float64))
        assert abs(cost[1, 2] - ref) <= SIZE_TOL * ref
    assert sizes[0] > O.embedding_size(Y0) and sizes[2] > sizes[0]


def test_layers_size_covers_every_layer(dev):
    """With layers the map holds L x n rows; the size spans all of them."""
    from oracle import oracle as O
    from paper_1812_09869_gb300 import ptsne
    n, L = 2000, 2
    X, _ = synth.gaussian_mixture(n, 6, 4, seed=41)
    off = synth.equal_chunk_offsets(n, 4)
    perms = synth.permutations(n, 1, seed=42)
    Y0 = synth.init_gaussian(L * n, 2, 1e-4, seed=43)
    cfg = ptsne.Config(n=n, d=6, offsets=off, perplexity=20.0, iters=20, layers=L)
    with ptsne.Context(cfg) as c:
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        cost = np.zeros((1, 3))
        c.run(torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev), 1, Yd, cost_out=cost)
        torch.cuda.synchronize()
        ref = O.embedding_size(Yd.cpu().numpy().astype(np.float64))
    assert abs(cost[0, 2] - ref) <= SIZE_TOL * ref


@pytest.mark.parametrize("k", [1, 10, 32])
def test_knn_preservation_matches_oracle(dev, k):
    """Neighbour sets in the input space (D = 50 mixture) and in a 2-D map,
    and their overlap, against the oracle's exact sort.  A query whose k-th
    and (k+1)-th FP64 distances lie within FP32 resolution of each other can
    legitimately differ at the boundary; such queries (if any) are only
    checked for a valid set."""
    from oracle import oracle as O
    from paper_1812_09869_gb300 import ptsne
    n, d = 20011, 50
    X, _ = synth.gaussian_mixture(n, d, 12, seed=51, anisotropic=True)
    rng = np.random.default_rng(52)
    R = rng.standard_normal((d, 2)).astype(np.float32)
    Y = (X @ R + rng.standard_normal((n, 2)).astype(np.float32)).astype(np.float32)   # a map that keeps some structure
    q = rng.choice(n, 300, replace=False).astype(np.int32)
    q[0], q[1] = 0, n - 1                                                             # first and last rows
    ov = torch.full((len(q),), -7, dtype=torch.int32, device=dev)
    nx = torch.full((len(q), k), -7, dtype=torch.int32, device=dev)
    ny = torch.full((len(q), k), -7, dtype=torch.int32, device=dev)
    ptsne.knn_preservation(torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev), torch.from_numpy(q).to(dev), k,
                           ov, nx, ny)
    torch.cuda.synchronize()
    ov, nx, ny = ov.cpu().numpy(), nx.cpu().numpy(), ny.cpu().numpy()
    sx, dxs = O.knn_sets(X[q], X, k, want_dist=True)
    sy, dys = O.knn_sets(Y[q], Y, k, want_dist=True)

    def near_tie(ds):
        return np.abs(ds[:, k] - ds[:, k - 1]) <= 1e-5 * np.maximum(ds[:, k], 1e-30)

    tie = near_tie(dxs) | near_tie(dys)
    assert tie.mean() < 0.05
    ok = ~tie
    assert np.array_equal(nx[ok], sx[ok]) and np.array_equal(ny[ok], sy[ok])
    ref = np.array([len(np.intersect1d(a, b)) for a, b in zip(sx, sy)])
    assert np.array_equal(ov[ok], ref[ok])
    # every set is valid: k distinct indices, the query excluded
    for i in range(len(q)):
        for s in (nx[i], ny[i]):
            assert len(set(s.tolist())) == k and q[i] not in s and s.min() >= 0 and s.max() < n
    # the mean preservation of the queries, as the oracle defines it
    assert abs(ov[ok].mean() / k - O.knn_preservation(X[q[ok]], X, Y[q[ok]], Y, k=k)) <= 1e-12


def test_knn_query_outside_the_points_is_reported(dev):
    from paper_1812_09869_gb300 import ptsne
    n = 1000
    X = torch.from_numpy(synth.init_gaussian(n, 5, 1.0, seed=53)).to(dev)
    Y = torch.from_numpy(synth.init_gaussian(n, 2, 1.0, seed=54)).to(dev)
    q = torch.tensor([3, n, -1, 7], dtype=torch.int32, device=dev)
    ov = torch.zeros(4, dtype=torch.int32, device=dev)
    ptsne.knn_preservation(X, Y, q, 5, ov)
    torch.cuda.synchronize()
    o = ov.cpu().numpy()
    assert o[1] == -1 and o[2] == -1 and 0 <= o[0] <= 5 and 0 <= o[3] <= 5
