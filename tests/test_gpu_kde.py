"""paKDE of a 2-D map: precisions from the perplexity search on the map's
own distances (ptsne_affinities on a 2-D context) and the grid density of
ptsne_kde_grid, against the oracle's search and its every-point-every-cell
density."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("grid", [(128, 96), (33, 257)])
def test_pakde_matches_oracle(dev, grid):
    from paper_1812_09869_gb300 import ptsne
    n = 3000
    Ymap, _ = synth.gaussian_mixture(n, 2, 5, seed=70, anisotropic=True)   # a 2-D point set standing in for a map
    Ymap = np.ascontiguousarray(Ymap / 4.0, dtype=np.float32)
    off = np.array([0, 1000, 1777, 3000])
    perm = synth.permutations(n, 1, seed=71)[0]
    gx, gy = grid
    box = (float(Ymap[:, 0].min() - 1), float(Ymap[:, 0].max() + 1), float(Ymap[:, 1].min() - 1),
           float(Ymap[:, 1].max() + 1))
    with ptsne.Context(ptsne.Config(n=n, d=2, offsets=off, perplexity=30.0, iters=1)) as ctx:
        Yd = torch.from_numpy(Ymap).to(dev)
        bd = torch.zeros(n, dtype=torch.float32, device=dev)
        ctx.affinities(Yd, torch.from_numpy(perm).to(dev), beta_out=bd)
        fd = torch.full((gy, gx), float("nan"), dtype=torch.float32, device=dev)
        ptsne.kde_grid(Yd, bd, gx, gy, box, fd)
        torch.cuda.synchronize()
        f = fd.cpu().numpy().astype(np.float64)
    beta_ref = np.empty(n)
    for c in range(len(off) - 1):
        idx = perm[off[c]:off[c + 1]]
        _, br, bad = O.affinities(Ymap[idx], 30.0)
        assert bad == 0
        beta_ref[idx] = br
    f_ref = O.kde_grid(Ymap, beta_ref, gx, gy, box)
    assert np.abs(f - f_ref).max() <= 1e-3 * f_ref.max()
    assert abs(f.sum() - f_ref.sum()) <= 1e-4
    assert abs(f_ref.sum() - 1.0) <= 2e-2            # the box holds almost all of the mass


def test_kernels_too_wide_for_the_grid_are_counted_and_left_out(dev):
    """A point whose precision is far too small for the grid (its kernel would
    cover more than PTSNE_KDE_MAX_CELLS cells) is left out and counted; the
    others are splatted as the oracle evaluates them."""
    from paper_1812_09869_gb300 import ptsne
    gx = gy = 2048
    Y = np.array([[0.1, 0.2], [0.5, 0.5], [-0.3, 0.4]], dtype=np.float32)
    beta = np.array([4.0e4, 1.0e-3, 2.5e4], dtype=np.float32)   # the middle kernel spans the whole box
    box = (-1.0, 1.0, -1.0, 1.0)
    fd = torch.full((gy, gx), float("nan"), dtype=torch.float32, device=dev)
    dropped = torch.full((1,), -1, dtype=torch.int64, device=dev)
    ptsne.kde_grid(torch.from_numpy(Y).to(dev), torch.from_numpy(beta).to(dev), gx, gy, box, fd,
                   dropped_out=dropped)
    torch.cuda.synchronize()
    assert dropped.item() == 1
    keep = np.array([0, 2])
    # the estimator's 1/n uses all three points; the dropped one adds nothing
    f_ref = O.kde_grid(Y[keep], beta[keep].astype(np.float64), gx, gy, box) * (2.0 / 3.0)
    f = fd.cpu().numpy().astype(np.float64)
    assert np.abs(f - f_ref).max() <= 1e-3 * f_ref.max()
