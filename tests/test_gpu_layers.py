"""ptSNE with layers (threads chained over L elementary chunks, L maps per
point) against the FP64 oracle: each thread's joint P and one gradient step,
then whole epochs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth

from parity import GRAD_TOL, P_TOL, chunk_blocks, p_error, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L = 3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _setup():
    n = 2500
    X, _ = synth.gaussian_mixture(n, 12, 6, seed=60, anisotropic=True)
    off = np.array([0, 430, 950, 1500, 1999, 2500])        # 5 elementary chunks, ragged
    perms = synth.permutations(n, 2, seed=61)
    Y0 = np.concatenate([synth.init_gaussian(n, 2, 1e-2, seed=62 + k) for k in range(L)])   # L layers
    return X, off, perms, Y0


def _thread_rows(off, perm, t, n):
    """(layer, point) of each row of thread t: slot k holds elementary chunk t + k."""
    T = len(off) - 1
    rows = []
    for k in range(L):
        c = (t + k) % T
        rows += [(k, int(p)) for p in perm[off[c]:off[c + 1]]]
    return rows


def test_thread_affinities_and_first_step_match_oracle(dev):
    from paper_1812_09869_gb300 import ptsne
    X, off, perms, Y0 = _setup()
    n, T = X.shape[0], len(off) - 1
    perm = perms[0]
    tz = [sum(off[(t + k) % T + 1] - off[(t + k) % T] for k in range(L)) for t in range(T)]
    toff = np.concatenate([[0], np.cumsum(tz)])
    cfg = ptsne.Config(n=n, d=X.shape[1], offsets=off, perplexity=30.0, iters=1, layers=L)
    with ptsne.Context(cfg) as ctx:
        pd = torch.from_numpy(perm).to(dev)
        Pd = torch.zeros(int(sum(z * z for z in tz)), dtype=torch.float32, device=dev)
        bd = torch.zeros(L * n, dtype=torch.float32, device=dev)
        ctx.affinities(torch.from_numpy(X).to(dev), pd, P_out=Pd, beta_out=bd)
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        gd = torch.zeros_like(Yd)
        Zd = torch.zeros(T, dtype=torch.float64, device=dev)
        ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
        torch.cuda.synchronize()
        st = ctx.stats()
        blocks = chunk_blocks(Pd.cpu().numpy(), toff)
        beta, g, Z = bd.cpu().numpy().astype(np.float64), gd.cpu().numpy(), Zd.cpu().numpy()
    assert st.bisect_failed_rows == 0 and st.bad_perm_entries == 0
    for t in range(T):
        rows = _thread_rows(off, perm, t, n)
        vi = np.array([k * n + p for k, p in rows])
        Pr, br, bad = O.affinities(X[[p for _, p in rows]], 30.0)
        assert bad == 0
        assert p_error(blocks[t], Pr) <= P_TOL, (t, p_error(blocks[t], Pr))
        assert np.abs(beta[vi] - br).max() <= 1e-4 * br.max()
        gr, Zr = O.gradient(Pr, Y0[vi])
        assert rel_max(g[vi], gr) <= GRAD_TOL, (t, rel_max(g[vi], gr))
        assert abs(Z[t] - Zr) <= 1e-6 * Zr


def test_layered_epochs_match_oracle(dev):
    from paper_1812_09869_gb300 import ptsne
    X, off, perms, Y0 = _setup()
    n = X.shape[0]
    cfg = ptsne.Config(n=n, d=X.shape[1], offsets=off, perplexity=30.0, iters=40, layers=L)
    with ptsne.Context(cfg) as ctx:
        Yd = torch.from_numpy(Y0.copy()).to(dev)
        cost = np.zeros((2, 3))
        ctx.run(torch.from_numpy(X).to(dev), torch.from_numpy(perms).to(dev), 2, Yd, cost_out=cost)
        torch.cuda.synchronize()
    _, cref = O.ptsne_run_layers(X, Y0, perms, off, L, O.params(perplexity=30.0, iters=40, epochs=2))
    assert abs(cost[0, 0] - cref[0, 0]) <= 1e-3 * cref[0, 0], (cost, cref)   # first epoch: tight
    assert abs(cost[1, 0] - cref[1, 0]) <= 1e-2 * cref[1, 0], (cost, cref)   # then within 1%
