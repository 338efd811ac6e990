"""ptsne_gradient_static, the entry point that allocates no device memory (its
scratch is a fixed array inside the library), for callers that cannot call
cudaMalloc: a host framework that owns the whole device memory pool, or code
that must not block on an allocation.  It is checked against the existing
entry point ptsne_step on the same chunk and against the FP64 oracle on the
oracle's own P, on two calls in a row (the second sees the scratch the first
left behind), with 2-D and 3-D maps, and at the largest chunk the fixed
scratch holds.  Kept in a file of its own, collected last, so that it runs
both in a fresh process and after every other test has used the library."""
import ctypes as C

import numpy as np
import pytest

from paper_1812_09869_gb300 import synth

from parity import GRAD_TOL, rel_max

torch = pytest.importorskip("torch")

MAX_ROWS = 32768   # PTSNE_STATIC_MAX_ROWS


@pytest.fixture(scope="module")
def lib():
    from paper_1812_09869_gb300 import build, ptsne
    build.build()
    return ptsne.lib()


def test_rejects_sizes_beyond_the_scratch(lib):
    """Host-side checks run before any device work (fake non-null pointers are
    never dereferenced)."""
    from paper_1812_09869_gb300 import ptsne
    fake = C.c_void_p(0x1000)
    rc = lib.ptsne_gradient_static(fake, MAX_ROWS + 1, fake, MAX_ROWS + 1, 2, fake, None, None)
    assert rc == ptsne.EINVAL
    msg = lib.ptsne_last_error(None).decode()
    assert str(MAX_ROWS) in msg and "scratch" in msg
    assert lib.ptsne_gradient_static(fake, 100, fake, 100, 4, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_gradient_static(fake, 99, fake, 100, 2, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_gradient_static(None, 100, fake, 100, 2, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_gradient_static(fake, 100, fake, 1, 2, fake, None, None) == ptsne.EINVAL


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.gpu
@pytest.mark.parametrize("out_dim", [2, 3])
def test_static_gradient_matches_step_and_oracle_on_two_calls_in_a_row(lib, out_dim):
    """z = 3001: several row blocks, a ragged tail, more rows than the
    1024-thread final pass."""
    _need_gpu()
    from oracle import oracle as O
    from paper_1812_09869_gb300 import ptsne
    dev = torch.device("cuda:0")
    z, d = 3001, 16
    X, _ = synth.gaussian_mixture(z, d, 6, seed=91, anisotropic=True)
    perm = synth.permutations(z, 1, seed=92)[0]
    Y0 = synth.init_gaussian(z, out_dim, 3.0, seed=93)
    # the oracle's own P of the chunk (rows in chunk order: row r is point perm[r])
    P_orc, _, _ = O.affinities(X[perm].astype(np.float64), 30.0)
    P_orc32 = torch.from_numpy(P_orc.astype(np.float32)).to(dev)
    ctx = ptsne.Context(ptsne.Config(n=z, d=d, offsets=[0, z], perplexity=30.0, iters=1, out_dim=out_dim))
    Pd = torch.zeros((z, z), dtype=torch.float32, device=dev)
    pd = torch.from_numpy(perm).to(dev)
    ctx.affinities(torch.from_numpy(X).to(dev), pd, P_out=Pd)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    idx = pd.long()
    for call in range(2):            # the second call sees the scratch the first one left behind
        Yc = Yd[idx].contiguous()    # chunk order
        # against the existing entry point, on the context's P
        g_ref = torch.zeros_like(Yd)
        Z_ref = torch.zeros(1, dtype=torch.float64, device=dev)
        ctx.step(pd, Yd, grad_out=g_ref, Z_out=Z_ref)   # gradient at the input Y, then Y moves
        g = torch.full((z, out_dim), float("nan"), dtype=torch.float32, device=dev)
        Zs = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        ptsne.gradient_static(Pd, Yc, g, Zs)
        torch.cuda.synchronize()
        gs, gr = g.cpu().numpy(), g_ref[idx].cpu().numpy()
        assert np.isfinite(gs).all()
        assert rel_max(gs, gr) <= GRAD_TOL, (call, rel_max(gs, gr))
        assert abs(Zs.item() - Z_ref.item()) <= 1e-6 * Z_ref.item(), (call, Zs.item(), Z_ref.item())
        # against the oracle, on the oracle's P rounded to FP32 (the kernel's input)
        g2 = torch.full((z, out_dim), float("nan"), dtype=torch.float32, device=dev)
        Z2 = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        ptsne.gradient_static(P_orc32, Yc, g2, Z2)
        torch.cuda.synchronize()
        Yh = Yc.cpu().numpy().astype(np.float64)
        g_orc, Z_orc = O.gradient(P_orc.astype(np.float32).astype(np.float64), Yh)
        assert rel_max(g2.cpu().numpy(), g_orc) <= GRAD_TOL, (call, rel_max(g2.cpu().numpy(), g_orc))
        assert abs(Z2.item() - Z_orc) <= 1e-6 * Z_orc, (call, Z2.item(), Z_orc)
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("out_dim", [2, 3])
def test_static_gradient_at_the_largest_chunk_allocates_nothing(lib, out_dim):
    """z = PTSNE_STATIC_MAX_ROWS (the per-row accumulators fill the scratch
    exactly) with a padded leading dimension; sampled rows and Z against the
    oracle, and the device's free memory is unchanged across a call."""
    _need_gpu()
    from oracle import oracle as O
    from paper_1812_09869_gb300 import ptsne
    dev = torch.device("cuda:0")
    z, ld, seed = MAX_ROWS, MAX_ROWS + 64, 95 + out_dim
    P = torch.empty((z, ld), dtype=torch.float32, device=dev)
    P[:, z:] = float("nan")          # padding beyond z is never read
    blk = 2048
    for r0 in range(0, z, blk):      # 4 GB drawn block by block on the host
        rows = np.arange(r0, min(z, r0 + blk))
        P[r0:r0 + len(rows), :z] = torch.from_numpy(synth.lowrank_affinity_rows(z, seed, rows)).to(dev)
    Y = synth.init_gaussian(z, out_dim, 5.0, seed=seed + 1)
    Yd = torch.from_numpy(Y).to(dev)
    g = torch.full((z, out_dim), float("nan"), dtype=torch.float32, device=dev)
    Zs = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    ptsne.gradient_static(P, Yd, g, Zs, ld=ld)      # warm-up: module and scratch address set up
    torch.cuda.synchronize()
    g.fill_(float("nan"))
    free0, _ = torch.cuda.mem_get_info()
    ptsne.gradient_static(P, Yd, g, Zs, ld=ld)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    gs = g.cpu().numpy()
    assert np.isfinite(gs).all()
    sample = np.unique(np.concatenate([[0, 1, z - 2, z - 1],
                                       np.random.default_rng(seed).integers(0, z, 60)]))
    Yh = Y.astype(np.float64)
    Z_orc = O.cauchy_Z(Yh)
    g_orc = O.gradient_rows(synth.lowrank_affinity_rows(z, seed, sample), sample, Yh, Z_orc)
    assert rel_max(gs[sample], g_orc) <= GRAD_TOL, rel_max(gs[sample], g_orc)
    assert abs(Zs.item() - Z_orc) <= 1e-6 * Z_orc, (Zs.item(), Z_orc)
    # every row of a symmetric P: the gradient sums to zero (pairwise antisymmetry)
    assert np.abs(gs.astype(np.float64).sum(0)).max() <= 1e-3 * np.abs(gs).max() * np.sqrt(z)
