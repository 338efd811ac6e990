"""ptsne_gradient_static, the entry point that allocates no device memory
(its scratch is a fixed array inside the library), against ptsne_step on the
same chunk.  Kept in a file of its own, collected last, so that it runs both
in a fresh process and after every other test has used the library."""
import ctypes as C

import numpy as np
import pytest

from paper_1812_09869_gb300 import synth

from parity import GRAD_TOL, rel_max

torch = pytest.importorskip("torch")


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
    max_rows = 32768
    rc = lib.ptsne_gradient_static(fake, max_rows + 1, fake, max_rows + 1, 2, fake, None, None)
    assert rc == ptsne.EINVAL
    msg = lib.ptsne_last_error(None).decode()
    assert str(max_rows) in msg and "scratch" in msg
    assert lib.ptsne_gradient_static(fake, 100, fake, 100, 4, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_gradient_static(fake, 99, fake, 100, 2, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_gradient_static(None, 100, fake, 100, 2, fake, None, None) == ptsne.EINVAL


@pytest.mark.gpu
def test_static_gradient_matches_step_on_two_calls_in_a_row(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import ptsne
    dev = torch.device("cuda:0")
    z, d = 3001, 16                  # several row blocks and a ragged tail; z > the 1024-thread final pass
    X, _ = synth.gaussian_mixture(z, d, 6, seed=91, anisotropic=True)
    perm = synth.permutations(z, 1, seed=92)[0]
    Y0 = synth.init_disk(z, seed=93)
    ctx = ptsne.Context(ptsne.Config(n=z, d=d, offsets=[0, z], perplexity=30.0, iters=1))
    Pd = torch.zeros((z, z), dtype=torch.float32, device=dev)
    pd = torch.from_numpy(perm).to(dev)
    ctx.affinities(torch.from_numpy(X).to(dev), pd, P_out=Pd)
    Yd = torch.from_numpy(Y0.copy()).to(dev)
    idx = pd.long()
    for call in range(2):            # the second call sees the scratch the first one left behind
        Yc = Yd[idx].contiguous()    # chunk order: row r is point perm[r]
        g_ref = torch.zeros_like(Yd)
        Z_ref = torch.zeros(1, dtype=torch.float64, device=dev)
        ctx.step(pd, Yd, grad_out=g_ref, Z_out=Z_ref)   # gradient at the input Y, then Y moves
        g = torch.full((z, 2), float("nan"), dtype=torch.float32, device=dev)
        Zs = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        ptsne.gradient_static(Pd, Yc, g, Zs)
        torch.cuda.synchronize()
        gr = g_ref[idx].cpu().numpy()
        assert np.isfinite(g.cpu().numpy()).all()
        assert rel_max(g.cpu().numpy(), gr) <= GRAD_TOL, (call, rel_max(g.cpu().numpy(), gr))
        assert abs(Zs.item() - Z_ref.item()) <= 1e-6 * Z_ref.item(), (call, Zs.item(), Z_ref.item())
    ctx.close()
