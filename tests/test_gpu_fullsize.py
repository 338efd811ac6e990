"""Parity at the benchmark's full size and launch configuration: the
1,000,000-point, D = 64 uneven-chunk workload (324 chunks of 1027..4998
points) with BF16 distances and FP32 window recompute, the batched persistent
schedule and the launch shape the library's autotuner picks, exactly as
bench.py runs it.  Sampled chunks (the smallest, the largest and one in
between) are compared with the FP64 oracle element by element; properties
that hold at any size are checked on every chunk."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth

from parity import GRAD_TOL, P_TOL, p_error, rel_max

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_09869_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("form", ["autotuned", "all_mixed"])
def test_full_size_bench_configuration(dev, form):
    """form "autotuned": the distance form ptsne_autotune picks (as the bench
    runs it); "all_mixed": every chunk through the BF16 Gram matrix, the
    coarse search and the window recompute."""
    from paper_1812_09869_gb300 import ptsne
    w = synth.workload("uneven-1m-d64", epochs=1)
    sizes = np.diff(w.offsets)
    cfg = ptsne.Config(n=w.n, d=w.d, offsets=w.offsets, perplexity=w.perplexity, iters=w.iters, lr=w.lr,
                       momentum=w.momentum, precision=w.precision, schedule="batched")
    perm = w.perms[0]
    with ptsne.Context(cfg) as ctx:
        Xd = torch.from_numpy(w.X).to(dev)
        pd = torch.from_numpy(perm).to(dev)
        Yd = torch.from_numpy(w.Y0.copy()).to(dev)
        ctx.autotune(Xd, pd, Yd, iters=3)                      # the bench's launch shape and form
        if form == "all_mixed":
            ctx.set_form_threshold(2.0)
            ctx.set_locality_order(False)
        Pd = torch.zeros(int((sizes.astype(np.int64) ** 2).sum()), dtype=torch.float32, device=dev)
        bd = torch.zeros(w.n, dtype=torch.float32, device=dev)
        ctx.affinities(Xd, pd, P_out=Pd, beta_out=bd)
        st = ctx.stats()
        assert st.bisect_failed_rows == 0 and st.wait_timeouts == 0 and st.bad_perm_entries == 0
        # every chunk: exactly symmetric, zero diagonal, total mass 1 (Eq. 3)
        worst_sum = 0.0
        blocks = torch.split(Pd, [int(z) * int(z) for z in sizes])
        for z, blk in zip(sizes, blocks):
            v = blk.view(int(z), int(z))
            assert torch.equal(v, v.T)
            assert float(v.diagonal().abs().max()) == 0.0
            worst_sum = max(worst_sum, abs(float(v.double().sum()) - 1.0))
        assert worst_sum <= 1e-5, worst_sum
        # one gradient step of every chunk
        gd = torch.zeros_like(Yd)
        Zd = torch.zeros(len(sizes), dtype=torch.float64, device=dev)
        ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
        torch.cuda.synchronize()
        beta = bd.cpu().numpy().astype(np.float64)
        g = gd.cpu().numpy()
        Z = Zd.cpu().numpy()
        sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), len(sizes) // 2})
        for c in sample:
            idx = perm[w.offsets[c]:w.offsets[c + 1]]
            Pr, br, bad = O.affinities(w.X[idx], w.perplexity)
            assert bad == 0
            Pg = blocks[c].view(int(sizes[c]), int(sizes[c])).cpu().numpy().astype(np.float64)
            assert p_error(Pg, Pr) <= P_TOL, (c, p_error(Pg, Pr))
            assert np.abs(beta[idx] - br).max() <= 1e-4 * br.max()
            gr, Zr = O.gradient(Pr, w.Y0[idx])
            assert rel_max(g[idx], gr) <= GRAD_TOL, (c, rel_max(g[idx], gr))
            assert abs(Z[c] - Zr) <= 1e-6 * Zr


@pytest.mark.parametrize("precision", ["bf16_window", "bf16_window_autotuned", "fp32"])
def test_full_size_precision_stress(dev, precision):
    """The precision-stress workload at full size: 200,000 sparse image-like
    vectors (D = 784, ~80% zeros, values in [0, 1]) in 64 chunks of 3125, with
    the BF16 tensor-core Gram matrix, FP32 window recompute and FP64 redo of
    stalled rows ("bf16_window": every chunk mixed in the caller's row order;
    "bf16_window_autotuned": the form and locality order ptsne_autotune_form
    picks, as the bench runs it), and for comparison FP32 distances
    throughout.  Three chunks (first, middle, last) against the FP64 oracle
    element by element; the errors are printed for the record."""
    from paper_1812_09869_gb300 import ptsne
    w = synth.workload("sparse-200k-d784", epochs=1)
    sizes = np.diff(w.offsets)
    cfg = ptsne.Config(n=w.n, d=w.d, offsets=w.offsets, perplexity=w.perplexity, iters=w.iters, lr=w.lr,
                       momentum=w.momentum, precision=precision.replace("_autotuned", ""), schedule="batched")
    perm = w.perms[0]
    with ptsne.Context(cfg) as ctx:
        Xd = torch.from_numpy(w.X).to(dev)
        pd = torch.from_numpy(perm).to(dev)
        Yd = torch.from_numpy(w.Y0.copy()).to(dev)
        if precision.endswith("_autotuned"):
            ctx.autotune_form(Xd, pd)
        Pd = torch.zeros(int((sizes.astype(np.int64) ** 2).sum()), dtype=torch.float32, device=dev)
        bd = torch.zeros(w.n, dtype=torch.float32, device=dev)
        ctx.affinities(Xd, pd, P_out=Pd, beta_out=bd)
        st = ctx.stats()
        assert st.bisect_failed_rows == 0 and st.wait_timeouts == 0 and st.nonfinite_inputs == 0
        gd = torch.zeros_like(Yd)
        Zd = torch.zeros(len(sizes), dtype=torch.float64, device=dev)
        ctx.step(pd, Yd, grad_out=gd, Z_out=Zd)
        torch.cuda.synchronize()
        blocks = torch.split(Pd, [int(z) * int(z) for z in sizes])
        beta = bd.cpu().numpy().astype(np.float64)
        g, Z = gd.cpu().numpy(), Zd.cpu().numpy()
        errs = {"P": 0.0, "beta": 0.0, "grad": 0.0, "Z": 0.0}
        for c in (0, len(sizes) // 2, len(sizes) - 1):
            idx = perm[w.offsets[c]:w.offsets[c + 1]]
            Pr, br, bad = O.affinities(w.X[idx], w.perplexity)
            assert bad == 0
            Pg = blocks[c].view(int(sizes[c]), int(sizes[c])).cpu().numpy().astype(np.float64)
            gr, Zr = O.gradient(Pr, w.Y0[idx])
            e = {"P": p_error(Pg, Pr), "beta": np.abs(beta[idx] - br).max() / br.max(),
                 "grad": rel_max(g[idx], gr), "Z": abs(Z[c] - Zr) / Zr}
            errs = {k: max(errs[k], e[k]) for k in errs}
        print(f"\n[precision stress {precision}] max over chunks 0, 32, 63: P {errs['P']:.2e} (of row max / "
              f"relative), beta {errs['beta']:.2e}, gradient {errs['grad']:.2e}, Z {errs['Z']:.2e}; "
              f"max |H - ln perp| {st.max_abs_entropy_err:.2e} nats; FP64 rows {st.bisect_fp64_rows}, "
              f"window pairs {st.window_pairs}, FP32-whole chunks {st.fp32_chunks}, locality order "
              f"{st.locality_order}")
        assert errs["P"] <= P_TOL and errs["beta"] <= 1e-4 and errs["grad"] <= GRAD_TOL and errs["Z"] <= 1e-6, errs
