"""The C-ABI library builds, loads and exports every declared entry point, and
its host-side argument validation rejects bad parameters before any device
work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    import glob
    text = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(ptsne_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_09869_gb300 import build, ptsne
    build.build()
    return ptsne.lib()


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for s in ("ptsne_create", "ptsne_destroy", "ptsne_affinities", "ptsne_step", "ptsne_run",
              "ptsne_run_host", "ptsne_cost", "ptsne_get_stats", "ptsne_last_error", "ptsne_gradient_static",
              "ptsne_mlp_create", "ptsne_mlp_train", "ptsne_mlp_grad", "ptsne_mlp_infer", "ptsne_embedding_size",
              "ptsne_knn_preservation", "ptsne_mlp_warm_start"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in _declared_symbols():
        assert hasattr(lib, s), f"libptsne.so does not export {s}"


def _params(**kw):
    from paper_1812_09869_gb300 import ptsne
    off = np.asarray(kw.pop("offsets", [0, 100, 200]), dtype=np.int64)
    base = dict(n=int(off[-1]), d=8, out_dim=2, perplexity=10.0, n_chunks=len(off) - 1, iters=10, lr=200.0,
                momentum=0.5, lr_mode=0, use_gains=1, precision=0, schedule=0, use_graph=1, layers=1)
    base.update(kw)
    p = ptsne.Params(base["n"], base["d"], base["out_dim"], base["perplexity"], base["n_chunks"],
                     off.ctypes.data_as(C.POINTER(C.c_int64)), base["iters"], base["lr"], base["momentum"],
                     base["lr_mode"], base["use_gains"], base["precision"], base["schedule"], base["use_graph"],
                     base["layers"])
    return p, off


@pytest.mark.parametrize("bad", [
    dict(d=0), dict(d=5000), dict(out_dim=4), dict(perplexity=1.0), dict(perplexity=99.0),
    dict(perplexity=float("nan")), dict(offsets=[0, 1, 200]), dict(offsets=[0, 100, 9000]),
    dict(n=150), dict(iters=-1), dict(lr=0.0), dict(momentum=1.0), dict(lr_mode=7), dict(use_gains=2),
    dict(precision=9), dict(schedule=3), dict(offsets=[0, 9000, 9100], perplexity=5.0), dict(use_graph=2),
    dict(layers=0), dict(layers=3), dict(offsets=[0, 5000, 9000], layers=2),
])
def test_create_rejects_bad_parameters_on_the_host(lib, bad):
    p, off = _params(**bad)
    h = C.c_void_p()
    rc = lib.ptsne_create(C.byref(h), C.byref(p))
    assert rc == -1, (bad, rc)
    assert not h.value
    assert lib.ptsne_last_error(None).decode().startswith("invalid parameter")


def test_null_arguments_are_rejected(lib):
    h = C.c_void_p()
    assert lib.ptsne_create(None, None) == -1
    assert lib.ptsne_create(C.byref(h), None) == -1
    assert lib.ptsne_affinities(None, None, None, None, None, None) == -1
    assert lib.ptsne_step(None, None, None, None, None, None) == -1
    assert lib.ptsne_run(None, None, None, 1, None, None, None) == -1
    assert lib.ptsne_set_form_threshold(None, 0.5) == -1
    assert lib.ptsne_autotune_form(None, None, None, None) == -1
    lib.ptsne_destroy(None)


def test_bindings_fail_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_1812_09869_gb300 import ptsne
    monkeypatch.setattr(ptsne, "_lib", None)
    monkeypatch.setattr(ptsne, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        ptsne.lib()


@pytest.mark.parametrize("field,value", [("d_in", 65), ("d_in", 0), ("out_dim", 4), ("batch", 100),
                                         ("batch", 0), ("infer_rows", 1000), ("lr", 0.0), ("beta2", 1.0)])
def test_mapper_create_rejects_bad_parameters(lib, field, value):
    """Checked on the host before any device allocation."""
    from paper_1812_09869_gb300 import mapper as M
    from paper_1812_09869_gb300 import ptsne
    L = M.lib()
    p = M.MlpParams(50, 2, 4096, 1 << 16, 1e-3, 0.9, 0.999, 1e-8, 1e-4)
    setattr(p, field, value)
    init = np.zeros(M.n_params(50, 2), np.float32)
    h = C.c_void_p()
    assert L.ptsne_mlp_create(C.byref(h), C.byref(p), init.ctypes.data_as(C.c_void_p)) == ptsne.EINVAL
    assert not h.value
    assert "invalid parameter" in L.ptsne_mlp_last_error(None).decode()


def test_mapper_pack_roundtrip():
    from paper_1812_09869_gb300 import mapper as M
    from paper_1812_09869_gb300 import synth
    W = synth.mlp_init(50, 3, seed=5)
    flat = M.pack(W)
    assert flat.size == M.n_params(50, 3) == 256 * 50 + 256 + 256 * 256 + 256 + 3 * 256 + 3
    back = M.unpack(flat, 50, 3)
    for k in M.PARAM_ORDER:
        assert np.array_equal(back[k], W[k])


def test_kde_grid_rejects_bad_arguments_on_the_host(lib):
    from paper_1812_09869_gb300 import ptsne
    fake = C.c_void_p(0x1000)
    box = (C.c_float * 4)(0.0, 1.0, 0.0, 1.0)
    bad_box = (C.c_float * 4)(1.0, 0.0, 0.0, 1.0)
    assert lib.ptsne_kde_grid(fake, fake, 10, 0, 8, box, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_kde_grid(fake, fake, 0, 8, 8, box, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_kde_grid(fake, fake, 10, 8, 8, bad_box, fake, None, None) == ptsne.EINVAL
    assert lib.ptsne_kde_grid(None, fake, 10, 8, 8, box, fake, None, None) == ptsne.EINVAL
    assert "ptsne_kde_grid" in lib.ptsne_last_error(None).decode()


def test_knn_preservation_rejects_bad_arguments_on_the_host(lib):
    from paper_1812_09869_gb300 import ptsne
    fake = C.c_void_p(0x1000)
    assert lib.ptsne_knn_preservation(fake, fake, 100, 50, 2, fake, 10, 0, fake, None, None, None) == ptsne.EINVAL
    assert lib.ptsne_knn_preservation(fake, fake, 100, 50, 2, fake, 10, 33, fake, None, None, None) == ptsne.EINVAL
    assert lib.ptsne_knn_preservation(fake, fake, 10, 50, 2, fake, 10, 10, fake, None, None, None) == ptsne.EINVAL
    assert lib.ptsne_knn_preservation(fake, fake, 100, 0, 2, fake, 10, 10, fake, None, None, None) == ptsne.EINVAL
    assert lib.ptsne_knn_preservation(None, fake, 100, 50, 2, fake, 10, 10, fake, None, None, None) == ptsne.EINVAL
    assert "ptsne_knn_preservation" in lib.ptsne_last_error(None).decode()
    assert lib.ptsne_knn_preservation(fake, fake, 100, 50, 2, fake, 0, 10, fake, None, None, None) == ptsne.OK


def test_warm_start_rejects_a_mismatched_context(lib):
    from paper_1812_09869_gb300 import mapper as M
    from paper_1812_09869_gb300 import ptsne
    fake = C.c_void_p(0x1000)
    ML = M.lib()
    assert ML.ptsne_mlp_warm_start(None, fake, fake, fake, fake, fake, None, None, None) == ptsne.EINVAL
