"""Thin ctypes binding of libptsne.so (argument marshalling only).

Every function forwards to the C entry point of the same name declared in
include/ptsne.h; all arithmetic runs in the library's CUDA kernels.  Tensors
are torch CUDA tensors (PyTorch supplies device memory and streams only).
The library must have been built (``paper_1812_09869_gb300.build.build()``):
nothing here falls back to any other implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptsne.so")

OK, EINVAL, ENONFINITE, ENOMEM, ECUDA, ESTATE, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
WBISECT = 1
LR_FIXED, LR_PAPER = 0, 1
PREC_FP32, PREC_BF16_WINDOW = 0, 1
SCHED_BATCHED, SCHED_PER_CHUNK = 0, 1

_PRECISION = {"fp32": PREC_FP32, "bf16_window": PREC_BF16_WINDOW}
_SCHEDULE = {"batched": SCHED_BATCHED, "per_chunk": SCHED_PER_CHUNK}


class PtsneError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ptsne error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("d", C.c_int32),
        ("out_dim", C.c_int32),
        ("perplexity", C.c_double),
        ("n_chunks", C.c_int32),
        ("chunk_offsets", C.POINTER(C.c_int64)),
        ("iters", C.c_int32),
        ("lr", C.c_float),
        ("momentum", C.c_float),
        ("lr_mode", C.c_int32),
        ("use_gains", C.c_int32),
        ("precision", C.c_int32),
        ("schedule", C.c_int32),
        ("use_graph", C.c_int32),
        ("layers", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("bisect_rows", C.c_int64),
        ("bisect_fp64_rows", C.c_int64),
        ("bisect_failed_rows", C.c_int64),
        ("window_pairs", C.c_int64),
        ("nonfinite_inputs", C.c_int64),
        ("bad_perm_entries", C.c_int64),
        ("wait_timeouts", C.c_int64),
        ("max_abs_entropy_err", C.c_double),
        ("kernel_launches", C.c_int64),
        ("stage_ms", C.c_double * 7),
        ("stage_calls", C.c_int64 * 7),
        ("bisect_evals", C.c_int64),
        ("ptiles_total", C.c_int64),
        ("ptiles_nonzero", C.c_int64),
        ("fp32_chunks", C.c_int64),
        ("form_threshold", C.c_double),
        ("window_fraction", C.c_double * 8),
        ("form_ms_mixed", C.c_double),
        ("form_ms_fp32", C.c_double),
        ("form_ms_window", C.c_double),
        ("locality_order", C.c_int64),
    ]


STAGES = ("gather", "distances", "perplexity", "joint_p", "iterate", "pool", "cost")


class Tuning(C.Structure):
    _fields_ = [("cluster", C.c_int32), ("group", C.c_int32), ("consumer_warps", C.c_int32)]


class TuneTrial(C.Structure):
    _fields_ = [("tuning", Tuning), ("ms_per_iter", C.c_double)]


_lib = None


def lib():
    """Load libptsne.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1812_09869_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.ptsne_create.argtypes = [C.POINTER(vp), C.POINTER(Params)]
        L.ptsne_destroy.argtypes = [vp]
        L.ptsne_destroy.restype = None
        L.ptsne_last_error.argtypes = [vp]
        L.ptsne_last_error.restype = C.c_char_p
        L.ptsne_affinities.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ptsne_step.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ptsne_distances.argtypes = [vp, vp, vp, vp, vp]
        L.ptsne_affinities_from_distances.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp]
        L.ptsne_cost.argtypes = [vp, vp, vp, vp, vp]
        L.ptsne_embedding_size.argtypes = [vp, vp, vp, vp]
        L.ptsne_run.argtypes = [vp, vp, vp, C.c_int32, vp, C.POINTER(C.c_double), vp]
        L.ptsne_run_host.argtypes = [vp, vp, vp, C.c_int32, vp, C.POINTER(C.c_double), vp]
        L.ptsne_get_stats.argtypes = [vp, C.POINTER(Stats), vp]
        L.ptsne_workspace_bytes.argtypes = [vp]
        L.ptsne_workspace_bytes.restype = C.c_size_t
        L.ptsne_set_profiling.argtypes = [vp, C.c_int]
        L.ptsne_reset_counters.argtypes = [vp]
        L.ptsne_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.ptsne_set_locality_order.argtypes = [vp, C.c_int]
        L.ptsne_set_deterministic.argtypes = [vp, C.c_int]
        L.ptsne_set_form_threshold.argtypes = [vp, C.c_double]
        L.ptsne_autotune_form.argtypes = [vp, vp, vp, vp]
        L.ptsne_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.ptsne_autotune.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_char_p, C.POINTER(TuneTrial), C.c_int32,
                                     C.POINTER(C.c_int32), vp]
        L.ptsne_gradient_static.argtypes = [vp, C.c_int64, vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.ptsne_kde_grid.argtypes = [vp, vp, C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_float), vp, vp, vp]
        L.ptsne_knn_preservation.argtypes = [vp, vp, C.c_int64, C.c_int32, C.c_int32, vp, C.c_int32, C.c_int32, vp,
                                             vp, vp, vp]
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class Config:
    n: int
    d: int
    offsets: "object"            # sequence of n_chunks + 1 int64 offsets
    perplexity: float = 30.0
    out_dim: int = 2
    iters: int = 100
    lr: float = 200.0
    momentum: float = 0.5
    lr_mode: int = LR_FIXED
    use_gains: int = 1
    precision: str = "fp32"
    schedule: str = "batched"
    use_graph: int = 1
    layers: int = 1              # > 1: threads chain `layers` elementary chunks; maps hold layers x n rows


class Context:
    """Owns one ptsne_ctx (device workspace for one problem shape)."""

    def __init__(self, cfg: Config):
        import numpy as np
        self.cfg = cfg
        self._off = np.ascontiguousarray(np.asarray(cfg.offsets, dtype=np.int64))
        p = Params(cfg.n, cfg.d, cfg.out_dim, cfg.perplexity, len(self._off) - 1,
                   self._off.ctypes.data_as(C.POINTER(C.c_int64)), cfg.iters, cfg.lr, cfg.momentum,
                   cfg.lr_mode, cfg.use_gains, _PRECISION[cfg.precision], _SCHEDULE[cfg.schedule], cfg.use_graph,
                   cfg.layers)
        h = C.c_void_p()
        rc = lib().ptsne_create(C.byref(h), C.byref(p))
        if rc != OK:
            raise PtsneError(rc, lib().ptsne_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ptsne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, warn_ok=False):
        if rc < 0 or (rc > 0 and not warn_ok):
            raise PtsneError(rc, lib().ptsne_last_error(self.h).decode())
        return rc

    @property
    def workspace_bytes(self) -> int:
        return int(lib().ptsne_workspace_bytes(self.h))

    @property
    def n_chunks(self) -> int:
        return len(self._off) - 1

    # --- entry points -------------------------------------------------------
    def affinities(self, X, perm, P_out=None, beta_out=None, stream=None):
        return self._check(lib().ptsne_affinities(self.h, _ptr(X), _ptr(perm), _ptr(P_out), _ptr(beta_out),
                                                  _stream(stream)))

    def affinities_from_distances(self, D, perm, P_out=None, beta_out=None, ldd=None, stream=None):
        """D: n x n float32 dissimilarities in original point order."""
        ldd = int(D.shape[-1]) if ldd is None else int(ldd)
        return self._check(lib().ptsne_affinities_from_distances(self.h, _ptr(D), ldd, _ptr(perm), _ptr(P_out),
                                                                 _ptr(beta_out), _stream(stream)))

    def distances(self, X, perm, D_out, stream=None):
        return self._check(lib().ptsne_distances(self.h, _ptr(X), _ptr(perm), _ptr(D_out), _stream(stream)))

    def step(self, perm, Y, grad_out=None, Z_out=None, stream=None):
        return self._check(lib().ptsne_step(self.h, _ptr(perm), _ptr(Y), _ptr(grad_out), _ptr(Z_out),
                                            _stream(stream)))

    def cost(self, perm, Y, out, stream=None):
        return self._check(lib().ptsne_cost(self.h, _ptr(perm), _ptr(Y), _ptr(out), _stream(stream)))

    def embedding_size(self, Y, out, stream=None):
        """ptsne_embedding_size: the diagonal of Y's bounding box into out (1 float64, device)."""
        return self._check(lib().ptsne_embedding_size(self.h, _ptr(Y), _ptr(out), _stream(stream)))

    @staticmethod
    def _cost_ptr(cost_out, epochs):
        if cost_out is None:
            return None
        if cost_out.dtype != np.float64 or cost_out.size < 3 * epochs or not cost_out.flags.c_contiguous:
            raise ValueError("cost_out must be a C-contiguous float64 array of epochs x 3")
        return cost_out.ctypes.data_as(C.POINTER(C.c_double))

    def run(self, X, perms, epochs, Y, cost_out=None, stream=None):
        """cost_out: optional float64 numpy array (epochs x 3): avg KL, avg
        normalised cost and embedding size after each epoch."""
        cp = self._cost_ptr(cost_out, epochs)
        return self._check(lib().ptsne_run(self.h, _ptr(X), _ptr(perms), epochs, _ptr(Y), cp, _stream(stream)),
                           warn_ok=True)

    def run_host(self, X_host, perms_host, epochs, Y_host, cost_out=None, stream=None):
        """Host tensors (ideally pinned); Y_host is updated in place."""
        cp = self._cost_ptr(cost_out, epochs)
        return self._check(lib().ptsne_run_host(self.h, _ptr(X_host), _ptr(perms_host), epochs, _ptr(Y_host),
                                                cp, _stream(stream)), warn_ok=True)

    def stats(self, stream=None) -> Stats:
        st = Stats()
        self._check(lib().ptsne_get_stats(self.h, C.byref(st), _stream(stream)))
        return st

    def set_profiling(self, on: bool):
        return self._check(lib().ptsne_set_profiling(self.h, int(bool(on))))

    def reset_counters(self):
        return self._check(lib().ptsne_reset_counters(self.h))

    def set_tuning(self, cluster: int, group: int, consumer_warps: int):
        t = Tuning(cluster, group, consumer_warps)
        return self._check(lib().ptsne_set_tuning(self.h, C.byref(t)))

    def set_locality_order(self, on: bool):
        return self._check(lib().ptsne_set_locality_order(self.h, int(bool(on))))

    def set_deterministic(self, on: bool):
        """Fixed-point accumulation in the batched kernel: bitwise repeatable runs."""
        return self._check(lib().ptsne_set_deterministic(self.h, int(bool(on))))

    def set_form_threshold(self, threshold: float):
        """BF16_WINDOW: chunks whose size bin's window fraction is >= threshold
        are computed in FP32 whole (2: never, negative: always)."""
        return self._check(lib().ptsne_set_form_threshold(self.h, C.c_double(threshold)))

    def tuning(self) -> tuple:
        t = Tuning()
        self._check(lib().ptsne_get_tuning(self.h, C.byref(t)))
        return (t.cluster, t.group, t.consumer_warps)

    def autotune_form(self, X, perm, stream=None):
        """BF16_WINDOW: time both forms of the distances (and the locality
        order) on this partition and set the form threshold."""
        return self._check(lib().ptsne_autotune_form(self.h, _ptr(X), _ptr(perm), _stream(stream)))

    def form_record(self) -> dict:
        """The form choice of a BF16_WINDOW context, for reports."""
        st = self.stats()
        return {"threshold": st.form_threshold, "ms_all_mixed": st.form_ms_mixed, "ms_all_fp32": st.form_ms_fp32,
                "ms_window": st.form_ms_window, "locality_order": bool(st.locality_order),
                "window_fraction_by_size_bin": [round(v, 4) for v in st.window_fraction]}

    def autotune(self, X, perm, Y, iters=3, cache_path=None, stream=None):
        """Returns [((cluster, group, consumer_warps), ms_per_iter), ...] of the timed trials."""
        cap = 64
        arr = (TuneTrial * cap)()
        n = C.c_int32(0)
        cp = None if cache_path is None else os.fsencode(cache_path)
        self._check(lib().ptsne_autotune(self.h, _ptr(X), _ptr(perm), _ptr(Y), iters, cp, arr, cap, C.byref(n),
                                         _stream(stream)))
        return [((t.tuning.cluster, t.tuning.group, t.tuning.consumer_warps), t.ms_per_iter)
                for t in arr[:n.value]]


def gradient_static(P, Y, grad_out, Z_out=None, ld=None, stream=None):
    """ptsne_gradient_static: the gradient of one chunk with no device
    allocation (fixed library scratch).  P: z x ld float32, Y and grad_out:
    z x out_dim float32, Z_out: optional 1-element float64 tensor."""
    z, od = int(Y.shape[0]), int(Y.shape[1])
    ld = int(P.shape[-1]) if ld is None else int(ld)
    rc = lib().ptsne_gradient_static(_ptr(P), ld, _ptr(Y), z, od, _ptr(grad_out), _ptr(Z_out), _stream(stream))
    if rc != OK:
        raise PtsneError(rc, lib().ptsne_last_error(None).decode())
    return rc


def kde_grid(Y, beta, gx, gy, box, density_out, dropped_out=None, stream=None):
    """ptsne_kde_grid: paKDE of the map Y (n x 2) with precisions beta (n) on a
    gx x gy grid over box = (xmin, xmax, ymin, ymax) into density_out (gy x gx);
    dropped_out (optional, 1 int64 device tensor) counts the points left out
    because their kernel covers more than PTSNE_KDE_MAX_CELLS cells."""
    b = (C.c_float * 4)(*[float(v) for v in box])
    rc = lib().ptsne_kde_grid(_ptr(Y), _ptr(beta), int(Y.shape[0]), int(gx), int(gy), b, _ptr(density_out),
                              _ptr(dropped_out), _stream(stream))
    if rc != OK:
        raise PtsneError(rc, lib().ptsne_last_error(None).decode())
    return rc


def knn_preservation(X, Y, queries, k, overlap_out, nbr_x_out=None, nbr_y_out=None, stream=None):
    """ptsne_knn_preservation: per query, the overlap of its k nearest
    neighbours in X (n x d) and in Y (n x od); optional neighbour sets."""
    n, d = int(X.shape[0]), int(X.shape[1])
    rc = lib().ptsne_knn_preservation(_ptr(X), _ptr(Y), n, d, int(Y.shape[1]), _ptr(queries), int(queries.shape[0]),
                                      int(k), _ptr(overlap_out), _ptr(nbr_x_out), _ptr(nbr_y_out), _stream(stream))
    if rc != OK:
        raise PtsneError(rc, lib().ptsne_last_error(None).decode())
    return rc
