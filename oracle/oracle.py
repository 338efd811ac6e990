"""Python face of the ptSNE oracle (test infrastructure only).

The ptSNE arithmetic lives in plain C (ptsne_oracle.c, FP64); this module loads
it with ctypes and adds the FP64 numpy oracle of the learned out-of-sample
mapper (an MLP that the paper does not have; see mlp_* below) and brute-force
k-NN preservation.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module; the product path never does.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


class OrcParams(C.Structure):
    _fields_ = [
        ("perplexity", C.c_double),
        ("lr", C.c_double),
        ("momentum", C.c_double),
        ("lr_mode", C.c_int32),
        ("use_gains", C.c_int32),
        ("iters", C.c_int32),
        ("epochs", C.c_int32),
        ("bisect_tol", C.c_double),
        ("bisect_maxit", C.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_sqdist.argtypes = [_D, C.c_int64, C.c_int32, _D]
        L.orc_row_beta.argtypes = [_D, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                   C.c_int32, _D, _D, _I32]
        L.orc_affinities.argtypes = [_D, C.c_int64, C.c_int32, C.c_double, C.c_double,
                                     C.c_int32, _D, _D, _D]
        L.orc_affinities_from_distances.argtypes = [_D, C.c_int64, C.c_double, C.c_double, C.c_int32, _D, _D, _D]
        L.orc_cauchy_Z.argtypes = [_D, C.c_int64, C.c_int32]
        L.orc_cauchy_Z.restype = C.c_double
        L.orc_gradient.argtypes = [_D, _D, C.c_int64, C.c_int32, _D, _D]
        L.orc_gradient_rows.argtypes = [_D, _I64, C.c_int64, _D, C.c_int64, C.c_int32, C.c_double, _D]
        L.orc_kl.argtypes = [_D, _D, C.c_int64, C.c_int32]
        L.orc_kl.restype = C.c_double
        L.orc_normalized_cost.argtypes = [_D, _D, C.c_int64, C.c_int32]
        L.orc_normalized_cost.restype = C.c_double
        L.orc_embedding_size.argtypes = [_D, C.c_int64, C.c_int32]
        L.orc_embedding_size.restype = C.c_double
        L.orc_paper_lr.argtypes = [_D, C.c_int64, C.c_int32]
        L.orc_paper_lr.restype = C.c_double
        L.orc_update.argtypes = [_D, _D, _D, _D, C.c_int64, C.c_int32, C.c_double,
                                 C.c_double, C.c_int32, C.c_int32]
        L.orc_update.restype = None
        L.orc_partial_tsne.argtypes = [_D, C.c_int64, C.c_int32, C.c_int32,
                                       C.POINTER(OrcParams), _D, _D, _D, _D]
        L.orc_ptsne_run.argtypes = [_D, C.c_int64, C.c_int32, C.c_int32, _I32, _I64,
                                    C.c_int32, C.POINTER(OrcParams), _D, _D]
        L.orc_ptsne_run_layers.argtypes = [_D, C.c_int64, C.c_int32, C.c_int32, _I32, _I64, C.c_int32,
                                           C.c_int32, C.POINTER(OrcParams), _D, _D]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


BISECT_TOL = 1e-10   # |H - ln perp| in nats
BISECT_MAXIT = 200


def num_threads() -> int:
    return int(lib().orc_num_threads())


def sqdist(X):
    X = _f64(X)
    z, d = X.shape
    D = np.empty((z, z))
    assert lib().orc_sqdist(_d(X), z, d, _d(D)) == 0
    return D


def row_beta(drow, i, perp, tol=BISECT_TOL, maxit=BISECT_MAXIT):
    """(status, beta, H_nats, iterations) of the perplexity search for row i."""
    drow = _f64(drow)
    b, h, it = C.c_double(), C.c_double(), C.c_int32()
    st = lib().orc_row_beta(_d(drow), drow.shape[0], i, perp, tol, maxit,
                            C.byref(b), C.byref(h), C.byref(it))
    return st, b.value, h.value, it.value


def affinities(Xc, perp, tol=BISECT_TOL, maxit=BISECT_MAXIT, want_cond=False):
    """Joint P (z x z), beta (z), [p_{j|i} (z x z)], number of unconverged rows."""
    Xc = _f64(Xc)
    z, d = Xc.shape
    P = np.empty((z, z))
    beta = np.empty(z)
    cond = np.empty((z, z)) if want_cond else None
    st = lib().orc_affinities(_d(Xc), z, d, perp, tol, maxit, _d(P), _d(beta),
                              _d(cond) if want_cond else None)
    if st < 0:
        raise ValueError(f"orc_affinities failed: {st}")
    return (P, beta, cond, st) if want_cond else (P, beta, st)


def affinities_from_distances(D, perp, tol=BISECT_TOL, maxit=BISECT_MAXIT):
    """Joint P (z x z), beta (z) and the number of unconverged rows from a
    precomputed z x z dissimilarity matrix D."""
    D = _f64(D)
    z = D.shape[0]
    P = np.empty((z, z))
    beta = np.empty(z)
    st = lib().orc_affinities_from_distances(_d(D), z, perp, tol, maxit, _d(P), _d(beta), None)
    if st < 0:
        raise ValueError(f"orc_affinities_from_distances failed: {st}")
    return P, beta, st


def cauchy_Z(Y):
    Y = _f64(Y)
    return lib().orc_cauchy_Z(_d(Y), Y.shape[0], Y.shape[1])


def gradient(P, Y):
    P, Y = _f64(P), _f64(Y)
    z, od = Y.shape
    g = np.empty((z, od))
    Z = C.c_double()
    assert lib().orc_gradient(_d(P), _d(Y), z, od, _d(g), C.byref(Z)) == 0
    return g, Z.value


def gradient_rows(Prows, rows, Y, Z):
    """Eq. 6 at the chunk rows `rows` from their P rows (len(rows) x z) and the
    chunk's Z (cauchy_Z(Y)), for chunks too large for a dense FP64 P."""
    Prows, Y = _f64(Prows), _f64(Y)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    z, od = Y.shape
    assert Prows.shape == (len(rows), z)
    g = np.empty((len(rows), od))
    rc = lib().orc_gradient_rows(_d(Prows), rows.ctypes.data_as(_I64), len(rows), _d(Y), z, od, float(Z), _d(g))
    if rc != 0:
        raise ValueError(f"orc_gradient_rows failed: {rc}")
    return g


def kl(P, Y):
    P, Y = _f64(P), _f64(Y)
    return lib().orc_kl(_d(P), _d(Y), Y.shape[0], Y.shape[1])


def normalized_cost(P, Y):
    P, Y = _f64(P), _f64(Y)
    return lib().orc_normalized_cost(_d(P), _d(Y), Y.shape[0], Y.shape[1])


def embedding_size(Y):
    Y = _f64(Y)
    return lib().orc_embedding_size(_d(Y), Y.shape[0], Y.shape[1])


def paper_lr(Y):
    Y = _f64(Y)
    return lib().orc_paper_lr(_d(Y), Y.shape[0], Y.shape[1])


def update(Y, vel, gains, grad, lr=200.0, momentum=0.5, lr_mode=0, use_gains=1):
    """In-place update of float64 arrays Y, vel, gains (see orc_update)."""
    for a in (Y, vel, gains):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = _f64(grad)
    z, od = Y.shape
    lib().orc_update(_d(Y), _d(vel), _d(gains), _d(grad), z, od, lr, momentum,
                     lr_mode, use_gains)


def params(perplexity=30.0, lr=200.0, momentum=0.5, lr_mode=0, use_gains=1,
           iters=100, epochs=1, tol=BISECT_TOL, maxit=BISECT_MAXIT) -> OrcParams:
    return OrcParams(perplexity, lr, momentum, lr_mode, use_gains, iters, epochs, tol, maxit)


def partial_tsne(Xc, Yc, prm: OrcParams, want_P=False):
    """One partial t-SNE; returns (Y_final, kl, ncost, status[, P])."""
    Xc = _f64(Xc)
    Y = _f64(Yc).copy()
    z, d = Xc.shape
    od = Y.shape[1]
    P = np.empty((z, z)) if want_P else None
    k, nc = C.c_double(), C.c_double()
    st = lib().orc_partial_tsne(_d(Xc), z, d, od, C.byref(prm), _d(Y),
                                _d(P) if want_P else None, C.byref(k), C.byref(nc))
    if st < 0:
        raise ValueError(f"orc_partial_tsne failed: {st}")
    out = (Y, k.value, nc.value, st)
    return out + (P,) if want_P else out


def ptsne_run(X, Y0, perms, offsets, prm: OrcParams):
    """Full ptSNE epoch cycle; returns (Y, cost[epochs, 2] = (avg KL, avg ncost))."""
    X = _f64(X)
    Y = _f64(Y0).copy()
    n, d = X.shape
    od = Y.shape[1]
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    assert perms.shape[0] >= prm.epochs and perms.shape[1] == n
    cost = np.empty((prm.epochs, 2))
    st = lib().orc_ptsne_run(_d(X), n, d, od, perms.ctypes.data_as(_I32),
                             offsets.ctypes.data_as(_I64), len(offsets) - 1,
                             C.byref(prm), _d(Y), _d(cost))
    if st < 0:
        raise ValueError(f"orc_ptsne_run failed: {st}")
    return Y, cost


def ptsne_run_layers(X, Y0, perms, offsets, layers, prm: OrcParams):
    """ptSNE with layers: thread t runs elementary chunks t .. t+layers-1 (mod
    T); Y0 and the result hold `layers` maps of n points, layer-major
    (layers*n x out_dim).  Returns (Y, cost[epochs, 2])."""
    X = _f64(X)
    Y = _f64(Y0).copy()
    n, d = X.shape
    od = Y.shape[1]
    assert Y.shape[0] == layers * n
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    cost = np.empty((prm.epochs, 2))
    st = lib().orc_ptsne_run_layers(_d(X), n, d, od, perms.ctypes.data_as(_I32), offsets.ctypes.data_as(_I64),
                                    len(offsets) - 1, layers, C.byref(prm), _d(Y), _d(cost))
    if st < 0:
        raise ValueError(f"orc_ptsne_run_layers failed: {st}")
    return Y, cost


# ---------------------------------------------------------------------------
# Perplexity-adaptive kernel density estimate of a 2-D map (paKDE, the
# paper's Clustering section): the sample smoothing estimator with Gaussian
# kernels K_j = exp(-beta_j |c - y_j|^2) / pi and h_j^2 = 1 / beta_j, i.e.
#     f(c) = (S / n) sum_j (beta_j / pi) exp(-beta_j |c - y_j|^2)
# on a regular grid of cells c of area S; beta_j from the perplexity search on
# the map's own distances.  Plain numpy, every point against every cell.
# ---------------------------------------------------------------------------

def kde_grid(Y, beta, gx, gy, box):
    """Density of each cell of a gx x gy grid over box = (xmin, xmax, ymin,
    ymax), evaluated at the cell centres; returns (gy, gx) float64."""
    Y, beta = _f64(Y), _f64(beta)
    x0, x1, y0, y1 = map(float, box)
    dx, dy = (x1 - x0) / gx, (y1 - y0) / gy
    cx = x0 + (np.arange(gx) + 0.5) * dx
    cy = y0 + (np.arange(gy) + 0.5) * dy
    f = np.zeros((gy, gx))
    for j in range(Y.shape[0]):
        ex = np.exp(-beta[j] * (cx - Y[j, 0]) ** 2)
        ey = np.exp(-beta[j] * (cy - Y[j, 1]) ** 2)
        f += (beta[j] / math.pi) * np.outer(ey, ex)
    return f * (dx * dy) / Y.shape[0]


# ---------------------------------------------------------------------------
# Learned out-of-sample mapper (not in the paper): MLP d_in -> 256 -> 256 -> 2
# with exact (erf) GELU, trained by mean squared error on standardised ptSNE
# coordinates with AdamW.  FP64 numpy, written as the plain definition.
# ---------------------------------------------------------------------------

def gelu(u):
    return 0.5 * u * (1.0 + _erf(u / math.sqrt(2.0)))


def gelu_grad(u):
    return 0.5 * (1.0 + _erf(u / math.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)


def _erf(x):
    from scipy.special import erf
    return erf(x)


def mlp_forward(W, x):
    """W = dict(W1 (256 x din), b1, W2 (256 x 256), b2, W3 (2 x 256), b3).
    Returns (y, cache)."""
    u1 = x @ W["W1"].T + W["b1"]
    h1 = gelu(u1)
    u2 = h1 @ W["W2"].T + W["b2"]
    h2 = gelu(u2)
    y = h2 @ W["W3"].T + W["b3"]
    return y, (x, u1, h1, u2, h2)


def mlp_loss_grad(W, x, t):
    """Loss L = sum_b sum_k (y_bk - t_bk)^2 / (2B) and its gradient dict."""
    W = {k: np.asarray(v, dtype=np.float64) for k, v in W.items()}
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    y, (x, u1, h1, u2, h2) = mlp_forward(W, x)
    r = (y - t) / B
    L = 0.5 * float(np.sum((y - t) ** 2)) / B
    g = {}
    g["W3"] = r.T @ h2
    g["b3"] = r.sum(0)
    dh2 = r @ W["W3"]
    du2 = dh2 * gelu_grad(u2)
    g["W2"] = du2.T @ h1
    g["b2"] = du2.sum(0)
    dh1 = du2 @ W["W2"]
    du1 = dh1 * gelu_grad(u1)
    g["W1"] = du1.T @ x
    g["b1"] = du1.sum(0)
    return L, g


def adamw_step(W, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (decoupled weight decay on weights, not biases), in place."""
    for k in W:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        decay = wd * W[k] if k.startswith("W") else 0.0
        W[k] = W[k] - lr * (mh / (np.sqrt(vh) + eps) + decay)


def knn_sets(q, a, k, exclude_self=True, want_dist=False):
    """Indices of the k nearest rows of `a` to each row of `q` (squared
    Euclidean distances in FP64, exact by full sort; ties to the smaller
    index), nearest first; with exclude_self the nearest entry (the query
    itself, at distance 0) is dropped.  want_dist: also the sorted distances
    (k + 1 of them, the one after the k-th included)."""
    q, a = _f64(q), _f64(a)
    d = (q * q).sum(1)[:, None] + (a * a).sum(1)[None, :] - 2.0 * q @ a.T
    order = np.argsort(d, axis=1, kind="stable")
    sel = order[:, 1:k + 1] if exclude_self else order[:, :k]
    if not want_dist:
        return sel
    lo = 1 if exclude_self else 0
    return sel, np.take_along_axis(d, order[:, lo:lo + k + 1], axis=1)


def knn_preservation(Xq, Xall, Yq, Yall, k=10, exclude_self=True):
    """Mean fraction of each query's k nearest neighbours in X (exact, by full
    sort) that are also among its k nearest neighbours in Y."""
    nx, ny = knn_sets(Xq, Xall, k, exclude_self), knn_sets(Yq, Yall, k, exclude_self)
    return float(np.mean([len(np.intersect1d(a, b)) / k for a, b in zip(nx, ny)]))
