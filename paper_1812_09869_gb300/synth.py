"""Seeded synthetic inputs for ptSNE (data, chunk layouts, partitions, initial maps).

This module holds no part of the method's arithmetic: it only draws the random
inputs that both the CUDA path and the FP64 oracle consume.  The random
partition of every epoch (the paper's "the master mixes the data and defines the
data chunks", ptSNE section, subsection "epochs") is drawn here and passed in as
an input array, so neither side implements a generator of its own.

The datasets of the paper (MNIST, GMM5, GMM7, dwt1005) are not available; the
generators below produce stand-ins with the same structure: Gaussian mixtures
(like GMM5/GMM7) and sparse image-like vectors in [0, 1] (like MNIST's 784-pixel
intensities).  No item of any public dataset is reproduced.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "gaussian_mixture",
    "zipf_sizes",
    "sparse_images",
    "equal_chunk_offsets",
    "uniform_chunk_offsets",
    "permutations",
    "init_gaussian",
    "init_disk",
    "mlp_init",
    "Workload",
    "workload",
    "WORKLOADS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _haar_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    """Uniformly random rotation: QR of a Gaussian matrix with the sign fix."""
    a = rng.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    q *= np.sign(np.diag(r))[None, :]
    return q


def zipf_sizes(n: int, k: int, s: float = 1.2) -> np.ndarray:
    """Cluster sizes proportional to rank^-s (rank 1..k), rounded to sum to n."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    raw = w / w.sum() * n
    sizes = np.floor(raw).astype(np.int64)
    rest = n - int(sizes.sum())
    order = np.argsort(-(raw - sizes), kind="stable")
    sizes[order[:rest]] += 1
    return sizes


def gaussian_mixture(n: int, d: int, k: int, seed: int, *, sizes=None,
                     mean_var: float = 25.0, anisotropic: bool = False,
                     eig_range=(0.1, 2.0)) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian mixture X (n x d, float32, row-major) and its component labels.

    Means are drawn N(0, mean_var * I).  Isotropic components have unit
    variance; anisotropic ones have covariance Q^T diag(lambda) Q with Q a Haar
    rotation and lambda ~ U[eig_range].  Rows are shuffled so that labels are
    not contiguous.
    """
    rng = _rng(seed)
    if sizes is None:
        sizes = np.full(k, n // k, dtype=np.int64)
        sizes[: n - int(sizes.sum())] += 1
    sizes = np.asarray(sizes, dtype=np.int64)
    assert int(sizes.sum()) == n and len(sizes) == k
    means = rng.standard_normal((k, d)) * np.sqrt(mean_var)
    X = np.empty((n, d), dtype=np.float32)
    labels = np.empty(n, dtype=np.int32)
    row = 0
    for c in range(k):
        m = int(sizes[c])
        z = rng.standard_normal((m, d), dtype=np.float32)
        if anisotropic:
            q = _haar_orthogonal(rng, d)
            lam = rng.uniform(eig_range[0], eig_range[1], size=d)
            # x = mu + z diag(sqrt(lam)) Q  => cov = Q^T diag(lam) Q
            L = (np.sqrt(lam)[:, None] * q).astype(np.float32)
            z = z @ L
        X[row:row + m] = z + means[c].astype(np.float32)[None, :]
        labels[row:row + m] = c
        row += m
    order = rng.permutation(n)
    return np.ascontiguousarray(X[order]), labels[order]


def sparse_images(n: int, seed: int, *, side: int = 28, n_proto: int = 10,
                  coverage: float = 0.2, noise: float = 0.1):
    """Sparse image-like vectors in [0, 1]: prototype + noise on its support.

    Each of `n_proto` prototypes is a union of random rectangles covering about
    `coverage` of the side x side pixels, with intensities U[0.5, 1].  A sample
    is its prototype plus N(0, noise^2) on the prototype's non-zero pixels,
    clipped to [0, 1]; about 1 - coverage of the entries are exactly zero.
    """
    rng = _rng(seed)
    d = side * side
    protos = np.zeros((n_proto, side, side), dtype=np.float32)
    for p in range(n_proto):
        mask = np.zeros((side, side), dtype=bool)
        while mask.mean() < coverage:
            h, w = rng.integers(3, 10, size=2)
            r0 = rng.integers(0, side - h + 1)
            c0 = rng.integers(0, side - w + 1)
            mask[r0:r0 + h, c0:c0 + w] = True
        vals = rng.uniform(0.5, 1.0, size=(side, side)).astype(np.float32)
        protos[p][mask] = vals[mask]
    protos = protos.reshape(n_proto, d)
    labels = rng.integers(0, n_proto, size=n).astype(np.int32)
    X = protos[labels].copy()
    support = X > 0
    X += rng.standard_normal((n, d), dtype=np.float32) * np.float32(noise) * support
    np.clip(X, 0.0, 1.0, out=X)
    X[~support] = 0.0
    return np.ascontiguousarray(X), labels


def equal_chunk_offsets(n: int, c: int) -> np.ndarray:
    """Offsets of c near-equal chunks: the first n mod c chunks get one more."""
    sizes = np.full(c, n // c, dtype=np.int64)
    sizes[: n % c] += 1
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def uniform_chunk_offsets(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Chunk sizes drawn U{lo..hi} until they cover n points.

    The last draw is shrunk to fit.  If what is left for it is below `lo`, it is
    merged into the previous chunk, and if that merged chunk exceeds `hi` it is
    split into two halves, so every size stays within [lo, hi] (given n >= lo).
    """
    assert n >= lo and hi >= 2 * lo
    rng = _rng(seed)
    sizes: list[int] = []
    left = n
    while left > 0:
        s = int(rng.integers(lo, hi + 1))
        if s >= left:
            s = left
        sizes.append(s)
        left -= s
    if len(sizes) > 1 and sizes[-1] < lo:
        merged = sizes[-2] + sizes[-1]
        sizes = sizes[:-2]
        if merged > hi:
            sizes += [merged // 2, merged - merged // 2]
        else:
            sizes.append(merged)
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def permutations(n: int, epochs: int, seed: int) -> np.ndarray:
    """One random permutation of [0, n) per epoch, int32 array (epochs x n)."""
    rng = _rng(seed)
    out = np.empty((epochs, n), dtype=np.int32)
    for e in range(epochs):
        out[e] = rng.permutation(n).astype(np.int32)
    return out


def init_gaussian(n: int, out_dim: int, std: float, seed: int) -> np.ndarray:
    """Initial map Y ~ N(0, std^2 I), float32 (n x out_dim)."""
    rng = _rng(seed)
    return (rng.standard_normal((n, out_dim)) * std).astype(np.float32)


def init_disk(n: int, seed: int) -> np.ndarray:
    """Initial map uniform in the disk of radius 1 (the paper's ptSNE start)."""
    rng = _rng(seed)
    r = np.sqrt(rng.uniform(0.0, 1.0, size=n))
    t = rng.uniform(0.0, 2.0 * np.pi, size=n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1).astype(np.float32)


def lowrank_affinity_rows(z: int, seed: int, rows) -> np.ndarray:
    """Rows `rows` of a seeded symmetric non-negative z x z float32 matrix
    shaped like a joint P (entries ~1/z^2, varied over rows and columns):
    (u_i u_j + v_i v_j) / s with u ~ U[0.5, 1.5], v ~ U[0, 1]^3 and s the sum
    over all pairs.  Any subset of rows can be drawn on its own, bit for bit
    equal to the same rows of a full draw, so chunks too large for a dense
    host matrix can be generated block by block.  The diagonal is left as is
    (consumers ignore it)."""
    rng = _rng(seed)
    u = rng.uniform(0.5, 1.5, z)
    v = rng.uniform(0.0, 1.0, z) ** 3
    s = u.sum() ** 2 + v.sum() ** 2
    uf, vf = (u / np.sqrt(s)).astype(np.float32), (v / np.sqrt(s)).astype(np.float32)
    rows = np.asarray(rows, dtype=np.int64)
    return np.outer(uf[rows], uf) + np.outer(vf[rows], vf)


def mlp_init(d_in: int, out_dim: int, seed: int, hidden: int = 256) -> dict:
    """Initial mapper parameters: weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)),
    biases zero, float32 (W1 hidden x d_in, W2 hidden x hidden, W3 out x hidden)."""
    rng = _rng(seed)

    def u(rows, cols):
        a = 1.0 / np.sqrt(cols)
        return rng.uniform(-a, a, size=(rows, cols)).astype(np.float32)

    return {"W1": u(hidden, d_in), "b1": np.zeros(hidden, np.float32),
            "W2": u(hidden, hidden), "b2": np.zeros(hidden, np.float32),
            "W3": u(out_dim, hidden), "b3": np.zeros(out_dim, np.float32)}


@dataclasses.dataclass
class Workload:
    """A named synthetic workload: data, chunk layout, partitions and start map."""
    name: str
    X: np.ndarray            # n x d float32
    labels: np.ndarray       # n int32 (component / prototype id)
    offsets: np.ndarray      # n_chunks + 1 int64
    perms: np.ndarray        # epochs x n int32
    Y0: np.ndarray           # n x out_dim float32
    perplexity: float
    epochs: int
    iters: int
    lr: float = 200.0
    momentum: float = 0.5
    precision: str = "fp32"  # "fp32" or "bf16_window"

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def chunk_sizes(self) -> np.ndarray:
        return np.diff(self.offsets)


def _plain_2000():
    X, lab = gaussian_mixture(2000, 10, 8, seed=1)
    off = np.array([0, 2000], dtype=np.int64)
    perms = permutations(2000, 1, seed=101)
    Y0 = init_gaussian(2000, 2, 1e-4, seed=201)
    return Workload("plain-2000x10", X, lab, off, perms, Y0, 30.0, 1, 100)


def _chunks64_100k(epochs: int = 10):
    n, d, k = 100_000, 50, 20
    X, lab = gaussian_mixture(n, d, k, seed=2, anisotropic=True)
    off = equal_chunk_offsets(n, 64)
    perms = permutations(n, epochs, seed=102)
    Y0 = init_gaussian(n, 2, 1e-4, seed=202)
    return Workload("ptsne-100k-d50-64chunks", X, lab, off, perms, Y0, 30.0, epochs, 100)


def _uneven_1m(epochs: int = 10):
    n, d, k = 1_000_000, 64, 50
    X, lab = gaussian_mixture(n, d, k, seed=3, sizes=zipf_sizes(n, k, 1.2), anisotropic=True)
    off = uniform_chunk_offsets(n, 1000, 5000, seed=303)
    perms = permutations(n, epochs, seed=103)
    Y0 = init_gaussian(n, 2, 1e-4, seed=203)
    return Workload("uneven-1m-d64", X, lab, off, perms, Y0, 30.0, epochs, 100,
                    precision="bf16_window")


def _uneven_100k(epochs: int = 2):
    """The 1M workload's recipe at 100k points (about 33 chunks of U{1000..5000}):
    the same kernels at a size small enough for detailed profiler captures."""
    n, d, k = 100_000, 64, 50
    X, lab = gaussian_mixture(n, d, k, seed=3, sizes=zipf_sizes(n, k, 1.2), anisotropic=True)
    off = uniform_chunk_offsets(n, 1000, 5000, seed=303)
    perms = permutations(n, epochs, seed=103)
    Y0 = init_gaussian(n, 2, 1e-4, seed=203)
    return Workload("uneven-100k-d64", X, lab, off, perms, Y0, 30.0, epochs, 100,
                    precision="bf16_window")


def _sparse_200k(epochs: int = 1):
    n = 200_000
    X, lab = sparse_images(n, seed=4)
    off = equal_chunk_offsets(n, 64)
    perms = permutations(n, epochs, seed=104)
    Y0 = init_gaussian(n, 2, 1e-4, seed=204)
    return Workload("sparse-200k-d784", X, lab, off, perms, Y0, 30.0, epochs, 100,
                    precision="bf16_window")


def _mapper_2m(epochs: int = 10):
    """2 x 1M points of the 20-component, D=50 mixture: train half + held-out half."""
    n, d, k = 2_000_000, 50, 20
    X, lab = gaussian_mixture(n, d, k, seed=5, anisotropic=True)
    half = n // 2
    off = uniform_chunk_offsets(half, 1000, 5000, seed=305)
    perms = permutations(half, epochs, seed=105)
    Y0 = init_gaussian(half, 2, 1e-4, seed=205)
    return Workload("mapper-1m+1m-d50", X, lab, off, perms, Y0, 30.0, epochs, 100)


WORKLOADS = {
    "plain-2000x10": _plain_2000,
    "ptsne-100k-d50-64chunks": _chunks64_100k,
    "uneven-1m-d64": _uneven_1m,
    "uneven-100k-d64": _uneven_100k,
    "sparse-200k-d784": _sparse_200k,
    "mapper-1m+1m-d50": _mapper_2m,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
