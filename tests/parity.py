"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

# P: entries at least 1e-6 of their row's largest entry must match to 1e-4
# relative; every entry must match to 1e-4 of its row's largest entry (the
# "max-relative error <= 1e-4" of the requirement, with the 1e-6 floor below
# which FP32 exponentials lose relative accuracy).
P_TOL = 1e-4
P_FLOOR = 1e-6
GRAD_TOL = 1e-3   # max |g_gpu - g_ref| / max |g_ref| after one step
KL_TOL = 0.01     # final KL within 1%


def p_error(P_gpu, P_ref):
    """max over rows of the floor-relative error described above."""
    P_gpu = np.asarray(P_gpu, dtype=np.float64)
    P_ref = np.asarray(P_ref, dtype=np.float64)
    rowmax = P_ref.max(axis=1, keepdims=True)
    rowmax = np.where(rowmax > 0, rowmax, 1.0)
    diff = np.abs(P_gpu - P_ref)
    big = P_ref >= P_FLOOR * rowmax
    rel_big = np.max(np.where(big, diff / np.where(big, P_ref, 1.0), 0.0))
    rel_all = np.max(diff / rowmax)
    return float(max(rel_big, rel_all))


def chunk_blocks(P_flat, offsets):
    """Split the exported P (sum z^2 floats) into per-chunk z x z arrays."""
    out, base = [], 0
    for c in range(len(offsets) - 1):
        z = int(offsets[c + 1] - offsets[c])
        out.append(np.asarray(P_flat[base:base + z * z], dtype=np.float64).reshape(z, z))
        base += z * z
    return out


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
