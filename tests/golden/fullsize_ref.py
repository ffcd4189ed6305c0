"""Reader of the full-size oracle references (``vacancy9072.npz``, ``metal7200.npz``) written by
``make_fullsize.py``: the quantised columns and sketches back to float64, and the sketch matrix.
Holds no arithmetic of the method and imports neither the oracle nor the CUDA library, so the
GPU tests and the benchmark can read the stored values directly.

Quantisation: an entry v is stored as the integer rint(v * 2^40) (absolute error <= 2^-41),
its eight little-endian bytes split into planes so that the mostly constant high bytes deflate.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
QSCALE = 2.0 ** 40
SKETCH = 24                    # rows of the sketch matrix Omega


def sha256(a: np.ndarray) -> str:
    """SHA-256 of an array's row-major float64 bytes (the key of a stored reference)."""
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float64).tobytes()).hexdigest()


def quantise(cols: np.ndarray) -> np.ndarray:
    """(n, c) float64 -> (8, n * c) uint8 byte planes of rint(v * 2^40) as little-endian int64."""
    q = np.rint(np.ascontiguousarray(cols) * QSCALE).astype("<i8")
    return q.reshape(-1).view(np.uint8).reshape(-1, 8).T.copy()


def dequantise(planes: np.ndarray, n: int) -> np.ndarray:
    """Inverse of quantise: (8, n * c) byte planes -> (n, c) float64."""
    q = np.ascontiguousarray(planes.T).reshape(-1).view("<i8")
    return (q.astype(np.float64) / QSCALE).reshape(n, -1)


def sketch_matrix(n: int, seed: int) -> np.ndarray:
    """Omega (SKETCH x n) with seeded N(0, 1) entries (the workloads module's generator)."""
    import workloads as wl
    return wl.gaussian((SKETCH, n), seed=seed)


def path(name: str) -> str:
    return os.path.join(HERE, f"{name}.npz")


def load(name: str) -> dict:
    """The stored reference of workload ``name`` ("vacancy9072" or "metal7200") with the sampled
    columns and the sketch dequantised (keys V_cols, X_cols, sketch)."""
    with np.load(path(name)) as z:
        d = {k: z[k] for k in z.files}
    n = int(d["n"])
    d["V_cols"] = dequantise(d["Vq"], n)
    d["X_cols"] = dequantise(d["Xq"], n)
    d["sketch"] = dequantise(d["Sq"], SKETCH)
    return d
