"""Brute-force checker: the classical cyclic Jacobi eigenvalue algorithm (Golub & Van Loan,
Matrix Computations, Section 8.5), written independently of the oracle for tiny matrices.

Each rotation zeroes one off-diagonal pair exactly; sweeps repeat until the off-diagonal mass is
below 1e-30 of the total, so the result is the exact eigendecomposition up to rounding.
"""
import numpy as np


def jacobi_eigh(A, max_sweeps: int = 60):
    a = np.array(A, dtype=np.float64, copy=True)
    n = a.shape[0]
    v = np.eye(n)
    total = float(np.sum(a * a))
    for _ in range(max_sweeps):
        off = float(np.sum(np.triu(a, 1) ** 2) + np.sum(np.tril(a, -1) ** 2))
        if off <= 1e-30 * total or off == 0.0:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = a[p, q]
                if apq == 0.0:
                    continue
                theta = (a[q, q] - a[p, p]) / (2.0 * apq)
                t = (1.0 if theta >= 0 else -1.0) / (abs(theta) + np.sqrt(theta * theta + 1.0))
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                # A <- J^T A J with J the rotation in the (p, q) plane
                ap, aq = a[:, p].copy(), a[:, q].copy()
                a[:, p] = c * ap - s * aq
                a[:, q] = s * ap + c * aq
                ap, aq = a[p, :].copy(), a[q, :].copy()
                a[p, :] = c * ap - s * aq
                a[q, :] = s * ap + c * aq
                vp, vq = v[:, p].copy(), v[:, q].copy()
                v[:, p] = c * vp - s * vq
                v[:, q] = s * vp + c * vq
    w = np.diag(a).copy()
    order = np.argsort(w, kind="stable")
    return w[order], v[:, order]
