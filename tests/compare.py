"""Comparison helpers shared by the parity tests (sign- and cluster-aware)."""
import numpy as np


def spectral_scale(lam_ref) -> float:
    """||A|| for the tolerances: the largest |eigenvalue| of the reference."""
    return float(np.max(np.abs(lam_ref)))


def vector_projector_errors(U, V):
    """Per column ||u u^T - v v^T||_F for unit columns (no cancellation near 1)."""
    d = np.sum(U * V, axis=0)
    s = np.where(d < 0, -1.0, 1.0)
    diff = np.linalg.norm(U - V * s, axis=0)
    return diff * np.sqrt(1.0 + np.abs(d))


def clusters(lam, tol):
    """Index groups of the reference eigenvalues (in index order) whose sorted neighbours are
    closer than tol."""
    order = np.argsort(lam, kind="stable")
    groups, cur = [], [order[0]]
    for a, b in zip(order[:-1], order[1:]):
        if lam[b] - lam[a] < tol:
            cur.append(b)
        else:
            groups.append(cur)
            cur = [b]
    groups.append(cur)
    return groups


def projector_errors(Uref, V, lam_ref, cluster_tol=0.0):
    """Subspace projector error ||P_ref - P||_F per cluster (singletons: per vector)."""
    errs = []
    for g in clusters(lam_ref, cluster_tol) if cluster_tol > 0 else [[i] for i in range(len(lam_ref))]:
        if len(g) == 1:
            errs.append(float(vector_projector_errors(Uref[:, g], V[:, g])[0]))
        else:
            Pa = Uref[:, g] @ Uref[:, g].T
            Pb = V[:, g] @ V[:, g].T
            errs.append(float(np.linalg.norm(Pa - Pb)))
    return np.array(errs)
