"""PFSM oracle (plain FP64 CPU restatement of arXiv:1502.07806, Section II).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline leg, never by the GPU library or its binding. It shares no code with the GPU path.
The arithmetic lives in ``pfsm_oracle.c`` (straight loops); this module only marshals numpy
arrays through ctypes.

Parity status per function (what pins it; see ``tests/test_oracle_pins.py``):
  plan         pinned: sizes/containment invariants, hand-worked layouts, cluster snap cases
  gershgorin   pinned: contains every eigenvalue of random matrices, exact on diagonal ones
  symeig       pinned: 2x2 closed form, tridiagonal Toeplitz closed form, brute-force cyclic
               Jacobi, LAPACK (numpy) on random symmetric matrices, diagonal input exact
  fs_iterate   pinned: eigenbasis closed form of (I - alpha (A - eps I)^2)^K
  mgs          pinned: Householder QR with positive R diagonal (numpy), orthonormality
  rayleigh     pinned: exact eigenvectors give exact eigenvalues and zero residual
  pfsm         pinned: P=1 / halo>=N / block-diagonal inputs reduce to the exact
               eigendecomposition; E=0 gives V=I exactly; trace and Weyl-bound invariants;
               monotone error over an SCF-like sequence
  backward     pinned: sum(lambda) -> identity, occupied sum -> projector, central finite
               differences of the exact eigen-map
  gen_to_std   pinned: LAPACK solve(B, A) at convergence, the closed-form Neumann sum of the
               iteration after a fixed count, diagonal B exact in one update, divergence of a
               non-dominant B reported
  gen_to_std_sym pinned: eigendecomposition-based B^{-1/2}, LAPACK generalized eigenvalues
               (sygvd via scipy) of (A, B), B-orthonormal generalized eigenvectors x = S y
  guard        pinned: diagonal input 0, 2x2 closed form |b| / |a - d|, hand-worked 3x3, the
               paper's mixed-eigenvector counterexample far above the workloads' values
  full         pinned: LAPACK (numpy) eigenvalues and eigenvectors up to the sign rule, the sign
               rule itself, equality with the method for one block and no Eq. 11 iterations
  pfsm_guarded pinned through guard, full and pfsm
  fs_adaptive  pinned: an exact eigenbasis stops at once, zero steps give one exact Rayleigh
               quotient, a perturbed eigenvector converges to LAPACK's eigenvalue in a few steps,
               the method with it against LAPACK
  scf_step     pinned: exact eigenbasis in gives back the basis (A diagonal), the chained
               eigenvalues and projectors against LAPACK's eigendecomposition of each H_j,
               orthonormality of the carried basis
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfsm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# tests that plant mistakes load a mutated copy of the oracle through this variable
_OVERRIDE = os.environ.get("PFSM_ORACLE_LIB_OVERRIDE")

OK, INVALID_ARG, NOT_SPD, NAN_INPUT, NOT_CONVERGED = 0, 1, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable x86-64 code, IEEE semantics, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        if _OVERRIDE:
            lib = ctypes.CDLL(_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_plan.argtypes = [i64, i32, i32, f64, P, P, P, P, P, P]
        lib.oracle_gershgorin.argtypes = [i64, P, P, P]
        lib.oracle_symeig.argtypes = [i64, P, P, P]
        lib.oracle_fs_iterate.argtypes = [i64, i64, P, P, P, P, i32]
        lib.oracle_fs_iterate.restype = None
        lib.oracle_fs_iterate_adaptive.argtypes = [i64, i64, P, P, P, P, i32, f64, f64, f64, f64, P, P]
        lib.oracle_mgs.argtypes = [i64, i64, P, P]
        lib.oracle_rayleigh.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_rayleigh.restype = None
        lib.oracle_pfsm.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_backward.argtypes = [i64, P, P, P, P, f64, P]
        lib.oracle_backward.restype = None
        lib.oracle_gen_to_std.argtypes = [i64, P, P, P, i32, f64, P, P]
        lib.oracle_gen_to_std_sym.argtypes = [i64, P, P, P, P, i32, f64, P, P]
        lib.oracle_guard.argtypes = [i64, P, P]
        lib.oracle_guard.restype = None
        lib.oracle_full.argtypes = [i64, P, P, P, P]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} returned status {code}")
        self.code = code


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


class _Params(ctypes.Structure):
    _fields_ = [("halo", ctypes.c_int32), ("fs_iters", ctypes.c_int32),
                ("alpha_theta", ctypes.c_double), ("cluster_tol", ctypes.c_double),
                ("slice_sizes", ctypes.c_void_p), ("fs_adaptive", ctypes.c_int32), ("fs_tol", ctypes.c_double)]


def set_threads(n: int) -> None:
    """Limit OpenMP threads (results do not depend on the count)."""
    os.environ["OMP_NUM_THREADS"] = str(n)
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(ctypes.c_int(n))
    except OSError:
        pass


def plan(prev, nblocks: int, halo: int = -1, cluster_tol: float = 1e-5, slice_sizes=None):
    """Slices and windows: returns int32 arrays (k0, m, s, M) of length nblocks."""
    prev = _f64(prev)
    n = prev.size
    out = np.zeros((4, nblocks), dtype=np.int32)
    ss = None if slice_sizes is None else np.ascontiguousarray(slice_sizes, dtype=np.int32)
    st = _load().oracle_plan(n, nblocks, halo, cluster_tol, _p(prev), _p(ss),
                             _p(out[0]), _p(out[1]), _p(out[2]), _p(out[3]))
    if st:
        raise OracleError(st, "plan")
    return out[0].copy(), out[1].copy(), out[2].copy(), out[3].copy()


def gershgorin(A):
    A = _f64(A)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    st = _load().oracle_gershgorin(A.shape[0], _p(A), ctypes.byref(lo), ctypes.byref(hi))
    if st:
        raise OracleError(st, "gershgorin")
    return lo.value, hi.value


def symeig(B):
    """All eigenpairs of a symmetric matrix: (w ascending, Z with Z[:, j] the vector of w[j])."""
    B = _f64(B)
    n = B.shape[0]
    w = np.zeros(n)
    Z = np.zeros((n, n))
    st = _load().oracle_symeig(n, _p(B), _p(w), _p(Z))
    if st:
        raise OracleError(st, "symeig")
    return w, Z


def fs_iterate(A, X, eps, alpha, iters: int):
    """Eq. 11 applied ``iters`` times to the columns of X (n x cnt); returns the new X."""
    A = _f64(A)
    Xt = _f64(np.asarray(X).T)
    eps, alpha = _f64(eps), _f64(alpha)
    _load().oracle_fs_iterate(A.shape[0], Xt.shape[0], _p(A), _p(Xt), _p(eps), _p(alpha), iters)
    return Xt.T.copy()


def mgs(X):
    """Modified Gram-Schmidt of the columns of X: returns (Q, r_diag)."""
    Xt = _f64(np.asarray(X).T)
    rd = np.zeros(Xt.shape[0])
    st = _load().oracle_mgs(Xt.shape[1], Xt.shape[0], _p(Xt), _p(rd))
    if st:
        raise OracleError(st, "mgs")
    return Xt.T.copy(), rd


def rayleigh(A, Q):
    A = _f64(A)
    Qt = _f64(np.asarray(Q).T)
    lam = np.zeros(Qt.shape[0])
    res = np.zeros(Qt.shape[0])
    _load().oracle_rayleigh(A.shape[0], Qt.shape[0], _p(A), _p(Qt), _p(lam), _p(res))
    return lam, res


class Result:
    """Oracle outputs of one PFSM solve."""

    def __init__(self, n, nb):
        self.lam = np.zeros(n)
        self.V = np.zeros((n, n))
        self.res = np.zeros(n)
        self.xfs = np.zeros((n, n))
        self.eps = np.zeros(n)
        self.alpha = np.zeros(n)
        self.plan = np.zeros((4, nb), dtype=np.int32)


def pfsm(A, prev, nblocks: int, halo: int = -1, fs_iters: int = 3, alpha_theta: float = 1.0,
         cluster_tol: float = 1e-5, slice_sizes=None, keep_xfs: bool = True, fs_adaptive: bool = False,
         fs_tol: float = 0.0) -> Result:
    """The whole method on one matrix (Section II); fs_adaptive selects the Rayleigh-quotient
    variant of Eq. 11 with residual stopping (fs_iters is then the cap)."""
    A, prev = _f64(A), _f64(prev)
    n = A.shape[0]
    ss = None if slice_sizes is None else np.ascontiguousarray(slice_sizes, dtype=np.int32)
    prm = _Params(halo, fs_iters, alpha_theta, cluster_tol, _p(ss), int(bool(fs_adaptive)), fs_tol)
    r = Result(n, nblocks)
    xfs = r.xfs if keep_xfs else None
    st = _load().oracle_pfsm(n, nblocks, ctypes.byref(prm), _p(A), _p(prev), _p(r.lam), _p(r.V),
                             _p(r.res), _p(xfs), _p(r.eps), _p(r.alpha), _p(r.plan))
    if st:
        raise OracleError(st, "pfsm")
    if not keep_xfs:
        r.xfs = None
    return r


def backward(V, lam, dlam, dV, tau: float = 1e-8):
    """Eigen-adjoint dA for a loss with gradients dlam (N) and dV (N x N)."""
    V, lam = _f64(V), _f64(lam)
    n = V.shape[0]
    dlam = None if dlam is None else _f64(dlam)
    dV = np.zeros((n, n)) if dV is None else _f64(dV)
    dA = np.zeros((n, n))
    _load().oracle_backward(n, _p(V), _p(lam), _p(dlam), _p(dV), tau, _p(dA))
    return dA


def gen_to_std(A, B, max_iters: int = 50, tol: float = 1e-14):
    """Z = B^{-1} A by the Jacobi iteration of Eq. 14 (from Z_0 = 0). Returns (Z, iters, resid,
    status): status OK or NOT_CONVERGED (Z is then the last iterate)."""
    A, B = _f64(A), _f64(B)
    n = A.shape[0]
    Z = np.zeros((n, n))
    it, r = ctypes.c_int32(), ctypes.c_double()
    st = _load().oracle_gen_to_std(n, _p(A), _p(B), _p(Z), max_iters, tol, ctypes.byref(it), ctypes.byref(r))
    if st not in (OK, NOT_CONVERGED):
        raise OracleError(st, "gen_to_std")
    return Z, it.value, r.value, st


def gen_to_std_sym(A, B, max_iters: int = 50, tol: float = 1e-14):
    """Symmetric conversion C = B^{-1/2} A B^{-1/2} with S = B^{-1/2} by Newton-Schulz.
    Returns (C, S, iters, resid, status)."""
    A, B = _f64(A), _f64(B)
    n = A.shape[0]
    C, S = np.zeros((n, n)), np.zeros((n, n))
    it, r = ctypes.c_int32(), ctypes.c_double()
    st = _load().oracle_gen_to_std_sym(n, _p(A), _p(B), _p(C), _p(S), max_iters, tol, ctypes.byref(it),
                                       ctypes.byref(r))
    if st not in (OK, NOT_CONVERGED):
        raise OracleError(st, "gen_to_std_sym")
    return C, S, it.value, r.value, st


def guard(A) -> float:
    """Diagonal-dominance value g of A (largest l2 off-diagonal row norm / diagonal spread)."""
    A = _f64(A)
    g = ctypes.c_double()
    _load().oracle_guard(A.shape[0], _p(A), ctypes.byref(g))
    return g.value


def full(A):
    """Full diagonalization with the start-vector sign rule: (lam, V, res), V[:, k] vector k."""
    A = _f64(A)
    n = A.shape[0]
    lam, V, res = np.zeros(n), np.zeros((n, n)), np.zeros(n)
    st = _load().oracle_full(n, _p(A), _p(lam), _p(V), _p(res))
    if st:
        raise OracleError(st, "full")
    return lam, V, res


def pfsm_guarded(A, prev, nblocks: int, solve_index: int = 0, full_steps: int = 0, guard_max: float = 0.0,
                 **kw):
    """The method with the conventional first steps and the guard: solves with index below
    full_steps, and solves of an A whose guard value exceeds guard_max (> 0), are full
    diagonalizations. Returns (path, lam, V): path 0 method, 1 first-steps rule, 2 guard."""
    if solve_index < full_steps:
        lam, V, _ = full(A)
        return 1, lam, V
    if guard_max > 0.0 and guard(A) > guard_max:
        lam, V, _ = full(A)
        return 2, lam, V
    r = pfsm(A, prev, nblocks, **kw)
    return 0, r.lam, r.V


def scf_step(H, Vb, lam_prev, nblocks: int, solve_index: int = 1, full_steps: int = 0, guard_max: float = 0.0,
             **kw):
    """One step of the SCF loop the method assumes (the input "similar to the previous
    iteration"): A = sym(Vb^T H Vb) is the new Hamiltonian in the previous eigenbasis Vb (columns),
    solved with the previous eigenvalues as prev; the new basis is Vb V. Returns
    (path, lam, Vb_new). The products are library matrix products (numpy), the solve the oracle's."""
    H, Vb = _f64(H), _f64(Vb)
    A = Vb.T @ H @ Vb
    A = 0.5 * (A + A.T)
    path, lam, V = pfsm_guarded(A, lam_prev, nblocks, solve_index=solve_index, full_steps=full_steps,
                                guard_max=guard_max, **kw)
    return path, lam, Vb @ V


def fs_iterate_adaptive(A, X, eps, alpha, max_iters: int, tol_abs: float, theta: float = 1.0):
    """Rayleigh-quotient variant of Eq. 11 on the rows of X (copies). Returns (X, eps, alpha, iters,
    resid, status)."""
    A = _f64(A)
    X, eps, alpha = _f64(X).copy(), _f64(eps).copy(), _f64(alpha).copy()
    n = A.shape[0]
    lo, hi = gershgorin(A)
    it, r = ctypes.c_int32(), ctypes.c_double()
    st = _load().oracle_fs_iterate_adaptive(n, X.shape[0], _p(A), _p(X), _p(eps), _p(alpha), max_iters, tol_abs,
                                            theta, lo, hi, ctypes.byref(it), ctypes.byref(r))
    return X, eps, alpha, it.value, r.value, st
