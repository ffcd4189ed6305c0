"""B300-native partitioned folded spectrum method (PFSM, arXiv:1502.07806, Section II).

Thin Python binding over the C ABI in ``include/pfsm.h``: this module only marshals torch CUDA
tensors (device pointers, sizes, the current stream) into ``libpfsm.so``. Every step of the
method runs in the library's CUDA kernels; there is no CPU path. If the library is missing the
calls raise ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpfsm.so")

OK, INVALID_ARG, CUDA_ERROR, NOT_SPD, NAN_INPUT, NOT_CONVERGED, TIMEOUT, NO_SOLVE, OUT_OF_MEMORY = range(9)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA_ERROR", 3: "NOT_SPD", 4: "NAN_INPUT",
                5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "NO_SOLVE", 8: "OUT_OF_MEMORY"}
FP64, TF32_SPLIT, BF16_SPLIT = 0, 1, 2
DIAG_RESIDUALS, DIAG_XFS, DIAG_EPS, DIAG_ALPHA, DIAG_PLAN = range(5)

EXPORTED = ("pfsm_default_params", "pfsm_init", "pfsm_solve", "pfsm_backward", "pfsm_get_status",
            "pfsm_get_diagnostic", "pfsm_set_timing", "pfsm_get_profile", "pfsm_last_error",
            "pfsm_destroy", "pfsm_fs_iterate_noalloc", "pfsm_split_gemm", "pfsm_split_gemm_ex", "pfsm_batch_init",
            "pfsm_solve_batched", "pfsm_batch_get_status", "pfsm_batch_destroy", "pfsm_gen_to_std",
            "pfsm_gen_to_std_sym", "pfsm_scf_step", "pfsm_selftest_fp64_helpers", "pfsm_selftest_i64_to_f64")
PHASES = ("plan", "submatrix", "fs_iterations", "gram_schmidt", "rayleigh", "backward")
SUB_PHASES = ("tridiag", "bisect", "inverse_iter", "backtransform", "overlap", "cholesky")
# two-stage reduction (mixed forms, wide windows): inside "tridiag" and "backtransform"
BAND_PHASES = ("band_panels", "band_chase", "band_bt_chase", "band_bt_panels")


class PFSMError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}" + (f" ({detail})" if detail else ""))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("halo", ctypes.c_int32), ("fs_iters", ctypes.c_int32),
                ("alpha_theta", ctypes.c_double), ("cluster_tol", ctypes.c_double),
                ("degen_tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("recompute_v", ctypes.c_int32), ("slice_sizes", ctypes.POINTER(ctypes.c_int32)),
                ("guard_max", ctypes.c_double), ("full_steps", ctypes.c_int32),
                ("fs_adaptive", ctypes.c_int32), ("fs_tol", ctypes.c_double), ("reduction", ctypes.c_int32)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32), ("timed", ctypes.c_int32),
                ("phase_ms", ctypes.c_float * 12), ("gemm_tile_n", ctypes.c_int32),
                ("path", ctypes.c_int32), ("guard_value", ctypes.c_double),
                ("fs_steps", ctypes.c_int32), ("fs_residual", ctypes.c_double),
                ("gs_precond", ctypes.c_int32), ("gs_precond_residual", ctypes.c_double),
                ("band_ms", ctypes.c_float * 4)]


_lib = None


def load_library():
    """Loads libpfsm.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"PFSM CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_1502_07806_b300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.pfsm_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.pfsm_default_params.restype = None
    lib.pfsm_init.argtypes = [i64, i32, ctypes.POINTER(Params), ctypes.POINTER(P)]
    lib.pfsm_solve.argtypes = [P, P, P, P, P, P]
    lib.pfsm_backward.argtypes = [P, P, P, P, P]
    lib.pfsm_get_status.argtypes = [P, ctypes.POINTER(i32)]
    lib.pfsm_get_diagnostic.argtypes = [P, i32, P, P]
    lib.pfsm_fs_iterate_noalloc.argtypes = [i64, i64, P, P, P, P, i32, P]
    lib.pfsm_split_gemm.argtypes = [i64, i64, i64, P, P, P, i32, P]
    lib.pfsm_split_gemm_ex.argtypes = [i64, i64, i64, P, P, P, i32, i32, P]
    lib.pfsm_gen_to_std.argtypes = [i64, P, P, P, i32, ctypes.c_double, P, P, P]
    lib.pfsm_gen_to_std_sym.argtypes = [i64, P, P, P, P, i32, ctypes.c_double, P, P, P]
    lib.pfsm_scf_step.argtypes = [P, P, P, P, P, P]
    lib.pfsm_batch_init.argtypes = [i32, P, P, ctypes.POINTER(Params), ctypes.POINTER(P)]
    lib.pfsm_solve_batched.argtypes = [P, P, P, P, P, P]
    lib.pfsm_batch_get_status.argtypes = [P, P]
    lib.pfsm_batch_destroy.argtypes = [P]
    lib.pfsm_set_timing.argtypes = [P, i32]
    lib.pfsm_get_profile.argtypes = [P, ctypes.POINTER(Profile)]
    lib.pfsm_last_error.argtypes = []
    lib.pfsm_selftest_fp64_helpers.argtypes = [P, i64, P, P, P, P, P]
    lib.pfsm_selftest_i64_to_f64.argtypes = [P, P, i64, P, P]
    lib.pfsm_last_error.restype = ctypes.c_char_p
    lib.pfsm_destroy.argtypes = [P]
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != OK:
        raise PFSMError(rc, where, load_library().pfsm_last_error().decode())


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_params() -> Params:
    p = Params()
    load_library().pfsm_default_params(ctypes.byref(p))
    return p


class Handle:
    """Owns one pfsm_handle_t (workspace for N x N problems split into nblocks slices)."""

    def __init__(self, n: int, nblocks: int, halo: int = -1, fs_iters: int = 3,
                 alpha_theta: float = 1.0, cluster_tol: float = 1e-5, degen_tol: float = 1e-8,
                 precision: int = FP64, recompute_v: bool = False, slice_sizes=None,
                 guard_max: float = 0.0, full_steps: int = 0, fs_adaptive: bool = False, fs_tol: float = 0.0,
                 reduction: int = 0):
        lib = load_library()
        p = default_params()
        p.halo, p.fs_iters, p.alpha_theta = halo, fs_iters, alpha_theta
        p.cluster_tol, p.degen_tol, p.precision = cluster_tol, degen_tol, precision
        p.recompute_v = int(bool(recompute_v))
        p.guard_max, p.full_steps = guard_max, full_steps
        p.fs_adaptive, p.fs_tol = int(bool(fs_adaptive)), fs_tol
        p.reduction = reduction
        self._sizes = None
        if slice_sizes is not None:
            self._sizes = (ctypes.c_int32 * nblocks)(*[int(x) for x in slice_sizes])
            p.slice_sizes = ctypes.cast(self._sizes, ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        _check(lib.pfsm_init(n, nblocks, ctypes.byref(p), ctypes.byref(h)), "pfsm_init")
        self._h, self.n, self.nblocks = h, n, nblocks

    def close(self):
        if getattr(self, "_h", None):
            load_library().pfsm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, A: torch.Tensor, prev: torch.Tensor, eigvals_out: torch.Tensor | None = None,
              V_out: torch.Tensor | None = None):
        n = self.n
        if eigvals_out is None:
            eigvals_out = torch.empty(n, dtype=torch.float64, device=A.device)
        if V_out is None:
            V_out = torch.empty(n, n, dtype=torch.float64, device=A.device)
        _check(load_library().pfsm_solve(self._h, _ptr(A), _ptr(prev), _ptr(eigvals_out),
                                         _ptr(V_out), _stream()), "pfsm_solve")
        return eigvals_out, V_out

    def backward(self, dlam: torch.Tensor | None, dV: torch.Tensor | None,
                 dA_out: torch.Tensor | None = None):
        n = self.n
        if dA_out is None:
            dA_out = torch.empty(n, n, dtype=torch.float64, device="cuda")
        _check(load_library().pfsm_backward(self._h, _ptr(dlam), _ptr(dV), _ptr(dA_out), _stream()),
               "pfsm_backward")
        return dA_out

    def scf_step(self, H: torch.Tensor, Vb: torch.Tensor, lam_prev: torch.Tensor,
                 lam_out: torch.Tensor | None = None) -> torch.Tensor:
        """One chained SCF step: solve sym(Vb^T H Vb) with lam_prev, Vb <- Vb V in place.
        Returns the eigenvalues."""
        if lam_out is None:
            lam_out = torch.empty(self.n, dtype=torch.float64, device=H.device)
        _check(load_library().pfsm_scf_step(self._h, _ptr(H), _ptr(Vb), _ptr(lam_prev), _ptr(lam_out),
                                            _stream()), "pfsm_scf_step")
        return lam_out

    def status(self) -> int:
        s = ctypes.c_int32(-1)
        _check(load_library().pfsm_get_status(self._h, ctypes.byref(s)), "pfsm_get_status")
        return s.value

    def set_timing(self, enable: bool = True):
        _check(load_library().pfsm_set_timing(self._h, int(bool(enable))), "pfsm_set_timing")

    def profile(self) -> dict:
        """Launch count and per-phase CUDA-event times (ms) of the last call on this handle."""
        pr = Profile()
        _check(load_library().pfsm_get_profile(self._h, ctypes.byref(pr)), "pfsm_get_profile")
        out = {"launches": pr.launches, "gemm_tile_n": pr.gemm_tile_n, "path": pr.path,
               "guard_value": pr.guard_value, "fs_steps": pr.fs_steps, "fs_residual": pr.fs_residual,
               "gs_precond": pr.gs_precond, "gs_precond_residual": pr.gs_precond_residual}
        if pr.timed:
            out.update({name: float(pr.phase_ms[i]) for i, name in enumerate(PHASES)})
            out.update({name: float(pr.phase_ms[6 + i]) for i, name in enumerate(SUB_PHASES)})
            out.update({name: float(pr.band_ms[i]) for i, name in enumerate(BAND_PHASES)})
        return out

    def diagnostic(self, which: int) -> torch.Tensor:
        n = self.n
        if which == DIAG_XFS:
            out = torch.empty(n, n, dtype=torch.float64, device="cuda")
        elif which == DIAG_PLAN:
            out = torch.empty(max(1, (4 * self.nblocks + 1) // 2), dtype=torch.float64, device="cuda")
        else:
            out = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(load_library().pfsm_get_diagnostic(self._h, which, ctypes.c_void_p(out.data_ptr()), _stream()),
               "pfsm_get_diagnostic")
        if which == DIAG_PLAN:
            return out.view(torch.int32)[: 4 * self.nblocks].reshape(4, self.nblocks)
        return out


def fs_iterate_noalloc(A: torch.Tensor, X_rows: torch.Tensor, eps: torch.Tensor,
                       alpha: torch.Tensor, iters: int) -> torch.Tensor:
    """Eq. 11 in place on the rows of X_rows (count x N) with no device allocation in the
    library (its scratch is a fixed 8 MiB device array; count * N <= 2^20)."""
    n, count = A.shape[0], X_rows.shape[0]
    _check(load_library().pfsm_fs_iterate_noalloc(n, count, _ptr(A), _ptr(X_rows), _ptr(eps),
                                                  _ptr(alpha), iters, _stream()),
           "pfsm_fs_iterate_noalloc")
    return X_rows


class Batch:
    """Many independent problems of uneven N solved by one captured CUDA graph."""

    def __init__(self, sizes, nblocks, halo: int = -1, fs_iters: int = 3, precision: int = FP64,
                 alpha_theta: float = 1.0, cluster_tol: float = 1e-5):
        lib = load_library()
        p = default_params()
        p.halo, p.fs_iters, p.precision = halo, fs_iters, precision
        p.alpha_theta, p.cluster_tol = alpha_theta, cluster_tol
        self.sizes = [int(n) for n in sizes]
        self.count = len(self.sizes)
        ns = (ctypes.c_int64 * self.count)(*self.sizes)
        nb = (ctypes.c_int32 * self.count)(*[int(x) for x in nblocks])
        b = ctypes.c_void_p()
        _check(lib.pfsm_batch_init(self.count, ns, nb, ctypes.byref(p), ctypes.byref(b)), "pfsm_batch_init")
        self._b = b

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def solve(self, As, prevs, lams=None, Vs=None):
        if lams is None:
            lams = [torch.empty(n, dtype=torch.float64, device="cuda") for n in self.sizes]
        if Vs is None:
            Vs = [torch.empty(n, n, dtype=torch.float64, device="cuda") for n in self.sizes]
        for t in list(As) + list(prevs) + list(lams) + list(Vs):
            _ptr(t)   # type / device / layout checks
        _check(load_library().pfsm_solve_batched(self._b, self._ptrs(As), self._ptrs(prevs),
                                                 self._ptrs(lams), self._ptrs(Vs), _stream()),
               "pfsm_solve_batched")
        return lams, Vs

    def status(self):
        out = (ctypes.c_int32 * self.count)()
        _check(load_library().pfsm_batch_get_status(self._b, out), "pfsm_batch_get_status")
        return list(out)

    @classmethod
    def autotuned(cls, As, prevs, halo: int = -1, fs_iters: int = 3, precision: int = FP64,
                  cache_path: str | None = None, **kw):
        """A batch whose block counts are measured per size class (autotune.tune on the first
        problem of each class; later problems of the class reuse it)."""
        from . import autotune
        nblocks = [autotune.tune(A, prev, precision, halo=halo, fs_iters=fs_iters, cache_path=cache_path)
                   for A, prev in zip(As, prevs)]
        return cls([int(A.shape[0]) for A in As], nblocks, halo=halo, fs_iters=fs_iters,
                   precision=precision, **kw)

    def close(self):
        if getattr(self, "_b", None):
            load_library().pfsm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split_gemm(P: torch.Tensor, Q: torch.Tensor, precision: int = BF16_SPLIT, tile_n: int = 0) -> torch.Tensor:
    """C = P Q^T on the tensor cores in split BF16/TF32 or FP64-accurate digits (FP64 in and out);
    tile_n: output-tile width of the split products (64, 96, 128; 0 = autotuned)."""
    rows, K = P.shape
    cols = Q.shape[0]
    C = torch.empty(rows, cols, dtype=torch.float64, device=P.device)
    _check(load_library().pfsm_split_gemm_ex(rows, cols, K, _ptr(P), _ptr(Q), _ptr(C), precision, tile_n,
                                             _stream()), "pfsm_split_gemm_ex")
    return C


def gen_to_std(A: torch.Tensor, B: torch.Tensor, max_iters: int = 50, tol: float = 1e-12,
               check: bool = True):
    """Z = B^-1 A by the Jacobi iteration of Eq. 14 on the device. Returns (Z, iters, resid);
    with check=False a PFSM_ERR_NOT_CONVERGED result is returned instead of raised. The
    residual is itself a digit product, with a floor of about sqrt(N) 2^-46: tol should stay
    above it."""
    n = A.shape[0]
    Z = torch.empty(n, n, dtype=torch.float64, device=A.device)
    it, r = ctypes.c_int32(), ctypes.c_double()
    rc = load_library().pfsm_gen_to_std(n, _ptr(A), _ptr(B), _ptr(Z), max_iters, tol, ctypes.byref(it),
                                        ctypes.byref(r), _stream())
    if check or rc != 5:
        _check(rc, "pfsm_gen_to_std")
    return Z, it.value, r.value


def gen_to_std_sym(A: torch.Tensor, B: torch.Tensor, max_iters: int = 50, tol: float = 1e-11,
                   check: bool = True):
    """C = B^-1/2 A B^-1/2 and S = B^-1/2 (Newton-Schulz) on the device. Returns (C, S, iters, resid).
    The residual max|I - Q Y| has a floor of a few sqrt(N) 2^-46 (1.6e-12 at N = 200)."""
    n = A.shape[0]
    C = torch.empty(n, n, dtype=torch.float64, device=A.device)
    S = torch.empty(n, n, dtype=torch.float64, device=A.device)
    it, r = ctypes.c_int32(), ctypes.c_double()
    rc = load_library().pfsm_gen_to_std_sym(n, _ptr(A), _ptr(B), _ptr(C), _ptr(S), max_iters, tol,
                                            ctypes.byref(it), ctypes.byref(r), _stream())
    if check or rc != 5:
        _check(rc, "pfsm_gen_to_std_sym")
    return C, S, it.value, r.value


def solve(A: torch.Tensor, prev: torch.Tensor, nblocks: int, **kw):
    """One-shot solve: returns (eigvals, V, status)."""
    h = Handle(A.shape[0], nblocks, **kw)
    lam, V = h.solve(A, prev)
    st = h.status()
    h.close()
    return lam, V, st


class PFSMFunction(torch.autograd.Function):
    """(A, prev) -> (eigvals, V) through the PFSM kernels, with the eigen-adjoint backward."""

    @staticmethod
    def forward(ctx, A, prev, handle: Handle):
        lam, V = handle.solve(A.contiguous(), prev.contiguous())
        ctx.handle = handle
        return lam, V

    @staticmethod
    def backward(ctx, dlam, dV):
        dlam = None if dlam is None else dlam.contiguous()
        dV = None if dV is None else dV.contiguous()
        dA = ctx.handle.backward(dlam, dV)
        return dA, None, None
