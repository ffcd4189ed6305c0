"""The allocation-free Eq. 11 entry point (for callers that cannot allocate device memory at
call time: codes that reserve all device memory for their own pool, or latency-critical loops
that cudaMalloc's device-wide synchronisation would stall) against the regular solve path and
against the oracle's Eq. 11.

Kept in a file of its own that pytest collects last: it must pass both alone in a fresh
process and after every other test, and a failure here should not hide the others."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as wl

CAP = 1 << 20          # count * N limit of the entry point's fixed scratch array


def _lib():
    import paper_1502_07806_b300 as pf
    from paper_1502_07806_b300 import build
    build.build()
    return pf, pf.load_library()


def _call(lib, n, count, A, X, eps, alpha, iters=3):
    return lib.pfsm_fs_iterate_noalloc(n, count, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(alpha.data_ptr()), iters,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_rejects_oversized_input_without_a_gpu():
    pf, lib = _lib()
    # count * N above 2^20: refused before any device work
    rc = lib.pfsm_fs_iterate_noalloc(2048, 1024, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     ctypes.c_void_p(16), ctypes.c_void_p(16), 3, None)
    assert rc == pf.INVALID_ARG
    rc = lib.pfsm_fs_iterate_noalloc(1024, 1025, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     ctypes.c_void_p(16), ctypes.c_void_p(16), 3, None)
    assert rc == pf.INVALID_ARG
    rc = lib.pfsm_fs_iterate_noalloc(64, 8, None, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     ctypes.c_void_p(16), 3, None)
    assert rc == pf.INVALID_ARG


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _lib()


@pytest.mark.gpu
def test_noalloc_matches_regular_path_twice_in_a_row():
    pf, lib = _gpu()
    for call, step in enumerate((0, 3)):       # two calls in a row, different inputs
        p = wl.small_gapped(step)
        A = torch.from_numpy(p.A).cuda()
        prev = torch.from_numpy(p.prev).cuda()
        # start vectors, shifts and steps from the regular path (K = 0 exposes the start vectors)
        h0 = pf.Handle(p.n, p.nblocks, fs_iters=0)
        h0.solve(A, prev)
        X0 = h0.diagnostic(pf.DIAG_XFS)             # V layout: column k = vector k
        eps = h0.diagnostic(pf.DIAG_EPS)
        alpha = h0.diagnostic(pf.DIAG_ALPHA)
        assert h0.status() == 0
        # the regular path's vectors after K = 3 iterations
        h3 = pf.Handle(p.n, p.nblocks, fs_iters=3)
        h3.solve(A, prev)
        ref = h3.diagnostic(pf.DIAG_XFS).cpu().numpy()
        assert h3.status() == 0
        X = X0.t().contiguous()                     # rows = vectors
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call(lib, p.n, p.n, A, X, eps, alpha) == pf.OK, call
        torch.cuda.synchronize()
        if call == 1:
            # the module holding the scratch array is loaded by the first call; later calls
            # leave the device's free memory exactly as it was
            assert torch.cuda.mem_get_info()[0] == free0
        got = X.t().cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
        h0.close()
        h3.close()


@pytest.mark.gpu
def test_noalloc_matches_oracle_eq11_on_oracle_start_vectors(orc):
    pf, lib = _gpu()
    p = wl.small_gapped(1)
    start = orc.pfsm(p.A, p.prev, p.nblocks, fs_iters=0)       # start vectors, shifts, steps
    ref = orc.fs_iterate(p.A, start.xfs, start.eps, start.alpha, 3)
    A = torch.from_numpy(p.A).cuda()
    X = torch.from_numpy(np.ascontiguousarray(start.xfs.T)).cuda()
    eps = torch.from_numpy(start.eps).cuda()
    alpha = torch.from_numpy(start.alpha).cuda()
    assert _call(lib, p.n, p.n, A, X, eps, alpha) == pf.OK
    np.testing.assert_allclose(X.t().cpu().numpy(), ref, rtol=0, atol=1e-12)
    # fewer vectors than N (count != N): a contiguous subset of rows
    lo, c = 37, 50
    Xs = torch.from_numpy(np.ascontiguousarray(start.xfs[:, lo:lo + c].T)).cuda()
    es, als = eps[lo:lo + c].contiguous(), alpha[lo:lo + c].contiguous()
    assert _call(lib, p.n, c, A, Xs, es, als) == pf.OK
    np.testing.assert_allclose(Xs.t().cpu().numpy(), ref[:, lo:lo + c], rtol=0, atol=1e-12)


@pytest.mark.gpu
def test_noalloc_at_its_size_limit():
    pf, lib = _gpu()
    p = wl.random_nearly_diagonal(1024, seed=77, sigma=1e-3, nblocks=8)
    assert p.n * p.n == CAP                      # count * N exactly at the limit
    A = torch.from_numpy(p.A).cuda()
    prev = torch.from_numpy(p.prev).cuda()
    h0 = pf.Handle(p.n, p.nblocks, fs_iters=0)
    h0.solve(A, prev)
    X = h0.diagnostic(pf.DIAG_XFS).t().contiguous()
    eps, alpha = h0.diagnostic(pf.DIAG_EPS), h0.diagnostic(pf.DIAG_ALPHA)
    h3 = pf.Handle(p.n, p.nblocks, fs_iters=3)
    h3.solve(A, prev)
    ref = h3.diagnostic(pf.DIAG_XFS).cpu().numpy()
    assert h0.status() == 0 and h3.status() == 0
    assert _call(lib, p.n, p.n, A, X, eps, alpha) == pf.OK
    np.testing.assert_allclose(X.t().cpu().numpy(), ref, rtol=0, atol=1e-12)
    h0.close()
    h3.close()
