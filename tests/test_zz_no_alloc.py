"""The allocation-free Eq. 11 entry point (for callers that cannot allocate device memory at
call time) matches the regular solve path.

Kept in a file of its own that pytest collects last: it must pass both alone in a fresh
process and after every other test, and a failure here should not hide the others."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as wl


def test_noalloc_rejects_oversized_input_without_a_gpu():
    import paper_1502_07806_b300 as pf
    from paper_1502_07806_b300 import build
    build.build()
    lib = pf.load_library()
    # count * N above 2^20: refused before any device work
    rc = lib.pfsm_fs_iterate_noalloc(2048, 1024, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     ctypes.c_void_p(16), ctypes.c_void_p(16), 3, None)
    assert rc == pf.INVALID_ARG
    rc = lib.pfsm_fs_iterate_noalloc(64, 8, None, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     ctypes.c_void_p(16), 3, None)
    assert rc == pf.INVALID_ARG


@pytest.mark.gpu
def test_noalloc_matches_regular_path_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_07806_b300 as pf
    from paper_1502_07806_b300 import build
    build.build()
    lib = pf.load_library()
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
        rc = lib.pfsm_fs_iterate_noalloc(p.n, p.n, ctypes.c_void_p(A.data_ptr()),
                                         ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(eps.data_ptr()),
                                         ctypes.c_void_p(alpha.data_ptr()), 3,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == pf.OK, call
        torch.cuda.synchronize()
        got = X.t().cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
        h0.close()
        h3.close()
