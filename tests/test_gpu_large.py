"""GPU parity at full size: the silicon-vacancy-like N = 9072 matrix (36 slices, windows of 2068,
near-degenerate pairs) in the split-precision forms, and the aluminium-like metal N = 7200
(30 slices, windows of 1440) with the eigen-adjoint backward.

The oracle cannot redo a whole solve at these sizes in test time, so the checks are
  * sampled outputs the oracle computes one by one: the partition plan (bit-exact), and for one
    slice its window eigenpairs (oracle Householder + QR on that window) and its vectors after
    the Eq. 11 iterations (oracle Eq. 11 applied to those start vectors);
  * properties that hold at any size: orthonormality, the Gram-Schmidt relation between the
    vectors before and after orthonormalisation (V^T X upper triangular with positive diagonal),
    residuals equal to ||A v - lambda v||, trace(A) = sum(lambda), sorted eigenvalues within
    sqrt(sum r_k^2) of the exact spectrum (Weyl), the Hellmann-Feynman projector for an
    occupied-sum loss.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_07806_b300 as mod
    from paper_1502_07806_b300 import build
    build.build()
    mod.load_library()
    return mod


def _start_vectors_of_slice(orc, p, r_plan, b, eps_all):
    """Oracle start vectors, shifts and steps of slice b (Section II, readings R4-R6)."""
    k0, m, s, M = (int(v[b]) for v in r_plan)
    sub = p.A[s:s + M, s:s + M]
    w, Y = orc.symeig(sub)
    n = p.n
    X0 = np.zeros((n, m))
    eps = np.zeros(m)
    for t in range(m):
        col = k0 + t - s
        y = Y[:, col]
        yh = y[col]
        ref = yh if abs(yh) >= 0.1 else y[int(np.argmax(np.abs(y)))]
        X0[s:s + M, t] = y * (-1.0 if ref < 0 else 1.0)
        eps[t] = w[col]
    lo, hi = orc.gershgorin(p.A)
    dmax = np.maximum(hi - eps, eps - lo)
    alpha = np.minimum(1.0 / dmax ** 2, 1.0 - 2.0 ** -20)
    return k0, m, X0, eps, alpha


def _properties(p, lam, V, res, Xfs):
    n = p.n
    Vt = torch.from_numpy(V).cuda()
    A = torch.from_numpy(p.A).cuda()
    G = Vt.T @ Vt
    orth = float((G - torch.eye(n, dtype=torch.float64, device="cuda")).abs().max())
    assert orth < 1e-12, orth
    AV = A @ Vt
    R = torch.linalg.norm(AV - Vt * torch.from_numpy(lam).cuda(), dim=0).cpu().numpy()
    np.testing.assert_allclose(res, R, rtol=1e-5, atol=1e-12)
    assert abs(np.sum(lam) - np.trace(p.A)) < 1e-9 * n
    # Gram-Schmidt in index order: V^T Xfs is upper triangular with positive diagonal
    Rgs = (Vt.T @ torch.from_numpy(Xfs).cuda()).cpu().numpy()
    low = np.tril(Rgs, -1)
    assert np.max(np.abs(low)) < 1e-10 * np.max(np.abs(Rgs))
    assert np.all(np.diag(Rgs) > 0)
    return orth


@pytest.mark.parametrize("prec_name", ["bf16", "tf32"])
def test_vacancy_like_full_size(pf, orc, prec_name):
    p = wl.vacancy_like()
    prec = {"bf16": pf.BF16_SPLIT, "tf32": pf.TF32_SPLIT}[prec_name]
    h = pf.Handle(p.n, p.nblocks, precision=prec)
    lam, V = h.solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.prev).cuda())
    assert h.status() == 0
    plan = h.diagnostic(pf.DIAG_PLAN).cpu().numpy()
    ref_plan = orc.plan(p.prev, p.nblocks)
    for a, b in zip(plan, ref_plan):
        np.testing.assert_array_equal(a, b)
    eps = h.diagnostic(pf.DIAG_EPS).cpu().numpy()
    alpha = h.diagnostic(pf.DIAG_ALPHA).cpu().numpy()
    Xfs = h.diagnostic(pf.DIAG_XFS).cpu().numpy()
    res = h.diagnostic(pf.DIAG_RESIDUALS).cpu().numpy()
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    # sampled: one slice in the middle, recomputed by the oracle
    k0, m, X0, eps_ref, alpha_ref = _start_vectors_of_slice(orc, p, ref_plan, 17, eps)
    np.testing.assert_allclose(eps[k0:k0 + m], eps_ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(alpha[k0:k0 + m], alpha_ref, rtol=1e-10)
    X_ref = orc.fs_iterate(p.A, X0, eps_ref, alpha_ref, p.fs_iters)
    dx = np.max(np.abs(Xfs[:, k0:k0 + m] - X_ref))
    print(f"vacancy9072 {prec_name}: slice 17 vectors after Eq. 11 vs oracle: {dx:.2e}")
    # split products accumulate in FP32 over K = 9072 terms: ~sqrt(K) 2^-24 of sum |E||x|,
    # propagated by alpha (A - eps I); held to the eigenvector bar (projectors <= 1e-8)
    assert dx < 1e-8
    orth = _properties(p, lam, V, res, Xfs)
    # V^T A V = diag(lambda) + F with column norms of F equal to the residuals, so by Weyl the
    # sorted Rayleigh quotients lie within ||F||_2 <= sqrt(sum r_k^2) of the sorted spectrum
    ev = torch.linalg.eigvalsh(torch.from_numpy(p.A).cuda()).cpu().numpy()
    err = np.abs(np.sort(lam) - ev)
    bound = float(np.sqrt(np.sum(res ** 2)))
    print(f"vacancy9072 {prec_name}: orth {orth:.1e}, max |lambda - exact| {np.max(err):.2e}, "
          f"max residual {np.max(res):.2e}, Weyl bound {bound:.2e}")
    assert np.max(err) <= bound + 1e-12


def test_metal_like_full_size_with_backward(pf, orc):
    p = wl.metal_like()
    n = p.n
    h = pf.Handle(n, p.nblocks, halo=p.halo, precision=pf.BF16_SPLIT, recompute_v=True)
    A = torch.from_numpy(p.A).cuda()
    prev = torch.from_numpy(p.prev).cuda()
    lam, V = h.solve(A, prev)
    assert h.status() == 0
    np.testing.assert_array_equal(h.diagnostic(pf.DIAG_PLAN).cpu().numpy(),
                                  np.stack(orc.plan(p.prev, p.nblocks, halo=p.halo)))
    res = h.diagnostic(pf.DIAG_RESIDUALS).cpu().numpy()
    Xfs = h.diagnostic(pf.DIAG_XFS).cpu().numpy()
    lam_h, V_h = lam.cpu().numpy(), V.cpu().numpy()
    _properties(p, lam_h, V_h, res, Xfs)
    # occupied-sum loss: dA = V_occ V_occ^T (Hellmann-Feynman), V recomputed inside backward
    occ = 6000
    dlam = torch.zeros(n, dtype=torch.float64, device="cuda")
    dlam[:occ] = 1.0
    dA = h.backward(dlam, None)
    assert h.status() == 0
    P = V[:, :occ] @ V[:, :occ].T
    err = float((dA - P).abs().max())
    print(f"metal7200: |dA - V_occ V_occ^T| = {err:.2e}")
    assert err < 1e-11
    # full loss sum_occ lambda + <V, W>: symmetric result, and the adjoint identity
    # <dA, D> = d/dh L(A + h D) on the exact eigen-map is covered at small size in
    # test_gpu_parity.py / test_oracle_pins.py
    W = torch.from_numpy(wl.gaussian((n, n), seed=55)).cuda()
    dA = h.backward(dlam, W)
    assert h.status() == 0
    assert float((dA - dA.T).abs().max()) == 0.0
