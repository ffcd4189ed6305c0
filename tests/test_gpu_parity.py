"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs. Tolerances for the FP64 form: eigenvalues |dlambda| <= 1e-10 ||A|| (||A|| = largest
|eigenvalue|), eigenvectors by projector ||P_gpu - P_ref||_F <= 1e-8 (per vector; per cluster of
near-degenerate eigenvalues where a cluster exists)."""
import numpy as np
import pytest
import torch

import workloads as wl
from compare import projector_errors, spectral_scale

pytestmark = pytest.mark.gpu

LAM_TOL = 1e-10
PROJ_TOL = 1e-8


@pytest.fixture(scope="module")
def pf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_07806_b300 as mod
    from paper_1502_07806_b300 import build
    build.build()
    mod.load_library()
    return mod


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _run(pf, p, nblocks=None, **kw):
    nb = p.nblocks if nblocks is None else nblocks
    kw.setdefault("halo", p.halo)
    h = pf.Handle(p.n, nb, **kw)
    lam, V = h.solve(_dev(p.A), _dev(p.prev))
    st = h.status()
    out = dict(lam=lam.cpu().numpy(), V=V.cpu().numpy(), status=st,
               res=h.diagnostic(pf.DIAG_RESIDUALS).cpu().numpy(),
               xfs=h.diagnostic(pf.DIAG_XFS).cpu().numpy(),
               eps=h.diagnostic(pf.DIAG_EPS).cpu().numpy(),
               alpha=h.diagnostic(pf.DIAG_ALPHA).cpu().numpy(),
               plan=h.diagnostic(pf.DIAG_PLAN).cpu().numpy())
    out["handle"] = h
    return out


def _check(orc_res, g, lam_tol=LAM_TOL, proj_tol=PROJ_TOL, cluster_tol=0.0):
    assert g["status"] == 0
    np.testing.assert_array_equal(g["plan"], orc_res.plan)
    scale = spectral_scale(orc_res.lam)
    dl = np.max(np.abs(g["lam"] - orc_res.lam))
    assert dl <= lam_tol * scale, f"max |dlambda| = {dl:.3e}"
    pe = projector_errors(orc_res.V, g["V"], orc_res.lam, cluster_tol)
    assert np.max(pe) <= proj_tol, f"max projector error = {np.max(pe):.3e}"
    return dl / scale, float(np.max(pe))


def test_small_gapped_matches_oracle(pf, orc):
    p = wl.small_gapped(0)
    r = orc.pfsm(p.A, p.prev, p.nblocks)
    g = _run(pf, p)
    _check(r, g)
    # intermediate stages: shifts, steps, vectors after Eq. 11 (same sign rule on both sides)
    np.testing.assert_allclose(g["eps"], r.eps, rtol=0, atol=1e-13)
    np.testing.assert_allclose(g["alpha"], r.alpha, rtol=1e-12)
    np.testing.assert_allclose(g["xfs"], r.xfs, rtol=0, atol=1e-11)
    np.testing.assert_allclose(g["res"], r.res, rtol=1e-6, atol=1e-13)


@pytest.mark.parametrize("step", range(5))
def test_scf_sequence_matches_oracle(pf, orc, step):
    p = wl.small_gapped(step)
    r = orc.pfsm(p.A, p.prev, p.nblocks)
    _check(r, _run(pf, p))


@pytest.mark.parametrize("n,nb,halo,K", [
    (1, 1, -1, 3), (2, 1, -1, 3), (2, 2, 0, 2), (8, 3, 1, 3), (17, 4, 2, 1), (64, 5, -1, 3),
    (130, 7, 9, 4), (130, 1, -1, 3), (97, 6, 200, 3), (200, 9, 13, 0), (333, 11, 31, 5),
])
def test_ragged_and_edge_sizes(pf, orc, n, nb, halo, K):
    """Odd sizes that leave ragged GEMM tiles, slices of unequal size, windows clamped at both
    ends, a single slice (full eigendecomposition), halo >= N, K = 0."""
    p = wl.random_nearly_diagonal(n, seed=1000 + n + nb, sigma=2e-3, decay=12.0, nblocks=nb, halo=halo)
    r = orc.pfsm(p.A, p.prev, nb, halo=halo, fs_iters=K)
    g = _run(pf, p, fs_iters=K)
    _check(r, g)


def test_explicit_slice_sizes(pf, orc):
    p = wl.random_nearly_diagonal(150, seed=77, sigma=1e-3, nblocks=4, halo=10)
    sizes = [10, 70, 33, 37]
    r = orc.pfsm(p.A, p.prev, 4, halo=10, slice_sizes=sizes)
    g = _run(pf, p, slice_sizes=sizes)
    _check(r, g)


def test_cluster_snap_matches_oracle(pf, orc):
    """Near-degenerate pairs of previous eigenvalues on nominal slice boundaries."""
    p = wl.random_nearly_diagonal(256, seed=91, sigma=1e-3, nblocks=4)
    prev = p.prev.copy()
    for k in (64, 128, 129, 192):
        prev[k] = prev[k - 1] + 1e-7
    prev = np.maximum.accumulate(prev)
    A = p.A.copy()
    A[np.diag_indices(256)] = prev
    p.A, p.prev = A, prev
    r = orc.pfsm(A, prev, 4)
    assert list(r.plan[0]) != [0, 64, 128, 192]
    g = _run(pf, p)
    _check(r, g, cluster_tol=1e-6)


def test_zero_coupling_gives_identity(pf):
    lam = np.sort(np.random.default_rng(9).uniform(-1, 1, 96))
    p = wl.Problem("diag", np.diag(lam), lam, 4)
    g = _run(pf, p)
    assert g["status"] == 0
    np.testing.assert_allclose(g["V"], np.eye(96), rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["lam"], lam, rtol=0, atol=1e-15)


def test_diamond_like_matches_oracle(pf, orc):
    """N = 1280 in 10 slices of 128 (windows of 384): the benchmarked workload."""
    p = wl.diamond_like(0)
    r = orc.pfsm(p.A, p.prev, p.nblocks)
    g = _run(pf, p)
    dl, pe = _check(r, g)
    print(f"diamond1280: max|dlam|/||A|| = {dl:.2e}, max projector err = {pe:.2e}")


@pytest.mark.parametrize("step", [4, 6, 7])
@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_late_diamond_steps_match_oracle(pf, orc, step, prec):
    """Later SCF steps of the diamond-like workload (couplings 5e-6, 5e-7, 1.6e-7): nearly
    diagonal windows whose eigenvalue pairs about 5e-7 of the span apart share one FP32 bracket,
    so some lanes of the eigenvalue kernel stay uncertified after three Newton steps and take the
    retries and the lane-parallel multisection."""
    p = wl.diamond_like(step)
    r = orc.pfsm(p.A, p.prev, p.nblocks)
    g = _run(pf, p, precision=pf.FP64 if prec == "fp64" else pf.BF16_SPLIT)
    dl, pe = _check(r, g)
    print(f"diamond1280 step {step} {prec}: max|dlam|/||A|| = {dl:.2e}, max projector err = {pe:.2e}")


def test_invariants_on_gpu_result(pf):
    p = wl.diamond_like(3)
    g = _run(pf, p)
    V = g["V"]
    orth = np.max(np.abs(V.T @ V - np.eye(p.n)))
    assert orth < 1e-13
    assert abs(np.sum(g["lam"]) - np.trace(p.A)) < 1e-11
    R = p.A @ V - V * g["lam"]
    np.testing.assert_allclose(np.linalg.norm(R, axis=0), g["res"], rtol=1e-6, atol=1e-13)


# ------------------------------------------------------------------------------- errors --

def test_nan_input_is_reported(pf):
    p = wl.random_nearly_diagonal(40, seed=5, nblocks=2)
    A = p.A.copy()
    A[3, 7] = np.nan
    h = pf.Handle(40, 2)
    h.solve(_dev(A), _dev(p.prev))
    assert h.status() == pf.NAN_INPUT


def test_unsorted_prev_is_reported(pf):
    p = wl.random_nearly_diagonal(40, seed=6, nblocks=2)
    prev = p.prev.copy()
    prev[[5, 6]] = prev[[6, 5]]
    h = pf.Handle(40, 2)
    h.solve(_dev(p.A), _dev(prev))
    assert h.status() == pf.INVALID_ARG


def test_randomly_mixed_matrix_breaks_like_the_oracle(pf, orc):
    """The paper's failure mode (Section II): a randomly rotated spectrum."""
    n = 64
    rng = np.random.default_rng(13)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-1, 1, n))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    prev = np.sort(np.diag(A))
    h = pf.Handle(n, 8, halo=2)
    lg, _ = h.solve(_dev(A), _dev(prev))
    st = h.status()
    try:
        orc.pfsm(A, prev, 8, halo=2)
        oracle_breaks = False
    except orc.OracleError:
        oracle_breaks = True
    if oracle_breaks:
        assert st == pf.NOT_SPD
    else:
        assert st == 0 and np.max(np.abs(np.sort(lg.cpu().numpy()) - lam)) > 1e-2


def test_backward_before_solve(pf):
    h = pf.Handle(16, 2)
    with pytest.raises(pf.PFSMError) as e:
        h.backward(None, None)
    assert e.value.code == pf.NO_SOLVE


# ----------------------------------------------------------------------------- backward --

def test_backward_matches_oracle_gradient(pf, orc):
    p = wl.small_gapped(1)
    n = p.n
    r = orc.pfsm(p.A, p.prev, p.nblocks)
    W = wl.gaussian((n, n), seed=17)
    dlam = np.r_[np.ones(200), np.zeros(n - 200)]
    ref = orc.backward(r.V, r.lam, dlam, W, tau=1e-8)
    h = pf.Handle(n, p.nblocks)
    h.solve(_dev(p.A), _dev(p.prev))
    dA = h.backward(_dev(dlam), _dev(W)).cpu().numpy()
    assert h.status() == 0
    assert np.array_equal(dA, dA.T)
    err = np.max(np.abs(dA - ref)) / np.max(np.abs(ref))
    assert err < 1e-7, err


def test_backward_trace_loss_is_identity(pf):
    p = wl.small_gapped(2)
    h = pf.Handle(p.n, p.nblocks)
    h.solve(_dev(p.A), _dev(p.prev))
    dA = h.backward(_dev(np.ones(p.n)), None).cpu().numpy()
    np.testing.assert_allclose(dA, np.eye(p.n), rtol=0, atol=1e-12)


def test_backward_recompute_matches_kept(pf):
    p = wl.small_gapped(1)
    W = wl.gaussian((p.n, p.n), seed=3)
    outs = []
    for rec in (False, True):
        h = pf.Handle(p.n, p.nblocks, recompute_v=rec)
        A, prev = _dev(p.A), _dev(p.prev)
        h.solve(A, prev)
        outs.append(h.backward(None, _dev(W)).cpu().numpy())
        assert h.status() == 0
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", [2, 1], ids=["bf16", "tf32"])
def test_mixed_backward_matches_oracle(pf, orc, prec):
    """The mixed forms' backward (its three N^3 products as FP64-accurate digit products): against
    the oracle's adjoint evaluated at the GPU's own (lambda, V), which isolates the backward's
    arithmetic, and against the oracle's gradient from its own forward (the FP64 form's bar)."""
    p = wl.small_gapped(1)
    n = p.n
    W = wl.gaussian((n, n), seed=17)
    dlam = np.r_[np.ones(200), np.zeros(n - 200)]
    h = pf.Handle(n, p.nblocks, precision=prec)
    lam, V = h.solve(_dev(p.A), _dev(p.prev))
    dA = h.backward(_dev(dlam), _dev(W)).cpu().numpy()
    assert h.status() == 0
    assert np.array_equal(dA, dA.T)
    same = orc.backward(V.cpu().numpy(), lam.cpu().numpy(), dlam, W, tau=1e-8)
    err_same = np.max(np.abs(dA - same)) / np.max(np.abs(same))
    r = orc.pfsm(p.A, p.prev, p.nblocks)
    ref = orc.backward(r.V, r.lam, dlam, W, tau=1e-8)
    err = np.max(np.abs(dA - ref)) / np.max(np.abs(ref))
    print(f"mixed backward: vs oracle adjoint at the same (lambda, V) {err_same:.2e}, vs oracle gradient {err:.2e}")
    assert err_same < 1e-12, err_same
    assert err < 1e-7, err
    # sum of all eigenvalues: dA = I exactly up to the products' rounding
    dI = h.backward(_dev(np.ones(n)), None).cpu().numpy()
    np.testing.assert_allclose(dI, np.eye(n), rtol=0, atol=1e-12)
    # recomputing (lambda, V) inside the backward gives the kept result bit for bit (the last
    # solve's A and prev must stay valid for it)
    h2 = pf.Handle(n, p.nblocks, precision=prec, recompute_v=True)
    A2, prev2 = _dev(p.A), _dev(p.prev)
    h2.solve(A2, prev2)
    np.testing.assert_array_equal(h2.backward(_dev(dlam), _dev(W)).cpu().numpy(), dA)


def test_autograd_function(pf):
    p = wl.small_gapped(3)
    h = pf.Handle(p.n, p.nblocks)
    A = _dev(p.A).requires_grad_(True)
    lam, V = pf.PFSMFunction.apply(A, _dev(p.prev), h)
    loss = lam[:100].sum()
    loss.backward()
    Vn = V.detach().cpu().numpy()
    np.testing.assert_allclose(A.grad.cpu().numpy(), Vn[:, :100] @ Vn[:, :100].T, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------- mixed forms, edges --

@pytest.mark.parametrize("prec", [2, 1], ids=["bf16", "tf32"])
@pytest.mark.parametrize("n,nb,halo,K", [
    (1, 1, -1, 3), (2, 1, -1, 3), (2, 2, 0, 2), (8, 3, 1, 3), (17, 4, 2, 1), (64, 5, -1, 3),
    (130, 7, 9, 4), (130, 1, -1, 3), (97, 6, 200, 3), (200, 9, 13, 0),
])
def test_mixed_ragged_and_edge_sizes(pf, orc, n, nb, halo, K, prec):
    """The mixed forms on the same edge cases: windows of one or two rows (no reflectors), a single
    slice, halo >= N, K = 0, products far smaller than one tensor-core tile. Same FP64 bars."""
    p = wl.random_nearly_diagonal(n, seed=1000 + n + nb, sigma=2e-3, decay=12.0, nblocks=nb, halo=halo)
    r = orc.pfsm(p.A, p.prev, nb, halo=halo, fs_iters=K)
    g = _run(pf, p, fs_iters=K, precision=prec)
    _check(r, g)


@pytest.mark.parametrize("prec", [2, 1], ids=["bf16", "tf32"])
@pytest.mark.parametrize("n,nb,halo,K", [
    (120, 1, -1, 3), (200, 3, 40, 3), (333, 4, 50, 2), (513, 1, -1, 3), (700, 5, -1, 3), (450, 7, 90, 0),
    (301, 2, 150, 1),
])
def test_two_stage_reduction_matches_oracle(pf, orc, n, nb, halo, K, prec):
    """The two-stage window reduction (dense -> band of half-width 32 by digit products, FP64 bulge
    chasing with every task split over a warp pair, the bulge reflectors applied in float-float, the
    panel back-transformation by digit products) forced on windows from 66 to 700 rows: ragged
    windows and slices, one window covering the matrix, a window whose width is not a multiple of
    32, K = 0. Same FP64 bars as every other form."""
    p = wl.random_nearly_diagonal(n, seed=2000 + n + nb, sigma=1e-3, decay=24.0, nblocks=nb, halo=halo)
    r = orc.pfsm(p.A, p.prev, nb, halo=halo, fs_iters=K)
    g = _run(pf, p, fs_iters=K, precision=prec, reduction=2)
    _check(r, g)
    np.testing.assert_allclose(g["eps"], r.eps, rtol=0, atol=1e-12)


@pytest.fixture(scope="module")
def wide(orc):
    p = wl.random_nearly_diagonal(1800, seed=4242, sigma=1e-3, decay=24.0, nblocks=2)
    return p, orc.pfsm(p.A, p.prev, 2, fs_iters=p.fs_iters)       # ~20 s of CPU, once


@pytest.mark.parametrize("prec", [0, 2, 1], ids=["fp64", "bf16", "tf32"])
def test_wide_windows_match_oracle(pf, wide, prec):
    """Windows of 1260 rows (N = 1800, two slices, default halo): in the mixed forms the two-stage
    reduction by default, with bulge-chasing sweeps of both kinds (the first 106 with more tasks
    than warp pairs, one warp per task; the rest split over warp pairs), and in every form the
    inverse iteration that keeps its iterates in global memory (windows wider than 731 rows)."""
    p, r = wide
    g = _run(pf, p, precision=prec)
    assert int(np.max(g["plan"][3])) == 1260
    _check(r, g)


@pytest.mark.parametrize("prec", [2, 1], ids=["bf16", "tf32"])
def test_mixed_explicit_slices_cluster_snap_and_zero_coupling(pf, orc, prec):
    """Explicit uneven slices, near-degenerate previous eigenvalues on slice boundaries (the plan
    moves them), and a diagonal A (start vectors are unit vectors, V = I) in the mixed forms."""
    p = wl.random_nearly_diagonal(150, seed=77, sigma=1e-3, nblocks=4, halo=10)
    sizes = [10, 70, 33, 37]
    _check(orc.pfsm(p.A, p.prev, 4, halo=10, slice_sizes=sizes), _run(pf, p, slice_sizes=sizes, precision=prec))
    q = wl.random_nearly_diagonal(256, seed=91, sigma=1e-3, nblocks=4)
    prev = q.prev.copy()
    for k in (64, 128, 129, 192):
        prev[k] = prev[k - 1] + 1e-7
    prev = np.maximum.accumulate(prev)
    A = q.A.copy()
    A[np.diag_indices(256)] = prev
    q.A, q.prev = A, prev
    _check(orc.pfsm(A, prev, 4), _run(pf, q, precision=prec), cluster_tol=1e-6)
    lam = np.sort(np.random.default_rng(9).uniform(-1, 1, 96))
    d = wl.Problem("diag", np.diag(lam), lam, 4)
    g = _run(pf, d, precision=prec)
    assert g["status"] == 0
    np.testing.assert_allclose(g["V"], np.eye(96), rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["lam"], lam, rtol=0, atol=1e-15)
