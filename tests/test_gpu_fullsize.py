"""GPU parity at full size against the FP64 oracle's own outputs for the same inputs.

The oracle needs tens of CPU-minutes per solve at these sizes, so its outputs were computed once by
``tests/golden/make_fullsize.py`` (which calls only ``oracle/``) and stored under ``tests/golden/``
keyed by the SHA-256 of the input. Compared here, for every precision form:
  * the partition plan, bit for bit;
  * every shift eps_k (window eigenvalue) and step alpha_k, and every eigenvalue lambda_k
    (|dlambda| <= 1e-10 ||A||, ||A|| = max |lambda_ref|);
  * every residual ||A v_k - lambda_k v_k||;
  * a sample of eigenvectors in full (projector error <= 1e-8), including near-degenerate pairs of
    previous eigenvalues (1e-6 apart), and a sketch of EVERY eigenvector: with Omega the seeded
    24 x N Gaussian matrix, ||Omega (v - v_ref)|| / sqrt(24) estimates ||v - v_ref|| (a chi
    variable with 24 degrees of freedom: within a factor 0.5 .. 1.6 of the true value except with
    probability 1.1e-4), held to the same 1e-8;
  * a sample of the vectors after the Eq. 11 iterations (before Gram-Schmidt), <= 1e-8.
The per-eigenvalue errors of each form are printed (max, median, 99th percentile).
"""
import os
import sys

import numpy as np
import pytest
import torch

import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import fullsize_ref as fr  # noqa: E402

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


def _golden(name, p):
    g = fr.load(name)
    assert str(g["sha256_A"]) == fr.sha256(p.A), f"{name}: input differs from the stored one (rerun make_fullsize.py)"
    assert str(g["sha256_prev"]) == fr.sha256(p.prev)
    return g


def _vector_errors(U, V):
    """Per column ||u u^T - v v^T||_F of unit columns (sign-free)."""
    d = np.sum(U * V, axis=0)
    return np.linalg.norm(U - V * np.where(d < 0, -1.0, 1.0), axis=0) * np.sqrt(1.0 + np.abs(d))


def check_against_golden(pf, p, g, h, lam, V, tag):
    n = p.n
    assert h.status() == 0
    np.testing.assert_array_equal(h.diagnostic(pf.DIAG_PLAN).cpu().numpy(), g["plan"])
    np.testing.assert_allclose(h.diagnostic(pf.DIAG_EPS).cpu().numpy(), g["eps"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(h.diagnostic(pf.DIAG_ALPHA).cpu().numpy(), g["alpha"], rtol=1e-10)
    lam_h = lam.cpu().numpy()
    scale = float(np.max(np.abs(g["lam"])))
    dl = np.abs(lam_h - g["lam"]) / scale
    res = h.diagnostic(pf.DIAG_RESIDUALS).cpu().numpy()
    np.testing.assert_allclose(res, g["res"], rtol=1e-4, atol=1e-12)
    cols = torch.from_numpy(g["cols"]).cuda()
    pe = _vector_errors(g["V_cols"], V.index_select(1, cols).cpu().numpy())
    Om = torch.from_numpy(fr.sketch_matrix(n, int(g["sketch_seed"]))).cuda()
    Sg = (Om @ V).cpu().numpy()
    Sr = g["sketch"]
    sgn = np.where(np.sum(Sg * Sr, axis=0) < 0, -1.0, 1.0)
    est = np.linalg.norm(Sg * sgn - Sr, axis=0) / np.sqrt(fr.SKETCH)
    xcols = torch.from_numpy(g["xcols"]).cuda()
    Xfs = h.diagnostic(pf.DIAG_XFS)
    dx = float(np.max(np.abs(Xfs.index_select(1, xcols).cpu().numpy() - g["X_cols"])))
    print(f"{tag}: |dlambda|/||A|| max {dl.max():.2e} median {np.median(dl):.2e} p99 {np.quantile(dl, 0.99):.2e}; "
          f"projector (sampled {pe.size}) {pe.max():.2e}; vector error sketch (all {n}) max {est.max():.2e} "
          f"median {np.median(est):.2e}; vectors after Eq. 11 {dx:.2e}")
    assert dl.max() <= LAM_TOL, dl.max()
    assert pe.max() <= PROJ_TOL, pe.max()
    assert est.max() <= PROJ_TOL, est.max()
    assert dx <= 1e-8, dx


@pytest.fixture(scope="module")
def vacancy():
    p = wl.vacancy_like()
    return p, _golden("vacancy9072", p)


@pytest.mark.parametrize("prec_name", ["bf16", "tf32", "fp64"])
def test_vacancy_like_full_size_matches_oracle(pf, vacancy, prec_name):
    """N = 9072, 36 slices, windows of 2068: the mixed forms reduce the windows in two stages (dense
    to band with digit products, bulge chasing), the FP64 form in one."""
    p, g = vacancy
    prec = {"bf16": pf.BF16_SPLIT, "tf32": pf.TF32_SPLIT, "fp64": pf.FP64}[prec_name]
    h = pf.Handle(p.n, p.nblocks, precision=prec)
    A, prev = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.prev).cuda()
    lam, V = h.solve(A, prev)
    check_against_golden(pf, p, g, h, lam, V, f"vacancy9072 {prec_name}")
    h.close()


def test_vacancy_like_one_stage_reduction_matches_oracle(pf, vacancy):
    """The mixed form with the one-stage window reduction forced (the automatic choice for windows
    narrower than 1024 rows) gives the oracle's outputs on the same full-size input too."""
    p, g = vacancy
    h = pf.Handle(p.n, p.nblocks, precision=pf.BF16_SPLIT, reduction=1)
    A, prev = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.prev).cuda()
    lam, V = h.solve(A, prev)
    check_against_golden(pf, p, g, h, lam, V, "vacancy9072 bf16 one-stage")
    h.close()


# ---------------------------------------------------------------------------------------------
# Metal-like N = 7200 (30 slices, halo 600, windows of 1440): forward and eigen-adjoint backward of
# the loss sum_{k < 6000} lambda_k + <V, W>, V recomputed inside the backward.

@pytest.fixture(scope="module")
def metal():
    p = wl.metal_like()
    return p, _golden("metal7200", p)


@pytest.fixture(scope="module")
def metal_directions(metal):
    """The 32 unit-Frobenius symmetric directions the oracle's directional derivatives used."""
    p, g = metal
    return [wl.symmetric_direction(p.n, int(s)) for s in g["dir_seeds"]]


def _loss_grads(p, g):
    dlam = np.zeros(p.n)
    dlam[:int(g["occupied"])] = 1.0
    W = wl.gaussian((p.n, p.n), seed=int(g["w_seed"]))
    return dlam, W


@pytest.mark.parametrize("prec_name", ["bf16", "fp64"])
def test_metal_like_full_size_forward_and_gradient_match_oracle(pf, metal, metal_directions, prec_name):
    """Forward against the oracle as for the vacancy-like matrix; the gradient against the oracle's
    gradient (from the oracle's own eigenpairs) on 8192 sampled entries, the whole diagonal and 32
    directional derivatives <dA, D_d>. The gradient amplifies eigenvector differences by the
    coupling factors 1/(lambda_j - lambda_i) (up to 5e5 here), so its bar is 1e-6 of max |dA|
    (measured: see the printed errors)."""
    p, g = metal
    prec = {"bf16": pf.BF16_SPLIT, "fp64": pf.FP64}[prec_name]
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, precision=prec, recompute_v=True)
    A, prev = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.prev).cuda()
    lam, V = h.solve(A, prev)
    check_against_golden(pf, p, g, h, lam, V, f"metal7200 {prec_name}")
    del V
    dlam, W = _loss_grads(p, g)
    dA = h.backward(torch.from_numpy(dlam).cuda(), torch.from_numpy(W).cuda())
    assert h.status() == 0
    assert float((dA - dA.T).abs().max()) == 0.0
    dA = dA.cpu().numpy()
    scale = float(np.max(np.abs(g["dA_diag"])))
    e_s = float(np.max(np.abs(dA[g["dA_rows"], g["dA_cols"]] - g["dA_vals"]))) / scale
    e_d = float(np.max(np.abs(np.diag(dA) - g["dA_diag"]))) / scale
    dots = np.array([float(np.sum(dA * D)) for D in metal_directions])
    e_dot = float(np.max(np.abs(dots - g["dA_dot_dir"]) / np.maximum(np.abs(g["dA_dot_dir"]), 1e-300)))
    print(f"metal7200 {prec_name} gradient vs oracle: sampled entries {e_s:.2e}, diagonal {e_d:.2e} (of max |dA_ii| "
          f"{scale:.3e}), directional derivatives (relative) {e_dot:.2e}")
    assert e_s <= 1e-6 and e_d <= 1e-6, (e_s, e_d)
    assert e_dot <= 1e-6, e_dot
    h.close()


@pytest.fixture(scope="module")
def exact_map_fd(metal, metal_directions):
    """Central differences of the loss on the exact eigen-map (torch.linalg.eigh, FP64, as a
    library test tool) along the 32 directions: eigenvectors ascending, signed by the start-vector
    rule (home component positive when >= 0.1 in size, else the largest), h = 1e-6."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p, g = metal
    dlam, W = _loss_grads(p, g)
    A = torch.from_numpy(p.A).cuda()
    Wt = torch.from_numpy(W).cuda()
    idx = torch.arange(p.n, device="cuda")
    occ = int(g["occupied"])

    def loss(Ap):
        lam, V = torch.linalg.eigh(Ap)
        home = V[idx, idx]
        big = V.gather(0, V.abs().argmax(dim=0, keepdim=True))[0]
        ref = torch.where(home.abs() >= 0.1, home, big)
        V = V * torch.where(ref < 0, -1.0, 1.0)
        return float(lam[:occ].sum() + (V * Wt).sum())

    hstep = 1e-6
    fd = []
    for D in metal_directions:
        Dt = torch.from_numpy(D).cuda()
        fd.append((loss(A + hstep * Dt) - loss(A - hstep * Dt)) / (2 * hstep))
    return np.array(fd)


@pytest.mark.parametrize("prec_name", ["bf16", "fp64"])
def test_metal_like_backward_matches_exact_map_finite_differences(pf, metal, metal_directions, exact_map_fd,
                                                                   prec_name):
    """The adjoint differentiates the exact eigendecomposition, so it is checked where it is exact:
    the handle's first solve is a full diagonalisation (full_steps = 1; cuSOLVER syevd, the
    start-vector sign rule), the backward runs on those eigenpairs (FP64 products, or the mixed
    forms' digit products), and <dA, D_d> is compared with central differences of the exact map.
    No pair of this spectrum is closer than 1.8e-6, so the degenerate-pair mask (1e-8) is unused."""
    p, g = metal
    prec = {"bf16": pf.BF16_SPLIT, "fp64": pf.FP64}[prec_name]
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, precision=prec, full_steps=1)
    A, prev = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.prev).cuda()
    h.solve(A, prev)
    assert h.profile()["path"] == 1
    dlam, W = _loss_grads(p, g)
    dA = h.backward(torch.from_numpy(dlam).cuda(), torch.from_numpy(W).cuda())
    assert h.status() == 0
    dA = dA.cpu().numpy()
    dots = np.array([float(np.sum(dA * D)) for D in metal_directions])
    # relative to the largest directional derivative: a direction whose derivative nearly cancels
    # keeps the differences' absolute error (truncation (h d / gap)^2 ~ 1e-8 and eigh's rounding
    # ~1e-5 absolute) against a small value
    err = np.abs(dots - exact_map_fd) / np.max(np.abs(exact_map_fd))
    rel = np.abs(dots - exact_map_fd) / np.abs(exact_map_fd)
    print(f"metal7200 {prec_name} backward vs central differences of the exact map: max |error| / max |derivative| "
          f"{err.max():.2e}; per direction relative max {rel.max():.2e}, median {np.median(rel):.2e}")
    assert err.max() <= 1e-6, err.max()
    h.close()
