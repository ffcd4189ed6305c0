"""GPU: the generalized -> standard conversion (Eq. 14-15) against the FP64 oracle and LAPACK.

Both forms use FP64-accurate digit products, whose error is about sqrt(K) 2^-46 of
max|P_r| max|Q_c| per product (tests/test_gpu_mixed.py): the GPU iterates follow the oracle's
within that per update, the computed residuals have that floor (so the stopping tolerance is
1e-12, above it at every size tested), and the converged results are compared with LAPACK's
solve and generalized eigensolver within a few times sqrt(N) 2^-46."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

U46 = 2.0 ** -46
TOL = 1e-12                # Jacobi: residual floor ~6.5e-13 at N = 1280
TOL_SYM = 1e-11            # Newton-Schulz: max|I - Q Y| floor ~1.6e-12 at N = 200


@pytest.fixture(scope="module")
def pf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_07806_b300 as mod
    from paper_1502_07806_b300 import build
    build.build()
    mod.load_library()
    return mod


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("n,seed", [(1, 1), (77, 2), (130, 3), (257, 4)])
def test_jacobi_fixed_count_follows_the_oracle(pf, orc, n, seed):
    """tol = 0: exactly max_iters updates on both sides; the iterates agree element by element."""
    A, B = wl.generalized_pair(n, seed, sigma_b=2e-2)
    for k in (0, 1, 4):
        Zo, ito, ro, sto = orc.gen_to_std(A, B, max_iters=k, tol=0.0)
        Zg, itg, rg = pf.gen_to_std(_dev(A), _dev(B), max_iters=k, tol=0.0, check=False)
        Zg = Zg.cpu().numpy()
        scale = max(np.max(np.abs(Zo)), 1e-300)
        err = np.max(np.abs(Zg - Zo)) / scale
        print(f"n={n} k={k}: |Z_gpu - Z_oracle| / max|Z| = {err:.2e}, resid {rg:.3e} vs {ro:.3e}")
        # tol = 0 runs every update, unless the oracle's exact FP64 residual reached 0 (N = 1)
        assert itg == k and (ito == k or ro == 0.0)
        assert err <= 4.0 * max(k, 1) * np.sqrt(n) * U46
        # the residual itself is a product: equal up to the digit products' error (2^-46 sqrt(K) class)
        assert rg == pytest.approx(ro, rel=1e-6, abs=4.0 * np.sqrt(n) * U46)


@pytest.mark.parametrize("n,seed", [(96, 5), (1280, 6)])
def test_jacobi_converges_to_lapack_solve(pf, orc, n, seed):
    A, B = wl.generalized_pair(n, seed)
    Zg, itg, rg = pf.gen_to_std(_dev(A), _dev(B), max_iters=100, tol=TOL)
    Zg = Zg.cpu().numpy()
    ref = np.linalg.solve(B, A)
    err = np.max(np.abs(Zg - ref)) / np.max(np.abs(ref))
    print(f"n={n}: {itg} updates, resid {rg:.2e}, |Z - solve(B, A)| / max|Z| = {err:.2e}")
    assert rg <= TOL and err <= 2 * TOL + 8.0 * np.sqrt(n) * U46
    if n <= 128:
        Zo, ito, ro, sto = orc.gen_to_std(A, B, max_iters=100, tol=TOL)
        assert abs(itg - ito) <= 1
        assert np.max(np.abs(Zg - Zo)) <= (2 * TOL + 8.0 * np.sqrt(n) * U46) * np.max(np.abs(Zo))


def test_jacobi_rejects_zero_diagonal_and_leaves_z(pf):
    n = 16
    A, B = wl.generalized_pair(n, 7)
    B[3, 3] = 0.0
    Z = torch.full((n, n), 7.0, dtype=torch.float64, device="cuda")
    dA, dB = _dev(A), _dev(B)                      # keep the operands alive across the call
    lib = pf.load_library()
    rc = lib.pfsm_gen_to_std(n, dA.data_ptr(), dB.data_ptr(), Z.data_ptr(), 10, 1e-14, None, None, None)
    torch.cuda.synchronize()
    assert rc == 1 and bool(torch.all(Z == 7.0))
    with pytest.raises(pf.PFSMError):
        pf.gen_to_std(_dev(A), _dev(B))


def test_jacobi_reports_non_convergence(pf):
    n = 24
    A = np.eye(n)
    B = np.full((n, n), 0.5) + 0.1 * np.eye(n)                      # not diagonally dominant
    Z, it, r = pf.gen_to_std(_dev(A), _dev(B), max_iters=20, tol=TOL, check=False)
    assert it == 20 and r > 1.0
    with pytest.raises(pf.PFSMError):
        pf.gen_to_std(_dev(A), _dev(B), max_iters=20, tol=TOL)


@pytest.mark.parametrize("n,seed", [(1, 8), (65, 9), (200, 10)])
def test_symmetric_form_follows_the_oracle(pf, orc, n, seed):
    A, B = wl.generalized_pair(n, seed, sigma_b=2e-2)
    Co, So, ito, ro, sto = orc.gen_to_std_sym(A, B, max_iters=60, tol=TOL_SYM)
    Cg, Sg, itg, rg = pf.gen_to_std_sym(_dev(A), _dev(B), max_iters=60, tol=TOL_SYM)
    Cg, Sg = Cg.cpu().numpy(), Sg.cpu().numpy()
    eC = np.max(np.abs(Cg - Co)) / np.max(np.abs(Co))
    eS = np.max(np.abs(Sg - So)) / np.max(np.abs(So))
    print(f"n={n}: {itg} vs {ito} updates, |C - C_oracle| {eC:.2e}, |S - S_oracle| {eS:.2e}")
    bound = 4 * TOL_SYM + 16.0 * np.sqrt(n) * U46
    assert abs(itg - ito) <= 1 and eC <= bound and eS <= bound


@pytest.mark.parametrize("n,seed", [(300, 11), (1280, 12)])
def test_symmetric_form_gives_the_generalized_eigenpairs(pf, n, seed):
    """Eigenvalues of C against LAPACK's generalized solver (sygvd); x = S y B-orthonormal."""
    A, B = wl.generalized_pair(n, seed)
    Cg, Sg, it, r = pf.gen_to_std_sym(_dev(A), _dev(B), max_iters=60, tol=TOL_SYM)
    C, S = Cg.cpu().numpy(), Sg.cpu().numpy()
    lam, Y = np.linalg.eigh(0.5 * (C + C.T))
    lam_ref = sla.eigh(A, B, eigvals_only=True)
    X = S @ Y
    e_lam = np.max(np.abs(lam - lam_ref)) / np.max(np.abs(lam_ref))
    e_orth = np.max(np.abs(X.T @ B @ X - np.eye(n)))
    e_sym = np.max(np.abs(C - C.T)) / np.max(np.abs(C))
    print(f"n={n}: {it} updates, eig {e_lam:.2e}, B-orth {e_orth:.2e}, asym {e_sym:.2e}")
    bound = 4 * TOL_SYM + 16.0 * np.sqrt(n) * U46
    assert e_lam <= bound and e_orth <= bound and e_sym <= bound


def test_symmetric_form_stays_put_after_convergence(pf, orc):
    """Thirty updates past convergence (tol = 0) leave S where it converged: the products are true
    products X Y, not X Y^T, so rounding asymmetry cannot grow."""
    n = 200
    A, B = wl.generalized_pair(n, 10, sigma_b=2e-2)
    C0, S0, it0, r0 = pf.gen_to_std_sym(_dev(A), _dev(B), max_iters=60, tol=TOL_SYM)
    C1, S1, it1, r1 = pf.gen_to_std_sym(_dev(A), _dev(B), max_iters=it0 + 30, tol=0.0, check=False)
    d = float((S1 - S0).abs().max() / S0.abs().max())
    print(f"after {it1} updates: residual {r1:.2e}, |S - S_converged| {d:.2e}")
    assert r1 <= TOL_SYM and d <= 4 * TOL_SYM
