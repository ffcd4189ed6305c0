"""GPU: the conventional path around the method (Section II): the first solves of a handle as full
diagonalizations (the paper's conventional first SCF steps) and the diagonal-dominance guard,
against the oracle's full diagonalization, guard value and method."""
import numpy as np
import pytest
import torch

import workloads as wl
from compare import projector_errors

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


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _mixed(n, seed):
    """The paper's counterexample: eigenvectors mixed by a random orthogonal matrix."""
    Q, _ = np.linalg.qr(wl.gaussian((n, n), seed=seed))
    lam = np.linspace(-1.0, 1.5, n)
    return (Q * lam) @ Q.T, lam


@pytest.mark.parametrize("prec", [0, 2])
def test_first_steps_rule(pf, orc, prec):
    p = wl.small_gapped(0)
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, precision=prec, full_steps=2)
    lam_f, V_f, _ = orc.full(p.A)
    ref = orc.pfsm(p.A, p.prev, p.nblocks, halo=p.halo)
    scale = np.max(np.abs(p.A))
    for step, want in enumerate((1, 1, 0)):
        lam, V = h.solve(_dev(p.A), _dev(p.prev))
        assert h.status() == 0
        prof = h.profile()
        lam, V = lam.cpu().numpy(), V.cpu().numpy()
        assert prof["path"] == want
        if want:
            dl = np.max(np.abs(lam - lam_f)) / scale
            dv = np.max(np.abs(V - V_f))
            print(f"prec {prec} step {step}: full diagonalization |dlam| {dl:.2e} |dV| {dv:.2e}")
            assert dl <= 1e-12 and dv <= 1e-10
        else:
            dl = np.max(np.abs(lam - ref.lam)) / scale
            pe = np.max(projector_errors(ref.V, V, ref.lam))
            print(f"prec {prec} step {step}: method |dlam| {dl:.2e} projector {pe:.2e}")
            assert dl <= 1e-10 and pe <= 1e-8
    h.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_guard_falls_back_on_the_counterexample(pf, orc, prec):
    n = 160
    A, lam0 = _mixed(n, 41)
    g_ref = orc.guard(A)
    h = pf.Handle(n, 4, precision=prec, guard_max=0.05)
    lam, V = h.solve(_dev(A), _dev(lam0))
    prof = h.profile()
    assert h.status() == 0 and prof["path"] == 2
    assert prof["guard_value"] == pytest.approx(g_ref, rel=1e-12)
    lam_f, V_f, _ = orc.full(A)
    assert np.max(np.abs(lam.cpu().numpy() - lam_f)) <= 1e-12
    assert np.max(np.abs(V.cpu().numpy() - V_f)) <= 1e-10
    # a nearly diagonal matrix passes the guard and takes the method
    p = wl.small_gapped(0)
    h2 = pf.Handle(p.n, p.nblocks, halo=p.halo, precision=prec, guard_max=0.05)
    h2.solve(_dev(p.A), _dev(p.prev))
    prof2 = h2.profile()
    print(f"prec {prec}: guard {prof['guard_value']:.3f} (counterexample), {prof2['guard_value']:.2e} (workload)")
    assert prof2["path"] == 0 and prof2["guard_value"] == pytest.approx(orc.guard(p.A), rel=1e-12)
    h.close()
    h2.close()


def test_backward_after_a_full_diagonalization(pf, orc):
    p = wl.small_gapped(1)
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, full_steps=1)
    lam, V = h.solve(_dev(p.A), _dev(p.prev))
    assert h.profile()["path"] == 1
    occ = p.n // 2
    dlam = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dlam[:occ] = 1.0
    dA = h.backward(dlam, None).cpu().numpy()
    ref = orc.backward(V.cpu().numpy(), lam.cpu().numpy(), dlam.cpu().numpy(), None)
    assert np.max(np.abs(dA - ref)) <= 1e-10
    h.close()


def test_nan_input_is_reported_on_the_conventional_path(pf):
    p = wl.small_gapped(0)
    A = p.A.copy()
    A[3, 5] = A[5, 3] = np.nan
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, full_steps=1)
    h.solve(_dev(A), _dev(p.prev))
    assert h.status() == 4          # PFSM_ERR_NAN_INPUT
    h.close()
