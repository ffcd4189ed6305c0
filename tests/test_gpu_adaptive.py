"""GPU: the adaptive variant of Eq. 11 (Rayleigh-quotient shifts, residual stopping) against the
oracle's, in both forms (it runs its products in FP64 in every form)."""
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


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("name,make", [("gapped256", lambda: wl.small_gapped(0)),
                                       ("ragged333", lambda: wl.random_nearly_diagonal(333, seed=9, sigma=2e-3,
                                                                                     nblocks=5))])
def test_adaptive_matches_the_oracle(pf, orc, prec, name, make):
    p = make()
    K = 6
    ref = orc.pfsm(p.A, p.prev, p.nblocks, halo=p.halo, fs_iters=K, fs_adaptive=True, fs_tol=0.0)
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, fs_iters=K, precision=prec, fs_adaptive=True, fs_tol=0.0)
    lam, V = h.solve(_dev(p.A), _dev(p.prev))
    assert h.status() == 0
    prof = h.profile()
    eps = h.diagnostic(2).cpu().numpy()
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    scale = np.max(np.abs(ref.lam))
    dl = np.max(np.abs(lam - ref.lam)) / scale
    de = np.max(np.abs(eps - ref.eps)) / scale
    pe = np.max(projector_errors(ref.V, V, ref.lam))
    print(f"{name} prec {prec}: steps {prof['fs_steps']} residual {prof['fs_residual']:.2e} "
          f"|dlam| {dl:.2e} |deps| {de:.2e} projector {pe:.2e}")
    assert prof["fs_steps"] == K
    assert dl <= 1e-10 and de <= 1e-12 and pe <= 1e-8
    h.close()


def test_adaptive_stops_on_the_residual(pf, orc):
    p = wl.small_gapped(0)
    h = pf.Handle(p.n, p.nblocks, halo=p.halo, fs_iters=3, fs_adaptive=True, fs_tol=0.0)
    h.solve(_dev(p.A), _dev(p.prev))
    r3 = h.profile()["fs_residual"]
    lo, hi = orc.gershgorin(p.A)
    # a tolerance (relative to the Gershgorin bound) that the residual of the third step meets
    tol = 1.5 * r3 / max(abs(lo), abs(hi))
    h2 = pf.Handle(p.n, p.nblocks, halo=p.halo, fs_iters=50, fs_adaptive=True, fs_tol=tol)
    h2.solve(_dev(p.A), _dev(p.prev))
    prof = h2.profile()
    print(f"steps {prof['fs_steps']} residual {prof['fs_residual']:.3e} (3-step residual {r3:.3e})")
    assert prof["fs_steps"] <= 3 and prof["fs_residual"] <= 1.5 * r3 * (1 + 1e-9)
    h.close()
    h2.close()
