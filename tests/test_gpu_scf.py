"""GPU: the chained SCF loop (pfsm_scf_step) against the oracle's chain, step by step: the first
step conventionally (the Hamiltonian is dense), then the method in the previous eigenbasis."""
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


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("n,nb", [(96, 4), (256, 4)])
def test_chain_follows_the_oracle(pf, orc, prec, n, nb):
    steps = 5
    Hs = wl.scf_sequence(n, steps, seed=53 + n)
    h = pf.Handle(n, nb, precision=prec, full_steps=1)
    Vb = torch.eye(n, dtype=torch.float64, device="cuda")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    Vo, lamo = np.eye(n), np.zeros(n)
    for j, H in enumerate(Hs):
        lam = h.scf_step(torch.from_numpy(H).cuda(), Vb, lam.clone())
        assert h.status() == 0 and h.profile()["path"] == (1 if j == 0 else 0)
        path, lamo, Vo = orc.scf_step(H, Vo, lamo, nb, solve_index=j, full_steps=1)
        l, V = lam.cpu().numpy(), Vb.cpu().numpy()
        scale = np.max(np.abs(lamo))
        dl = np.max(np.abs(l - lamo)) / scale
        pe = np.max(projector_errors(Vo, V, lamo))
        orth = np.max(np.abs(V.T @ V - np.eye(n)))
        print(f"prec {prec} n {n} step {j}: |dlam| {dl:.2e} projector {pe:.2e} orth {orth:.2e}")
        assert dl <= 1e-10 and pe <= 1e-8 and orth <= 1e-12
    h.close()


def test_step_rejects_recompute_backward(pf):
    n = 64
    H = wl.scf_sequence(n, 1, seed=60)[0]
    h = pf.Handle(n, 2, full_steps=1, recompute_v=True)
    Vb = torch.eye(n, dtype=torch.float64, device="cuda")
    h.scf_step(torch.from_numpy(H).cuda(), Vb, torch.zeros(n, dtype=torch.float64, device="cuda"))
    with pytest.raises(pf.PFSMError):
        h.backward(torch.ones(n, dtype=torch.float64, device="cuda"), None)
    h.close()
