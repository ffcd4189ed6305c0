"""GPU: batches of independent problems of uneven order (64 k-point/spin-like matrices with N in
200..3000, slices clamp(N/10, 64, 256) wide) solved by one captured CUDA graph.

Checks: every problem of the batch equals the same problem solved alone through pfsm_solve
(bit-exact: same kernels, same inputs, deterministic arithmetic; BF16, TF32 and FP64 forms); a replay of the captured graph
and a re-capture for new buffers reproduce it; the smallest problems match the FP64 oracle at the
FP64 bar; all device status words are clear."""
import numpy as np
import pytest
import torch

import workloads as wl
from compare import projector_errors, spectral_scale

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
def problems():
    sizes = wl.batch_sizes(64)
    return [wl.batch_problem(i, int(n)) for i, n in enumerate(sizes)]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("name,prec", [("bf16", 2), ("tf32", 1), ("fp64", 0)])
def test_batch_equals_individual_solves(pf, problems, name, prec):
    probs = problems if name != "fp64" else problems[:12]
    As = [_dev(p.A) for p in probs]
    prevs = [_dev(p.prev) for p in probs]
    b = pf.Batch([p.n for p in probs], [p.nblocks for p in probs], precision=prec)
    lams, Vs = b.solve(As, prevs)
    assert b.status() == [0] * len(probs)
    lams2, Vs2 = b.solve(As, prevs, lams=[torch.empty_like(x) for x in lams],
                         Vs=[torch.empty_like(x) for x in Vs])          # new buffers: re-capture
    lams3, Vs3 = b.solve(As, prevs, lams2, Vs2)                          # same buffers: replay
    assert b.status() == [0] * len(probs)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        h = pf.Handle(p.n, p.nblocks, precision=prec)
        lam, V = h.solve(As[i], prevs[i])
        assert h.status() == 0
        assert torch.equal(lams[i], lam) and torch.equal(Vs[i], V), f"problem {i} (N={p.n})"
        assert torch.equal(lams3[i], lam) and torch.equal(Vs3[i], V), f"problem {i} replay"
        h.close()
    b.close()


@pytest.mark.parametrize("prec", [2, 1])
def test_batch_small_problems_match_oracle(pf, orc, problems, prec):
    order = np.argsort([p.n for p in problems])[:4]
    probs = [problems[i] for i in order]
    b = pf.Batch([p.n for p in probs], [p.nblocks for p in probs], precision=prec)
    lams, Vs = b.solve([_dev(p.A) for p in probs], [_dev(p.prev) for p in probs])
    assert b.status() == [0] * len(probs)
    for p, lam, V in zip(probs, lams, Vs):
        r = orc.pfsm(p.A, p.prev, p.nblocks)
        dl = np.max(np.abs(lam.cpu().numpy() - r.lam)) / spectral_scale(r.lam)
        pe = np.max(projector_errors(r.V, V.cpu().numpy(), r.lam))
        print(f"batch N={p.n}: |dlam|/||A|| = {dl:.2e}, projector = {pe:.2e}")
        assert dl <= 1e-10 and pe <= 1e-8
    b.close()


def test_autotuned_batch(pf, problems, tmp_path):
    """Block counts measured per size class; each problem still equals its solo solve with the
    chosen layout and stays within the FP64 bars of the oracle-checked default."""
    from paper_1502_07806_b300 import autotune
    order = np.argsort([p.n for p in problems])
    probs = [problems[i] for i in order[:3]] + [problems[order[-1]]]
    As = [_dev(p.A) for p in probs]
    prevs = [_dev(p.prev) for p in probs]
    path = str(tmp_path / "tune.json")
    nbs = []
    for A, prev, p in zip(As, prevs, probs):
        best, meas = autotune.tune(A, prev, pf.BF16_SPLIT, cache_path=path, return_measurements=True)
        print(f"N={p.n}: " + ", ".join(f"{k} slices {v[0]:.2f} ms res {v[1]:.1e}" for k, v in sorted(meas.items()))
              + f" -> {best}")
        assert best in autotune.candidates(p.n) and best in meas
        nbs.append(best)
    b = pf.Batch.autotuned(As, prevs, precision=pf.BF16_SPLIT, cache_path=path)
    lams, Vs = b.solve(As, prevs)
    assert b.status() == [0] * len(probs)
    for i, p in enumerate(probs):
        h = pf.Handle(p.n, nbs[i], precision=pf.BF16_SPLIT)
        lam, V = h.solve(As[i], prevs[i])
        assert h.status() == 0
        assert torch.equal(lams[i], lam) and torch.equal(Vs[i], V)
        h.close()
    b.close()
