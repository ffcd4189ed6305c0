"""The hand-written FP64 helpers of the serial paths against CUDA's correctly rounded arithmetic.

Reciprocals and inverse square roots on the window eigensolves, the bulge chase and the panel QR are
FP32 seeds refined by two Newton steps (instead of the IEEE FP64 divide and square-root sequences),
and the digit products' epilogue rounds an exact 64-bit level sum to FP64 by integer operations.
Here they run through the library's test entry points on inputs that span the exponent range and
the mantissa interval [1, 2) (its ends included), against:
  1/x           IEEE division (numpy's and CUDA's are both correctly rounded);
  1/sqrt(x)     the correctly rounded value, from 60-digit decimal arithmetic;
  t 2^e         the exact rational rounded once (Python's Fraction -> float is correctly rounded).
The bit-pattern inverse square root is the one the panel QR and the bulge chase use. Bounds: the
Newton helpers within 2 ulp of the correctly rounded result (two steps from a 2^-22
seed leave ~2^-88 of approximation error, so only the last steps' roundings remain); the integer
conversion bit for bit."""
import ctypes
import decimal
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_07806_b300 as pf
    from paper_1502_07806_b300 import build
    build.build()
    return pf, pf.load_library()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _inputs(lo_exp, hi_exp, seed):
    rng = random.Random(seed)
    xs = []
    for e in range(lo_exp, hi_exp + 1):
        for m in (1.0, 1.5, float(np.nextafter(2.0, 0.0)), float(np.nextafter(1.0, 2.0)),
                  1.0 + rng.random(), 1.0 + rng.random(), 1.0 + rng.random()):
            xs.append(m * 2.0 ** e)
    return np.array(xs, dtype=np.float64)


def _ulps(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_newton_reciprocal_and_rsqrt_within_two_ulp():
    pf, lib = _lib()
    x = _inputs(-1020, 1020, 3)                      # positive, results normal
    xd = torch.from_numpy(x).cuda()
    r1, r2, r3, r4 = (torch.empty_like(xd) for _ in range(4))
    assert lib.pfsm_selftest_fp64_helpers(_ptr(xd), x.size, _ptr(r1), _ptr(r2), _ptr(r3), _ptr(r4), None) == pf.OK
    torch.cuda.synchronize()
    rcp_ref = 1.0 / x
    decimal.getcontext().prec = 60
    rsq_ref = np.array([float(1 / decimal.Decimal(v).sqrt()) for v in x])
    e_rcp = _ulps(r1.cpu().numpy(), rcp_ref)
    e_rsq = _ulps(r2.cpu().numpy(), rsq_ref)
    e_fast = _ulps(r3.cpu().numpy(), rcp_ref)
    e_frsq = _ulps(r4.cpu().numpy(), rsq_ref)
    print(f"max ulp: scaled_rcp {e_rcp.max():.2f}, scaled_rsqrt {e_rsq.max():.2f}, fast_rcp {e_fast.max():.2f}, "
          f"fast_rsqrt {e_frsq.max():.2f}")
    assert e_rcp.max() <= 2.0
    assert e_rsq.max() <= 2.0
    assert e_fast.max() <= 2.0
    assert e_frsq.max() <= 2.0


def test_fast_reciprocal_negative_and_outside_its_fast_range():
    pf, lib = _lib()
    x = np.concatenate([-_inputs(-1020, 1020, 5), _inputs(-1020, -126, 6), _inputs(126, 1020, 7)])
    xd = torch.from_numpy(x).cuda()
    r1, r2, r3, r4 = (torch.empty_like(xd) for _ in range(4))
    assert lib.pfsm_selftest_fp64_helpers(_ptr(xd), x.size, _ptr(r1), _ptr(r2), _ptr(r3), _ptr(r4), None) == pf.OK
    torch.cuda.synchronize()
    got = r3.cpu().numpy()
    assert _ulps(got, 1.0 / x).max() <= 2.0
    outside = np.abs(x) < 2.0 ** -125
    outside |= np.abs(x) >= 2.0 ** 126
    np.testing.assert_array_equal(got[outside], 1.0 / x[outside])      # CUDA's own division there
    # the inverse square roots outside the bit-pattern range fall back to the scaled helper
    pos = x > 0
    decimal.getcontext().prec = 60
    rsq_ref = np.array([float(1 / decimal.Decimal(v).sqrt()) for v in x[pos]])
    assert _ulps(r4.cpu().numpy()[pos], rsq_ref).max() <= 2.0
    # the square-root and scaled helpers are defined for positive arguments only: zero elsewhere
    for r in (r1, r2, r4):
        assert np.all(r.cpu().numpy()[x <= 0] == 0.0)


def test_integer_sum_to_fp64_is_correctly_rounded():
    pf, lib = _lib()
    rng = random.Random(11)
    ts = [0, 1, -1, 3, -5, (1 << 53) + 1, (1 << 54) + 2, (1 << 54) + 6, -((1 << 54) + 2), (1 << 63) - 1,
          -(1 << 63), 0x7FFFFFFFFFFFFC00, 0x7FFFFFFFFFFFFE00, 0x7FFFFFFFFFFFFDFF, (1 << 62) - 1, -(1 << 62) + 1]
    for _ in range(60000):
        b = rng.randint(1, 63)
        ts.append(rng.randint(-(1 << b) + 1, (1 << b) - 1))
    es = [rng.randint(-960, 900) for _ in ts]
    t = torch.tensor(ts, dtype=torch.int64).cuda()
    e = torch.tensor(es, dtype=torch.int32).cuda()
    out = torch.empty(len(ts), dtype=torch.float64, device="cuda")
    assert lib.pfsm_selftest_i64_to_f64(_ptr(t), _ptr(e), len(ts), _ptr(out), None) == pf.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = np.array([float(Fraction(a) * Fraction(2) ** b) for a, b in zip(ts, es)])
    np.testing.assert_array_equal(got, ref)


def test_selftest_entry_points_reject_bad_arguments():
    pf, lib = _lib()
    assert lib.pfsm_selftest_fp64_helpers(None, 4, None, None, None, None, None) == pf.INVALID_ARG
    assert lib.pfsm_selftest_fp64_helpers(None, -1, None, None, None, None, None) == pf.INVALID_ARG
    assert lib.pfsm_selftest_i64_to_f64(None, None, 3, None, None) == pf.INVALID_ARG
    assert lib.pfsm_selftest_fp64_helpers(None, 0, None, None, None, None, None) == pf.OK
