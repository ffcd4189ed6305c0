"""Pins for the oracle: each check ties the oracle to something other than itself -- a closed
form, a textbook routine written independently (brute-force Jacobi), a library routine used as a
reference (LAPACK through numpy), a hand-worked layout, or an invariant the mathematics fixes.

Paper passages: Section II (Eq. 11 and the partitioned scheme, Fig. 1), the Gram-Schmidt step
after the iterations, and the gamma / slice-size rule at the end of Section II.
"""
import os

import numpy as np
import pytest

import workloads as wl
from jacobi_ref import jacobi_eigh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _projector_err(U, V):
    """Largest ||u u^T - v v^T||_F over matching unit columns (sign-free comparison).
    Uses ||u u^T - v v^T||_F = ||u - s v|| sqrt(1 + |u.v|), s = sign(u.v), which avoids the
    cancellation of sqrt(2 - 2 (u.v)^2) near 1."""
    return float(np.max(_projector_errs(U, V)))


def _projector_errs(U, V):
    d = np.sum(U * V, axis=0)
    s = np.where(d < 0, -1.0, 1.0)
    diff = np.linalg.norm(U - V * s, axis=0)
    return diff * np.sqrt(1.0 + np.abs(d))


def _gap_bound(w, scale, c=100.0):
    """Per-vector rounding bound c * u * ||B|| / gap_k (Davis-Kahan with a backward-stable solver)."""
    gaps = np.full(w.size, np.inf)
    if w.size > 1:
        dw = np.diff(w)
        gaps[:-1] = np.minimum(gaps[:-1], dw)
        gaps[1:] = np.minimum(gaps[1:], dw)
    return c * 2.2e-16 * scale / gaps


# ------------------------------------------------------------------------------------ plan --

def _golden_plans():
    rows = []
    with open(os.path.join(GOLDEN, "plan_layouts.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            head, tail = line.split("|")
            n, p, h = (int(x) for x in head.split())
            parts = [np.array([int(x) for x in seg.split()]) for seg in tail.split(";")]
            rows.append((n, p, h, parts))
    return rows


@pytest.mark.parametrize("row", _golden_plans(), ids=lambda r: f"N{r[0]}P{r[1]}")
def test_plan_matches_hand_worked_layouts(orc, row):
    n, p, h, (k0, m, s, M) = row
    prev = np.linspace(-1.0, 1.0, n)
    got = orc.plan(prev, p, halo=h)
    for g, e in zip(got, (k0, m, s, M)):
        np.testing.assert_array_equal(g, e)


def test_plan_invariants_random(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = int(rng.integers(1, 400))
        p = int(rng.integers(1, min(n, 40) + 1))
        h = int(rng.integers(-1, n + 3))
        prev = np.sort(rng.uniform(-1, 1, n))
        k0, m, s, M = orc.plan(prev, p, halo=h, cluster_tol=0.0)
        assert m.sum() == n and k0[0] == 0 and np.all(m >= 1)
        assert np.all(k0[1:] == k0[:-1] + m[:-1])
        hh = (n + 9) // 10 if h < 0 else h
        assert np.all(M == np.minimum(n, m + 2 * hh))
        assert np.all(s >= 0) and np.all(s + M <= n)
        assert np.all(s <= k0) and np.all(k0 + m <= s + M)   # the window contains its slice


def test_plan_cluster_snap(orc):
    # 16 values, 2 slices: nominal boundary 8 sits inside a cluster {7, 8}; reach = 8 // 4 = 2
    prev = np.arange(16, dtype=float)
    prev[8] = prev[7] + 1e-7
    k0, m, _, _ = orc.plan(prev, 2, halo=0, cluster_tol=1e-5)
    # d=1: down candidate 7 has gap prev[7]-prev[6] = 1 >= tol -> boundary 7
    assert list(k0) == [0, 7] and list(m) == [7, 9]
    # cluster {6, 7, 8}: d=1 down (7) fails, d=1 up (9) succeeds
    prev = np.arange(16, dtype=float)
    prev[7] = prev[6] + 1e-7
    prev[8] = prev[7] + 1e-7
    k0, _, _, _ = orc.plan(prev, 2, halo=0, cluster_tol=1e-5)
    assert list(k0) == [0, 9]
    # cluster wider than the reach on both sides: boundary stays nominal
    prev = np.arange(16, dtype=float)
    prev[5:12] = prev[5] + 1e-7 * np.arange(7)
    k0, _, _, _ = orc.plan(prev, 2, halo=0, cluster_tol=1e-5)
    assert list(k0) == [0, 8]
    # tolerance 0 disables the snap
    prev = np.arange(16, dtype=float)
    prev[8] = prev[7]
    k0, _, _, _ = orc.plan(prev, 2, halo=0, cluster_tol=0.0)
    assert list(k0) == [0, 8]


def test_plan_rejects_bad_input(orc):
    with pytest.raises(orc.OracleError):
        orc.plan(np.array([0.0, 2.0, 1.0]), 1)          # not ascending
    with pytest.raises(orc.OracleError):
        orc.plan(np.arange(3.0), 4)                     # more slices than indices
    with pytest.raises(orc.OracleError):
        orc.plan(np.arange(6.0), 2, slice_sizes=[2, 3])  # sizes do not cover N
    with pytest.raises(orc.OracleError):
        orc.plan(np.array([0.0, np.nan]), 1)
    k0, m, _, _ = orc.plan(np.arange(6.0), 2, slice_sizes=[1, 5], halo=0)
    assert list(k0) == [0, 1] and list(m) == [1, 5]


# ------------------------------------------------------------------------------ gershgorin --

def test_gershgorin_contains_spectrum(orc):
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 40):
        B = rng.standard_normal((n, n))
        B = B + B.T
        lo, hi = orc.gershgorin(B)
        ev = np.linalg.eigvalsh(B)
        assert lo <= ev[0] + 1e-12 and ev[-1] <= hi + 1e-12
        r = np.sum(np.abs(B), axis=1) - np.abs(np.diag(B))
        assert lo == pytest.approx(np.min(np.diag(B) - r), abs=1e-12)
    assert orc.gershgorin(np.diag([3.0, -2.0, 5.0])) == (-2.0, 5.0)


# ---------------------------------------------------------------------------------- symeig --

def test_symeig_2x2_closed_form(orc):
    for a, b, c in [(2.0, 1.0, 3.0), (1.0, 1e-9, 1.0), (-5.0, 2.0, 7.0), (0.0, 1.0, 0.0)]:
        w, Z = orc.symeig(np.array([[a, b], [b, c]]))
        mid, rad = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
        np.testing.assert_allclose(w, [mid - rad, mid + rad], rtol=0, atol=1e-14 * (1 + abs(mid) + rad))
        for j, lam in enumerate(w):
            # (A - lam I) z = 0 row by row
            assert abs((a - lam) * Z[0, j] + b * Z[1, j]) < 1e-13 * (1 + rad)
            assert abs(b * Z[0, j] + (c - lam) * Z[1, j]) < 1e-13 * (1 + rad)


def test_symeig_tridiagonal_toeplitz_closed_form(orc):
    # T = tridiag(b, a, b): lambda_j = a + 2 b cos(j pi/(n+1)), u_j[i] = sin(i j pi/(n+1))
    n, a, b = 60, 0.3, -0.7
    T = np.diag(np.full(n, a)) + np.diag(np.full(n - 1, b), 1) + np.diag(np.full(n - 1, b), -1)
    w, Z = orc.symeig(T)
    j = np.arange(1, n + 1)
    exact = np.sort(a + 2 * b * np.cos(j * np.pi / (n + 1)))
    np.testing.assert_allclose(w, exact, rtol=0, atol=1e-13)
    i = np.arange(1, n + 1)[:, None]
    lam_j = a + 2 * b * np.cos(j * np.pi / (n + 1))
    U = np.sin(i * j[None, :] * np.pi / (n + 1))
    U /= np.linalg.norm(U, axis=0)
    U = U[:, np.argsort(lam_j)]
    assert _projector_err(U, Z) < 1e-12


@pytest.mark.parametrize("n", [1, 3, 8, 17, 24])
def test_symeig_matches_bruteforce_jacobi(orc, n):
    rng = np.random.default_rng(100 + n)
    B = rng.standard_normal((n, n))
    B = 0.5 * (B + B.T)
    w, Z = orc.symeig(B)
    wj, Vj = jacobi_eigh(B)
    scale = max(1.0, np.max(np.abs(wj)))
    np.testing.assert_allclose(w, wj, rtol=0, atol=1e-13 * scale)
    assert np.all(_projector_errs(Vj, Z) <= _gap_bound(wj, scale))
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) < 1e-13


def test_symeig_matches_lapack_on_nearly_diagonal(orc):
    p = wl.random_nearly_diagonal(150, seed=11, sigma=2e-3)
    w, Z = orc.symeig(p.A)
    wl_, Vl = np.linalg.eigh(p.A)
    np.testing.assert_allclose(w, wl_, rtol=0, atol=1e-13)
    assert np.all(_projector_errs(Vl, Z) <= _gap_bound(wl_, 1.0))
    assert np.max(np.abs(p.A @ Z - Z * w)) < 1e-13


def test_symeig_diagonal_and_degenerate(orc):
    d = np.array([3.0, -1.0, 2.0, -1.0, 0.5])
    w, Z = orc.symeig(np.diag(d))
    assert list(w) == sorted(d)                          # exact
    assert np.array_equal(np.abs(Z), np.eye(5)[:, [1, 3, 4, 2, 0]])
    w, Z = orc.symeig(np.eye(6) * 2.5)
    assert np.all(w == 2.5) and np.max(np.abs(Z.T @ Z - np.eye(6))) < 1e-15


# ------------------------------------------------------------------- folded-spectrum step --

def test_fs_iterate_eigenbasis_closed_form(orc):
    # Eq. 11: x_K = (I - alpha (A - eps I)^2)^K x_0 = U diag(f^K) U^T x_0, f = 1 - alpha (lam - eps)^2
    p = wl.random_nearly_diagonal(40, seed=21, sigma=5e-2, decay=None)
    lam, U = np.linalg.eigh(p.A)
    rng = np.random.default_rng(4)
    X0 = rng.standard_normal((40, 6))
    eps = np.array([lam[3], lam[10] + 1e-3, -0.5, 0.0, 0.7, lam[39]])
    alpha = np.array([0.2, 0.1, 0.3, 0.05, 0.25, 0.15])
    for K in (0, 1, 3):
        X = orc.fs_iterate(p.A, X0, eps, alpha, K)
        for c in range(6):
            f = (1.0 - alpha[c] * (lam - eps[c]) ** 2) ** K
            exact = U @ (f * (U.T @ X0[:, c]))
            np.testing.assert_allclose(X[:, c], exact, rtol=0, atol=1e-12)


# -------------------------------------------------------------------------- Gram-Schmidt --

def test_mgs_equals_householder_qr(orc):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((30, 12))
    Q, rd = orc.mgs(X)
    Qh, Rh = np.linalg.qr(X)
    sgn = np.sign(np.diag(Rh))
    np.testing.assert_allclose(Q, Qh * sgn, rtol=0, atol=1e-13)
    np.testing.assert_allclose(rd, np.abs(np.diag(Rh)), rtol=1e-13)
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) < 1e-14


def test_mgs_rank_deficient_is_not_spd(orc):
    X = np.random.default_rng(8).standard_normal((10, 4))
    X[:, 3] = X[:, 1] * 2.0 + 1e-12 * X[:, 0]
    with pytest.raises(orc.OracleError) as e:
        orc.mgs(X)
    assert e.value.code == orc.NOT_SPD


def test_rayleigh_exact_on_eigenvectors(orc):
    p = wl.random_nearly_diagonal(25, seed=31, sigma=1e-2)
    lam, U = np.linalg.eigh(p.A)
    l, r = orc.rayleigh(p.A, U)
    np.testing.assert_allclose(l, lam, rtol=0, atol=1e-14)
    assert np.max(r) < 1e-13
    v = np.random.default_rng(2).standard_normal(25)
    v /= np.linalg.norm(v)
    l, r = orc.rayleigh(p.A, v[:, None])
    assert l[0] == pytest.approx(v @ p.A @ v, abs=1e-14)
    assert r[0] == pytest.approx(np.linalg.norm(p.A @ v - l[0] * v), abs=1e-14)


# ------------------------------------------------------------------------ whole method --

def _exact(A):
    return np.linalg.eigh(A)


@pytest.mark.parametrize("n,nb,halo", [(37, 1, -1), (37, 3, 40), (64, 4, 64)])
def test_pfsm_full_window_is_exact(orc, n, nb, halo):
    """P = 1 or halo >= N: every window is A itself, the start vectors are exact eigenvectors,
    Eq. 11 leaves them fixed (up to scale <= 1) and the result is the full eigendecomposition."""
    p = wl.random_nearly_diagonal(n, seed=41 + n, sigma=3e-2, decay=8.0)
    r = orc.pfsm(p.A, p.prev, nb, halo=halo)
    lam, U = _exact(p.A)
    np.testing.assert_allclose(r.lam, lam, rtol=0, atol=1e-13)
    assert _projector_err(U, r.V) < 1e-10
    assert np.max(r.res) < 1e-12


def test_pfsm_zero_coupling_is_identity(orc):
    lam = np.sort(np.random.default_rng(9).uniform(-1, 1, 50))
    r = orc.pfsm(np.diag(lam), lam, 5)
    assert np.array_equal(r.V, np.eye(50))
    assert np.array_equal(r.lam, lam)
    assert np.all(r.res == 0.0)


def test_pfsm_block_diagonal_inside_windows_is_exact(orc):
    """A block-diagonal A whose blocks each lie inside one window: window eigenvectors are
    exact eigenvectors of A, so the method reproduces the exact decomposition."""
    n, nb = 48, 4
    rng = np.random.default_rng(12)
    lam = np.sort(rng.uniform(-1, 1, n))
    A = np.diag(lam)
    for b in range(nb):              # 12x12 blocks aligned with the slices
        sl = slice(12 * b, 12 * b + 12)
        E = 5e-3 * rng.standard_normal((12, 12))
        A[sl, sl] += E + E.T - 2 * np.diag(np.diag(E))
    r = orc.pfsm(A, lam, nb, halo=2)
    ev, U = _exact(A)
    np.testing.assert_allclose(np.sort(r.lam), ev, rtol=0, atol=1e-13)
    assert np.max(r.res) < 1e-12
    # index k stays tied to its slice: vectors of block b live in block b's rows
    for b in range(nb):
        rows = np.r_[0:12 * b, 12 * b + 12:n]
        assert np.max(np.abs(r.V[rows, 12 * b:12 * b + 12])) == 0.0


def test_pfsm_start_vectors_and_shifts(orc):
    """K = 0 exposes the start vectors: zero-padded window eigenvectors at the slice's own
    ascending positions, shifts equal to the window eigenvalues (Section II, reading R4)."""
    p = wl.random_nearly_diagonal(90, seed=51, sigma=4e-3)
    r = orc.pfsm(p.A, p.prev, 3, halo=7, fs_iters=0)
    k0, m, s, M = r.plan
    for b in range(3):
        sub = p.A[s[b]:s[b] + M[b], s[b]:s[b] + M[b]]
        w, Y = np.linalg.eigh(sub)
        for t in range(m[b]):
            k = k0[b] + t
            pos = k - s[b]
            assert r.eps[k] == pytest.approx(w[pos], abs=1e-14)
            x = r.xfs[:, k]
            assert np.all(x[:s[b]] == 0.0) and np.all(x[s[b] + M[b]:] == 0.0)
            y = Y[:, pos]
            assert abs(abs(x[s[b]:s[b] + M[b]] @ y) - 1.0) < 1e-12
            # sign reading R5: the home component is positive when it is >= 0.1 in size
            if abs(y[pos]) >= 0.1:
                assert x[k] > 0


def test_pfsm_alpha_keeps_every_factor_in_unit_interval(orc):
    """Reading R6 of Eq. 7-11: 0 <= 1 - alpha (lambda_n - eps)^2 <= 1 for every eigenvalue
    (1 exactly where an eigenvalue equals the shift), and the farthest eigenvalue is damped
    hardest."""
    p = wl.small_gapped(0)
    r = orc.pfsm(p.A, p.prev, 4)
    lam = np.linalg.eigvalsh(p.A)
    f = 1.0 - r.alpha[None, :] * (lam[:, None] - r.eps[None, :]) ** 2
    assert np.all(f >= -1e-12) and np.all(f <= 1.0)
    assert np.all(r.alpha > 0) and np.all(r.alpha < 1.0)
    assert np.all(np.min(f, axis=0) < 0.2)


def test_pfsm_iterations_then_gram_schmidt(orc):
    """Stage chain: xfs equals the eigenbasis closed form of Eq. 11 applied to the start
    vectors, and V equals the Householder QR (positive diagonal) of xfs."""
    p = wl.random_nearly_diagonal(60, seed=61, sigma=5e-3)
    r0 = orc.pfsm(p.A, p.prev, 3, halo=8, fs_iters=0)
    r = orc.pfsm(p.A, p.prev, 3, halo=8, fs_iters=4)
    lam, U = _exact(p.A)
    f = (1.0 - r.alpha[None, :] * (lam[:, None] - r.eps[None, :]) ** 2) ** 4
    exact = U @ (f * (U.T @ r0.xfs))
    np.testing.assert_allclose(r.xfs, exact, rtol=0, atol=1e-12)
    Qh, Rh = np.linalg.qr(r.xfs)
    np.testing.assert_allclose(r.V, Qh * np.sign(np.diag(Rh)), rtol=0, atol=1e-12)


def test_pfsm_invariants_small_gapped(orc):
    p = wl.small_gapped(0)
    r = orc.pfsm(p.A, p.prev, 4)
    n = p.n
    orth = np.max(np.abs(r.V.T @ r.V - np.eye(n)))
    assert orth < 1e-13
    # trace(A) = sum of Rayleigh quotients for any orthonormal V
    assert abs(np.sum(r.lam) - np.trace(p.A)) < 10 * n * orth * np.max(np.abs(r.lam)) + 1e-12
    # Weyl / Krylov-Bogoliubov: each lambda_k lies within r_k of an exact eigenvalue
    ev = np.linalg.eigvalsh(p.A)
    dist = np.min(np.abs(r.lam[:, None] - ev[None, :]), axis=1)
    assert np.all(dist <= r.res + 1e-13)
    # the method's premise: Rayleigh quotients stay close to the previous eigenvalues
    assert np.max(np.abs(r.lam - p.prev)) < 0.05


def test_pfsm_scf_sequence_error_shrinks(orc):
    """As E shrinks along the SCF-like sequence, the error against the exact eigenvalues falls
    monotonically (first-order perturbation: vector error ~ ||E outside window|| / gap)."""
    errs = []
    for step in range(5):
        p = wl.small_gapped(step)
        r = orc.pfsm(p.A, p.prev, 4)
        errs.append(np.max(np.abs(np.sort(r.lam) - np.linalg.eigvalsh(p.A))))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-8      # gamma ~ 0.45 here: "identical" to full diagonalisation


def test_pfsm_randomly_mixed_matrix_breaks(orc):
    """Section II: the method needs diagonal dominance; a randomly rotated spectrum makes the
    window solves return nearly identical shifts that do not span the spectrum. The symptom is
    either Gram-Schmidt breakdown (NOT_SPD) or eigenvalue estimates far from the exact ones."""
    n = 64
    rng = np.random.default_rng(13)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-1, 1, n))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    prev = np.sort(np.diag(A))
    try:
        r = orc.pfsm(A, prev, 8, halo=2, fs_iters=3)
    except orc.OracleError as e:
        assert e.code == orc.NOT_SPD
        return
    assert np.max(np.abs(np.sort(r.lam) - lam)) > 1e-2


def test_pfsm_rejects_nan(orc):
    p = wl.random_nearly_diagonal(10, seed=3)
    A = p.A.copy()
    A[2, 5] = np.nan
    with pytest.raises(orc.OracleError) as e:
        orc.pfsm(A, p.prev, 2)
    assert e.value.code == orc.NAN_INPUT


# ----------------------------------------------------------------------------- backward --

def test_backward_trace_loss_gives_identity(orc):
    p = wl.random_nearly_diagonal(30, seed=71, sigma=1e-2)
    lam, V = np.linalg.eigh(p.A)
    rng = np.random.default_rng(1)
    dA = orc.backward(V, lam, np.ones(30), None)
    np.testing.assert_allclose(dA, np.eye(30), rtol=0, atol=1e-13)
    # occupied sum -> projector onto the occupied subspace (Hellmann-Feynman)
    occ = 11
    dl = np.r_[np.ones(occ), np.zeros(30 - occ)]
    dA = orc.backward(V, lam, dl, None)
    np.testing.assert_allclose(dA, V[:, :occ] @ V[:, :occ].T, rtol=0, atol=1e-13)
    # a random dV orthogonal to nothing in particular keeps dA symmetric
    dA = orc.backward(V, lam, None, rng.standard_normal((30, 30)))
    assert np.array_equal(dA, dA.T)


def _gauge_eigh(A, ref):
    lam, V = np.linalg.eigh(A)
    s = np.sign(np.sum(V * ref, axis=0))
    s[s == 0] = 1.0
    return lam, V * s


def test_backward_matches_central_differences(orc):
    n, occ = 14, 6
    p = wl.random_nearly_diagonal(n, seed=81, sigma=3e-2, decay=None)
    A = p.A
    lam0, V0 = np.linalg.eigh(A)
    W = wl.gaussian((n, n), seed=5)

    def loss(M):
        lam, V = _gauge_eigh(M, V0)
        return np.sum(lam[:occ]) + np.sum(V * W)

    dlam = np.r_[np.ones(occ), np.zeros(n - occ)]
    dA = orc.backward(V0, lam0, dlam, W, tau=1e-12)
    h = 1e-6
    for d in range(8):
        D = wl.symmetric_direction(n, seed=900 + d)
        fd = (loss(A + h * D) - loss(A - h * D)) / (2 * h)
        assert np.sum(dA * D) == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_backward_masks_degenerate_pairs(orc):
    V = np.eye(4)
    lam = np.array([0.0, 1.0, 1.0 + 1e-12, 2.0])
    dV = np.ones((4, 4))
    dA = orc.backward(V, lam, None, dV, tau=1e-8)
    # with V = I, dA = sym(F o dV); the masked pair (1, 2) contributes nothing
    assert dA[1, 2] == 0.0 and dA[2, 1] == 0.0
    assert dA[0, 1] == pytest.approx(0.5 * (1.0 / (1.0 - 0.0) + 1.0 / (0.0 - 1.0)))
    assert np.all(np.diag(dA) == 0.0)


# ---- generalized -> standard conversion (Eq. 14-15) ---------------------------------------

def test_gen_to_std_reaches_lapack_solve(orc):
    """At convergence the Jacobi iterate is B^{-1} A, checked against LAPACK's LU solve."""
    for n, seed in ((12, 1), (57, 2), (96, 3)):
        A, B = wl.generalized_pair(n, seed)
        Z, it, r, st = orc.gen_to_std(A, B, max_iters=200, tol=1e-15)
        assert st == 0 and r <= 1e-15 and 3 <= it < 200
        ref = np.linalg.solve(B, A)
        assert np.max(np.abs(Z - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_gen_to_std_fixed_count_is_the_neumann_sum(orc):
    """After k updates from Z_0 = 0: Z_k = sum_{j<k} (I - D^-1 B)^j D^-1 A (closed form of Eq. 14)."""
    n = 20
    A, B = wl.generalized_pair(n, 4, sigma_b=3e-2)
    for k in (1, 2, 5):
        Z, it, r, st = orc.gen_to_std(A, B, max_iters=k, tol=0.0)
        assert it == k and st == 5 and r > 0.0
        Dinv = np.diag(1.0 / np.diag(B))
        G = np.eye(n) - Dinv @ B
        ref, term = np.zeros((n, n)), Dinv @ A
        for _ in range(k):
            ref += term
            term = G @ term
        assert np.max(np.abs(Z - ref)) <= 1e-14 * np.max(np.abs(ref))
        assert r == pytest.approx(np.max(np.abs(A - B @ ref)) / np.max(np.abs(A)), rel=1e-9, abs=1e-17)


def test_gen_to_std_diagonal_b_is_exact_in_one_update(orc):
    n = 9
    A = wl.random_nearly_diagonal(n, seed=5, sigma=0.1, decay=None).A
    d = 0.5 + np.arange(n) / n
    Z, it, r, st = orc.gen_to_std(A, np.diag(d), max_iters=10, tol=1e-15)
    assert st == 0 and it == 1
    assert np.array_equal(Z, A / d[:, None])


def test_gen_to_std_reports_divergence_and_bad_input(orc):
    n = 8
    A = np.eye(n)
    B = np.full((n, n), 0.5) + 0.1 * np.eye(n)             # not diagonally dominant
    Z, it, r, st = orc.gen_to_std(A, B, max_iters=30, tol=1e-14)
    assert st == 5 and it == 30 and r > 1.0
    with pytest.raises(orc.OracleError):
        orc.gen_to_std(A, B - np.diag(np.diag(B)))            # zero diagonal


def test_gen_to_std_sym_matches_eigendecomposition(orc):
    """S = B^{-1/2} against the eigendecomposition of B; C's eigenvalues against LAPACK's
    generalized eigensolver (sygvd); x = S y are B-orthonormal generalized eigenvectors."""
    import scipy.linalg as sla
    for n, seed in ((10, 6), (48, 7)):
        A, B = wl.generalized_pair(n, seed, sigma_b=2e-2)
        C, S, it, r, st = orc.gen_to_std_sym(A, B, max_iters=60, tol=1e-14)
        assert st == 0 and r <= 1e-14
        w, U = np.linalg.eigh(B)
        Sref = (U * w ** -0.5) @ U.T
        assert np.max(np.abs(S - Sref)) <= 1e-13
        assert np.max(np.abs(C - C.T)) <= 1e-13
        lam_g = sla.eigh(A, B, eigvals_only=True)
        lam, Y = np.linalg.eigh(C)
        assert np.max(np.abs(lam - lam_g)) <= 1e-13 * np.max(np.abs(lam_g))
        X = S @ Y
        assert np.max(np.abs(X.T @ B @ X - np.eye(n))) <= 1e-12
        assert np.max(np.abs(A @ X - (B @ X) * lam)) <= 1e-12


def test_gen_to_std_sym_identity_b_is_exact(orc):
    n = 7
    A = wl.random_nearly_diagonal(n, seed=8, sigma=0.2, decay=None).A
    C, S, it, r, st = orc.gen_to_std_sym(A, np.eye(n), max_iters=5, tol=0.0)
    # B = I: c = 1, Y_0 = Q_0 = I, T = I, the iterates never move and C = A exactly
    assert np.array_equal(S, np.eye(n)) and np.array_equal(C, A) and r == 0.0


# ---- diagonal-dominance guard and the conventional first steps --------------------------------

def test_guard_closed_forms(orc):
    assert orc.guard(np.diag([3.0, -1.0, 2.0])) == 0.0
    for a, b, d in ((1.0, 0.25, -1.0), (0.3, -0.02, 0.5), (-2.0, 1e-6, 7.0)):
        assert orc.guard(np.array([[a, b], [b, d]])) == pytest.approx(abs(b) / abs(a - d), rel=1e-15)
    A = np.array([[1.0, 0.1, 0.2], [0.1, 0.0, -0.3], [0.2, -0.3, 2.0]])
    # rows: sqrt(0.01 + 0.04), sqrt(0.01 + 0.09), sqrt(0.04 + 0.09); spread 2
    assert orc.guard(A) == pytest.approx(np.sqrt(0.13) / 2.0, rel=1e-15)
    assert orc.guard(np.ones((3, 3)) - np.eye(3) + 5 * np.eye(3)) == float("inf")


def test_guard_separates_the_papers_counterexample(orc):
    """Randomly mixed eigenvectors (the paper's failure example) against the workloads."""
    n = 96
    lam = np.linspace(-1.0, 1.5, n)
    Q, _ = np.linalg.qr(wl.gaussian((n, n), seed=31))
    mixed = (Q * lam) @ Q.T
    assert orc.guard(mixed) > 0.1
    assert orc.guard(wl.small_gapped(0).A) < 0.01
    assert orc.guard(wl.diamond_like(0).A) < 0.01


def test_full_diagonalization_matches_lapack_and_sign_rule(orc):
    for n, seed in ((1, 1), (9, 2), (64, 3)):
        A = wl.random_nearly_diagonal(n, seed=seed, sigma=0.05, decay=None).A
        lam, V, res = orc.full(A)
        w, U = np.linalg.eigh(A)
        assert np.max(np.abs(lam - w)) <= 1e-13 * max(1.0, np.max(np.abs(w)))
        d = np.sign(np.sum(U * V, axis=0))
        assert np.max(np.abs(V - U * d)) <= 1e-12
        assert np.max(res) <= 1e-12
        for k in range(n):
            v = V[:, k]
            if abs(v[k]) >= 0.1:
                assert v[k] > 0
            else:
                assert v[np.argmax(np.abs(v))] > 0


def test_full_equals_one_block_without_iterations(orc):
    n = 40
    p = wl.random_nearly_diagonal(n, seed=4, sigma=0.01)
    lam, V, _ = orc.full(p.A)
    r = orc.pfsm(p.A, p.prev, 1, halo=n, fs_iters=0)
    assert np.max(np.abs(lam - r.lam)) <= 1e-13
    assert np.max(np.abs(V - r.V)) <= 1e-12


def test_guarded_paths(orc):
    p = wl.small_gapped(0)
    assert orc.pfsm_guarded(p.A, p.prev, p.nblocks, solve_index=0, full_steps=2)[0] == 1
    assert orc.pfsm_guarded(p.A, p.prev, p.nblocks, solve_index=2, full_steps=2)[0] == 0
    n = 64
    Q, _ = np.linalg.qr(wl.gaussian((n, n), seed=32))
    lam = np.linspace(-1.0, 1.0, n)
    mixed = (Q * lam) @ Q.T
    path, l2, V2 = orc.pfsm_guarded(mixed, lam, 4, guard_max=0.05)
    assert path == 2 and np.max(np.abs(l2 - lam)) <= 1e-13


# ---- the chained SCF loop -------------------------------------------------------------------

def test_scf_step_keeps_an_exact_eigenbasis(orc):
    n = 48
    H = wl.scf_sequence(n, 1, seed=51)[0]
    w, U = np.linalg.eigh(H)
    path, lam, Vb = orc.scf_step(H, U, w, 4)
    assert path == 0
    assert np.max(np.abs(lam - w)) <= 1e-13
    assert np.max(np.abs(np.abs(np.sum(Vb * U, axis=0)) - 1.0)) <= 1e-12


def test_scf_chain_tracks_each_hamiltonian(orc):
    """Step 0 conventionally (H_0 is dense), then the method in the previous eigenbasis. Every
    step: the basis stays orthonormal, and each eigenvalue lies within Kahan's bound
    ||H V - V Lambda||_2 of LAPACK's (sorted pairing, V orthonormal); the method's own
    approximation error does not grow along the chain."""
    n, steps = 96, 5
    Hs = wl.scf_sequence(n, steps, seed=52)
    Vb, lam = np.eye(n), np.zeros(n)
    errs = []
    for j, H in enumerate(Hs):
        path, lam, Vb = orc.scf_step(H, Vb, lam, 4, solve_index=j, full_steps=1)
        assert path == (1 if j == 0 else 0)
        w = np.linalg.eigvalsh(H)
        assert np.max(np.abs(Vb.T @ Vb - np.eye(n))) <= 1e-12
        R = H @ Vb - Vb * lam
        bound = np.linalg.norm(R, 2) + 1e-14
        err = np.max(np.abs(lam - w))
        assert err <= bound
        errs.append(err)
    assert errs[0] <= 1e-13                      # the conventional step is exact
    assert max(errs[2:]) <= 2.0 * errs[1]        # no growth along the chain


# ---- adaptive variant of Eq. 11 (Rayleigh-quotient shifts, residual stopping) -------------------

def test_adaptive_stops_at_once_on_an_exact_eigenbasis(orc):
    n = 30
    A = wl.random_nearly_diagonal(n, seed=61, sigma=0.05).A
    w, U = np.linalg.eigh(A)
    X, eps, alpha, it, r, st = orc.fs_iterate_adaptive(A, U.T, w, np.full(n, 0.5), 10, 1e-13)
    assert st == 0 and it == 0 and r <= 1e-13
    assert np.array_equal(X, U.T)


def test_adaptive_zero_steps_is_one_rayleigh_quotient(orc):
    n = 20
    A = wl.random_nearly_diagonal(n, seed=62, sigma=0.1, decay=None).A
    X0 = wl.gaussian((3, n), seed=63)
    eps0 = np.array([0.1, -0.2, 0.3])
    X, eps, alpha, it, r, st = orc.fs_iterate_adaptive(A, X0, eps0, np.full(3, 0.5), 0, 0.0)
    rq = np.einsum("ki,ij,kj->k", X0, A, X0) / np.einsum("ki,ki->k", X0, X0)
    assert it == 0 and st == 5 and np.array_equal(X, X0)
    assert np.max(np.abs(eps - rq)) <= 1e-15
    res = [np.linalg.norm(A @ x - q * x) / np.linalg.norm(x) for x, q in zip(X0, rq)]
    assert r == pytest.approx(max(res), rel=1e-12)


def test_adaptive_residual_decreases_and_bounds_the_shift_error(orc):
    """Folded-spectrum steps contract slowly (1 - alpha (lambda - eps)^2 per neighbour), so the
    pin is the theory's: the residual decreases step by step, and each Rayleigh-quotient shift is
    within ||r||^2 / gap of its eigenvalue (gap to the rest of the spectrum)."""
    n = 40
    A = wl.random_nearly_diagonal(n, seed=64, sigma=0.02).A
    w, U = np.linalg.eigh(A)
    ks = [3, 17, 30]
    X0 = U[:, ks].T + 1e-3 * wl.gaussian((3, n), seed=65)
    prev = None
    for steps in (0, 1, 2, 4, 8, 16):
        X, eps, alpha, it, r, st = orc.fs_iterate_adaptive(A, X0, w[ks] + 1e-4, np.full(3, 0.3), steps, 0.0)
        assert it == steps
        if prev is not None:
            assert r < prev
        prev = r
        for k, e in zip(ks, eps):
            x = X[list(ks).index(k)]
            x = x / np.linalg.norm(x)
            res = np.linalg.norm(A @ x - (x @ A @ x) * x)
            gap = min(abs(w[j] - e) for j in range(n) if j != k)
            assert abs(e - w[k]) <= res ** 2 / gap * 1.01 + 1e-15


def test_method_with_adaptive_iterations_against_lapack(orc):
    """More capped steps lower the eigenvalue error; every result is within Kahan's residual
    bound; with the same count the adaptive variant is no worse than the fixed shifts."""
    p = wl.small_gapped(0)
    w = np.linalg.eigvalsh(p.A)
    fixed = orc.pfsm(p.A, p.prev, p.nblocks, halo=p.halo, fs_iters=3)
    errs = []
    for k in (3, 10, 20):
        r = orc.pfsm(p.A, p.prev, p.nblocks, halo=p.halo, fs_iters=k, fs_adaptive=True, fs_tol=0.0)
        err = np.max(np.abs(r.lam - w))
        R = p.A @ r.V - r.V * r.lam
        assert err <= np.linalg.norm(R, 2)
        errs.append(err)
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert errs[0] <= 1.01 * np.max(np.abs(fixed.lam - w))
