"""Seeded synthetic inputs for the PFSM hot path.

Test and benchmark infrastructure shared by the CUDA path and the oracle. This module draws
random numbers and assembles matrices; it holds none of the method's arithmetic.

The paper's matrices come from Kohn-Sham SCF runs (diamond, C60 cluster, Cu, a Si vacancy cell,
an Al supercell; Sections III-IV, Tables I-III). Those runs are not reproducible here, so each
workload is a seeded stand-in with the shape the paper describes: the reduced Hamiltonian
expressed in the previous SCF step's eigenbasis, i.e. nearly diagonal with its diagonal ordered
like the previous eigenvalues (abstract; Section II):

    A = diag(lam) + E,   E symmetric, zero diagonal, small off-diagonal entries,
    prev_eigvals = lam   (ascending).

Random numbers come from a counter-based splitmix64 stream (Steele, Lea, Flood 2014; the
standard 64-bit finaliser constants), turned into 53-bit uniforms and Box-Muller normals.
Value i of stream ``seed`` is ``mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)``, so any sub-range
can be regenerated without drawing the ones before it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def seed_for(cfg: int, idx: int = 0) -> int:
    """Stream seed of instance ``idx`` of workload family ``cfg``."""
    return 0x9F5D0000 + 1000 * cfg + idx


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw_u64(seed: int, start: int, count: int) -> np.ndarray:
    """Values start .. start+count-1 of the splitmix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN)


def uniform(seed: int, start: int, count: int) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    return (raw_u64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, start: int, count: int) -> np.ndarray:
    """Standard normals, one per pair of uniforms (Box-Muller, cosine branch)."""
    u = uniform(seed, 2 * start, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


class _Stream:
    """Sequential reader over one seeded stream."""

    def __init__(self, seed: int):
        self.seed, self.pos = seed, 0

    def uniform(self, n: int) -> np.ndarray:
        out = uniform(self.seed, self.pos, n)
        self.pos += n
        return out

    def normal(self, n: int) -> np.ndarray:
        # normals consume two uniforms each; keep the cursor in uniform units
        if self.pos % 2:
            self.pos += 1
        out = normal(self.seed, self.pos // 2, n)
        self.pos += 2 * n
        return out

    def u64(self, n: int) -> np.ndarray:
        out = raw_u64(self.seed, self.pos, n)
        self.pos += n
        return out


def coupling(n: int, sigma: float, decay: float | None, st: _Stream) -> np.ndarray:
    """Symmetric E with zero diagonal; upper triangle drawn row-major as
    sigma * N(0,1) * exp(-|i-j|/decay) (no decay factor when ``decay`` is None)."""
    iu, ju = np.triu_indices(n, k=1)
    vals = st.normal(iu.size) * sigma
    if decay is not None:
        vals *= np.exp(-(ju - iu) / decay)
    E = np.zeros((n, n))
    E[iu, ju] = vals
    E[ju, iu] = vals
    return E


@dataclasses.dataclass
class Problem:
    """One PFSM input: A (n x n, row-major float64), prev_eigvals (ascending) and the
    partitioning the workload prescribes."""
    name: str
    A: np.ndarray
    prev: np.ndarray
    nblocks: int
    halo: int = -1
    fs_iters: int = 3

    @property
    def n(self) -> int:
        return self.A.shape[0]


def _assemble(lam: np.ndarray, E: np.ndarray) -> np.ndarray:
    A = E.copy()
    A[np.diag_indices_from(A)] = lam
    return A


# --- workload families (sizes and distributions follow the paper's test systems) ---------

SEQ1_SIGMAS = (1e-3, 3e-4, 1e-4, 3e-5, 1e-5)


def small_gapped(step: int = 0, n: int = 256, nblocks: int = 4, sigma: float | None = None,
                 seed: int | None = None) -> Problem:
    """N=256 test matrix: lam sorted U[-0.8, 1.5] Ha, E ~ sigma N(0,1) exp(-|i-j|/32),
    4 slices of 64. ``step`` indexes the 5-step SCF-like sequence with sigma in
    (1e-3, 3e-4, 1e-4, 3e-5, 1e-5); lam is shared by the sequence, E is fresh per step."""
    base = seed_for(1, 0) if seed is None else seed
    lam = np.sort(-0.8 + 2.3 * _Stream(base).uniform(n))
    sig = SEQ1_SIGMAS[step] if sigma is None else sigma
    E = coupling(n, sig, 32.0, _Stream(base + 100 + step))
    return Problem(f"gapped{n}_s{step}", _assemble(lam, E), lam, nblocks)


SEQ2_STEPS = 8


def diamond_like(step: int = 0, n_occ: int = 1024, n_unocc: int = 256, nblocks: int = 10) -> Problem:
    """Diamond-cell-like N=1280: lam from a two-peak density of states (1024 values from
    N(-0.4, 0.25^2) and 256 from N(0.6, 0.3^2) Ha, merged and sorted);
    E ~ sigma_j N(0,1) exp(-|i-j|/64) with sigma_j = 5e-4 * 10^(-j/2), j = 0..7."""
    st = _Stream(seed_for(2, 0))
    lam = np.sort(np.concatenate([-0.4 + 0.25 * st.normal(n_occ), 0.6 + 0.3 * st.normal(n_unocc)]))
    n = n_occ + n_unocc
    E = coupling(n, 5e-4 * 10.0 ** (-step / 2.0), 64.0, _Stream(seed_for(2, 100 + step)))
    return Problem(f"diamond{n}_s{step}", _assemble(lam, E), lam, nblocks)


def vacancy_like(n: int = 9072, nblocks: int = 36, n_pairs: int | None = None) -> Problem:
    """Silicon-vacancy-like N=9072 (432 occupied + 8640 unoccupied): lam sorted U[-0.5, 3.0] Ha,
    then ~2% of the values placed in near-degenerate pairs (lam[i+1] = lam[i] + 1e-6 for 90
    disjoint seeded i); E ~ 1e-4 N(0,1), dense, no decay."""
    st = _Stream(seed_for(3, 0))
    lam = np.sort(-0.5 + 3.5 * st.uniform(n))
    n_pairs = max(1, round(0.01 * n)) if n_pairs is None else n_pairs
    taken = np.zeros(n + 1, dtype=bool)
    picked = 0
    while picked < n_pairs:
        i = int(st.u64(1)[0] % np.uint64(n - 1))
        if taken[i] or taken[i + 1] or (i > 0 and taken[i - 1]) or taken[i + 2]:
            continue
        taken[i] = taken[i + 1] = True
        lam[i + 1] = lam[i] + 1e-6
        picked += 1
    lam = np.sort(lam)
    E = coupling(n, 1e-4, None, _Stream(seed_for(3, 100)))
    return Problem(f"vacancy{n}", _assemble(lam, E), lam, nblocks)


def metal_like(n: int = 7200, nblocks: int = 30, halo: int = 600) -> Problem:
    """Aluminium-supercell-like N=7200 (6000 occupied + 1200 unoccupied), metallic: lam sorted
    U[-0.3, 0.5] Ha with no gap, E ~ 2e-4 N(0,1) exp(-|i-j|/128); submatrix width 0.2
    (halo 600 around slices of 240)."""
    lam = np.sort(-0.3 + 0.8 * _Stream(seed_for(5, 0)).uniform(n))
    E = coupling(n, 2e-4, 128.0, _Stream(seed_for(5, 100)))
    return Problem(f"metal{n}", _assemble(lam, E), lam, nblocks, halo=halo)


def batch_sizes(count: int = 64) -> np.ndarray:
    """Uneven k-point/spin problem sizes N_i = 200 + (u_i mod 2801), i.e. 200..3000."""
    u = raw_u64(seed_for(4, 0), 0, count)
    return (200 + (u % np.uint64(2801))).astype(np.int64)


def batch_problem(i: int, n: int) -> Problem:
    """Problem i of the uneven batch: built like the N=256 matrix (lam sorted U[-0.8, 1.5],
    sigma = 1e-3, decay 32) with its own seed; slices clamp(N/10, 64, 256) wide."""
    m = min(256, max(64, n // 10))
    nblocks = max(1, n // m)
    p = small_gapped(0, n=n, nblocks=nblocks, sigma=1e-3, seed=seed_for(4, 1 + i))
    p.name = f"batch{i}_n{n}"
    return p


def random_nearly_diagonal(n: int, seed: int, sigma: float = 1e-3, decay: float | None = 16.0,
                           lo: float = -1.0, hi: float = 1.0, nblocks: int = 1,
                           halo: int = -1) -> Problem:
    """Generic small test matrix for edge cases (odd sizes, ragged slices)."""
    lam = np.sort(lo + (hi - lo) * _Stream(seed).uniform(n))
    E = coupling(n, sigma, decay, _Stream(seed + 7))
    return Problem(f"rnd{n}_{seed}", _assemble(lam, E), lam, nblocks, halo=halo)


def generalized_pair(n: int, seed: int, sigma_a: float = 1e-3, sigma_b: float = 5e-3,
                     decay: float | None = 16.0, b_spread: float = 0.1):
    """Inputs A x = lambda B x of the generalized -> standard conversion (Eq. 14-15): A nearly
    diagonal like the reduced Hamiltonian (lam sorted U[-1, 1], coupling sigma_a), B an overlap
    matrix close to the identity (ultrasoft pseudopotentials): diagonal 1 + U[0, b_spread],
    off-diagonal sigma_b N(0,1) exp(-|i-j|/decay), diagonally dominant. Returns (A, B)."""
    A = random_nearly_diagonal(n, seed, sigma=sigma_a, decay=decay).A
    st = _Stream(seed + 11)
    d = 1.0 + b_spread * st.uniform(n)
    B = _assemble(d, coupling(n, sigma_b, decay, _Stream(seed + 13)))
    return A, B


def scf_sequence(n: int, steps: int, seed: int, sigma0: float = 3e-3, decay_per_step: float = 0.3,
                 lo: float = -1.0, hi: float = 1.5):
    """A chained SCF-like sequence of Hamiltonians in a fixed (non-eigen) basis: H_j = Q diag(lam) Q^T
    + sigma_j S_j with Q a seeded random orthogonal matrix (so H_0 is dense, not diagonally dominant),
    lam sorted U[lo, hi], S_j symmetric N(0,1) / sqrt(n) and sigma_j = sigma0 decay^j (the SCF
    changes shrinking). Returns the list [H_0, ..., H_{steps-1}]."""
    Qg = _Stream(seed).normal(n * n).reshape(n, n)
    Q, R = np.linalg.qr(Qg)
    Q = Q * np.sign(np.diag(R))
    lam = np.sort(lo + (hi - lo) * _Stream(seed + 1).uniform(n))
    H0 = (Q * lam) @ Q.T
    out = []
    for j in range(steps):
        S = symmetric_direction(n, seed + 100 + j) * np.sqrt(n)   # unit-Frobenius direction, rescaled
        out.append(0.5 * ((H0 + sigma0 * decay_per_step ** j * S / np.sqrt(n)) +
                          (H0 + sigma0 * decay_per_step ** j * S / np.sqrt(n)).T))
    return out


def symmetric_direction(n: int, seed: int) -> np.ndarray:
    """Random symmetric perturbation direction with unit Frobenius norm."""
    iu, ju = np.triu_indices(n)
    vals = _Stream(seed).normal(iu.size)
    D = np.zeros((n, n))
    D[iu, ju] = vals
    D[ju, iu] = vals
    return D / np.linalg.norm(D)


def gaussian(shape, seed: int) -> np.ndarray:
    """Seeded N(0,1) array (e.g. the W of a <V, W> loss)."""
    cnt = int(np.prod(shape))
    return _Stream(seed).normal(cnt).reshape(shape)
