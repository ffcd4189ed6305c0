"""Write the full-size oracle references used by the GPU parity tests at the two largest
workloads: the silicon-vacancy-like matrix (N = 9072, 36 slices, windows of 2068; Table II's
system) and the aluminium-like metal (N = 7200, 30 slices, halo 600, windows of 1440; Table III's
system) with the eigen-adjoint backward of the loss sum_{k < 6000} lambda_k + <V, W>.

Every stored value comes from ``oracle/`` (the plain FP64 CPU restatement of Section II); this
script only draws the seeded inputs, calls the oracle and packs a sample of its outputs. The whole
solve costs tens of minutes of CPU at these sizes, so it runs once and the results are kept,
keyed by the SHA-256 of the input bytes (A and prev, row-major float64).

Stored per workload (``tests/golden/<name>.npz``):
  sha256_A, sha256_prev, n, nblocks, halo, fs_iters   input identity and method parameters
  plan (4 x nblocks), lam, res, eps, alpha           every eigenvalue, residual, shift and step
  sketch_seed, Sq                                    the sketch Omega V of EVERY eigenvector
                                                     (Omega: SKETCH x n seeded N(0, 1)), quantised
  cols, Vq                                           sampled eigenvector columns, quantised
  xcols, Xq                                          sampled vectors after Eq. 11, quantised
The sketch lets a test check every vector and every cluster of close eigenvalues without storing
V: for unit vectors u, v, ||Omega (u - v)|| / sqrt(SKETCH) estimates ||u - v|| (a chi variable
with SKETCH degrees of freedom), and Omega P Omega^T = (Omega V_C)(Omega V_C)^T sketches the
projector P of a cluster C.
Metal workload only:
  dA_rows, dA_cols, dA_vals     sampled entries of the oracle gradient dA (FP64)
  dA_diag                       its whole diagonal
  dir_seeds, dA_dot_dir         <dA, D_d> for 32 unit-Frobenius symmetric directions D_d

Quantisation (fullsize_ref.py): a column entry v is stored as the integer rint(v * 2^40), byte
planes split so the (mostly constant) high bytes deflate well. The absolute error per entry is
<= 2^-41 (4.5e-13), so a stored unit column differs from the oracle's by < 2^-41 sqrt(N) = 4.3e-11
in norm, far below the 1e-8 projector bar the tests apply.

Usage: python tests/golden/make_fullsize.py [vacancy] [metal] [--threads T]
A raw dump of the full oracle outputs (several GB) goes to a cache directory outside the repository
($PFSM_ORACLE_CACHE, default <system temp dir>/pfsm_oracle_cache) so that the sample can be re-packed
without re-running the oracle.
"""
from __future__ import annotations

import argparse
import os
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402
from fullsize_ref import quantise, sha256, sketch_matrix  # noqa: E402

CACHE = os.environ.get("PFSM_ORACLE_CACHE", os.path.join(tempfile.gettempdir(), "pfsm_oracle_cache"))

# the <V, W> term of the metal loss and the directions of the directional-derivative check
W_SEED = 55
OCCUPIED = 6000
DIR_SEED0 = 0x5EED0000
N_DIRS = 32


def sample_columns(p, count: int, seed: int, pair_gap: float, max_pairs: int) -> np.ndarray:
    """Both members of up to max_pairs near-degenerate pairs of previous eigenvalues (gap <
    pair_gap; a seeded choice when there are more), then seeded distinct indices up to ``count``
    columns, ascending."""
    close = np.nonzero(np.diff(p.prev) < pair_gap)[0]
    if close.size > max_pairs:
        order = np.argsort(wl.raw_u64(seed + 1, 0, close.size), kind="stable")
        close = np.sort(close[order[:max_pairs]])
    pick = set(close.tolist()) | set((close + 1).tolist())
    u = wl.raw_u64(seed, 0, 8 * count)
    for v in u:
        if len(pick) >= count:
            break
        pick.add(int(v % np.uint64(p.n)))
    return np.array(sorted(pick), dtype=np.int64)


def run_oracle(p, threads: int):
    os.makedirs(CACHE, exist_ok=True)
    key = sha256(p.A)[:16]
    raw = os.path.join(CACHE, f"{p.name}_{key}.npz")
    if os.path.exists(raw):
        with np.load(raw) as z:
            return {k: z[k] for k in z.files}
    oracle.set_threads(threads)
    t0 = time.time()
    r = oracle.pfsm(p.A, p.prev, p.nblocks, halo=p.halo, fs_iters=p.fs_iters)
    print(f"{p.name}: oracle solve {time.time() - t0:.0f} s", flush=True)
    out = dict(lam=r.lam, res=r.res, eps=r.eps, alpha=r.alpha, plan=r.plan, V=r.V, xfs=r.xfs)
    np.savez(raw, **out)
    return out


def metal_gradient(p, r: dict, threads: int):
    oracle.set_threads(threads)
    n = p.n
    dlam = np.zeros(n)
    dlam[:OCCUPIED] = 1.0
    W = wl.gaussian((n, n), seed=W_SEED)
    t0 = time.time()
    dA = oracle.backward(r["V"], r["lam"], dlam, W, tau=1e-8)
    print(f"{p.name}: oracle backward {time.time() - t0:.0f} s", flush=True)
    return dA


def pack(p, r: dict, ncols: int, nx: int, seed: int, pair_gap: float, max_pairs: int,
         extra: dict | None = None) -> str:
    cols = sample_columns(p, ncols, seed, pair_gap, max_pairs)
    xcols = cols[np.linspace(0, cols.size - 1, nx).round().astype(np.int64)]
    sketch_seed = seed + 7
    Om = sketch_matrix(p.n, sketch_seed)
    out = dict(sha256_A=sha256(p.A), sha256_prev=sha256(p.prev), n=p.n, nblocks=p.nblocks,
               halo=p.halo, fs_iters=p.fs_iters, plan=r["plan"], lam=r["lam"], res=r["res"],
               eps=r["eps"], alpha=r["alpha"], sketch_seed=sketch_seed, Sq=quantise(Om @ r["V"]),
               cols=cols, Vq=quantise(r["V"][:, cols]), xcols=xcols, Xq=quantise(r["xfs"][:, xcols]))
    if extra:
        out.update(extra)
    path = os.path.join(HERE, f"{p.name}.npz")
    np.savez_compressed(path, **out)
    print(f"{p.name}: wrote {path} ({os.path.getsize(path) / 1e6:.2f} MB, {cols.size} columns)")
    return path


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="*", default=["vacancy", "metal"])
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    oracle.build()
    if "vacancy" in args.which:
        p = wl.vacancy_like()
        r = run_oracle(p, args.threads)
        # 24 of the 122 pairs of previous eigenvalues 1e-6 apart or closer (90 planted, 32 natural)
        # in full, every vector and pair through the sketch
        pack(p, r, ncols=64, nx=16, seed=wl.seed_for(3, 900), pair_gap=1.01e-6, max_pairs=24)
    if "metal" in args.which:
        p = wl.metal_like()
        r = run_oracle(p, args.threads)
        graw = os.path.join(CACHE, f"{p.name}_{sha256(p.A)[:16]}_dA.npy")
        if os.path.exists(graw):
            dA = np.load(graw)
        else:
            dA = metal_gradient(p, r, args.threads)
            np.save(graw, dA)
        n = p.n
        u = wl.raw_u64(wl.seed_for(5, 900), 0, 2 * 8192)
        rows = (u[0::2] % np.uint64(n)).astype(np.int64)
        cols = (u[1::2] % np.uint64(n)).astype(np.int64)
        seeds = np.array([DIR_SEED0 + d for d in range(N_DIRS)], dtype=np.int64)
        dots = np.array([float(np.sum(dA * wl.symmetric_direction(n, int(s)))) for s in seeds])
        pack(p, r, ncols=48, nx=16, seed=wl.seed_for(5, 901), pair_gap=1e-7, max_pairs=8,
             extra=dict(dA_rows=rows, dA_cols=cols, dA_vals=dA[rows, cols], dA_diag=np.diag(dA).copy(),
                        dir_seeds=seeds, dA_dot_dir=dots, w_seed=W_SEED, occupied=OCCUPIED))


if __name__ == "__main__":
    main()
