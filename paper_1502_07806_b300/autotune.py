"""Block-count (slice width) autotuner for PFSM solves.

The number of slices P, i.e. the slice width m = N / P, is a free parameter of the method
(Sec. II: each slice's eigenpairs come from a window of m + 2h rows; Fig. 1). It trades the
window eigensolves (P windows of M = m + 2h rows, ~P M^3 work, one thread-block cluster each)
against the start-vector quality the halo h sets, and its best value on a B300 depends on how
the windows pack into the GPU's clusters, so it is measured rather than modelled:

  * candidates: slice widths `WIDTHS` (64 .. 256, the batch workload's range), as block counts
    round(N / m) clipped to [1, N];
  * each candidate is timed on the caller's own matrix (CUDA events around `pfsm_solve`, after a
    warm-up solve), and rejected when its largest residual ||A v - lambda v|| exceeds the default
    layout's by more than `RESIDUAL_SLACK` (the autotuner may trade speed, not accuracy);
  * the fastest survivor wins; results are cached per (device, size class, form) in memory and,
    when a path is given, in a JSON file.

The selection logic (`choose`) is pure and takes the measurements as input; `tune` does the
measuring through the library.
"""
from __future__ import annotations

import json
import os
import threading

WIDTHS = (64, 96, 128, 160, 192, 256)
RESIDUAL_SLACK = 2.0
SIZE_CLASS = 64          # problems whose N agrees to this granularity share a tuned width

_lock = threading.Lock()
_memory: dict[str, int] = {}


def default_nblocks(n: int) -> int:
    """The untuned layout: slices clamp(N/10, 64, 256) wide (the batch workload's default)."""
    m = min(256, max(64, n // 10))
    return max(1, n // m)


def candidates(n: int) -> list[int]:
    """Distinct block counts for the candidate widths, default first."""
    out = [default_nblocks(n)]
    for m in WIDTHS:
        p = max(1, min(n, int(round(n / m))))
        if p not in out:
            out.append(p)
    return out


def choose(measured: dict[int, tuple[float, float]], default: int) -> int:
    """measured[nblocks] = (ms per solve, max residual). The fastest candidate whose residual is
    within RESIDUAL_SLACK of the default's (the default itself is always admissible)."""
    if default not in measured:
        raise ValueError("the default layout must be measured")
    bound = RESIDUAL_SLACK * max(measured[default][1], 1e-300)
    ok = {p: ms for p, (ms, res) in measured.items() if p == default or res <= bound}
    return min(ok, key=lambda p: (ok[p], p))


def size_class(n: int) -> int:
    return (int(n) + SIZE_CLASS // 2) // SIZE_CLASS


def cache_key(device: str, n: int, precision: int) -> str:
    return f"{device}|{size_class(n)}|{int(precision)}"


def _load_file(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _store_file(path: str, key: str, value: int) -> None:
    data = _load_file(path)
    data[key] = int(value)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(device: str, n: int, precision: int, path: str | None = None):
    key = cache_key(device, n, precision)
    with _lock:
        if key in _memory:
            return _memory[key]
    if path:
        v = _load_file(path).get(key)
        if isinstance(v, int) and v >= 1:
            with _lock:
                _memory[key] = v
            return v
    return None


def remember(device: str, n: int, precision: int, nblocks: int, path: str | None = None) -> None:
    key = cache_key(device, n, precision)
    with _lock:
        _memory[key] = int(nblocks)
    if path:
        _store_file(path, key, nblocks)


def tune(A, prev, precision: int, halo: int = -1, fs_iters: int = 3, repeats: int = 3,
         cache_path: str | None = None, return_measurements: bool = False):
    """Measured block count for the problem (A, prev) (device tensors); cached per size class."""
    import torch

    from . import DIAG_RESIDUALS, Handle

    n = int(A.shape[0])
    device = torch.cuda.get_device_name(A.device)
    hit = lookup(device, n, precision, cache_path)
    if hit is not None and not return_measurements:
        return hit
    measured = {}
    stream = torch.cuda.current_stream()
    for p in candidates(n):
        h = Handle(n, p, halo=halo, fs_iters=fs_iters, precision=precision)
        try:
            lam = torch.empty(n, dtype=torch.float64, device=A.device)
            V = torch.empty(n, n, dtype=torch.float64, device=A.device)
            h.solve(A, prev, lam, V)                       # warm-up (and graph-free first touch)
            if h.status() != 0:
                continue
            times = []
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.solve(A, prev, lam, V)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            if h.status() != 0:
                continue
            res = float(h.diagnostic(DIAG_RESIDUALS).max())
            measured[p] = (min(times), res)
        finally:
            h.close()
    default = default_nblocks(n)
    if default not in measured:
        raise RuntimeError(f"autotune: the default layout ({default} slices) failed for N={n}")
    best = choose(measured, default)
    remember(device, n, precision, best, cache_path)
    return (best, measured) if return_measurements else best
