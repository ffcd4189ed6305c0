"""The multi-rank timing logic of bench.py on CPU with the gloo backend (world size 2): every rank
sees the slowest rank's time, and the whole-job rate counts every rank's units over that time.
(On GPUs the same calls run over NCCL with the tensor on the device.)"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 1.5 + rank                      # rank 1 is the slow one
        slowest = bench.max_over_ranks(local, world, device="cpu")
        q.put((rank, local, slowest, bench.job_rate(20, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.5, 2.5]
    assert all(o[2] == 2.5 for o in out)                  # both ranks report the max
    assert all(o[3] == pytest.approx(2 * 20 / 2.5) for o in out)


def test_single_rank_is_local():
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(20, 1, 2.0) == 10.0
