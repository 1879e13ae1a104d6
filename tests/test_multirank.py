"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs an independent replica, the job time is the slowest rank's (all-reduce
MAX), and the throughput is world x per-rank work / that time (weak scaling).
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 1.5 + rank            # rank 1 is the slow one
        t = bench.max_over_ranks(local, dist)
        out[rank] = (t, bench.job_throughput(world, 100.0, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, 2 * 100.0 / 2.5)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.job_throughput(1, 50.0, 2.0) == 25.0
