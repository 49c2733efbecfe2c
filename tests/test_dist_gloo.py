"""The bench's multi-rank logic on CPU: two gloo ranks on 127.0.0.1.

The GPU work itself needs a GPU per rank; what is checked here is the host
side that a launch with N > 1 ranks relies on: the job's step time is the max
over ranks (every rank gets the same value), the whole-job rate counts every
rank's strings, and the reference arm runs on rank 0 only (the other ranks
return without work)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        got = bench.allmax(ms, world, "cpu")
        rate = bench.whole_job_rate(1000, world, got)
        # the reference arm: a rank other than 0 returns before any work
        if rank != 0:
            bench.run_reference(None)  # args are not read on a rank > 0
        out[rank] = (got, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (15.0, pytest.approx(2 * 1000 / 0.015))
