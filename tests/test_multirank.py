"""The multi-GPU path of bench.py is replicas only: each rank solves its own problems and the
job rate is all ranks' solves over the slowest rank's time.  Its aggregation is checked here
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends its 10 steps took 100 * (r + 1) ms
    value, t = bench.job_throughput(10, 100.0 * (rank + 1))
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        value, t = out[r]
        assert t == 200.0                      # max over ranks
        assert abs(value - 2 * 10 / 0.2) < 1e-9  # all ranks' steps / slowest time


def test_single_process_is_identity():
    import bench
    value, t = bench.job_throughput(5, 250.0)
    assert t == 250.0 and abs(value - 20.0) < 1e-12
