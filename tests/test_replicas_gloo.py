"""The N > 1 bench path runs independent replicas (no data-path collective):
each rank solves its own copy and the job's time is the max over ranks.
This checks that aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r "took" 1 + r seconds for 1000 units
        t = bench.rank_max(1.0 + rank, world, "cpu")
        out[rank] = (t, bench.job_throughput(world, 1000.0, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (2.0, 1000.0)  # 2 ranks x 1000 units in 2 s


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.rank_max(3.5, 1) == 3.5
    assert bench.job_throughput(1, 10.0, 2.0) == 5.0
