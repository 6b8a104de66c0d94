"""The N > 1 path of bench.py on CPU: ranks are independent replicas (a
single instance does not shard), the timed duration is the slowest rank's and
the reported rate counts the units of all ranks.  world_size 2 over gloo."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank)  # rank 1 is the slow one
        out[rank] = t
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_world2():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 2.5
    # 10 steps per replica on 2 replicas in 2.5 s of the slowest rank
    assert bench.whole_job_rate(10, 2, 2.5) == pytest.approx(8.0)


def test_single_process_is_identity():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(5, 1, 0.5) == 10.0
