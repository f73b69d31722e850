"""The bench's multi-process (replica) timing on the CPU: two gloo ranks
report different totals; both must get the slowest rank's time spread over
all ranks' batches."""
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
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.whole_job_ms(10.0 * (rank + 1), 5, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_time_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        got = dict(out)
    assert got == {0: pytest.approx(20.0 / 10), 1: pytest.approx(20.0 / 10)}


def test_whole_job_time_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_ms(12.0, 4, 1) == 3.0
