"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

With N GPUs the method runs N independent replicas (no exchange between them); the
bench takes the slowest rank's time and reports the whole job's node updates over it.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms, bench.job_mlups(world, 1000, 10, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        times = [3.0, 5.0]
        mp.start_processes(_rank, args=(2, _free_port(), times, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    ms, mlups = res[0]
    assert ms == 5.0
    assert mlups == pytest.approx(2 * 1000 * 10 / 5e-3 / 1e6)
