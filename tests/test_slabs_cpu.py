"""Host side of the z-slab decomposition, on CPU: the partition, the neighbour and ghost
plane rules, and the halo-exchange schedule, in one process (LocalTransport) and across
two gloo ranks (DistTransport, the path NCCL takes between GPUs). Fake slabs stand in for
the library: each packs messages that name the slab, face and round, and records what it
unpacks, so a message routed to the wrong slab or side fails.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2409_03401_gb300.slabs import (LocalTransport, ghost_range, halo_exchange,  # noqa: E402
                                          neighbours, split_planes)


def test_split_planes_is_contiguous_and_balanced():
    for nz in (1, 7, 37, 512):
        for n in range(1, min(nz, 9) + 1):
            parts = split_planes(nz, n)
            assert parts[0][0] == 0 and sum(m for _, m in parts) == nz
            assert all(a + m == b for (a, m), (b, _) in zip(parts, parts[1:]))
            assert max(m for _, m in parts) - min(m for _, m in parts) <= 1
    with pytest.raises(ValueError):
        split_planes(3, 4)


def test_neighbours_and_ghost_planes():
    assert neighbours(0, 3, True) == (None, 1) and neighbours(2, 3, True) == (1, None)
    assert neighbours(0, 3, False) == (2, 1) and neighbours(2, 3, False) == (1, 0)
    assert neighbours(0, 1, False) == (0, 0) and neighbours(0, 1, True) == (None, None)
    assert ghost_range(10, 0, 4, True) == [0, 1, 2, 3, 4]
    assert ghost_range(10, 0, 4, False) == [9, 0, 1, 2, 3, 4]
    assert ghost_range(10, 6, 4, True) == [5, 6, 7, 8, 9]
    assert ghost_range(10, 6, 4, False) == [5, 6, 7, 8, 9, 0]
    assert ghost_range(5, 0, 5, False) == [4, 0, 1, 2, 3, 4, 0]


class FakeSlab:
    """Stands in for paper_2409_03401_gb300.slabs.Slab: messages carry (slab, side, kind,
    round); unpacked messages are kept per (kind, side)."""

    def __init__(self, i, n, wall_z):
        lower, upper = neighbours(i, n, wall_z)
        self.i, self.has = i, (lower is not None, upper is not None)
        self.round = 0
        self.got = {}

    def _msg(self, side, kind):
        return torch.tensor([self.i, side, kind, self.round], dtype=torch.int64)

    def pack(self, side):
        return self._msg(side, 0)

    def phi_pack(self, side):
        return self._msg(side, 1)

    def unpack(self, side, m):
        self.got[(0, side)] = m.tolist()

    def phi_unpack(self, side, m):
        self.got[(1, side)] = m.tolist()


def _check(slabs, n, wall_z, rnd, flow):
    for i, s in slabs.items():
        lower, upper = neighbours(i, n, wall_z)
        for kind in ((0, 1) if flow else (0,)):
            if lower is not None:
                assert s.got[(kind, 0)] == [lower, 1, kind, rnd]    # lower neighbour's upper face
            else:
                assert (kind, 0) not in s.got
            if upper is not None:
                assert s.got[(kind, 1)] == [upper, 0, kind, rnd]    # upper neighbour's lower face
            else:
                assert (kind, 1) not in s.got


@pytest.mark.parametrize("n", [1, 2, 3, 5])
@pytest.mark.parametrize("wall_z", [True, False])
@pytest.mark.parametrize("flow", [True, False])
def test_local_schedule_routes_every_face(n, wall_z, flow):
    slabs = {i: FakeSlab(i, n, wall_z) for i in range(n)}
    tr = LocalTransport(n, wall_z)
    for rnd in range(3):
        for s in slabs.values():
            s.round, s.got = rnd, {}
        halo_exchange(slabs, tr, flow)
        _check(slabs, n, wall_z, rnd, flow)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, wall_z, out):
    sys.path.insert(0, ROOT)
    from paper_2409_03401_gb300.slabs import DistTransport, halo_exchange as hx
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = FakeSlab(rank, world, wall_z)
        tr = DistTransport(wall_z)
        res = []
        for rnd in range(3):
            s.round, s.got = rnd, {}
            hx({rank: s}, tr, True)
            res.append(dict(s.got))
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
@pytest.mark.parametrize("wall_z", [True, False])
def test_two_gloo_ranks_exchange_halos(wall_z):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), wall_z, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rnd in range(3):
        slabs = {}
        for r in range(world):
            s = FakeSlab(r, world, wall_z)
            s.got = res[r][rnd]
            slabs[r] = s
        _check(slabs, world, wall_z, rnd, True)
