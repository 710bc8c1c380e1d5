"""Host logic of bench.py's N > 1 path on CPU: world-size-2 gloo ranks (replicas, max-over-ranks timing)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [1.0 + rank, 10.0 - rank]          # rank 0 slower on the second timer, rank 1 on the first
    got = bench.reduce_max(local, dist)
    dist.barrier()
    out[rank] = (got, bench.aggregate_value(world, 100.0, got[0]))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_aggregate_units():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        got, value = res[rank]
        assert got == [2.0, 10.0]
        assert value == pytest.approx(2 * 100.0 / 2.0)


def test_reduce_without_process_group_is_identity():
    import bench
    assert bench.reduce_max([3.0, 4.0]) == [3.0, 4.0]
    assert bench.aggregate_value(1, 50.0, 2.0) == 25.0
