"""The multi-rank path of bench.py (independent replicas) on CPU with gloo.

Each rank times its own replica; the job's time is the slowest rank's and
its throughput counts the units of every rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank        # rank 1 is the slow one
    units_local = 1.0e9 * (rank + 1)
    ms, value = bench.aggregate_ranks(ms_local, units_local, dist, "cpu")
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 150.0                          # max over ranks
        assert value == pytest.approx(3.0e9 / 0.150)  # all units / slowest time


def test_single_rank_has_no_collective():
    import bench
    ms, value = bench.aggregate_ranks(200.0, 4.0e9, None)
    assert ms == 200.0 and value == pytest.approx(2.0e10)
