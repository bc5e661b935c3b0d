"""The N > 1 path of bench.py (independent replicas, one per GPU) aggregates
with a max over ranks of the timed milliseconds and a sum of particle-updates.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, upd = bench.aggregate(10.0 + rank, 1000 * (rank + 1), dist, device="cpu")
    out[rank] = (ms, upd)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (11.0, 3000.0)


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.aggregate(3.5, 42) == (3.5, 42.0)
