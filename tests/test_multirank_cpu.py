"""The N > 1 bench path on CPU ranks (gloo, world size 2): every rank runs its own
independent replica; the job time is the slowest rank's and the throughput counts all
ranks' particle-steps.  No collective touches simulation data."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [10.0, 14.0][rank]
    units = [1000, 3000][rank]
    q.put((rank, bench.aggregate(ms, units, dist, device="cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    got = dict(q.get() for _ in range(2))
    for rank in (0, 1):
        max_ms, units = got[rank]
        assert max_ms == 14.0
        assert units == 4000.0


def test_aggregate_single_process():
    import bench

    assert bench.aggregate(5.0, 7, None) == (5.0, 7.0)
