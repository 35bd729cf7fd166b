"""Multi-GPU is replicas only: every rank solves its own problems and the
job's throughput uses the slowest rank's time.  The aggregation runs here
with world size 2 over gloo on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 if rank == 0 else 250.0  # rank 1 is slower
    value, t = bench.aggregate(local_ms, units_per_rank=20, dist=dist, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, t = out[r]
        assert t == pytest.approx(250.0)
        assert value == pytest.approx(world * 20 / 0.25)


def test_single_process_aggregate():
    import bench
    value, t = bench.aggregate(500.0, units_per_rank=10)
    assert t == 500.0 and value == pytest.approx(20.0)
