"""The benchmark's multi-GPU reporting (replicas only): two gloo ranks on the
CPU with different step times; every rank must see the slowest one and the
job throughput must count both replicas' work."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, value = bench.replica_throughput(torch, [2.0, 3.0][rank], world, 1.0e6, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank_and_all_work():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 3.0
        assert value == pytest.approx(world * 1.0e6 / 3.0e-3)
