"""The multi-process path of bench.py (independent replicas, one per GPU):
max-over-ranks timing and the whole-job rate, run as two gloo ranks on CPU."""

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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    sec = 1.0 + rank  # rank 1 is the slow one
    m = bench.max_over_ranks(sec)
    rate = bench.replica_rate(4, m, world)
    out[rank] = (m, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        m, rate = out[r]
        assert m == 2.0
        assert rate == world * 4 / 2.0


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_rate(10, 2.0, 1) == 5.0
