"""Multi-GPU runs are independent replicas (no data-path collective); the bench reduces only the
time (max over ranks) and the processed points (sum).  Checked with 2 gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow one
    pts_local = 1000 * (rank + 1)
    ms, value = bench.replica_aggregate(ms_local, pts_local, dist, device="cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregate_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of this (threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    expect_ms = 15.0
    expect_value = 3000 / (expect_ms * 1e-3) / 1e9
    for r in range(world):
        ms, value = out[r]
        assert ms == expect_ms
        assert abs(value - expect_value) <= 1e-12 * expect_value


def test_replica_aggregate_single_process():
    import bench
    ms, value = bench.replica_aggregate(4.0, 2000)
    assert ms == 4.0 and abs(value - 2000 / 4e-3 / 1e9) < 1e-15
