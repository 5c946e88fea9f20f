"""Replica (N > 1) host logic of bench.py on CPU: two gloo ranks aggregate
their timings (max over ranks) and iteration counts (sum over ranks)."""
import os
import socket

import pytest
import torch
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
    ms, iters = bench.aggregate_replicas(10.0 + 5.0 * rank, 400 + rank, world)
    out[rank] = (ms, iters)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == (15.0, 801)


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_replicas(12.5, 400, 1) == (12.5, 400)
