"""The multi-GPU path of bench.py is replicas only (one scene per rank, no
collective on the data path); its host logic -- max-over-ranks time and
whole-job particle count -- is checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [10.0, 25.0][rank]
    n_local = [1000, 3000][rank]
    value, ms = bench.aggregate_ranks(ms_local, n_local, steps=4, dist=dist, device="cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank_and_all_particles():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        value, ms = out[r]
        assert ms == 25.0
        assert abs(value - (1000 + 3000) * 4 / 0.025) < 1e-6


def test_single_rank_aggregation():
    import bench
    value, ms = bench.aggregate_ranks(20.0, 5000, steps=10)
    assert ms == 20.0 and abs(value - 5000 * 10 / 0.02) < 1e-9
