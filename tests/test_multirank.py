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


def test_dam_break_and_transfer_lines_with_stand_in_contexts(monkeypatch):
    """The extra bench lines, driven by stand-ins for the context calls (no
    GPU): every row has both kernels, the speed-up and the CK step's fraction
    of the peak from the stated algorithmic bytes."""
    import types

    import bench
    from paper_2412_10399_gb300 import scenes as S
    made = []
    monkeypatch.setattr(bench, "_make_ctx", lambda ck, sc, kernel, stream: (made.append((sc.n, kernel)) or kernel, None))
    monkeypatch.setattr(bench, "_time_steps", lambda ck, ctx, steps, stream: steps * (2.0 if ctx & 1 else 1.0))
    fake = types.SimpleNamespace(KERNEL_CK=0, KERNEL_QUADRATIC=1, TRANSFER_PIC=2, TRANSFER_APIC_GRAD=4,
                                 ckmpm_step=lambda c, n: None, ckmpm_sync=lambda c: None,
                                 ckmpm_destroy=lambda c: None)
    dam = bench.dam_break_lines(fake, 0, 1, 10, sizes=(2000,), peak=1000.0)
    row = dam["2000"]
    assert row["ck"]["ms_per_step"] == 1.0 and row["quadratic"]["ms_per_step"] == 2.0 and row["ck_speedup"] == 2.0
    assert row["ck"]["step_frac"] == pytest.approx(218.0 * 2000 / 1e-3 / 1e9 / 1000.0)
    sc = S.elastic_cube()
    tr = bench.transfer_lines(fake, sc, 0, 1, 10, peak=1000.0)
    assert tr["pic"]["ck"]["step_frac"] == pytest.approx(218.0 * sc.n / 1e-3 / 1e9 / 1000.0)
    assert tr["apic_grad"]["ck"]["step_frac"] == pytest.approx(290.0 * sc.n / 1e-3 / 1e9 / 1000.0)
    assert (sc.n, 0 | 2) in made and (sc.n, 1 | 4) in made
    assert "step_frac" not in bench.dam_break_lines(fake, 0, 1, 10, sizes=(2000,))["2000"]["ck"]


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    """Under torchrun the oracle's reference arm runs and prints on rank 0
    alone; the other ranks exit 0 without work."""
    import argparse

    import bench
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda steps=2: called.append(steps) or
                        {"value": 1e5, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "s"})
    args = argparse.Namespace(steps=5, warmup=2, gpus=2)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(args) == 0
    assert called == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    assert bench.run_reference(args) == 0
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] == 1e5
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert called == [1, 3]
