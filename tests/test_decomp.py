"""Spatial decomposition (slabs along x, one per rank): the reverse halo sum
after P2G, the halo fill after the grid update and the particle migration
after G2P, exchanged between gloo ranks on CPU.  Each rank runs the FP64
oracle's arithmetic on its own particles; after several steps the union of
the ranks' particles must equal the single-rank run up to float64 rounding
(the node sums are added in a different order)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2412_10399_gb300 import decomp as DC


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene(kernel, model, n=1500, res=32, seed=81, box=None):
    from paper_2412_10399_gb300 import scenes as S
    x, v, B, F = S.random_state(n, res, seed, margin_cells=4.0, v_scale=40.0, f_scale=0.05, box=box)
    mat = S.Material(model, 1e5, 0.3, 1000.0, 30.0)
    sc = S.Scene("decomp", res, 1.0 / res, 1e-4, x, v, np.zeros(n, np.uint8), [mat], kernel=kernel)
    return sc, B, F


def _pack(grids, n):
    """oracle grids {k: (m (n^3,), p (n^3, 3))} -> (G, nz, ny, nx, 4)"""
    return torch.stack([torch.cat([m[:, None], p], 1).reshape(n, n, n, 4) for (m, p) in grids.values()])


def _step(st, prm, rank, ranges, O):
    """One step of this rank's particles; a rank without particles still takes
    part in both halo exchanges (its contributions are zero)."""
    n = prm.n_nodes
    ks = O.grid_ids(prm.kernel)
    empty = st.x.shape[0] == 0
    local = torch.zeros((len(ks), n, n, n, 4), dtype=torch.float64) if empty else _pack(O.p2g(st, prm), n)
    g = DC.halo_sum(local, rank, ranges, prm.res)
    grids = {k: (g[i, ..., 0].reshape(-1), g[i, ..., 1:].reshape(-1, 3)) for i, k in enumerate(ks)}
    vg = O.grid_update(grids, prm)
    vt = torch.stack([vg[k].reshape(n, n, n, 3) for k in ks])
    vt = DC.halo_fill(vt, rank, ranges, prm.res)
    vg = {k: vt[i].reshape(-1, 3) for i, k in enumerate(ks)}
    if empty:
        return st
    v, B, C = O.g2p(st, vg, prm)
    F = O.plasticity((torch.eye(3, dtype=torch.float64) + prm.dt * C) @ st.F, st, prm)
    return O.State(st.x + prm.dt * v, v, B, F, st.mat, st.E)


def _worker(rank, world, port, kernel, model, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import ckmpm_oracle as O
    sc, B, F = _scene(kernel, model)
    prm = O.params_from_scene(sc)
    st_all = O.make_state(torch.from_numpy(sc.x), torch.from_numpy(sc.v), torch.from_numpy(B),
                          torch.from_numpy(F), mat=torch.from_numpy(sc.mat.astype(np.int64)))
    ranges = DC.slab_ranges(sc.res, world)
    cell = torch.floor(st_all.x[:, 0] / prm.dx).to(torch.int64)
    mine = DC.owner_of_cells(cell, ranges) == rank
    ids = torch.arange(sc.n)[mine]
    st = O.State(st_all.x[mine], st_all.v[mine], st_all.B[mine], st_all.F[mine], st_all.mat[mine])
    moved = 0
    for _ in range(steps):
        st = _step(st, prm, rank, ranges, O)
        cx = torch.floor(st.x[:, 0] / prm.dx).to(torch.int64)
        moved += int((DC.owner_of_cells(cx, ranges) != rank).sum())
        f = DC.migrate({"x": st.x, "v": st.v, "B": st.B, "F": st.F, "mat": st.mat, "id": ids}, cx, rank, ranges)
        st = O.State(f["x"], f["v"], f["B"], f["F"], f["mat"])
        ids = f["id"]
    out[rank] = (ids.numpy(), st.x.numpy(), st.v.numpy(), st.F.numpy(), st.B.numpy(), moved)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,kernel,model", [(2, 0, 0), (3, 0, 1), (2, 1, 0)])
def test_slab_decomposition_matches_one_rank(world, kernel, model):
    from oracle import ckmpm_oracle as O
    steps = 4
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, kernel, model, steps, out), nprocs=world, join=True,
                       start_method="spawn")
    sc, B, F = _scene(kernel, model)
    ref = O.run(O.make_state(torch.from_numpy(sc.x), torch.from_numpy(sc.v), torch.from_numpy(B),
                             torch.from_numpy(F), mat=torch.from_numpy(sc.mat.astype(np.int64))),
                O.params_from_scene(sc), steps)
    got_ids = np.concatenate([out[r][0] for r in range(world)])
    assert np.array_equal(np.sort(got_ids), np.arange(sc.n))  # every particle on exactly one rank
    assert sum(out[r][5] for r in range(world)) > 0  # particles did cross slabs
    for j, field in ((1, ref.x), (2, ref.v), (3, ref.F), (4, ref.B)):
        got = np.concatenate([out[r][j] for r in range(world)])[np.argsort(got_ids)]
        want = field.numpy()
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_slab_ranges_cover_the_domain_in_whole_blocks():
    for res in (16, 30, 64, 512):
        for world in (1, 2, 3, 4):
            r = DC.slab_ranges(res, world)
            assert r[0][0] == 0 and r[-1][1] == res
            assert all(a % 4 == 0 and a < b for a, b in r)
            assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
    with pytest.raises(ValueError):
        DC.slab_ranges(8, 3)


def _balance_worker(rank, world, port, kernel, steps, n, res, box, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import ckmpm_oracle as O
    sc, B, F = _scene(kernel, 1, n=n, res=res, box=box)
    prm = O.params_from_scene(sc)
    st_all = O.make_state(torch.from_numpy(sc.x), torch.from_numpy(sc.v), torch.from_numpy(B),
                          torch.from_numpy(F), mat=torch.from_numpy(sc.mat.astype(np.int64)))
    # start on even slabs: the particles crowd the low cells, mostly on rank 0
    even = DC.slab_ranges(sc.res, world)
    cell = torch.floor(st_all.x[:, 0] / prm.dx).to(torch.int64)
    mine = DC.owner_of_cells(cell, even) == rank
    f = {"x": st_all.x[mine], "v": st_all.v[mine], "B": st_all.B[mine], "F": st_all.F[mine],
         "mat": st_all.mat[mine], "id": torch.arange(sc.n)[mine]}
    n_even = int(mine.sum())
    cx = torch.floor(f["x"][:, 0] / prm.dx).to(torch.int64)
    counts = DC.layer_counts(cx, sc.res)
    ranges = DC.balanced_slab_ranges(counts, world)
    f = DC.repartition(f, cx, rank, ranges)
    n_bal = int(f["id"].numel())
    st = O.State(f["x"], f["v"], f["B"], f["F"], f["mat"])
    ids = f["id"]
    for _ in range(steps):
        st = _step(st, prm, rank, ranges, O)
        cx = torch.floor(st.x[:, 0] / prm.dx).to(torch.int64)
        f = DC.migrate({"x": st.x, "v": st.v, "B": st.B, "F": st.F, "mat": st.mat, "id": ids}, cx, rank, ranges)
        st = O.State(f["x"], f["v"], f["B"], f["F"], f["mat"])
        ids = f["id"]
    out[rank] = (ids.numpy(), st.x.numpy(), st.v.numpy(), st.F.numpy(), st.B.numpy(), n_even, n_bal,
                 counts.numpy(), ranges)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,kernel,n,res,box", [(3, 0, 1200, 32, (4.0, 14.0)), (4, 1, 2000, 64, (4.0, 24.0)),
                                                    (4, 0, 1200, 32, (4.0, 14.0))])
def test_balanced_slabs_repartition_and_step_match_one_rank(world, kernel, n, res, box):
    """A scene crowded into the low cells (4..14 of 32, 4..24 of 64) starts on
    even slabs (most of it on the first rank), is repartitioned onto
    particle-balanced slabs, then stepped with the halo exchanges and
    migration: no rank holds more than n / world plus one block layer's
    particles, and the union equals the single-rank run.  In the last case
    the particles fill three blocks along x for four ranks, so one rank is
    left empty and takes part in the exchanges with nothing of its own."""
    from oracle import ckmpm_oracle as O
    steps = 3
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_balance_worker, args=(world, port, kernel, steps, n, res, box, out), nprocs=world,
                       join=True, start_method="spawn")
    sc, B, F = _scene(kernel, 1, n=n, res=res, box=box)
    counts = out[0][7]
    assert counts.sum() == sc.n and all(np.array_equal(out[r][7], counts) for r in range(world))
    ranges = out[0][8]
    block = np.add.reduceat(counts, np.arange(0, sc.res, 4))
    bound = -(-sc.n // world) + block.max()
    even_max = max(out[r][5] for r in range(world))
    bal_max = max(out[r][6] for r in range(world))
    assert bal_max < even_max  # the even slabs overload a rank
    assert bal_max <= bound
    filled = int((block > 0).sum())
    n_empty = sum(out[r][6] == 0 for r in range(world))
    assert n_empty == max(0, world - filled)
    assert sum(out[r][6] for r in range(world)) == sc.n
    ref = O.run(O.make_state(torch.from_numpy(sc.x), torch.from_numpy(sc.v), torch.from_numpy(B),
                             torch.from_numpy(F), mat=torch.from_numpy(sc.mat.astype(np.int64))),
                O.params_from_scene(sc), steps)
    got_ids = np.concatenate([out[r][0] for r in range(world)])
    assert np.array_equal(np.sort(got_ids), np.arange(sc.n))
    for j, field in ((1, ref.x), (2, ref.v), (3, ref.F), (4, ref.B)):
        got = np.concatenate([out[r][j] for r in range(world)])[np.argsort(got_ids)]
        want = field.numpy()
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
    assert all(b - a >= 4 for a, b in ranges)


def test_balanced_slab_ranges_properties():
    rng = np.random.default_rng(3)
    for res in (16, 30, 64, 512):
        for world in (1, 2, 3, 5, 8):
            if world > -(-res // 4):
                continue
            counts = torch.from_numpy(rng.integers(0, 50, res) * (rng.random(res) < 0.6))
            r = DC.balanced_slab_ranges(counts, world)
            assert r[0][0] == 0 and r[-1][1] == res
            assert all(a % 4 == 0 and a < b for a, b in r)
            assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
            loads = [int(counts[a:b].sum()) for a, b in r]
            assert sum(loads) == int(counts.sum())
            block = torch.zeros(-(-res // 4), dtype=torch.int64).index_add_(0, torch.arange(res) // 4, counts)
            # no boundary had to move when every block edge is reachable: the load bound holds
            if world <= int((block > 0).sum()):
                assert max(loads) <= -(-int(counts.sum()) // world) + int(block.max())
    # all particles in the last block: every rank still keeps one block
    c = torch.zeros(16, dtype=torch.int64)
    c[15] = 10
    assert DC.balanced_slab_ranges(c, 4) == [(0, 4), (4, 8), (8, 12), (12, 16)]
    assert DC.balanced_slab_ranges(torch.zeros(30, dtype=torch.int64), 3) == DC.slab_ranges(30, 3)
    with pytest.raises(ValueError):
        DC.balanced_slab_ranges(torch.ones(8, dtype=torch.int64), 3)


def _drift_worker(rank, world, port, steps, every, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import ckmpm_oracle as O
    sc, B, F = _drift_scene()
    prm = O.params_from_scene(sc)
    st_all = O.make_state(torch.from_numpy(sc.x), torch.from_numpy(sc.v), torch.from_numpy(B),
                          torch.from_numpy(F), mat=torch.from_numpy(sc.mat.astype(np.int64)))
    cell = torch.floor(st_all.x[:, 0] / prm.dx).to(torch.int64)
    ranges = DC.balanced_slab_ranges(DC.layer_counts(cell, sc.res) // world, world)  # same on every rank
    mine = DC.owner_of_cells(cell, ranges) == rank
    f = {"x": st_all.x[mine], "v": st_all.v[mine], "B": st_all.B[mine], "F": st_all.F[mine],
         "mat": st_all.mat[mine], "id": torch.arange(sc.n)[mine]}
    changes, worst = 0, 1.0
    for k in range(steps):
        st = O.State(f["x"], f["v"], f["B"], f["F"], f["mat"])
        st = _step(st, prm, rank, ranges, O)
        cx = torch.floor(st.x[:, 0] / prm.dx).to(torch.int64)
        f = DC.migrate({"x": st.x, "v": st.v, "B": st.B, "F": st.F, "mat": st.mat, "id": f["id"]}, cx, rank, ranges)
        if (k + 1) % every == 0:
            cx = torch.floor(f["x"][:, 0] / prm.dx).to(torch.int64)
            worst = max(worst, DC.load_imbalance(DC.layer_counts(cx, sc.res), ranges))
            f, ranges, changed = DC.rebalance(f, cx, rank, ranges, sc.res, tolerance=0.1)
            changes += int(changed)
    out[rank] = (f["id"].numpy(), f["x"].numpy(), f["v"].numpy(), f["F"].numpy(), f["B"].numpy(), changes, worst,
                 ranges)
    dist.barrier()
    dist.destroy_process_group()


def _drift_scene():
    """The crowded scene of the balance test moving along +x at 150 m/s
    (0.48 cells per step; with the elastic wave speed the CFL number is 0.5)."""
    sc, B, F = _scene(0, 0, n=1200, res=32, box=(4.0, 12.0))
    sc.v = sc.v * 0.1 + np.array([150.0, 0.0, 0.0])
    return sc, B, F


def test_rebalance_follows_a_drifting_scene_and_matches_one_rank():
    """Particles drift across the slab boundaries; every two steps the ranks
    measure the imbalance and move to particle-balanced slabs when the
    largest rank exceeds the mean by more than 10%.  At least one rebalance
    happens, and after 16 steps (about 7.7 cells of drift) the union equals
    the single-rank run."""
    from oracle import ckmpm_oracle as O
    world, steps, every = 3, 16, 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_drift_worker, args=(world, port, steps, every, out), nprocs=world, join=True,
                       start_method="spawn")
    sc, B, F = _drift_scene()
    changes = {out[r][5] for r in range(world)}
    assert len(changes) == 1 and changes.pop() >= 1  # every rank took the same decisions, at least once
    assert all(out[r][7] == out[0][7] for r in range(world))
    ref = O.run(O.make_state(torch.from_numpy(sc.x), torch.from_numpy(sc.v), torch.from_numpy(B),
                             torch.from_numpy(F), mat=torch.from_numpy(sc.mat.astype(np.int64))),
                O.params_from_scene(sc), steps)
    got_ids = np.concatenate([out[r][0] for r in range(world)])
    assert np.array_equal(np.sort(got_ids), np.arange(sc.n))
    for j, field in ((1, ref.x), (2, ref.v), (3, ref.F), (4, ref.B)):
        got = np.concatenate([out[r][j] for r in range(world)])[np.argsort(got_ids)]
        want = field.numpy()
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
