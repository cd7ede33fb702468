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


def _scene(kernel, model, n=1500, res=32, seed=81):
    from paper_2412_10399_gb300 import scenes as S
    x, v, B, F = S.random_state(n, res, seed, margin_cells=4.0, v_scale=40.0, f_scale=0.05)
    mat = S.Material(model, 1e5, 0.3, 1000.0, 30.0)
    sc = S.Scene("decomp", res, 1.0 / res, 1e-4, x, v, np.zeros(n, np.uint8), [mat], kernel=kernel)
    return sc, B, F


def _pack(grids, n):
    """oracle grids {k: (m (n^3,), p (n^3, 3))} -> (G, nz, ny, nx, 4)"""
    return torch.stack([torch.cat([m[:, None], p], 1).reshape(n, n, n, 4) for (m, p) in grids.values()])


def _step(st, prm, rank, ranges, O):
    n = prm.n_nodes
    ks = O.grid_ids(prm.kernel)
    g = DC.halo_sum(_pack(O.p2g(st, prm), n), rank, ranges, prm.res)
    grids = {k: (g[i, ..., 0].reshape(-1), g[i, ..., 1:].reshape(-1, 3)) for i, k in enumerate(ks)}
    vg = O.grid_update(grids, prm)
    vt = torch.stack([vg[k].reshape(n, n, n, 3) for k in ks])
    vt = DC.halo_fill(vt, rank, ranges, prm.res)
    vg = {k: vt[i].reshape(-1, 3) for i, k in enumerate(ks)}
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
