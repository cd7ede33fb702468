"""Shared helpers for the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import numpy as np
import pytest
import torch

from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2412_10399_gb300 import ckmpm
    return ckmpm


def f32(a):
    return np.asarray(a, np.float64).astype(np.float32)


def random_scene(n, res, seed, model=S.FIXED_COROTATED, kernel=S.KERNEL_CK, dt=1e-4, E=1e5, box=None,
                 v_scale=1.0, b_scale=1.0, f_scale=0.05, gravity=(0.0, -9.8, 0.0), bc_cells=3.0):
    """A scene with a random (x, v, B, F) state, all rounded to float32."""
    x, v, B, F = S.random_state(n, res, seed, margin_cells=4.0, v_scale=v_scale, b_scale=b_scale,
                                f_scale=f_scale, box=box)
    mat = S.Material(model, E, 0.3, 1600.0 if model == S.DRUCKER_PRAGER else 1000.0, 30.0)
    sc = S.Scene("random", res, 1.0 / res, dt, f32(x).astype(np.float64), f32(v).astype(np.float64),
                 np.zeros(n, np.uint8), [mat], gravity=gravity, bc_cells=bc_cells, kernel=kernel)
    return sc, f32(B), f32(F)


def oracle_state(sc, B=None, F=None):
    st = O.make_state(torch.from_numpy(sc.x.astype(np.float32).astype(np.float64)),
                      torch.from_numpy(sc.v.astype(np.float32).astype(np.float64)),
                      None if B is None else torch.from_numpy(B.astype(np.float64)),
                      None if F is None else torch.from_numpy(F.astype(np.float64)),
                      mat=torch.from_numpy(sc.mat.astype(np.int64)))
    return st


def rel(gpu, ref):
    ref = np.asarray(ref, np.float64)
    d = np.abs(np.asarray(gpu, np.float64) - ref).max()
    s = np.abs(ref).max()
    return d / s if s > 0 else d


def window_step(x, v, B, F, mat, cell, p, prm_local, dx, halo=3):
    """One oracle step of particle p computed on a small local domain: every
    particle within `halo` cells of p (all that reach p's stencil nodes)
    shifted by a whole number of cells so that p's cell lands at the centre
    of a prm_local.res^3 domain, stepped without walls; returns p's
    (x, v, F, B) in the original frame and the neighbourhood's indices.
    Exact for p as long as the original domain's walls touch none of p's
    nodes (the shift is a multiple of dx, a power of two)."""
    near = np.flatnonzero(np.all(np.abs(cell - cell[p]) <= halo, axis=1))
    shift = (cell[p].astype(np.int64) - prm_local.res // 2) * dx
    st = O.make_state(torch.from_numpy(np.asarray(x[near], np.float64) - shift),
                      torch.from_numpy(np.asarray(v[near], np.float64)),
                      torch.from_numpy(np.asarray(B[near], np.float64)),
                      torch.from_numpy(np.asarray(F[near], np.float64)),
                      mat=torch.from_numpy(np.asarray(mat[near]).astype(np.int64)))
    new = O.step(st, prm_local, bc=False)
    i = int(np.flatnonzero(near == p)[0])
    return (new.x[i].numpy() + shift, new.v[i].numpy(), new.F[i].numpy(), new.B[i].numpy()), near, new, st
