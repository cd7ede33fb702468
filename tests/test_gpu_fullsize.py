"""Parity at the benchmark's full size, in the launch configuration bench.py
times: the large-impact scene (16,273,664 particles on the 512^3 virtual
grid) in a CK context made by ckmpm_create, stepped 80 times so that the
balls are in contact with the keep (stress, Drucker-Prager plasticity and the
fixed-corotated path all active), then one more step compared with the FP64
oracle on sampled particles.

The oracle cannot run the whole scene in a test, but one particle's step
depends only on the particles whose stencils reach its nodes, all within 3
cells of it.  For each sampled particle the test takes every particle within
3 cells (about 2,700), shifts them by a whole number of cells into a 14^3
local domain (an exact shift: dx is a power of two, and the kernel weights
depend only on offsets from nodes), and runs one oracle step there without
walls; the sampled particle's result is compared with the GPU's.  Samples
are at least 8 cells from every wall, so the big domain's sticky walls
(3 cells) touch none of their nodes.

Both sides start from the same state: the GPU state after 80 steps is read
back and uploaded again (so the stored M is rebuilt from the same B and F the
oracle receives).  Tolerances, per sampled particle: x within 1e-6 dx + 2e-7;
v within 2e-5 of its neighbourhood's velocity scale, the largest speed plus
the largest one-step velocity a node can get from one particle's stress,
dt max|tau| / (rho dx) (P2G rounds each block's sums to a unit set by the
largest contribution, and at rest the stress contributions are large and
cancel); F within 2e-5 of max(1, |F|); B within 5e-5 of the largest |B| over
the samples' neighbourhoods.
"""
import numpy as np
import pytest

from gpu_helpers import need_gpu, window_step
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu

R_LOCAL = 14
HALO = 3


def _pick_samples(x, v, F, mat, res, dx, rng):
    cell = np.floor(x / dx).astype(np.int32)
    inner = np.all((cell >= 8) & (cell < res - 8), axis=1)
    ball = np.flatnonzero(inner & (mat == 1))
    moving_sand = np.flatnonzero(inner & (mat == 0) & (np.linalg.norm(v, axis=1) > 0.5))
    strained_sand = np.flatnonzero(inner & (mat == 0) & (np.abs(F - np.eye(3)).reshape(len(F), 9).max(1) > 1e-4))
    any_sand = np.flatnonzero(inner & (mat == 0))
    picks = []
    for pool, k in ((ball, 16), (moving_sand, 16), (strained_sand, 8), (any_sand, 8)):
        if len(pool):
            picks.append(rng.choice(pool, size=min(k, len(pool)), replace=False))
    return np.unique(np.concatenate(picks)), cell


def test_large_impact_one_step_sampled_parity():
    ck = need_gpu()
    sc = S.large_impact()
    assert sc.n == 16273664
    sim = ck.Simulation(sc, ck.KERNEL_CK)
    sim.step(80)
    sim.sync()
    x0, v0 = sim.read(ck.FIELD_X), sim.read(ck.FIELD_V)
    B0, F0 = sim.read(ck.FIELD_B), sim.read(ck.FIELD_F)
    sim.write(ck.FIELD_F, F0)
    sim.write(ck.FIELD_B, B0)
    sim.step(1)
    sim.sync()
    x1, v1 = sim.read(ck.FIELD_X), sim.read(ck.FIELD_V)
    B1, F1 = sim.read(ck.FIELD_B), sim.read(ck.FIELD_F)
    sim.close()

    rng = np.random.default_rng(2024)
    mat = sc.mat
    samples, cell = _pick_samples(x0, v0, F0, mat, sc.res, sc.dx, rng)
    assert len(samples) >= 40
    assert np.any(mat[samples] == 1) and np.any(mat[samples] == 0)
    prm = O.params_from_scene(sc)
    prm.res, prm.bc_cells = R_LOCAL, 0.0
    got, want, vscale, bscale = [], [], [], 0.0
    rho_min = min(m.rho for m in prm.materials)
    for p in samples:
        w, near, new, st = window_step(x0, v0, B0, F0, mat, cell, p, prm, sc.dx, HALO)
        want.append(w)
        got.append((x1[p], v1[p], F1[p], B1[p]))
        tau = O.kirchhoff_stress(st, prm)
        vscale.append(max(np.abs(v0[near]).max(), float(new.v.abs().max()))
                      + prm.dt * float(tau.abs().max()) / (rho_min * sc.dx))
        bscale = max(bscale, float(np.abs(B0[near]).max()), float(new.B.abs().max()))
    for (gx, gv, gF, gB), (wx, wv, wF, wB), vs, p in zip(got, want, vscale, samples):
        assert np.abs(gx - wx).max() <= 1e-6 * sc.dx + 2e-7, p
        assert np.abs(gv - wv).max() <= 2e-5 * vs + 1e-7, p
        assert np.abs(gF - wF).max() <= 2e-5 * max(1.0, np.abs(wF).max()), p
        assert np.abs(gB - wB).max() <= 5e-5 * bscale + 1e-9, p


@pytest.mark.parametrize("kernel", [S.KERNEL_CK, S.KERNEL_QUADRATIC])
def test_granular_column_last_step_sampled_parity(kernel):
    """The granular-column configuration (346,112 Drucker-Prager particles on
    128^3, dt 5e-5) over its whole length: 499 steps on the GPU, then step 500
    compared with the FP64 oracle on sampled particles by the same local-window
    step and tolerances as the large-impact test.  A whole 500-step trajectory
    cannot be compared particle by particle: the float32 stress noise at rest
    (a few ulp of the stretches) grows over the collapse, so the check is that
    every step of the configuration, here its last and most deformed, is the
    oracle's step of the state it starts from."""
    ck = need_gpu()
    sc = S.granular_column()
    sc.kernel = kernel
    assert sc.n == 346112
    sim = ck.Simulation(sc, kernel)
    sim.step(499)
    sim.sync()
    x0, v0 = sim.read(ck.FIELD_X), sim.read(ck.FIELD_V)
    B0, F0 = sim.read(ck.FIELD_B), sim.read(ck.FIELD_F)
    sim.write(ck.FIELD_F, F0)
    sim.write(ck.FIELD_B, B0)
    sim.step(1)
    sim.sync()
    x1, v1 = sim.read(ck.FIELD_X), sim.read(ck.FIELD_V)
    B1, F1 = sim.read(ck.FIELD_B), sim.read(ck.FIELD_F)
    sim.close()

    rng = np.random.default_rng(500)
    mat = sc.mat
    cell = np.floor(x0 / sc.dx).astype(np.int32)
    inner = np.all((cell >= 8) & (cell < sc.res - 8), axis=1)
    dev = np.abs(F0 - np.eye(3)).reshape(len(F0), 9).max(1)
    strained = np.flatnonzero(inner & (dev > np.quantile(dev[inner], 0.99)))
    top = np.flatnonzero(inner & (cell[:, 1] >= cell[inner, 1].max() - 1))
    low = np.flatnonzero(inner & (cell[:, 1] <= 9))
    picks = [rng.choice(pool, size=min(k, len(pool)), replace=False)
             for pool, k in ((strained, 16), (top, 12), (low, 12), (np.flatnonzero(inner), 8)) if len(pool)]
    samples = np.unique(np.concatenate(picks))
    assert len(samples) >= 36
    prm = O.params_from_scene(sc)
    prm.res, prm.bc_cells = R_LOCAL, 0.0
    rho = prm.materials[0].rho
    for p in samples:
        (wx, wv, wF, wB), near, new, st = window_step(x0, v0, B0, F0, mat, cell, p, prm, sc.dx, HALO)
        tau = O.kirchhoff_stress(st, prm)
        vs = max(np.abs(v0[near]).max(), float(new.v.abs().max())) + prm.dt * float(tau.abs().max()) / (rho * sc.dx)
        bs = max(float(np.abs(B0[near]).max()), float(new.B.abs().max()))
        assert np.abs(x1[p] - wx).max() <= 1e-6 * sc.dx + 2e-7, p
        assert np.abs(v1[p] - wv).max() <= 2e-5 * vs + 1e-7, p
        assert np.abs(F1[p] - wF).max() <= 2e-5 * max(1.0, np.abs(wF).max()), p
        # B = 1/2 sum_k sum_i w v~_i (x_i - x_p)^T weighs the same node
        # velocities as v by offsets of at most 2 dx, so the node-velocity
        # noise the v bound allows reaches B as up to 2 dx times that bound;
        # the column moves slowly, so its B (about 1e-8) is of that order
        assert np.abs(B1[p] - wB).max() <= 5e-5 * bs + 2 * sc.dx * 2e-5 * vs + 1e-9, p
