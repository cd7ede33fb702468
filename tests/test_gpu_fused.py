"""Parity of the fused G2P2G step (CKMPM_STEP_G2P2G) with the FP64 oracle.

The fused kernel gathers step n and scatters the particles that stay in
their block into the grid of step n + 1; particles that change block (or take
the float64 pass) are scattered by the leftover P2G.  The grid a fused step
leaves behind is read back (mass and velocity) and compared with the oracle's
P2G + grid update of the state it was built from, and whole trajectories are
compared with the oracle under the same tolerances as the split step.
Velocities of ~60 m/s move particles about 0.2 cells per step, so that many
cross block boundaries and the leftover path is exercised.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import f32, need_gpu, oracle_state, random_scene, rel
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu

KERNELS = [S.KERNEL_CK, S.KERNEL_QUADRATIC]


def _fused(ck, sc, B=None, F=None, **kw):
    sim = ck.Simulation(sc, sc.kernel | ck.STEP_G2P2G, **kw)
    if F is not None:
        sim.write(ck.FIELD_F, F)
    if B is not None:
        sim.write(ck.FIELD_B, B)
    return sim


def _grid_check(gm, gv, st, prm, tol_m=1e-5, tol_v=2e-5):
    grids = O.p2g(st, prm)
    vg = O.grid_update(grids, prm)
    nn = prm.res + 1
    for gi, k in enumerate(O.grid_ids(prm.kernel)):
        mo = grids[k][0].numpy().reshape(nn, nn, nn)
        po = grids[k][1].numpy().reshape(nn, nn, nn, 3)
        vo = vg[k].numpy().reshape(nn, nn, nn, 3)
        assert rel(gm[gi], mo) <= tol_m, f"grid {k} mass"
        err = np.abs(mo[..., None] * (gv[gi] - vo)).max()
        assert err <= tol_v * max(np.abs(po).max(), 1e-30) + 1e-12, f"grid {k} velocity"
        assert np.all(gv[gi][mo == 0] == 0)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model", [S.FIXED_COROTATED, S.DRUCKER_PRAGER])
def test_grid_left_by_fused_steps_matches_oracle(kernel, model):
    ck = need_gpu()
    sc, B, F = random_scene(6000, 32, 41, model=model, kernel=kernel, f_scale=0.05, v_scale=60.0)
    sim = _fused(ck, sc, B, F)
    prm = O.params_from_scene(sc)
    st = oracle_state(sc, B, F)
    leftovers = []
    for _ in range(2):  # the first step starts with the prologue, the second is fused throughout
        sim.step(1)
        sim.sync()
        st = O.step(st, prm)
        leftovers.append(int(sim.stats().leftover_particles))
        gm = sim.read(ck.FIELD_GRID_M)
        gv = sim.read(ck.FIELD_GRID_V)
        # the oracle state carries float64 rounding of two steps; the grid is
        # compared against the GPU's own particle state one step on
        stg = O.make_state(torch.from_numpy(sim.read(ck.FIELD_X).astype(np.float64)),
                           torch.from_numpy(sim.read(ck.FIELD_V).astype(np.float64)),
                           torch.from_numpy(sim.read(ck.FIELD_B).astype(np.float64)),
                           torch.from_numpy(sim.read(ck.FIELD_F).astype(np.float64)),
                           mat=torch.from_numpy(sc.mat.astype(np.int64)))
        _grid_check(gm, gv, stg, prm, tol_m=2e-5, tol_v=1e-4)
    sim.close()
    assert min(leftovers) > 0, "no particle changed block: the leftover P2G was not exercised"
    with pytest.raises(ck.CKMPMError):
        sim2 = _fused(ck, sc, B, F)
        sim2.step(1)
        try:
            sim2.read(ck.FIELD_GRID_P)
        finally:
            sim2.close()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model", [S.FIXED_COROTATED, S.DRUCKER_PRAGER])
def test_fused_steps_match_oracle(kernel, model):
    ck = need_gpu()
    sc, B, F = random_scene(5000, 32, 42, model=model, kernel=kernel, f_scale=0.05, v_scale=60.0)
    sim = _fused(ck, sc, B, F)
    sim.step(3)
    sim.sync()
    got = {f: sim.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_B, ck.FIELD_F)}
    sim.close()
    new = O.run(oracle_state(sc, B, F), O.params_from_scene(sc), 3)
    assert np.abs(got[ck.FIELD_X] - new.x.numpy()).max() <= 1e-5 * sc.dx
    assert rel(got[ck.FIELD_V], new.v.numpy()) <= 1e-4
    assert rel(got[ck.FIELD_F], new.F.numpy()) <= 1e-5
    assert rel(got[ck.FIELD_B], new.B.numpy()) <= 2e-4


def test_fused_elastic_cube_100_steps_positions():
    """Configuration 1 with the fused step: positions within 1e-3 dx of the
    FP64 oracle after 100 steps."""
    ck = need_gpu()
    sc = S.elastic_cube()
    sim = ck.Simulation(sc, ck.KERNEL_CK | ck.STEP_G2P2G)
    sim.step(100)
    sim.sync()
    x = sim.read(ck.FIELD_X)
    F = sim.read(ck.FIELD_F)
    sim.close()
    st = O.run(O.state_from_scene(sc), O.params_from_scene(sc), 100)
    assert np.abs(x - st.x.numpy()).max() <= 1e-3 * sc.dx
    assert rel(F, st.F.numpy()) <= 1e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_fused_granular_column_steps(kernel):
    """Configuration 2 geometry (346,112 Drucker-Prager particles, 128^3), 10
    fused steps; the velocity bound is the float32 stress noise of the split
    step's test."""
    ck = need_gpu()
    sc = S.granular_column()
    sc.kernel = kernel
    sim = ck.Simulation(sc, kernel | ck.STEP_G2P2G)
    sim.step(10)
    sim.sync()
    x = sim.read(ck.FIELD_X)
    v = sim.read(ck.FIELD_V)
    sim.close()
    st = O.run(O.state_from_scene(sc), O.params_from_scene(sc), 10)
    assert np.abs(x - st.x.numpy()).max() <= 1e-4 * sc.dx
    mat = sc.materials[0]
    mu = mat.E / (2 * (1 + mat.nu))
    lam = mat.E * mat.nu / ((1 + mat.nu) * (1 - 2 * mat.nu))
    assert np.abs(v - st.v.numpy()).max() <= 10 * sc.dt * (2 * mu + 3 * lam) * 4.8e-7 / (mat.rho * sc.dx)


@pytest.mark.parametrize("model", [S.FIXED_COROTATED, S.DRUCKER_PRAGER])
def test_fused_float64_pass_two_steps(model):
    """Every other particle has a nearly singular F, so it takes the float64
    pass: the fused kernel leaves it to the leftover P2G, which scatters it
    after the pass has written its stress."""
    ck = need_gpu()
    sc, B, F = random_scene(3000, 16, 43, model=model, f_scale=0.02)
    F = F.astype(np.float64)
    F[::2, :, 2] *= 1e-3
    F = f32(F)
    sim = _fused(ck, sc, B, F)
    sim.step(1)
    sim.sync()
    st1 = sim.stats()
    sim.step(1)
    sim.sync()
    Fg = sim.read(ck.FIELD_F)
    vg = sim.read(ck.FIELD_V)
    sim.close()
    assert st1.fp64_particles >= sc.n // 2 - 5
    assert st1.leftover_particles >= st1.fp64_particles
    st2 = O.run(oracle_state(sc, B, F), O.params_from_scene(sc), 2)
    assert rel(Fg, st2.F.numpy()) <= 5e-6
    assert rel(vg, st2.v.numpy()) <= 2e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_fused_steps_around_probe_and_upload(kernel):
    """A probe (split P2G into the grid arrays) and an upload between fused
    steps make the next step rebuild the current grid first; the trajectory
    stays the oracle's."""
    ck = need_gpu()
    sc, B, F = random_scene(4000, 32, 44, kernel=kernel, f_scale=0.05, v_scale=30.0)
    sim = _fused(ck, sc, B, F)
    sim.step(2)
    sim.probe_grids()
    v2 = sim.read(ck.FIELD_V)
    sim.write(ck.FIELD_V, v2)
    sim.step(2)
    sim.sync()
    x = sim.read(ck.FIELD_X)
    v = sim.read(ck.FIELD_V)
    sim.close()
    new = O.run(oracle_state(sc, B, F), O.params_from_scene(sc), 4)
    assert np.abs(x - new.x.numpy()).max() <= 1e-5 * sc.dx
    assert rel(v, new.v.numpy()) <= 2e-4


def test_fused_server_admit_and_release():
    """Two scenes of different size and material in one fused context; the
    smaller is released after two steps and the other keeps stepping; each
    result matches the scene stepped alone by the split step."""
    ck = need_gpu()
    from paper_2412_10399_gb300 import serving as SV
    a, Ba, Fa = random_scene(3000, 32, 45, model=S.FIXED_COROTATED, f_scale=0.05, v_scale=20.0)
    b, Bb, Fb = random_scene(1500, 16, 46, model=S.DRUCKER_PRAGER, f_scale=0.05, v_scale=20.0)
    cfg = ck.ckmpm_config()
    cfg.kernel = ck.KERNEL_CK | ck.STEP_G2P2G
    cfg.max_particles = a.n + b.n
    cfg.max_keys = 8 ** 3 + 4 ** 3
    cfg.max_virtual_blocks = 9 ** 3 + 5 ** 3
    cfg.max_grid_blocks = 9 ** 3 + 5 ** 3
    cfg.max_scenes = 2
    cfg.max_materials = 2
    cfg.stream = torch.cuda.current_stream().cuda_stream
    srv = ck.ckmpm_create_server(cfg)
    sa, ka = ck.scene_struct(a)
    sb, kb = ck.scene_struct(b)
    ia = ck.ckmpm_admit(srv, sa)
    ib = ck.ckmpm_admit(srv, sb)

    def put(sid, sc, B, F):
        for fld, arr in ((ck.FIELD_F, F), (ck.FIELD_B, B)):
            x = np.ascontiguousarray(arr, np.float32)
            ck.ckmpm_upload(srv, sid, fld, x.ctypes.data, x.nbytes, False)

    def get(sid, n, fld):
        out = np.empty((n, 3), np.float32)
        ck.ckmpm_readback(srv, sid, fld, out.ctypes.data, out.nbytes, False)
        return out

    put(ia, a, Ba, Fa)
    put(ib, b, Bb, Fb)
    ck.ckmpm_step(srv, 2)
    xb = get(ib, b.n, ck.FIELD_X)
    ck.ckmpm_release(srv, ib)
    ck.ckmpm_step(srv, 2)
    xa = get(ia, a.n, ck.FIELD_X)
    ck.ckmpm_destroy(srv)
    for sc, B, F, steps, got in ((a, Ba, Fa, 4, xa), (b, Bb, Fb, 2, xb)):
        alone = ck.Simulation(sc, sc.kernel)
        alone.write(ck.FIELD_F, F)
        alone.write(ck.FIELD_B, B)
        alone.step(steps)
        want = alone.read(ck.FIELD_X)
        alone.close()
        assert np.abs(got - want).max() <= 1e-6 * sc.dx + 2e-7
