"""Parity of the CUDA CK-MPM step (through the C ABI) with the FP64 oracle.

Tolerances (from the float32 arithmetic of the CUDA path):
  * grid mass and momentum after P2G: max|gpu - oracle| / max|oracle| <= 1e-5,
    per field and per grid;
  * particle positions after 100 steps of the elastic cube: <= 1e-3 dx;
  * one-step particle fields: float32 round-off bounds derived from the
    magnitudes (about 1e-6 relative for v and F, 2e-5 for B).
Both sides start from the same float32-rounded input state.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import f32, need_gpu, oracle_state, random_scene, rel
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu

KERNELS = [S.KERNEL_CK, S.KERNEL_QUADRATIC]
MODELS = [S.FIXED_COROTATED, S.DRUCKER_PRAGER]


def _sim(ck, sc, B=None, F=None, **kw):
    sim = ck.Simulation(sc, sc.kernel, **kw)
    if F is not None:
        sim.write(ck.FIELD_F, F)
    if B is not None:
        sim.write(ck.FIELD_B, B)
    return sim


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("n,res,seed", [(1, 16, 1), (777, 16, 2), (6000, 32, 3)])
def test_p2g_grid_parity(kernel, model, n, res, seed):
    ck = need_gpu()
    sc, B, F = random_scene(n, res, seed, model=model, kernel=kernel, f_scale=0.08)
    sim = _sim(ck, sc, B, F)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    gv = sim.read(ck.FIELD_GRID_V)
    sim.close()
    prm = O.params_from_scene(sc)
    st = oracle_state(sc, B, F)
    grids = O.p2g(st, prm)
    vg = O.grid_update(grids, prm)
    nn = res + 1
    for gi, k in enumerate(O.grid_ids(kernel)):
        mo = grids[k][0].numpy().reshape(nn, nn, nn)
        po = grids[k][1].numpy().reshape(nn, nn, nn, 3)
        vo = vg[k].numpy().reshape(nn, nn, nn, 3)
        assert rel(gm[gi], mo) <= 1e-5, f"grid {k} mass"
        for a in range(3):
            assert rel(gp[gi][..., a], po[..., a]) <= 1e-5 or np.abs(gp[gi][..., a] - po[..., a]).max() <= 1e-5 * np.abs(po).max(), f"grid {k} momentum {a}"
        # velocity on nodes with mass, weighted by mass (momentum units)
        err = np.abs(mo[..., None] * (gv[gi] - vo)).max()
        assert err <= 2e-5 * max(np.abs(po).max(), 1e-30) + 1e-12, f"grid {k} velocity"
        assert np.all(gv[gi][mo == 0] == 0)


@pytest.mark.parametrize("kernel", KERNELS)
def test_p2g_grid_parity_dense_blocks(kernel):
    """8 particles per cell over cells [8, 24)^3: 64 particle blocks hold about
    512 particles each, so P2G takes its large-block fixed-point path."""
    ck = need_gpu()
    sc, B, F = random_scene(32768, 32, 4, model=S.DRUCKER_PRAGER, kernel=kernel, f_scale=0.08, box=(8.0, 24.0))
    sim = _sim(ck, sc, B, F)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    st = sim.stats()
    sim.close()
    assert st.n_particle_blocks >= 64
    prm = O.params_from_scene(sc)
    grids = O.p2g(oracle_state(sc, B, F), prm)
    nn = sc.res + 1
    for gi, k in enumerate(O.grid_ids(kernel)):
        mo = grids[k][0].numpy().reshape(nn, nn, nn)
        po = grids[k][1].numpy().reshape(nn, nn, nn, 3)
        assert rel(gm[gi], mo) <= 1e-5, f"grid {k} mass"
        assert rel(gp[gi], po) <= 1e-5, f"grid {k} momentum"


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model,f_scale", [(S.FIXED_COROTATED, 0.08), (S.DRUCKER_PRAGER, 0.08),
                                           (S.DRUCKER_PRAGER, 0.008), (S.DRUCKER_PRAGER, 0.002),
                                           (S.DRUCKER_PRAGER, 1e-4)])
def test_one_step_particle_parity(kernel, model, f_scale):
    """f_scale 0.008 keeps F F^T within 1/32 of I for nearly every particle, so
    Drucker-Prager takes the small-stretch matrix-series update (elastic,
    plastic and tip cases all occur) through the fourth power; 0.002 and 1e-4
    bring most warps to the third and second powers the series takes at
    smaller strains; 0.08 takes the eigen-decomposition."""
    ck = need_gpu()
    sc, B, F = random_scene(5000, 32, 7, model=model, kernel=kernel, f_scale=f_scale)
    sim = _sim(ck, sc, B, F)
    sim.step(1)
    sim.sync()
    got = {f: sim.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_B, ck.FIELD_F, ck.FIELD_C)}
    sim.close()
    prm = O.params_from_scene(sc)
    new = O.step(oracle_state(sc, B, F), prm)
    dx = sc.dx
    assert np.abs(got[ck.FIELD_X] - new.x.numpy()).max() <= 1e-6 * dx + 2e-7
    assert rel(got[ck.FIELD_V], new.v.numpy()) <= 2e-5
    assert rel(got[ck.FIELD_F], new.F.numpy()) <= 2e-6
    assert rel(got[ck.FIELD_B], new.B.numpy()) <= 5e-5
    C = new.B @ torch.linalg.inv(O.apic_D(new.x, prm))
    assert rel(got[ck.FIELD_C], C.numpy()) <= 1e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_fluid_one_step_particle_parity(kernel):
    """J-based fluid (B = 1e4 Pa so the pressure force is felt; F within 5% of
    I, so J covers compression and expansion): one step against the oracle,
    including the projection of F onto J^(1/3) I."""
    ck = need_gpu()
    sc, B, F = random_scene(5000, 32, 21, model=S.J_FLUID, kernel=kernel, E=1e4, f_scale=0.05)
    sim = _sim(ck, sc, B, F)
    sim.step(1)
    sim.sync()
    got = {f: sim.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_B, ck.FIELD_F)}
    sim.close()
    new = O.step(oracle_state(sc, B, F), O.params_from_scene(sc))
    assert np.abs(got[ck.FIELD_X] - new.x.numpy()).max() <= 1e-6 * sc.dx + 2e-7
    assert rel(got[ck.FIELD_V], new.v.numpy()) <= 2e-5
    assert rel(got[ck.FIELD_F], new.F.numpy()) <= 2e-6
    assert rel(got[ck.FIELD_B], new.B.numpy()) <= 5e-5
    off = got[ck.FIELD_F] - np.einsum("nii->ni", got[ck.FIELD_F])[:, :, None] * np.eye(3)[None]
    assert np.abs(off).max() == 0.0


@pytest.mark.parametrize("kernel", KERNELS)
def test_fluid_dam_break_40_steps_positions(kernel):
    """A small dam break (24,576 fluid particles uniform in a 16 x 12 x 16-cell
    cuboid on 64^3, the paper's B = 10 Pa and gamma = 7.15, dt 1e-4): positions
    within 1e-3 dx of the oracle after 40 steps from the same initial state."""
    ck = need_gpu()
    res, n = 64, 16 * 12 * 16 * 8
    dx = 1.0 / res
    u = S.uniform01(np.arange(3 * n, dtype=np.uint64) + np.uint64(1 << 50), 3).reshape(n, 3)
    x = (4.0 + u * np.array([16.0, 12.0, 16.0])) * dx
    sc = S.Scene("small_dam_break", res, dx, 1e-4, f32(x).astype(np.float64), np.zeros_like(x), np.zeros(n, np.uint8),
                 [S.FLUID], kernel=kernel)
    sim = ck.Simulation(sc, kernel)
    sim.step(40)
    sim.sync()
    xg = sim.read(ck.FIELD_X)
    sim.close()
    st = O.run(O.state_from_scene(sc), O.params_from_scene(sc), 40)
    assert np.abs(xg - st.x.numpy()).max() <= 1e-3 * dx


def test_elastic_cube_100_steps_positions():
    """Configuration 1 (32,768 particles, 64^3, dt 1e-4): positions within
    1e-3 dx of the FP64 oracle after 100 steps from the same initial state."""
    ck = need_gpu()
    sc = S.elastic_cube()
    sim = ck.Simulation(sc, ck.KERNEL_CK)
    sim.step(100)
    sim.sync()
    x = sim.read(ck.FIELD_X)
    F = sim.read(ck.FIELD_F)
    sim.close()
    prm = O.params_from_scene(sc)
    st = O.run(O.state_from_scene(sc), prm, 100)
    assert np.abs(x - st.x.numpy()).max() <= 1e-3 * sc.dx
    assert rel(F, st.F.numpy()) <= 1e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_granular_column_steps(kernel):
    """Configuration 2 geometry (346,112 Drucker-Prager particles, 128^3), 10 steps."""
    ck = need_gpu()
    sc = S.granular_column()
    sc.kernel = kernel
    sim = ck.Simulation(sc, kernel)
    sim.step(10)
    sim.sync()
    x = sim.read(ck.FIELD_X)
    v = sim.read(ck.FIELD_V)
    sim.close()
    prm = O.params_from_scene(sc)
    st = O.run(O.state_from_scene(sc), prm, 10)
    assert np.abs(x - st.x.numpy()).max() <= 1e-4 * sc.dx
    # float32 singular values of F ~ I carry a few ulp (4 ulp of 1.0 = 4.8e-7) of
    # noise, so the Hencky stress carries (2 mu + 3 lam) * 4.8e-7 ~ 0.4 Pa of
    # noise; at a free surface that accelerates particles by ~tau / (rho dx) and
    # over n steps moves v by n dt tau / (rho dx) ~ 3e-5 m/s here (the oracle,
    # in float64, has exact zeros for the lateral velocity of the falling column).
    mat = sc.materials[0]
    mu = mat.E / (2 * (1 + mat.nu))
    lam = mat.E * mat.nu / ((1 + mat.nu) * (1 - 2 * mat.nu))
    bound = 10 * sc.dt * (2 * mu + 3 * lam) * 4.8e-7 / (mat.rho * sc.dx)
    assert np.abs(v - st.v.numpy()).max() <= bound


@pytest.mark.parametrize("kernel", KERNELS)
def test_free_fall_single_particle(kernel):
    ck = need_gpu()
    x0 = np.array([[0.43, 0.61, 0.52]], np.float32)
    v0 = np.array([[0.2, 0.1, -0.3]], np.float32)
    sc = S.Scene("one", 32, 1 / 32, 1e-3, x0.astype(np.float64), v0.astype(np.float64), np.zeros(1, np.uint8),
                 [S.ELASTIC], kernel=kernel)
    sim = ck.Simulation(sc, kernel)
    n = 25
    sim.step(n)
    sim.sync()
    x = sim.read(ck.FIELD_X)[0].astype(np.float64)
    v = sim.read(ck.FIELD_V)[0].astype(np.float64)
    F = sim.read(ck.FIELD_F)[0]
    sim.close()
    g = np.array([0, -9.8, 0])
    assert np.abs(v - (v0[0] + n * 1e-3 * g)).max() < 2e-6
    assert np.abs(x - (x0[0] + n * 1e-3 * v0[0] + 1e-6 * g * n * (n + 1) / 2)).max() < 2e-6
    assert np.abs(F - np.eye(3)).max() < 1e-5


def test_fp64_svd_path_is_taken_and_matches():
    """Precision extension: forcing the float64 SVD (gap criterion 1.0) on
    degenerate F (J ~ 1e-3) keeps F and stress parity with the oracle."""
    ck = need_gpu()
    sc, B, F = random_scene(2000, 16, 9, f_scale=0.02)
    # squash F towards rank deficiency: F = R diag(1, 1, 1e-3)
    F = F.astype(np.float64)
    F[:, :, 2] *= 1e-3
    F = f32(F)
    sim = ck.Simulation(sc, sc.kernel, fp64_gap_tol=1.0)
    sim.write(ck.FIELD_F, F)
    sim.write(ck.FIELD_B, B)
    sim.step(1)
    sim.sync()
    st_gpu = sim.stats()
    Fg = sim.read(ck.FIELD_F)
    vg = sim.read(ck.FIELD_V)
    sim.close()
    assert st_gpu.fp64_particles == sc.n
    new = O.step(oracle_state(sc, B, F), O.params_from_scene(sc))
    assert rel(Fg, new.F.numpy()) <= 2e-6
    assert rel(vg, new.v.numpy()) <= 1e-4


@pytest.mark.parametrize("model", MODELS)
def test_fp64_pass_mixed_blocks_two_steps(model):
    """Every other particle has a nearly singular F (J ~ 1e-3 < j_tol), so the
    default criteria send it to the float64 pass while its neighbours in the
    same blocks stay in float32.  The pass rewrites M after G2P recorded the
    block bounds, so the next P2G (checked on the grids) relies on the pass
    raising them; two steps are then compared with the oracle."""
    ck = need_gpu()
    sc, B, F = random_scene(3000, 16, 13, model=model, f_scale=0.02)
    F = F.astype(np.float64)
    F[::2, :, 2] *= 1e-3
    F = f32(F)
    sim = _sim(ck, sc, B, F)
    sim.step(1)
    sim.sync()
    n64 = int(sim.stats().fp64_particles)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.step(1)
    sim.sync()
    Fg = sim.read(ck.FIELD_F)
    vg = sim.read(ck.FIELD_V)
    sim.close()
    assert n64 >= sc.n // 2 - 5 and n64 <= sc.n // 2 + 5
    prm = O.params_from_scene(sc)
    st1 = O.step(oracle_state(sc, B, F), prm)
    grids = O.p2g(st1, prm)
    nn = sc.res + 1
    for gi, k in enumerate(O.grid_ids(sc.kernel)):
        assert rel(gm[gi], grids[k][0].numpy().reshape(nn, nn, nn)) <= 1e-5
        assert rel(gp[gi], grids[k][1].numpy().reshape(nn, nn, nn, 3)) <= 1e-5
    st2 = O.step(st1, prm)
    assert rel(Fg, st2.F.numpy()) <= 5e-6
    assert rel(vg, st2.v.numpy()) <= 2e-4


@pytest.mark.parametrize("c,path", [(0.995, "series"), (0.9995, "series"), (1.002, "series"),
                                    (0.99999, "series"), (1.0001, "series"),
                                    (0.9, "eigen"), (0.97, "eigen"), (1.05, "eigen"),
                                    (0.9, "fp64"), (1.05, "fp64")])
def test_drucker_prager_isotropic_states_each_path(c, path):
    """Exactly isotropic F = c I through each float path of the sand update:
    the small-stretch matrix series (|c^2 - 1| <= 1/48), the eigen-
    decomposition of F F^T, and the float64 pass (forced by the gap
    criterion).  Every node is a sticky wall and gravity is off, so the grid
    velocities vanish, grad v = 0 and F reaches the return map unchanged:
    compression (c < 1) lies inside the cone and must stay c I, tension
    (c > 1) goes to the tip, F = I (klar2016 return map, as in the oracle)."""
    ck = need_gpu()
    n, res = 2000, 16
    sc, B, _ = random_scene(n, res, 31, model=S.DRUCKER_PRAGER, gravity=(0.0, 0.0, 0.0), bc_cells=float(res))
    F = np.broadcast_to(np.float32(c) * np.eye(3, dtype=np.float32), (n, 3, 3)).copy()
    kw = {"fp64_gap_tol": 1.0} if path == "fp64" else {}
    sim = ck.Simulation(sc, sc.kernel, **kw)
    sim.write(ck.FIELD_F, F)
    sim.step(1)
    sim.sync()
    n64 = int(sim.stats().fp64_particles)
    Fg = sim.read(ck.FIELD_F)
    vg = sim.read(ck.FIELD_V)
    sim.close()
    assert n64 == (n if path == "fp64" else 0)
    assert np.all(vg == 0.0)
    new = O.step(oracle_state(sc, np.zeros_like(B), F), O.params_from_scene(sc))
    want = (np.float64(np.float32(c)) if c < 1.0 else 1.0) * np.eye(3)
    assert np.abs(new.F.numpy() - want).max() <= 1e-15
    assert np.abs(Fg - want).max() <= 2e-7 * c


def test_upload_readback_roundtrip():
    ck = need_gpu()
    sc, B, F = random_scene(3000, 16, 11, f_scale=0.1)
    sim = _sim(ck, sc, B, F)
    assert np.array_equal(sim.read(ck.FIELD_X), f32(sc.x))
    assert np.array_equal(sim.read(ck.FIELD_V), f32(sc.v))
    assert np.array_equal(sim.read(ck.FIELD_F), F)
    assert rel(sim.read(ck.FIELD_B), B) <= 1e-5
    x2 = f32(sc.x + 0.25 * sc.dx)
    sim.write(ck.FIELD_X, x2)
    assert np.array_equal(sim.read(ck.FIELD_X), x2)
    sim.step(1)
    sim.sync()
    sim.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_probe_and_upload_leave_steps_unchanged(kernel):
    """P2G's per-block bounds are recorded when particles are binned and
    cleared once used.  Probing the grids (P2G without G2P) and re-uploading
    the same velocities (which re-bins the pool) must leave the following steps
    unchanged up to rounding: the cross-block flush of P2G adds floats with
    atomics, whose order varies from run to run."""
    ck = need_gpu()
    sc, B, F = random_scene(4000, 32, 12, kernel=kernel, f_scale=0.08)
    fields = (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F)
    ref = _sim(ck, sc, B, F)
    ref.step(1)
    want1 = [ref.read(f) for f in fields]
    ref.step(2)
    want3 = [ref.read(f) for f in fields]
    ref.close()
    sim = _sim(ck, sc, B, F)
    sim.probe_grids()
    sim.probe_grids()
    sim.step(1)
    got1 = [sim.read(f) for f in fields]
    _close(got1, want1, sc.dx)
    sim.write(ck.FIELD_V, got1[1])
    sim.probe_grids()
    sim.step(2)
    got3 = [sim.read(f) for f in fields]
    sim.close()
    _close(got3, want3, sc.dx)


def _close(got, want, dx):
    assert np.abs(got[0] - want[0]).max() <= 1e-6 * dx + 2e-7  # a few ulps of x in [0, 1)
    assert rel(got[1], want[1]) <= 1e-5
    assert rel(got[2], want[2]) <= 1e-6


def test_particle_leaving_domain_reports_edomain():
    ck = need_gpu()
    x0 = np.array([[0.52 / 16, 0.5, 0.5]], np.float32)
    v0 = np.array([[-100.0, 0.0, 0.0]], np.float32)
    sc = S.Scene("out", 16, 1 / 16, 1e-3, x0.astype(np.float64), v0.astype(np.float64), np.zeros(1, np.uint8),
                 [S.ELASTIC], bc_cells=0.0, gravity=(0.0, 0.0, 0.0))
    sim = ck.Simulation(sc, ck.KERNEL_CK)
    sim.step(1)
    with pytest.raises(ck.CKMPMError) as ei:
        sim.sync()
    assert ei.value.status == ck.EDOMAIN
    sim.close()


def test_empty_scene_is_rejected():
    ck = need_gpu()
    x = np.zeros((0, 3), np.float32)
    sc, keep = ck.make_scene(16, 1 / 16, 1e-4, [S.ELASTIC], x)
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_create(sc, 0, 0)
    assert ei.value.status == ck.EINVAL


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("fused", [False, True])
def test_nonfinite_state_reports_enonfinite(bad, fused):
    """One particle's F carries a NaN or an infinity: the step's finite check
    (one multiply-add by zero per value, NaN for any non-finite input) flags
    it and the next sync reports ENONFINITE; every loop of the
    decompositions is bounded, so the step itself completes."""
    ck = need_gpu()
    sc, B, F = random_scene(500, 16, 51, f_scale=0.05)
    F = F.copy()
    F[7, 1, 2] = bad
    sim = ck.Simulation(sc, sc.kernel | (ck.STEP_G2P2G if fused else 0))
    sim.write(ck.FIELD_F, F)
    sim.step(1)
    with pytest.raises(ck.CKMPMError) as ei:
        sim.sync()
    assert ei.value.status == ck.ENONFINITE
    sim.close()


def _rotation(g):
    q = g.normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("model,s1,s3", [(S.FIXED_COROTATED, 1.1, 0.9), (S.DRUCKER_PRAGER, 1.05, 0.85)])
def test_float32_error_on_clustered_singular_values(model, s1, s3):
    """Precision extension without the gap criterion: F = U diag(s1, s1 (1 +
    delta), s3) V^T with delta from 1e-7 to 1e-3 and random rotations, away
    from F = I, goes through the float32 eigen path (its pair of singular
    values is clustered, its eigenvectors ill-determined).  Every node is a
    wall, so F reaches the constitutive update unchanged; the projected F
    (Drucker-Prager) and the stress, through the next P2G's momentum (v = 0,
    B = 0), are compared with the float64 oracle.  The sand's strains
    (ln 1.05, ln 1.05, ln 0.85) lie outside the cone, so its F is projected.
    The measured errors are printed; the bounds are the float32 bounds of
    the one-step tests."""
    ck = need_gpu()
    n, res = 2000, 16
    sc, B, _ = random_scene(n, res, 71, model=model, gravity=(0.0, 0.0, 0.0), bc_cells=float(res), v_scale=0.0)
    g = np.random.default_rng(72)
    deltas = np.array([1e-7, 1e-6, 1e-5, 1e-4, 1e-3])
    F = np.empty((n, 3, 3))
    for p in range(n):
        d = deltas[p % len(deltas)]
        F[p] = _rotation(g) @ np.diag([s1, s1 * (1 + d), s3]) @ _rotation(g).T
    F = f32(F)
    sim = ck.Simulation(sc, sc.kernel)
    sim.write(ck.FIELD_F, F)
    sim.step(1)
    sim.sync()
    n64 = int(sim.stats().fp64_particles)
    Fg = sim.read(ck.FIELD_F)
    sim.probe_grids()
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    assert n64 == 0  # the default criteria (J, condition) leave these to float32
    prm = O.params_from_scene(sc)
    st1 = O.step(oracle_state(sc, np.zeros_like(B), F), prm)
    grids = O.p2g(st1, prm)
    nn = res + 1
    errF = rel(Fg, st1.F.numpy())
    errP = max(rel(gp[gi], grids[k][1].numpy().reshape(nn, nn, nn, 3)) for gi, k in enumerate(O.grid_ids(0)))
    per_delta = {float(d): float(np.abs(Fg[i::len(deltas)] - st1.F.numpy()[i::len(deltas)]).max())
                 for i, d in enumerate(deltas)}
    print(f"\nclustered sigma, model {model}: F rel err {errF:.3e}, stress-momentum rel err {errP:.3e}, "
          f"max |dF| by delta {per_delta}")
    assert errF <= 2e-6
    assert errP <= 1e-5
