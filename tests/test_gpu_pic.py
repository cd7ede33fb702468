"""Parity of the CUDA kernel-gradient transfers with the FP64 oracle, through
the C ABI: PIC (Sec. 4.3 with the kernel gradient, the oracle's reading R16)
and APIC with the kernel gradient (Sec. 4.4 momentum and B, the force and
grad v of Sec. 4.3; reading R17).

Tolerances are those of the APIC parity tests: grid mass and momentum after
P2G within 1e-5 of the largest oracle value per field and grid; one-step x
within 1e-6 dx, v within 2e-5 relative; positions of a 40-step dam break
within 1e-3 dx.  F: 99% of the particles within 2e-6 of max|F|, every one
within 1e-5.  The wider bound for the last few follows from the arithmetic:
P2G rounds a block's node sums to a fixed-point unit (absolute, the same for
every node of the block), and a node near the edge of a particle's support
has weight w ~ eps^3 (CK) but gradient |grad w| ~ eps^2 / dx, so when that
node's mass comes mostly from this particle its velocity error (unit / mass)
enters grad v multiplied by |grad w| / w ~ 3 / (eps dx).  The sparse random
states here (about 0.4 particles per cell, random velocities) make such nodes
common; APIC weights the same velocity by w and has no such factor.
The PIC state keeps no B: B and C read back as zeros and an upload of B is
refused.  The kernel-gradient APIC keeps B (within 5e-5 relative after one
step, as for APIC + MLS) and its stress term apart.
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


def _pic_scene(n, res, seed, model, kernel, **kw):
    sc, _, F = random_scene(n, res, seed, model=model, kernel=kernel, **kw)
    sc.transfer = S.TRANSFER_PIC
    return sc, np.zeros_like(F), F


def _sim(ck, sc, F):
    sim = ck.Simulation(sc, ck.kernel_code(sc))
    sim.write(ck.FIELD_F, F)
    return sim


def _grid_check(sc, gm, gp, grids):
    nn = sc.res + 1
    for gi, k in enumerate(O.grid_ids(sc.kernel)):
        mo = grids[k][0].numpy().reshape(nn, nn, nn)
        po = grids[k][1].numpy().reshape(nn, nn, nn, 3)
        assert rel(gm[gi], mo) <= 1e-5, f"grid {k} mass"
        for a in range(3):
            assert np.abs(gp[gi][..., a] - po[..., a]).max() <= 1e-5 * np.abs(po).max(), f"grid {k} momentum {a}"


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("n,res,seed", [(1, 16, 31), (777, 16, 32), (6000, 32, 33)])
def test_pic_p2g_grid_parity(kernel, model, n, res, seed):
    ck = need_gpu()
    sc, B, F = _pic_scene(n, res, seed, model, kernel, f_scale=0.08)
    sim = _sim(ck, sc, F)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    prm = O.params_from_scene(sc)
    assert prm.transfer == O.TRANSFER_PIC
    _grid_check(sc, gm, gp, O.p2g(oracle_state(sc, B, F), prm))


@pytest.mark.parametrize("kernel", KERNELS)
def test_pic_p2g_grid_parity_dense_blocks(kernel):
    """About 512 particles per particle block (the large-block path)."""
    ck = need_gpu()
    sc, B, F = _pic_scene(32768, 32, 34, S.DRUCKER_PRAGER, kernel, f_scale=0.08, box=(8.0, 24.0))
    sim = _sim(ck, sc, F)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    _grid_check(sc, gm, gp, O.p2g(oracle_state(sc, B, F), O.params_from_scene(sc)))


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model,f_scale", [(S.FIXED_COROTATED, 0.08), (S.DRUCKER_PRAGER, 0.08),
                                           (S.DRUCKER_PRAGER, 0.008), (S.J_FLUID, 0.05)])
def test_pic_one_step_particle_parity(kernel, model, f_scale):
    ck = need_gpu()
    E = 1e4 if model == S.J_FLUID else 1e5
    sc, B, F = _pic_scene(5000, 32, 35, model, kernel, f_scale=f_scale, E=E)
    sim = _sim(ck, sc, F)
    sim.step(1)
    sim.sync()
    got = {f: sim.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F, ck.FIELD_B, ck.FIELD_C)}
    sim.close()
    new = O.step(oracle_state(sc, B, F), O.params_from_scene(sc))
    assert np.abs(got[ck.FIELD_X] - new.x.numpy()).max() <= 1e-6 * sc.dx + 2e-7
    assert rel(got[ck.FIELD_V], new.v.numpy()) <= 2e-5
    Fo = new.F.numpy()
    err = np.abs(got[ck.FIELD_F] - Fo).reshape(-1, 9).max(1) / np.abs(Fo).max()
    assert np.quantile(err, 0.99) <= 2e-6 and err.max() <= 1e-5, (np.quantile(err, 0.99), err.max())
    assert float(np.abs(got[ck.FIELD_B]).max()) == 0.0 and float(np.abs(got[ck.FIELD_C]).max()) == 0.0


@pytest.mark.parametrize("kernel", KERNELS)
def test_pic_dam_break_40_steps_positions(kernel):
    """The small dam break of the APIC tests (24,576 fluid particles on 64^3,
    B = 10 Pa, gamma = 7.15, dt 1e-4) under the PIC transfer."""
    ck = need_gpu()
    res, n = 64, 16 * 12 * 16 * 8
    dx = 1.0 / res
    u = S.uniform01(np.arange(3 * n, dtype=np.uint64) + np.uint64(1 << 50), 3).reshape(n, 3)
    x = (4.0 + u * np.array([16.0, 12.0, 16.0])) * dx
    sc = S.Scene("small_dam_break_pic", res, dx, 1e-4, f32(x).astype(np.float64), np.zeros_like(x),
                 np.zeros(n, np.uint8), [S.FLUID], kernel=kernel, transfer=S.TRANSFER_PIC)
    sim = ck.Simulation(sc, ck.kernel_code(sc))
    sim.step(40)
    sim.sync()
    xg = sim.read(ck.FIELD_X)
    sim.close()
    st = O.run(O.state_from_scene(sc), O.params_from_scene(sc), 40)
    assert np.abs(xg - st.x.numpy()).max() <= 1e-3 * dx


def test_pic_refuses_B_upload():
    ck = need_gpu()
    sc, B, F = _pic_scene(100, 16, 36, S.FIXED_COROTATED, S.KERNEL_CK)
    sim = _sim(ck, sc, F)
    with pytest.raises(ck.CKMPMError) as e:
        sim.write(ck.FIELD_B, B + 1.0)
    assert e.value.status == ck.EINVAL
    sim.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_pic_static_p2g_matches_context_path(kernel):
    ck = need_gpu()
    sc, B, F = _pic_scene(7000, 32, 37, S.FIXED_COROTATED, kernel, f_scale=0.08)
    sim = _sim(ck, sc, F)
    sim.probe_grids()
    gm_ref = sim.read(ck.FIELD_GRID_M)
    gp_ref = sim.read(ck.FIELD_GRID_P)
    sim.close()
    dev = torch.device("cuda")
    x = torch.from_numpy(f32(sc.x)).to(dev)
    v = torch.from_numpy(f32(sc.v)).to(dev)
    mat = torch.from_numpy(sc.mat.copy()).to(dev)
    Fd = torch.from_numpy(F.reshape(-1, 9).copy()).to(dev)
    ng = 2 if kernel == S.KERNEL_CK else 1
    nn = sc.res + 1
    gm = torch.empty((ng, nn, nn, nn), dtype=torch.float32, device=dev)
    gp = torch.empty((ng, nn, nn, nn, 3), dtype=torch.float32, device=dev)
    scs, keep = ck.make_scene(sc.res, sc.dx, sc.dt, sc.materials, x, v, mat, gravity=sc.gravity,
                              bc_cells=sc.bc_cells, ppc=sc.ppc)
    stream = torch.cuda.current_stream().cuda_stream
    ck.ckmpm_p2g_grids_static(scs, ck.kernel_code(sc), 0, Fd.data_ptr(), gm.data_ptr(), gp.data_ptr(), stream)
    assert rel(gm.cpu().numpy(), gm_ref) <= 1e-5
    assert rel(gp.cpu().numpy(), gp_ref) <= 1e-5


# ------------------------------------------------- APIC with the kernel gradient

def _grad_scene(n, res, seed, model, kernel, **kw):
    sc, B, F = random_scene(n, res, seed, model=model, kernel=kernel, **kw)
    sc.transfer = S.TRANSFER_APIC_GRAD
    return sc, B, F


def _grad_sim(ck, sc, B, F):
    sim = ck.Simulation(sc, ck.kernel_code(sc))
    sim.write(ck.FIELD_F, F)
    sim.write(ck.FIELD_B, B)
    return sim


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("n,res,seed", [(1, 16, 51), (777, 16, 52), (6000, 32, 53)])
def test_apic_grad_p2g_grid_parity(kernel, model, n, res, seed):
    ck = need_gpu()
    sc, B, F = _grad_scene(n, res, seed, model, kernel, f_scale=0.08)
    sim = _grad_sim(ck, sc, B, F)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    prm = O.params_from_scene(sc)
    assert prm.transfer == O.TRANSFER_APIC_GRAD
    _grid_check(sc, gm, gp, O.p2g(oracle_state(sc, B, F), prm))


@pytest.mark.parametrize("kernel", KERNELS)
def test_apic_grad_p2g_grid_parity_dense_blocks(kernel):
    ck = need_gpu()
    sc, B, F = _grad_scene(32768, 32, 54, S.DRUCKER_PRAGER, kernel, f_scale=0.08, box=(8.0, 24.0))
    sim = _grad_sim(ck, sc, B, F)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    _grid_check(sc, gm, gp, O.p2g(oracle_state(sc, B, F), O.params_from_scene(sc)))


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model,f_scale", [(S.FIXED_COROTATED, 0.08), (S.DRUCKER_PRAGER, 0.08),
                                           (S.DRUCKER_PRAGER, 0.008), (S.J_FLUID, 0.05)])
def test_apic_grad_one_step_particle_parity(kernel, model, f_scale):
    ck = need_gpu()
    E = 1e4 if model == S.J_FLUID else 1e5
    sc, B, F = _grad_scene(5000, 32, 55, model, kernel, f_scale=f_scale, E=E)
    sim = _grad_sim(ck, sc, B, F)
    sim.step(1)
    sim.sync()
    got = {f: sim.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F, ck.FIELD_B, ck.FIELD_C)}
    sim.close()
    prm = O.params_from_scene(sc)
    new = O.step(oracle_state(sc, B, F), prm)
    assert np.abs(got[ck.FIELD_X] - new.x.numpy()).max() <= 1e-6 * sc.dx + 2e-7
    assert rel(got[ck.FIELD_V], new.v.numpy()) <= 2e-5
    Fo = new.F.numpy()
    err = np.abs(got[ck.FIELD_F] - Fo).reshape(-1, 9).max(1) / np.abs(Fo).max()
    assert np.quantile(err, 0.99) <= 2e-6 and err.max() <= 1e-5, (np.quantile(err, 0.99), err.max())
    assert rel(got[ck.FIELD_B], new.B.numpy()) <= 5e-5
    C = new.B @ torch.linalg.inv(O.apic_D(new.x, prm))
    assert rel(got[ck.FIELD_C], C.numpy()) <= 1e-4


@pytest.mark.parametrize("kernel", KERNELS)
def test_apic_grad_dam_break_40_steps_positions(kernel):
    ck = need_gpu()
    res, n = 64, 16 * 12 * 16 * 8
    dx = 1.0 / res
    u = S.uniform01(np.arange(3 * n, dtype=np.uint64) + np.uint64(1 << 50), 3).reshape(n, 3)
    x = (4.0 + u * np.array([16.0, 12.0, 16.0])) * dx
    sc = S.Scene("small_dam_break_apic_grad", res, dx, 1e-4, f32(x).astype(np.float64), np.zeros_like(x),
                 np.zeros(n, np.uint8), [S.FLUID], kernel=kernel, transfer=S.TRANSFER_APIC_GRAD)
    sim = ck.Simulation(sc, ck.kernel_code(sc))
    sim.step(40)
    sim.sync()
    xg = sim.read(ck.FIELD_X)
    sim.close()
    st = O.run(O.state_from_scene(sc), O.params_from_scene(sc), 40)
    assert np.abs(xg - st.x.numpy()).max() <= 1e-3 * dx


def test_apic_grad_B_roundtrip_and_static_entry_refuses():
    ck = need_gpu()
    sc, B, F = _grad_scene(500, 16, 56, S.FIXED_COROTATED, S.KERNEL_CK, f_scale=0.08)
    sim = _grad_sim(ck, sc, B, F)
    assert rel(sim.read(ck.FIELD_B), B) <= 1e-6  # B = M / m, no stress round trip
    assert rel(sim.read(ck.FIELD_F), F) == 0.0
    sim.close()
    scs, keep = ck.make_scene(sc.res, sc.dx, sc.dt, sc.materials, torch.from_numpy(f32(sc.x)).cuda(),
                              torch.from_numpy(f32(sc.v)).cuda(), torch.from_numpy(sc.mat.copy()).cuda())
    nn = sc.res + 1
    gm = torch.zeros((2, nn, nn, nn), dtype=torch.float32, device="cuda")
    gp = torch.zeros((2, nn, nn, nn, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ck.CKMPMError) as e:
        ck.ckmpm_p2g_grids_static(scs, ck.kernel_code(sc), 0, 0, gm.data_ptr(), gp.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert e.value.status == ck.EINVAL


@pytest.mark.parametrize("transfer", [S.TRANSFER_PIC, S.TRANSFER_APIC_GRAD])
@pytest.mark.parametrize("model", MODELS)
def test_kernel_gradient_transfers_float64_pass_two_steps(transfer, model):
    """Every other particle has a nearly singular F (J ~ 1e-3), so the default
    criteria send it to the float64 pass, which under PIC stores -dt V0 tau in
    the state's M slot and under the kernel-gradient APIC in the separate
    stress arrays; the next step's P2G reads them.  Two steps against the
    oracle: v within 2e-4 relative (the two-step float64-pass test of the
    APIC + MLS transfer), F within the 1e-5 this module states for the
    kernel-gradient transfers (a node at the edge of a particle's support
    carries its velocity error into grad v with the factor |grad w| / w)."""
    ck = need_gpu()
    sc, B, F = random_scene(3000, 16, 47, model=model, f_scale=0.02)
    sc.transfer = transfer
    F = F.astype(np.float64)
    F[::2, :, 2] *= 1e-3
    F = f32(F)
    sim = ck.Simulation(sc, ck.kernel_code(sc))
    sim.write(ck.FIELD_F, F)
    if transfer == S.TRANSFER_APIC_GRAD:
        sim.write(ck.FIELD_B, B)
    else:
        B = np.zeros_like(B)
    sim.step(1)
    sim.sync()
    n64 = int(sim.stats().fp64_particles)
    sim.step(1)
    sim.sync()
    Fg = sim.read(ck.FIELD_F)
    vg = sim.read(ck.FIELD_V)
    sim.close()
    assert n64 >= sc.n // 2 - 5
    st2 = O.run(oracle_state(sc, B, F), O.params_from_scene(sc), 2)
    assert rel(Fg, st2.F.numpy()) <= 1e-5
    assert rel(vg, st2.v.numpy()) <= 2e-4
