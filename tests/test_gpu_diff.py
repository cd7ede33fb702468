"""Hand-written adjoint of the CK-MPM step (CUDA) against the FP64 oracle's
autograd gradient and against central finite differences of the CUDA forward.

Tolerances: the float32 adjoint of one step matches the float64 VJP within
2e-3 of each field's largest entry; rollout gradients (16 steps) within 2e-2;
directional derivatives on the full 262,144-particle, 64-step configuration
within 3% of central differences (h = 1e-3 absolute for v, 1e-2 relative for E).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import f32, need_gpu, rel
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu
F64 = torch.float64


def _diff():
    need_gpu()
    from paper_2412_10399_gb300 import diff
    return diff


def _random_fc_state(n, res, seed):
    x, v, B, F = S.random_state(n, res, seed, margin_cells=5.0, f_scale=0.08)
    g = np.random.default_rng(seed)
    E = 1e5 * (0.5 + g.random(n))
    mat = S.Material(S.FIXED_COROTATED, 1e5, 0.3, 1000.0)
    sc = S.Scene("diff_random", res, 1.0 / res, 1e-4, f32(x).astype(np.float64), f32(v).astype(np.float64),
                 np.zeros(n, np.uint8), [mat])
    return sc, f32(B), f32(F), f32(E)


def _cuda(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def test_diff_forward_step_matches_oracle():
    diff = _diff()
    sc, B, F, E = _random_fc_state(4000, 32, 31)
    sim = diff.DiffSim(sc)
    x, v, Bd, Fd, Ed = _cuda(f32(sc.x), f32(sc.v), B, F, E)
    x1, v1, B1, F1 = sim.step(x, v, Bd, Fd, Ed)
    sim.sync()
    prm = O.params_from_scene(sc)
    st = O.make_state(torch.from_numpy(f32(sc.x).astype(np.float64)), torch.from_numpy(f32(sc.v).astype(np.float64)),
                      torch.from_numpy(B.astype(np.float64)), torch.from_numpy(F.astype(np.float64)),
                      E=torch.from_numpy(E.astype(np.float64)))
    new = O.step(st, prm)
    assert np.abs(x1.cpu().numpy() - new.x.numpy()).max() <= 1e-6 * sc.dx + 2e-7
    assert rel(v1.cpu().numpy(), new.v.numpy()) <= 2e-5
    assert rel(B1.cpu().numpy(), new.B.numpy()) <= 5e-5
    assert rel(F1.cpu().numpy(), new.F.numpy()) <= 2e-6
    sim.close()


def test_diff_step_vjp_matches_oracle_autograd():
    diff = _diff()
    sc, B, F, E = _random_fc_state(3000, 32, 32)
    prm = O.params_from_scene(sc)
    g = np.random.default_rng(5)
    n = sc.n
    adj = [g.standard_normal((n, 3)), g.standard_normal((n, 3)), g.standard_normal((n, 3, 3)) * 10.0,
           g.standard_normal((n, 3, 3))]
    # float64 oracle VJP
    t = [torch.from_numpy(a.astype(np.float64)).requires_grad_(True)
         for a in (f32(sc.x), f32(sc.v), B, F, E)]
    st = O.make_state(t[0], t[1], t[2], t[3], E=t[4])
    new = O.step(st, prm, newton=True)
    outs = (new.x, new.v, new.B, new.F)
    ref = torch.autograd.grad(outs, t, [torch.from_numpy(a) for a in adj])
    # CUDA VJP
    sim = diff.DiffSim(sc)
    x, v, Bd, Fd, Ed = _cuda(f32(sc.x), f32(sc.v), B, F, E)
    gx1, gv1, gB1, gF1 = _cuda(*[f32(a) for a in adj])
    gE = torch.zeros_like(Ed)
    got = sim.step_backward(x, v, Bd, Fd, Ed, gx1, gv1, gB1, gF1, gE)
    sim.sync()
    names = ("x", "v", "B", "F")
    for name, a, b in zip(names, got, ref[:4]):
        assert rel(a.cpu().numpy(), b.numpy()) <= 2e-3, name
    assert rel(gE.cpu().numpy(), ref[4].numpy()) <= 2e-3, "E"
    sim.close()


def _cube(seed=0, res=32, lo=12, hi=20):
    sc = S.differentiable_cube(seed=seed, res=res, lo=lo, hi=hi)
    E = np.full(sc.n, sc.materials[0].E, np.float32)
    return sc, E


def _gpu_losses(diff, sim, x0, v0, E, steps, k, target):
    """Centre-of-mass distance and spread of the final positions, evaluated in
    float64 from the float32 rollout (so the loss itself adds no rounding)."""
    xT, vT = diff.Rollout.apply(x0, v0, E, sim, steps, k)
    xT = xT.double()
    com = xT.mean(0)
    L1 = torch.linalg.vector_norm(com - target.double())
    L2 = ((xT - com) ** 2).sum(1).mean()
    return L1, L2


def test_rollout_gradient_matches_oracle_autograd():
    """A 4,096-particle cube, 16 steps, checkpoints every 4: dL/dv0 and dL/dE of
    the centre-of-mass loss and of the spread loss against float64 autograd."""
    diff = _diff()
    sc, E = _cube()
    steps, k = 16, 4
    target = torch.tensor(sc.x.mean(0) + np.array([0.01, -0.005, 0.0]), dtype=F64)
    # oracle
    x0 = torch.from_numpy(f32(sc.x).astype(np.float64))
    v0 = torch.from_numpy(f32(sc.v).astype(np.float64)).requires_grad_(True)
    Et = torch.from_numpy(E.astype(np.float64)).requires_grad_(True)
    st = O.run(O.make_state(x0, v0, E=Et), O.params_from_scene(sc), steps, newton=True)
    com = st.x.mean(0)
    L1o = torch.linalg.vector_norm(com - target)
    L2o = ((st.x - com) ** 2).sum(1).mean()
    g1v, g1E = torch.autograd.grad(L1o, [v0, Et], retain_graph=True)
    g2v, g2E = torch.autograd.grad(L2o, [v0, Et])
    # CUDA adjoint
    sim = diff.DiffSim(sc)
    xg, vg, Eg = _cuda(f32(sc.x), f32(sc.v), E)
    vg.requires_grad_(True)
    Eg.requires_grad_(True)
    tg = target.float().cuda()
    L1, L2 = _gpu_losses(diff, sim, xg, vg, Eg, steps, k, tg)
    a1v, a1E = torch.autograd.grad(L1, [vg, Eg], retain_graph=True)
    L1b, L2b = _gpu_losses(diff, sim, xg, vg, Eg, steps, k, tg)
    a2v, a2E = torch.autograd.grad(L2b, [vg, Eg])
    sim.close()
    assert abs(float(L1) - float(L1o)) <= 1e-4 * float(L1o)
    assert rel(a1v.cpu().numpy(), g1v.numpy()) <= 2e-2
    assert rel(a2v.cpu().numpy(), g2v.numpy()) <= 2e-2
    assert rel(a2E.cpu().numpy(), g2E.numpy()) <= 2e-2
    # the centre of mass moves independently of stiffness (exact momentum bookkeeping)
    assert float(a1E.abs().max()) <= 1e-3 * float(a2E.abs().max())


def test_rollout_directional_derivatives_full_configuration():
    """Differentiable configuration: 262,144 particles on 128^3, 64 steps,
    checkpoints every 8; adjoint directional derivatives against central
    differences of the CUDA forward (h = 1e-3)."""
    diff = _diff()
    sc = S.differentiable_cube()
    E = np.full(sc.n, sc.materials[0].E, np.float32)
    steps, k = 64, 8
    target = torch.tensor(sc.x.mean(0) + np.array([0.01, -0.005, 0.0]), dtype=torch.float32).cuda()
    sim = diff.DiffSim(sc)
    x0, v0, Eg = _cuda(f32(sc.x), f32(sc.v), E)
    g = np.random.default_rng(11)
    # directions: a near-uniform velocity shift moves the centre of mass; an
    # expansion field (plus noise) changes the spread; a stiffness scaling
    # (plus noise) changes the spread through the elastic response
    dv = torch.from_numpy((1.0 + 0.5 * g.standard_normal((sc.n, 3))).astype(np.float32)).cuda()
    xc = sc.x - sc.x.mean(0)
    dv2 = torch.from_numpy((20.0 * xc + 0.5 * g.standard_normal((sc.n, 3))).astype(np.float32)).cuda()
    dE = torch.from_numpy((1.0 + 0.5 * g.standard_normal(sc.n)).astype(np.float32)).cuda()
    vr = v0.clone().requires_grad_(True)
    Er = Eg.clone().requires_grad_(True)
    L1, L2 = _gpu_losses(diff, sim, x0, vr, Er, steps, k, target)
    g1v = torch.autograd.grad(L1, [vr])[0]
    L1, L2 = _gpu_losses(diff, sim, x0, vr, Er, steps, k, target)
    g2v, g2E = torch.autograd.grad(L2, [vr, Er])
    h = 1e-3
    with torch.no_grad():
        def losses(v, Ev):
            return _gpu_losses(diff, sim, x0, v, Ev, steps, k, target)
        p1, _ = losses(v0 + h * dv, Eg)
        m1, _ = losses(v0 - h * dv, Eg)
        fd1v = (float(p1) - float(m1)) / (2 * h)
        _, p2 = losses(v0 + h * dv2, Eg)
        _, m2 = losses(v0 - h * dv2, Eg)
        fd2v = (float(p2) - float(m2)) / (2 * h)
        # a 1e-3 relative stiffness change moves L by ~6e-8 of its value, the
        # float32 resolution of the positions; 1e-2 keeps the difference well
        # above it (truncation error ~ h^2)
        hE = 1e-2
        pE = losses(v0, Eg * (1 + hE * dE))[1]
        mE = losses(v0, Eg * (1 - hE * dE))[1]
        fd2E = (float(pE) - float(mE)) / (2 * hE)
    an1v = float((g1v * dv).sum())
    an2v = float((g2v * dv2).sum())
    an2E = float((g2E * Eg * dE).sum())
    sim.close()
    assert abs(an1v - fd1v) <= 3e-2 * abs(fd1v)
    assert abs(an2v - fd2v) <= 3e-2 * abs(fd2v)
    assert abs(an2E - fd2E) <= 3e-2 * abs(fd2E)
