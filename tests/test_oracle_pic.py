"""Pins of the oracle's PIC transfer (reading R16: the scheme of Sec. 4.3 with
the kernel gradient, used by the paper's Taichi comparison).

What fixes it: the kernel derivatives against central differences of the
kernels, the derivative of the partition of unity (sum_i grad w = 0 on each
grid), the gradient's first moment (1/2 sum_k sum_i grad w (x_i - x_p)^T = I
on the dual grid, = I on the single quadratic grid), exact reproduction of an
affine grid velocity (v and grad v), linear momentum conservation of P2G with
stress, and the P2G force equal to minus twice the gradient of the stored
energy of F^ = (I + grad v(x^ - x)) F built by the PIC G2P itself.

The APIC transfer with the kernel gradient (reading R17: Sec. 4.4's momentum
transfer and B, the force and grad v of Sec. 4.3) is pinned by P2G linear and
angular momentum (sum x x m v + sum m eps:B, Supplement Thm 2.1/2.2: the
kernel-gradient force carries no torque because sum_k sum_i (x_i - x_p)
grad w^T = |K| I), by a full step conserving both, and by the affine field
giving B = A D and grad v = A.
"""
import pytest
import torch

from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

F64 = torch.float64
KERNELS = [O.KERNEL_CK, O.KERNEL_QUADRATIC]


def _prm(kernel, res=12, dt=1e-3):
    return O.Params(res=res, dx=1.0 / res, dt=dt, materials=[O.Mat(O.FIXED_COROTATED, 1e5, 0.3, 1000.0)],
                    kernel=kernel, transfer=O.TRANSFER_PIC)


def _state(n, res, seed, **kw):
    x, v, B, F = S.random_state(n, res, seed, **kw)
    return O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.zeros(n, 3, 3, dtype=F64), torch.from_numpy(F))


def test_kernel_derivatives_match_central_differences():
    t = torch.linspace(-1.7, 1.7, 3401, dtype=F64)
    # the B-spline's second derivative jumps at 1/2 and 3/2, where a central
    # difference is off by O(h)
    t = t[((t.abs() - 0.5).abs() > 1e-5) & ((t.abs() - 1.5).abs() > 1e-5)]
    h = 1e-6
    for k, kp in ((O.K1, O.K1_prime), (O.quadratic_bspline, O.quadratic_bspline_prime)):
        fd = (k(t + h) - k(t - h)) / (2 * h)
        assert torch.allclose(kp(t), fd, atol=1e-8, rtol=0)
    # K1 is C^2, so its derivative vanishes at 0 and at the support's ends
    assert float(O.K1_prime(torch.tensor([0.0, 1.0, -1.0], dtype=F64)).abs().max()) == 0.0


@pytest.mark.parametrize("kernel", KERNELS)
def test_gradient_sums_and_first_moment(kernel):
    dx = 1.0 / 16
    x = (4.0 + 8.0 * torch.rand(300, 3, dtype=F64, generator=torch.Generator().manual_seed(1))) * dx
    tot = torch.zeros(300, 3, 3, dtype=F64)
    ks = O.grid_ids(kernel)
    for k in ks:
        _, _, d, g = O.stencil_grad(x, dx, kernel, k)
        assert float(g.sum(1).abs().max()) < 1e-10 / dx  # d/dx_p of sum_i w = 1
        tot = tot + torch.einsum("nsa,nsb->nab", d, g)
    tot = tot / len(ks)
    assert torch.allclose(tot, torch.eye(3, dtype=F64).expand_as(tot), atol=1e-12, rtol=0)


@pytest.mark.parametrize("kernel", KERNELS)
def test_affine_grid_velocity_is_reproduced(kernel):
    prm = _prm(kernel, res=16)
    st = _state(200, 16, 4, margin_cells=4.0)
    A = torch.tensor([[0.3, -1.2, 0.5], [0.7, 0.1, -0.4], [-0.2, 0.9, 0.6]], dtype=F64)
    b = torch.tensor([0.5, -0.25, 1.0], dtype=F64)
    vg = {k: b + O.grid_nodes(prm, k) @ A.T for k in O.grid_ids(kernel)}
    v, B, C = O.g2p(st, vg, prm)
    assert torch.allclose(v, b + st.x @ A.T, atol=1e-12, rtol=0)
    assert torch.allclose(C, A.expand_as(C), atol=1e-10, rtol=0)
    assert float(B.abs().max()) == 0.0


@pytest.mark.parametrize("kernel", KERNELS)
def test_p2g_conserves_linear_momentum_with_stress(kernel):
    prm = _prm(kernel, res=16)
    st = _state(300, 16, 5, margin_cells=4.0, f_scale=0.2)
    grids = O.p2g(st, prm)
    assert torch.allclose(O.grid_momentum(grids, prm), O.particle_momentum(st, prm), atol=1e-14, rtol=1e-12)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("transfer", [O.TRANSFER_PIC, O.TRANSFER_APIC_GRAD])
def test_pic_force_is_minus_twice_energy_gradient(kernel, transfer):
    prm = _prm(kernel)
    prm.transfer = transfer
    st = _state(60, 12, 13, f_scale=0.15)
    if transfer == O.TRANSFER_APIC_GRAD:  # the B term cancels in the difference below
        st.B = 0.3 * torch.randn(60, 3, 3, dtype=F64, generator=torch.Generator().manual_seed(3))
    st.v.zero_()
    g_s = O.p2g(st, prm)
    g_0 = O.p2g(st, prm, stress=False)
    mu, lam = O.particle_lame(st, prm)
    disp = {k: torch.zeros(prm.n_nodes ** 3, 3, dtype=F64, requires_grad=True) for k in O.grid_ids(kernel)}
    _, _, C = O.g2p(st, disp, prm)
    Fh = (torch.eye(3, dtype=F64) + C) @ st.F
    E = (prm.V0 * O.fc_energy(Fh, mu, lam, newton=True)).sum()
    grads = torch.autograd.grad(E, [disp[k] for k in O.grid_ids(kernel)])
    scale = 2.0 if kernel == O.KERNEL_CK else 1.0  # each CK grid carries the full mass; totals are averaged
    for k, gk in zip(O.grid_ids(kernel), grads):
        f = (g_s[k][1] - g_0[k][1]) / prm.dt
        assert torch.allclose(f, -scale * gk, atol=1e-9 * float(gk.abs().max()), rtol=0)


def test_pic_step_keeps_B_zero_and_momentum():
    prm = _prm(O.KERNEL_CK, res=16)
    prm.gravity = (0.0, 0.0, 0.0)
    st = _state(300, 16, 8, margin_cells=5.0, f_scale=0.1)
    new = O.step(st, prm, bc=False)
    assert float(new.B.abs().max()) == 0.0
    assert torch.allclose(O.particle_momentum(new, prm), O.particle_momentum(st, prm), atol=1e-13, rtol=1e-11)


def _prm_grad(kernel, res=16, dt=1e-3, model=O.FIXED_COROTATED):
    prm = _prm(kernel, res=res, dt=dt)
    prm.materials = [O.Mat(model, 1e5, 0.3, 1000.0, 30.0)]
    prm.transfer = O.TRANSFER_APIC_GRAD
    return prm


def _state_B(n, res, seed, **kw):
    x, v, B, F = S.random_state(n, res, seed, **kw)
    return O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.from_numpy(B), torch.from_numpy(F))


@pytest.mark.parametrize("kernel", KERNELS)
def test_apic_grad_p2g_conserves_linear_and_angular_momentum(kernel):
    prm = _prm_grad(kernel)
    st = _state_B(300, 16, 41, margin_cells=4.0, f_scale=0.2)
    grids = O.p2g(st, prm)
    P, L = O.particle_momentum(st, prm), O.particle_angular_momentum(st, prm)
    assert torch.allclose(O.grid_momentum(grids, prm), P, atol=1e-13 * float(P.abs().max()), rtol=0)
    assert torch.allclose(O.grid_angular_momentum(grids, prm), L, atol=1e-12 * float(L.abs().max()), rtol=0)
    # the B term is really there: dropping B changes the grid momentum
    st0 = O.State(st.x, st.v, torch.zeros_like(st.B), st.F, st.mat)
    k0 = O.grid_ids(kernel)[0]
    assert not torch.allclose(O.p2g(st0, prm)[k0][1], grids[k0][1])


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("model", [O.FIXED_COROTATED, O.DRUCKER_PRAGER])
def test_apic_grad_step_conserves_momentum(kernel, model):
    prm = _prm_grad(kernel, dt=1e-4, model=model)
    st = _state_B(400, 16, 42, margin_cells=4.0, f_scale=0.1)
    P0, L0 = O.particle_momentum(st, prm), O.particle_angular_momentum(st, prm)
    new = O.step(st, prm, gravity=(0.0, 0.0, 0.0), bc=False)
    assert torch.allclose(O.particle_momentum(new, prm), P0, atol=1e-12 * float(P0.abs().max()), rtol=0)
    assert torch.allclose(O.particle_angular_momentum(new, prm), L0, atol=1e-11 * float(L0.abs().max()), rtol=0)
    assert float(new.B.abs().max()) > 0.0


@pytest.mark.parametrize("kernel", KERNELS)
def test_apic_grad_affine_field_gives_B_and_grad_v(kernel):
    prm = _prm_grad(kernel)
    st = _state_B(200, 16, 43, margin_cells=4.0)
    A = torch.tensor([[0.3, -1.2, 0.5], [0.7, 0.1, -0.4], [-0.2, 0.9, 0.6]], dtype=F64)
    b = torch.tensor([0.5, -0.25, 1.0], dtype=F64)
    vg = {k: b + O.grid_nodes(prm, k) @ A.T for k in O.grid_ids(kernel)}
    v, B, C = O.g2p(st, vg, prm)
    assert torch.allclose(v, b + st.x @ A.T, atol=1e-12, rtol=0)
    assert torch.allclose(B, A @ O.apic_D(st.x, prm), atol=1e-12, rtol=0)
    assert torch.allclose(C, A.expand_as(C), atol=1e-10, rtol=0)
