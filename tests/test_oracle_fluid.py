"""Pins of the oracle's J-based fluid (reading R15: p = B (J^-gamma - 1),
tau = -J p I, F projected to J^(1/3) I after each update).

The paper only cites the equation of state, so the model is pinned by what
the mathematics fixes: closed values of the pressure, the Kirchhoff stress as
the derivative of a stored energy of J alone (autograd through det F, for
general non-isotropic F), the projection keeping det F, and, at grid level,
the P2G force of a fluid equal to minus twice the gradient of the total stored
energy (the same variational identity the solids satisfy).
"""
import math

import numpy as np
import torch

from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

F64 = torch.float64
B_EOS, GAMMA = 10.0, 7.15


def _fluid_prm(res=12, dt=1e-3):
    return O.Params(res=res, dx=1.0 / res, dt=dt, materials=[O.Mat(O.J_FLUID, B_EOS, 0.0, 1000.0, 0.0, GAMMA)])


def test_fluid_pressure_closed_values():
    J = torch.tensor([1.0, 0.5, 2.0, 0.9], dtype=F64)
    p = O.fluid_pressure(J, B_EOS, GAMMA)
    want = torch.tensor([0.0, B_EOS * (2.0 ** GAMMA - 1.0), B_EOS * (0.5 ** GAMMA - 1.0),
                         B_EOS * (0.9 ** -GAMMA - 1.0)], dtype=F64)
    assert torch.allclose(p, want, rtol=1e-14, atol=0)
    assert p[1] > 0 and p[2] < 0  # compression pushes, expansion pulls


def test_fluid_kirchhoff_is_energy_derivative_for_general_F():
    """tau = dpsi/dF F^T with psi(F) = fluid_energy(det F), for F with shear."""
    g = torch.Generator().manual_seed(2)
    F = (torch.eye(3, dtype=F64) + 0.2 * torch.randn(40, 3, 3, generator=g, dtype=F64)).requires_grad_(True)
    assert bool((torch.det(F) > 0).all())
    psi = O.fluid_energy(torch.det(F), B_EOS, GAMMA).sum()
    (P,) = torch.autograd.grad(psi, [F])
    tau_ad = P @ F.detach().transpose(-1, -2)
    tau = O.fluid_kirchhoff(F.detach(), torch.full((40,), B_EOS, dtype=F64), torch.full((40,), GAMMA, dtype=F64))
    assert torch.allclose(tau, tau_ad, rtol=1e-12, atol=1e-12 * float(tau_ad.abs().max()))
    # isotropic whatever the shear
    off = tau - torch.diag_embed(torch.diagonal(tau, dim1=-2, dim2=-1))
    assert float(off.abs().max()) == 0.0
    assert torch.allclose(tau[:, 0, 0], tau[:, 1, 1]) and torch.allclose(tau[:, 0, 0], tau[:, 2, 2])
    # psi(1) = 0 and psi'(1) = -p(1) = 0: a fluid at rest volume stores nothing
    assert float(O.fluid_energy(torch.tensor(1.0, dtype=F64), B_EOS, GAMMA)) == 0.0


def test_fluid_projection_keeps_volume_and_is_idempotent():
    prm = _fluid_prm()
    x, v, B, F = S.random_state(30, 12, 3, f_scale=0.2)
    st = O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.from_numpy(B), torch.from_numpy(F))
    Fp = O.plasticity(st.F, st, prm)
    J = torch.det(st.F)
    assert torch.allclose(torch.det(Fp), J, rtol=1e-13, atol=0)
    c = J ** (1.0 / 3.0)
    assert torch.allclose(Fp, c[:, None, None] * torch.eye(3, dtype=F64), rtol=1e-14, atol=0)
    assert torch.allclose(O.plasticity(Fp, st, prm), Fp, rtol=0, atol=0)


def test_fluid_grid_force_is_minus_twice_energy_gradient():
    """As for the solids: with F^(xh) = (I + grad v(xh - x)) F from the oracle's
    G2P of grid displacements, the fluid's P2G force on each grid equals
    -2 dE/dxh, E = sum_p V0 psi(det F^_p)."""
    prm = _fluid_prm(res=12, dt=1e-3)
    x, v, B, F = S.random_state(60, 12, 14, f_scale=0.1)
    st = O.make_state(torch.from_numpy(x), torch.zeros(60, 3, dtype=F64), torch.zeros(60, 3, 3, dtype=F64),
                      torch.from_numpy(F))
    st.F = O.plasticity(st.F, st, prm)  # a fluid's F is volumetric
    g_s = O.p2g(st, prm)
    g_0 = O.p2g(st, prm, stress=False)
    disp = {k: torch.zeros(prm.n_nodes ** 3, 3, dtype=F64, requires_grad=True) for k in O.grid_ids(prm.kernel)}
    _, _, C = O.g2p(st, disp, prm)
    Fh = (torch.eye(3, dtype=F64) + C) @ st.F
    E = (prm.V0 * O.fluid_energy(torch.det(Fh), B_EOS, GAMMA)).sum()
    grads = torch.autograd.grad(E, [disp[k] for k in O.grid_ids(prm.kernel)])
    for k, gk in zip(O.grid_ids(prm.kernel), grads):
        f = (g_s[k][1] - g_0[k][1]) / prm.dt
        assert torch.allclose(f, -2.0 * gk, atol=1e-9 * float(gk.abs().max()), rtol=0)


def test_fluid_step_conserves_momentum_without_gravity():
    """One full step of a compressed fluid blob away from the walls: the total
    momentum is unchanged (internal pressure forces cancel) and F stays
    volumetric."""
    prm = _fluid_prm(res=16, dt=1e-3)
    prm.gravity = (0.0, 0.0, 0.0)
    x, v, B, F = S.random_state(200, 16, 5, margin_cells=5.0, f_scale=0.0)
    n = x.shape[0]
    Fc = np.eye(3)[None].repeat(n, 0) * 0.9  # J = 0.729: compressed
    st = O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.from_numpy(B), torch.from_numpy(Fc))
    p0 = O.particle_momentum(st, prm)
    new = O.step(st, prm, bc=False)
    p1 = O.particle_momentum(new, prm)
    assert torch.allclose(p1, p0, atol=1e-12 * float(O.particle_mass(st, prm).sum()), rtol=0)
    off = new.F - torch.diag_embed(torch.diagonal(new.F, dim1=-2, dim2=-1))
    assert float(off.abs().max()) == 0.0
    assert math.isfinite(float(new.x.sum()))
