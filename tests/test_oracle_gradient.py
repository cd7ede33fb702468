"""Pins of the FP64 oracle gradient used to check the CUDA adjoint.

The oracle gradient is torch autograd through the float64 oracle step (with
the Newton polar iteration for the fixed-corotated rotation, so F = I is
differentiable).  It is pinned here by float64 central finite differences of
the oracle itself, and by the exact momentum bookkeeping of the scheme: the
centre of mass moves by dt * mean(v) per step plus gravity, whatever the
stiffness, so d(COM loss)/dE vanishes and d(COM loss)/dv0 is the same for
every particle.
"""
import math

import numpy as np
import pytest
import torch

from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

F64 = torch.float64


def _tiny(seed=0, steps=3):
    sc = S.differentiable_cube(seed=seed, res=16, lo=6, hi=8)  # 8 cells -> 64 particles
    prm = O.params_from_scene(sc)
    prm.dt = 2e-4
    x0 = torch.from_numpy(sc.x.astype(np.float32).astype(np.float64))
    v0 = torch.from_numpy(sc.v.astype(np.float32).astype(np.float64))
    E = torch.full((sc.n,), sc.materials[0].E, dtype=F64)
    return sc, prm, x0, v0, E, steps


def _losses(x0, v0, E, prm, steps, target):
    st = O.make_state(x0, v0, E=E)
    st = O.run(st, prm, steps, newton=True)
    com = st.x.mean(0)
    L1 = torch.linalg.vector_norm(com - target)
    L2 = ((st.x - com) ** 2).sum(1).mean()
    return L1, L2


def test_oracle_gradient_matches_central_differences():
    sc, prm, x0, v0, E, steps = _tiny()
    target = x0.mean(0) + torch.tensor([0.01, -0.005, 0.0], dtype=F64)
    v0r = v0.clone().requires_grad_(True)
    Er = E.clone().requires_grad_(True)
    _, L2 = _losses(x0, v0r, Er, prm, steps, target)
    gv, gE = torch.autograd.grad(L2, [v0r, Er])
    g = torch.Generator().manual_seed(3)
    for _ in range(3):
        dv = torch.randn(v0.shape, generator=g, dtype=F64)
        dE = torch.randn(E.shape, generator=g, dtype=F64)
        hv, hE = 1e-6, 1e-4  # hE: the E-sensitivity is small, so a larger step keeps roundoff below 1e-6
        with torch.no_grad():
            fd_v = (_losses(x0, v0 + hv * dv, E, prm, steps, target)[1]
                    - _losses(x0, v0 - hv * dv, E, prm, steps, target)[1]) / (2 * hv)
            fd_E = (_losses(x0, v0, E * (1 + hE * dE), prm, steps, target)[1]
                    - _losses(x0, v0, E * (1 - hE * dE), prm, steps, target)[1]) / (2 * hE)
        an_v = float((gv * dv).sum())
        an_E = float((gE * E * dE).sum())
        assert abs(an_v - float(fd_v)) <= 1e-6 * abs(an_v) + 1e-12
        assert abs(an_E - float(fd_E)) <= 1e-5 * abs(an_E) + 1e-14
    # the spread loss does depend on stiffness
    assert float((gE * E).abs().max()) > 1e-10


def test_com_loss_gradient_is_stiffness_free_and_uniform():
    sc, prm, x0, v0, E, steps = _tiny(steps=4)
    target = x0.mean(0) + torch.tensor([0.01, -0.005, 0.0], dtype=F64)
    v0r = v0.clone().requires_grad_(True)
    Er = E.clone().requires_grad_(True)
    L1, _ = _losses(x0, v0r, Er, prm, steps, target)
    gv, gE = torch.autograd.grad(L1, [v0r, Er])
    # COM_T = COM_0 + T dt mean(v0) + gravity terms: dL/dv0_p = T dt / N * unit(COM_T - target)
    with torch.no_grad():
        st = O.run(O.make_state(x0, v0, E=E), prm, steps, newton=True)
        u = st.x.mean(0) - target
        u = u / torch.linalg.vector_norm(u)
    want = steps * prm.dt / sc.n * u
    assert torch.allclose(gv, want.expand_as(gv), rtol=1e-8, atol=1e-14)
    # stiffness enters only through internal forces, which carry no net momentum
    assert float(gE.abs().max()) < 1e-12 * float(gv.abs().max()) / sc.materials[0].E * 1e6
