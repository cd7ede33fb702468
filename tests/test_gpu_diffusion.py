"""Numerical diffusion, compact kernel against the quadratic B-spline (the
paper's comparison: a 20 x 10 x 140-cell elastic cuboid with the initial
velocity v_y = 0.2 sin(500 z), 500 steps of 2e-5 s, no gravity).  The paper
reports that the compact kernel loses energy noticeably slower; this checks
that behaviour on the CUDA path: the total (kinetic + fixed-corotated elastic)
energy kept by CK exceeds the quadratic twin's at every checkpoint."""
import numpy as np
import pytest

from gpu_helpers import need_gpu
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _energies(ck, sim, sc):
    m = sc.materials[0]
    V0 = sc.dx ** 3 / sc.ppc
    v = sim.read(ck.FIELD_V).astype(np.float64)
    F = sim.read(ck.FIELD_F).astype(np.float64)
    kin = 0.5 * m.rho * V0 * (v ** 2).sum()
    U, s, Vt = np.linalg.svd(F)
    R = U @ Vt
    mu = m.E / (2 * (1 + m.nu))
    lam = m.E * m.nu / ((1 + m.nu) * (1 - 2 * m.nu))
    J = np.linalg.det(F)
    psi = mu * ((F - R) ** 2).sum(axis=(1, 2)) + 0.5 * lam * (J - 1) ** 2
    return kin, V0 * psi.sum()


def test_compact_kernel_keeps_more_energy_than_quadratic():
    ck = need_gpu()
    sc = S.diffusion_bar()
    hist = {}
    for kernel in (ck.KERNEL_CK, ck.KERNEL_QUADRATIC):
        sim = ck.Simulation(sc, kernel)
        e = [sum(_energies(ck, sim, sc))]
        for _ in range(5):
            sim.step(100)
            sim.sync()
            e.append(sum(_energies(ck, sim, sc)))
        sim.close()
        hist[kernel] = np.array(e)
    eck, eq = hist[ck.KERNEL_CK], hist[ck.KERNEL_QUADRATIC]
    print("total energy CK", eck, "quadratic", eq)
    assert eck[0] == pytest.approx(eq[0], rel=1e-6)  # same initial state
    assert np.all(eck[1:] > eq[1:])
    assert np.all(np.diff(eck) <= 1e-6 * eck[0]) and np.all(np.diff(eq) <= 1e-6 * eq[0])  # both dissipate
