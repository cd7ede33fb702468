"""Numerical diffusion, compact kernel against the quadratic B-spline (the
paper's comparison: a 20 x 10 x 140-cell elastic cuboid with the initial
velocity v_y = 0.2 sin(500 z), 500 steps of 2e-5 s, no gravity).  The paper
reports that the compact kernel loses energy noticeably slower; this checks
that behaviour on the CUDA path: the total (kinetic + fixed-corotated elastic)
energy kept by CK exceeds the quadratic twin's at every checkpoint.

The paper does not say which transfer its comparison used, so the kernel-
gradient transfers are run too: APIC with the kernel gradient keeps the same
ordering at every checkpoint; PIC, which drops the affine part of the
velocity at every G2P, loses energy faster than either APIC form with either
kernel, and there CK keeps more than the quadratic twin over the first 200
steps (about 2.8x and 1.6x; by step 400 both have lost all but about 0.05% of
the initial energy and the ordering is no longer resolved)."""
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


def _history(ck, kernel, transfer):
    sc = S.diffusion_bar()
    sc.kernel = kernel
    sc.transfer = transfer
    sim = ck.Simulation(sc, ck.kernel_code(sc))
    e = [sum(_energies(ck, sim, sc))]
    for _ in range(5):
        sim.step(100)
        sim.sync()
        e.append(sum(_energies(ck, sim, sc)))
    sim.close()
    return np.array(e)


@pytest.mark.parametrize("transfer", [S.TRANSFER_APIC_MLS, S.TRANSFER_APIC_GRAD])
def test_compact_kernel_keeps_more_energy_than_quadratic(transfer):
    ck = need_gpu()
    hist = {kernel: _history(ck, kernel, transfer) for kernel in (ck.KERNEL_CK, ck.KERNEL_QUADRATIC)}
    eck, eq = hist[ck.KERNEL_CK], hist[ck.KERNEL_QUADRATIC]
    print("total energy CK", eck, "quadratic", eq)
    assert eck[0] == pytest.approx(eq[0], rel=1e-6)  # same initial state
    assert np.all(eck[1:] > eq[1:])
    assert np.all(np.diff(eck) <= 1e-6 * eck[0]) and np.all(np.diff(eq) <= 1e-6 * eq[0])  # both dissipate


def test_pic_dissipates_faster_and_ck_leads_early():
    ck = need_gpu()
    pic = {k: _history(ck, k, S.TRANSFER_PIC) for k in (ck.KERNEL_CK, ck.KERNEL_QUADRATIC)}
    apic = {k: _history(ck, k, S.TRANSFER_APIC_MLS) for k in (ck.KERNEL_CK, ck.KERNEL_QUADRATIC)}
    print("PIC total energy CK", pic[ck.KERNEL_CK], "quadratic", pic[ck.KERNEL_QUADRATIC])
    for k in pic:
        assert pic[k][0] == pytest.approx(apic[k][0], rel=1e-6)
        assert np.all(pic[k][1:] < apic[k][1:])
        assert np.all(np.diff(pic[k]) <= 1e-6 * pic[k][0])
    assert np.all(pic[ck.KERNEL_CK][1:3] > 1.3 * pic[ck.KERNEL_QUADRATIC][1:3])
