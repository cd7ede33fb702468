"""Host-side conserved quantities (diagnostics.conserved) against the oracle's
particle momentum and angular momentum (Supplement eq. 3, pinned in the oracle
tests), and Simulation.diagnostics on read-back fields (a stand-in for the
context's readback; no GPU)."""
import numpy as np
import pytest
import torch

from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import ckmpm as ck
from paper_2412_10399_gb300 import diagnostics as D
from paper_2412_10399_gb300 import scenes as S


def _state(seed):
    x, v, B, F = S.random_state(500, 16, seed)
    mat = (np.arange(500) % 2).astype(np.uint8)
    mats = [S.ELASTIC, S.SAND]
    return x, v, B, F, mat, mats


def test_conserved_matches_the_oracle():
    x, v, B, F, mat, mats = _state(3)
    prm = O.Params(res=16, dx=1 / 16, dt=1e-4, materials=[O.Mat(m.model, m.E, m.nu, m.rho, m.friction_deg) for m in mats])
    st = O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.from_numpy(B), torch.from_numpy(F),
                      mat=torch.from_numpy(mat.astype(np.int64)))
    d = D.conserved(x, v, mat, mats, prm.dx, prm.ppc, B)
    assert d["mass"] == pytest.approx(float(O.particle_mass(st, prm).sum()), rel=1e-14)
    assert np.allclose(d["momentum"], O.particle_momentum(st, prm).numpy(), rtol=1e-13, atol=0)
    assert np.allclose(d["angular_momentum"], O.particle_angular_momentum(st, prm).numpy(), rtol=1e-12, atol=1e-18)
    m = O.particle_mass(st, prm).numpy()
    assert d["kinetic_energy"] == pytest.approx(0.5 * float((m * (v ** 2).sum(1)).sum()), rel=1e-14)
    # no B: orbital part only
    d0 = D.conserved(x, v, mat, mats, prm.dx, prm.ppc)
    st0 = O.State(st.x, st.v, torch.zeros_like(st.B), st.F, st.mat)
    assert np.allclose(d0["angular_momentum"], O.particle_angular_momentum(st0, prm).numpy(), rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("kernel", [ck.KERNEL_CK, ck.KERNEL_CK | ck.TRANSFER_PIC])
def test_simulation_diagnostics_reads_the_fields_the_transfer_keeps(kernel):
    x, v, B, F, mat, mats = _state(4)
    sc = S.Scene("s", 16, 1 / 16, 1e-4, x, v, mat, mats)
    sim = object.__new__(ck.Simulation)
    sim.scene, sim.kernel, sim.n = sc, kernel, len(x)
    fields = {ck.FIELD_X: x.astype(np.float32), ck.FIELD_V: v.astype(np.float32), ck.FIELD_B: B.astype(np.float32)}
    reads = []
    sim.read = lambda f, scene_id=0: reads.append(f) or fields[f]
    d = sim.diagnostics()
    want = D.conserved(fields[ck.FIELD_X], fields[ck.FIELD_V], mat, mats, sc.dx, sc.ppc,
                       None if kernel & ck.TRANSFER_PIC else fields[ck.FIELD_B])
    assert np.array_equal(d["angular_momentum"], want["angular_momentum"])
    assert (ck.FIELD_B in reads) == (not kernel & ck.TRANSFER_PIC)
