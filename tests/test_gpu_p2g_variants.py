"""Every P2G form the launch configuration can select, against the FP64 oracle.

The APIC + MLS P2G has three switches, read from the environment when a
context is created: CKMPM_P2G_REP (one or two copies of the shared
accumulators), CKMPM_P2G_ROT (components issued in order or in the
lane-rotated order, one copy only) and CKMPM_P2G_FMA (contributions rounded to
fixed point by a conversion or, in blocks of 256 or more particles, by a fused
multiply-add).  The defaults are the compact kernel's (one copy, rotated, FMA)
and the quadratic twin's (two copies, in order, FMA); the other forms are
measured alternatives.  Each form must give the oracle's grids after one P2G
(Sec. 4.3.1-4.5) within the parity tolerance, on dense blocks (about 512
particles each: the FMA rounding) and on a sparse state (blocks of a few
particles: the conversion), and the forms must agree with one another far more
closely than that, since they add the same fixed-point contributions.
"""
import os

import numpy as np
import pytest

from gpu_helpers import need_gpu, oracle_state, random_scene, rel
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu

# (copies, rotated, fma)
FORMS = [(1, 0, 0), (1, 0, 1), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 0, 1)]
ENV = ("CKMPM_P2G_REP", "CKMPM_P2G_ROT", "CKMPM_P2G_FMA")

_oracle_cache = {}


def _grids_with(ck, sc, B, F, form):
    old = {k: os.environ.get(k) for k in ENV}
    try:
        for k, val in zip(ENV, form):
            os.environ[k] = str(val)
        sim = ck.Simulation(sc, sc.kernel)
        sim.write(ck.FIELD_F, F)
        sim.write(ck.FIELD_B, B)
        sim.probe_grids()
        gm = sim.read(ck.FIELD_GRID_M)
        gp = sim.read(ck.FIELD_GRID_P)
        st = sim.stats()
        sim.close()
    finally:
        for k, val in old.items():
            if val is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = val
    return gm, gp, st


def _case(kernel, dense):
    if dense:
        return random_scene(32768, 32, 4, model=S.DRUCKER_PRAGER, kernel=kernel, f_scale=0.08, box=(8.0, 24.0))
    return random_scene(777, 16, 2, model=S.FIXED_COROTATED, kernel=kernel, f_scale=0.08)


def _oracle(kernel, dense, sc, B, F):
    key = (kernel, dense)
    if key not in _oracle_cache:
        _oracle_cache[key] = O.p2g(oracle_state(sc, B, F), O.params_from_scene(sc))
    return _oracle_cache[key]


@pytest.mark.parametrize("kernel", [S.KERNEL_CK, S.KERNEL_QUADRATIC])
@pytest.mark.parametrize("dense", [True, False])
def test_every_p2g_form_matches_the_oracle_and_the_others(kernel, dense):
    ck = need_gpu()
    sc, B, F = _case(kernel, dense)
    grids = _oracle(kernel, dense, sc, B, F)
    nn = sc.res + 1
    results = {}
    for form in FORMS:
        gm, gp, st = _grids_with(ck, sc, B, F, form)
        if dense:
            # about 512 particles per block: the FMA rounding's blocks
            assert st.n_particle_blocks >= 64 and sc.n / st.n_particle_blocks >= 256
        for gi, k in enumerate(O.grid_ids(kernel)):
            mo = grids[k][0].numpy().reshape(nn, nn, nn)
            po = grids[k][1].numpy().reshape(nn, nn, nn, 3)
            assert rel(gm[gi], mo) <= 1e-5, f"form {form}: grid {k} mass"
            assert rel(gp[gi], po) <= 1e-5, f"form {form}: grid {k} momentum"
        results[form] = (np.asarray(gm, np.float64), np.asarray(gp, np.float64))
    # The forms add the same contributions; they differ only in the order of
    # float32 operations before the rounding to fixed point and in that
    # rounding (one unit, cnt x bound / 2^30, about 6e-8 of a dense node's sum),
    # so a node's sums may differ by a few units: 2e-6 of the largest value is
    # five times tighter than the oracle tolerance.
    ref_m, ref_p = results[FORMS[0]]
    for form, (gm, gp) in results.items():
        assert np.abs(gm - ref_m).max() <= 2e-6 * np.abs(ref_m).max(), f"form {form} mass"
        assert np.abs(gp - ref_p).max() <= 2e-6 * np.abs(ref_p).max(), f"form {form} momentum"
