"""Checkpoint and resume through the C ABI: a run interrupted by save() and
continued in a fresh context after load() follows the uninterrupted run.
The two agree to rounding, not bitwise: blocks meet in float atomics whose
order varies from run to run, and B travels as m B - dt V0 tau(F) recovered
and rebuilt in float32.  Tolerances after 5 steps: x within 1e-5 dx, v and
F within 1e-4 and 1e-5 relative; a checkpoint that lost B (APIC's affine
velocity) misses by orders of magnitude more."""
import numpy as np
import pytest

from gpu_helpers import need_gpu, random_scene, rel
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", [S.KERNEL_CK, S.KERNEL_QUADRATIC])
def test_resume_from_checkpoint_follows_the_uninterrupted_run(tmp_path, kernel):
    ck = need_gpu()
    sc, B, F = random_scene(4000, 32, 81, kernel=kernel, f_scale=0.05)
    path = str(tmp_path / "ckpt.npz")
    a = ck.Simulation(sc, ck.kernel_code(sc))
    a.write(ck.FIELD_F, F)
    a.write(ck.FIELD_B, B)
    a.step(10)
    a.sync()
    a.save(path)
    a.step(5)
    a.sync()
    want = [a.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F)]
    a.close()
    b = ck.Simulation(sc, ck.kernel_code(sc))
    b.load(path)
    b.step(5)
    b.sync()
    got = [b.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F)]
    b.close()
    assert np.abs(got[0] - want[0]).max() <= 1e-5 * sc.dx
    assert rel(got[1], want[1]) <= 1e-4
    assert rel(got[2], want[2]) <= 1e-5
