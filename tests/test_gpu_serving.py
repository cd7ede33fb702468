"""Serving extension: scenes run in one continuously batched context give the
same result as each scene run alone (positions within 1e-3 dx, the position
tolerance of the parity tests), while arriving at different times and with
different sizes and materials."""
import numpy as np
import pytest

from gpu_helpers import need_gpu
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


class StepClock:
    """Deterministic clock: 10 ms per poll, so arrivals map to global steps."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.01
        return self.t


def test_each_scene_alone_equals_in_the_mix():
    ck = need_gpu()
    from paper_2412_10399_gb300 import serving as SV
    reqs = S.served_mix(n_scenes=5, seed=7, n_max=3e5, steps=30)
    # stagger arrivals by global steps: 0, 0, 4, 9, 15 polls
    arrivals = [0.0, 0.0, 0.045, 0.095, 0.155]
    budget = SV.Budget.from_bytes(2 << 30, max_res=128, max_scenes=3)  # at most 3 resident at once
    eng = SV.EngineCK(budget)
    srv = SV.Server(eng, budget, clock=StepClock())
    for r, t in zip(reqs, arrivals):
        srv.submit(SV.Request(r.scene, r.scene.steps, arrival_s=t, read_fields=(ck.FIELD_X, ck.FIELD_F)))
    results = srv.run(sleep=lambda s: None)
    eng.close()
    assert len(results) == 5
    assert any(r.admitted_at_step > 0 for r in results)
    st = srv.stats()
    assert st["p99_ms"] is not None and st["p50_ms"] <= st["p99_ms"]
    for res in results:
        sc = res.request.scene
        sim = ck.Simulation(sc, ck.KERNEL_CK)
        sim.step(sc.steps)
        sim.sync()
        x = sim.read(ck.FIELD_X)
        F = sim.read(ck.FIELD_F)
        sim.close()
        assert np.abs(res.fields[ck.FIELD_X] - x).max() <= 1e-3 * sc.dx, sc.name
        assert np.abs(res.fields[ck.FIELD_F] - F).max() <= 1e-4, sc.name
