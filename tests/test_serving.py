"""Host logic of the serving loop (admission under a budget, FIFO, continuous
batching, latency accounting) with a fake engine: no GPU needed."""
import numpy as np
import pytest

from paper_2412_10399_gb300 import scenes as S
from paper_2412_10399_gb300 import serving as SV


class FakePending:
    """A step in flight: done after `lag` polls of done(); ms() waits for it."""

    def __init__(self, eng, ms, lag=2):
        self.eng, self._ms, self.left = eng, ms, lag
        self.harvested = False

    def done(self):
        self.left -= 1
        return self.left < 0

    def ms(self):
        self.eng.waits += 0 if self.left < 0 else 1
        self.harvested = True
        return self._ms


class FakeEngine:
    def __init__(self):
        self.pending = []
        self.waits = 0
        self.next_id = 0
        self.resident = set()
        self.max_resident = 0
        self.steps_of = {}
        self.admit_order = []

    def admit(self, scene):
        sid = self.next_id
        self.next_id += 1
        self.resident.add(sid)
        self.steps_of[sid] = 0
        self.admit_order.append(scene.name)
        self.max_resident = max(self.max_resident, len(self.resident))
        return sid

    def release(self, sid):
        self.resident.remove(sid)

    def step_async(self):
        for s in self.resident:
            self.steps_of[s] += 1
        p = FakePending(self, 0.5 + 0.1 * len(self.resident))
        self.pending.append(p)
        return p

    def read(self, sid, field, n):
        return np.full((n, 3), float(self.steps_of[sid]), np.float32)


class FakeClock:
    def __init__(self, dt=0.01):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def _scene(name, n, res=32):
    x = np.full((n, 3), 0.5, np.float64)
    return S.Scene(name, res, 1.0 / res, 1e-4, x, np.zeros_like(x), np.zeros(n, np.uint8), [S.ELASTIC])


def _budget_for(k, n, res=32):
    r = SV.scene_resources(n, res)
    return SV.Budget(**{key: k * v for key, v in r.items()})


def test_at_most_budget_many_scenes_are_resident_and_fifo_holds():
    eng = FakeEngine()
    srv = SV.Server(eng, _budget_for(2, 1000), clock=FakeClock())
    for i, steps in enumerate((5, 3, 4, 2)):
        srv.submit(SV.Request(_scene(f"s{i}", 1000), steps))
    res = srv.run(sleep=lambda s: None)
    assert eng.max_resident == 2
    assert eng.admit_order == ["s0", "s1", "s2", "s3"]
    assert sorted(r.request.scene.name for r in res) == ["s0", "s1", "s2", "s3"]
    for r in res:  # every scene ran exactly its steps, and its result was read before release
        assert float(r.fields[0][0, 0]) == r.request.steps
        assert r.finished_at_step - r.admitted_at_step == r.request.steps
    assert len(srv.latencies_ms) == 5 + 3 + 4 + 2
    # s2 waits for the first free slot (s1 finishes after 3 global steps)
    s2 = [r for r in res if r.request.scene.name == "s2"][0]
    assert s2.admitted_at_step == 3


def test_arrivals_join_running_work():
    eng = FakeEngine()
    clock = FakeClock(dt=0.01)
    srv = SV.Server(eng, _budget_for(3, 1000), clock=clock)
    srv.submit(SV.Request(_scene("early", 1000), 10, arrival_s=0.0))
    srv.submit(SV.Request(_scene("late", 1000), 3, arrival_s=0.045))
    res = srv.run(sleep=lambda s: None)
    late = [r for r in res if r.request.scene.name == "late"][0]
    early = [r for r in res if r.request.scene.name == "early"][0]
    assert 0 < late.admitted_at_step < early.finished_at_step  # admitted while 'early' was running
    assert eng.max_resident == 2
    st = srv.stats()
    assert st["scene_steps"] == 13 and st["scenes_finished"] == 2
    assert st["p50_ms"] <= st["p99_ms"]


def test_oversized_request_is_refused():
    srv = SV.Server(FakeEngine(), _budget_for(1, 1000), clock=FakeClock())
    with pytest.raises(ValueError):
        srv.submit(SV.Request(_scene("big", 100000), 1))


@pytest.mark.parametrize("kernel", [0, 1, 2, 4, 5])
def test_budget_from_bytes_stays_within_the_budget(kernel):
    b = SV.Budget.from_bytes(8 << 30, max_res=128, max_scenes=16, kernel=kernel)
    used = (b.particles * SV.bytes_per_particle(kernel) + b.keys * SV.BYTES_PER_KEY
            + b.virtual_blocks * SV.BYTES_PER_VIRTUAL_BLOCK + b.pool_blocks * SV.bytes_per_pool_block(kernel))
    assert used <= (8 << 30)
    assert used >= (8 << 30) * 0.999
    assert b.particles > 10_000_000
    # every scene that fits alone fits the pool reservation
    assert b.fits({}, SV.scene_resources(2_000_000, 128))


def test_steps_are_enqueued_without_waiting_and_bounded_in_flight():
    """The loop enqueues global steps ahead of the device and waits only when
    max_inflight steps are queued (or at the end): never more than that many
    are un-harvested, every step's time is accounted once, and what a request
    sees (arrival to result, wall time per resident step) is reported."""
    eng = FakeEngine()
    srv = SV.Server(eng, _budget_for(2, 1000), clock=FakeClock(), max_inflight=3)
    for i, steps in enumerate((12, 7, 9)):
        srv.submit(SV.Request(_scene(f"s{i}", 1000), steps))
    peak = 0
    while srv.poll():
        peak = max(peak, len(srv.inflight))
    assert peak <= 3
    assert all(p.harvested for p in eng.pending)
    assert len(srv.latencies_ms) == 12 + 7 + 9
    assert eng.waits < len(eng.pending)  # most steps were harvested after they finished, not waited for
    st = srv.stats()
    assert st["request_latency_p50_s"] is not None and st["request_latency_p50_s"] <= st["request_latency_p99_s"]
    assert st["resident_wall_ms_per_step_p50"] > 0
    assert abs(st["aggregate_particle_steps_per_s"] - 1000 * 28 / (srv.busy_ms / 1e3)) < 1e-6
