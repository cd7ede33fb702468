"""Serving loop over a multi-scene CK-MPM context (continuous batching).

Requests (a scene and a number of steps) arrive over time.  All resident
scenes advance together: every global step is one launch per kernel over the
concatenated block lists of every scene in the context.  The loop does not
wait for a global step: it enqueues the step with a pair of CUDA events
around it and goes on admitting and retiring while the device runs, with at
most ``max_inflight`` steps queued ahead; finished event pairs are harvested
by polling.  Waiting requests are admitted first come first served as soon as
the device-memory budget they need is free (admission is stream-ordered, so
it takes effect at the next enqueued step); a scene whose last step has been
enqueued is retired by reading back its final state, the one point where the
host waits for the device.  Reported: the device time of the global step
each scene-step belonged to (p50 / p99), and what a request sees: the wall
time from its arrival to its result and its wall time per step while
resident (p50 / p99), beside device-busy and wall throughput.

The admission arithmetic is plain host code (``Budget``); the engine is any
object with the ``admit / release / step / read`` methods of ``EngineCK``.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Sequence

# Device bytes per unit of each engine resource (see the layout in common.cuh):
BYTES_PER_PARTICLE = 2 * (16 + 48 + 16 + 16 + 4 + 4) + 2 * 4 + 4 + 4  # two pools, keys x2, perm, float64 list
BYTES_PER_KEY = 6 * 4 + 2 * 2 * 4                                  # histograms x2, offset, cursor, block list x2, P2G bounds x2
BYTES_PER_VIRTUAL_BLOCK = 2 * 4                                    # flag, table entry
BYTES_PER_POOL_BLOCK_CK = 2 * 2 * 64 * 16 + 2 * 4                  # Gacc + Gvel for both grids, list entries
BYTES_PER_PARTICLE_APIC_GRAD = 2 * 36                              # the separate stress term, both pools


def bytes_per_particle(kernel: int = 0) -> int:
    """Device bytes per particle for a kernel argument (kernel | transfer flag):
    APIC with the kernel gradient (flag 4) keeps its stress term in 36 more
    bytes per pool buffer."""
    return BYTES_PER_PARTICLE + (BYTES_PER_PARTICLE_APIC_GRAD if kernel & 4 else 0)


def bytes_per_pool_block(kernel: int = 0) -> int:
    """Device bytes per grid pool block: two grids for CK, one for the quadratic twin."""
    return BYTES_PER_POOL_BLOCK_CK if (kernel & 1) == 0 else BYTES_PER_POOL_BLOCK_CK // 2 + 4


def scene_resources(n: int, res: int) -> Dict[str, int]:
    """Engine resources a scene of n particles on a res^3 grid reserves.

    Pool blocks are reserved generously: a compact scene at 8 particles per
    cell touches about n/340 grid blocks; n/64 + 64 leaves room for it to
    spread, and the total over resident scenes stays below the pool size, so
    a step can never overflow the pool."""
    npb = -(-res // 4)
    nb = npb + 1
    return {"particles": n, "keys": npb ** 3, "virtual_blocks": nb ** 3,
            "pool_blocks": min(nb ** 3, n // 64 + 64), "scenes": 1}


@dataclasses.dataclass
class Budget:
    """Capacities of one context derived from a device-memory budget."""
    particles: int
    keys: int
    virtual_blocks: int
    pool_blocks: int
    scenes: int

    @staticmethod
    def from_bytes(budget: int, max_res: int = 128, max_scenes: int = 64, kernel: int = 0) -> "Budget":
        """Split a byte budget: key space and block tables sized for max_scenes
        scenes of max_res^3; the rest shared by particles and pool blocks in the
        ratio a compact 8-ppc scene uses them (n/64 pool blocks per particle).
        kernel: the context's kernel argument (kernel | transfer flag)."""
        r = scene_resources(0, max_res)
        keys = r["keys"] * max_scenes
        vblocks = r["virtual_blocks"] * max_scenes
        rest = budget - keys * BYTES_PER_KEY - vblocks * BYTES_PER_VIRTUAL_BLOCK
        if rest <= 0:
            raise ValueError("budget too small for the key space and block tables")
        pool_blocks_extra = 64 * max_scenes
        rest -= pool_blocks_extra * bytes_per_pool_block(kernel)
        if rest <= 0:
            raise ValueError("budget too small for the key space and block tables")
        per_particle = bytes_per_particle(kernel) + bytes_per_pool_block(kernel) / 64.0
        particles = int(rest // per_particle)
        return Budget(particles, keys, vblocks, particles // 64 + pool_blocks_extra, max_scenes)

    def fits(self, used: Dict[str, int], need: Dict[str, int]) -> bool:
        cap = dataclasses.asdict(self)
        return all(used.get(k, 0) + v <= cap[k] for k, v in need.items())


@dataclasses.dataclass
class Request:
    scene: object            # paper_2412_10399_gb300.scenes.Scene
    steps: int
    arrival_s: float = 0.0
    read_fields: Sequence[int] = (0,)  # fields read back when finished (default: positions)


@dataclasses.dataclass
class Result:
    request: Request
    admitted_at_step: int
    finished_at_step: int
    queue_s: float
    fields: Dict[int, object]
    admitted_s: float = 0.0   # wall time (from the server's start) of admission
    finished_s: float = 0.0   # wall time at which the result was read back


class EngineCK:
    """The C-ABI multi-scene context behind the serving loop."""

    def __init__(self, budget: Budget, kernel: int = 0, stream: Optional[int] = None):
        import torch

        from . import ckmpm as ck
        self.ck = ck
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream_ptr = stream
        self.stream = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
        cfg = ck.ckmpm_config()
        cfg.kernel = kernel
        cfg.max_particles = budget.particles
        cfg.max_keys = budget.keys
        cfg.max_grid_blocks = budget.pool_blocks
        cfg.max_virtual_blocks = budget.virtual_blocks
        cfg.max_scenes = budget.scenes
        cfg.max_materials = 4 * budget.scenes
        cfg.stream = stream
        self.ctx = ck.ckmpm_create_server(cfg)
        self.kernel = kernel
        self._events = []

    def admit(self, scene) -> int:
        sc, keep = self.ck.scene_struct(scene)
        try:
            return self.ck.ckmpm_admit(self.ctx, sc)
        except self.ck.CKMPMError as e:
            if e.status == self.ck.ENOMEM:
                raise MemoryError(str(e)) from e
            raise

    def release(self, sid: int):
        self.ck.ckmpm_release(self.ctx, sid)

    class _Pending:
        """A global step in flight: its event pair, returned to the engine's
        pool once its time has been read."""

        def __init__(self, eng, a, b):
            self.eng, self.a, self.b = eng, a, b

        def done(self) -> bool:
            return self.b.query()

        def ms(self) -> float:
            self.b.synchronize()
            t = self.a.elapsed_time(self.b)
            self.eng._events.append((self.a, self.b))
            return t

    def step_async(self) -> "EngineCK._Pending":
        """Enqueue one global step between two CUDA events; does not wait."""
        a, b = self._events.pop() if self._events else (self.torch.cuda.Event(enable_timing=True),
                                                          self.torch.cuda.Event(enable_timing=True))
        a.record(self.stream)
        self.ck.ckmpm_step(self.ctx, 1)
        b.record(self.stream)
        return EngineCK._Pending(self, a, b)

    def step(self) -> float:
        """One global step; returns its device time in ms (waits for it)."""
        return self.step_async().ms()

    def read(self, sid: int, field: int, n: int):
        import numpy as np
        shape = (n,) + self.ck._FIELD_SHAPE[field]
        out = np.empty(shape, np.float32)
        self.ck.ckmpm_readback(self.ctx, sid, field, out.ctypes.data, out.nbytes, False)
        return out

    def close(self):
        if self.ctx:
            self.ck.ckmpm_destroy(self.ctx)
            self.ctx = None


class Server:
    """Continuous-batching loop: FIFO admission under a resource budget,
    global steps enqueued without waiting (at most max_inflight ahead)."""

    def __init__(self, engine, budget: Budget, clock: Callable[[], float] = time.perf_counter,
                 max_inflight: int = 8):
        self.engine = engine
        self.budget = budget
        self.clock = clock
        self.max_inflight = max(1, max_inflight)
        self.waiting: List[Request] = []
        self.resident: Dict[int, dict] = {}
        self.used: Dict[str, int] = {}
        self.results: List[Result] = []
        self.latencies_ms: List[float] = []
        self.inflight = collections.deque()  # (pending step, number of scenes it advanced)
        self.step_count = 0
        self.particle_steps = 0
        self.busy_ms = 0.0
        self.t0 = clock()

    def submit(self, req: Request):
        need = scene_resources(req.scene.n, req.scene.res)
        if not self.budget.fits({}, need):
            raise ValueError("request larger than the whole budget")
        self.waiting.append(req)

    def _admit_ready(self, now: float):
        while self.waiting and self.waiting[0].arrival_s <= now:
            req = self.waiting[0]
            need = scene_resources(req.scene.n, req.scene.res)
            if not self.budget.fits(self.used, need):
                break  # FIFO: later requests wait behind the head
            try:
                sid = self.engine.admit(req.scene)
            except MemoryError:
                self._blocked = True  # released scenes' particles leave the pool at the next step
                break
            for k, v in need.items():
                self.used[k] = self.used.get(k, 0) + v
            self.resident[sid] = {"req": req, "left": req.steps, "need": need, "admitted": self.step_count,
                                  "queue_s": max(0.0, now - req.arrival_s), "admitted_s": now}
            self.waiting.pop(0)

    def _harvest(self, wait: bool = False):
        """Account the device time of finished global steps (all of those in
        flight with wait=True, else only those already done)."""
        while self.inflight and (wait or self.inflight[0][0].done()):
            pending, k = self.inflight.popleft()
            ms = pending.ms()
            self.busy_ms += ms
            self.latencies_ms.extend([ms] * k)

    def _retire_finished(self):
        for sid in [s for s, r in self.resident.items() if r["left"] == 0]:
            r = self.resident.pop(sid)
            req = r["req"]
            fields = {f: self.engine.read(sid, f, req.scene.n) for f in req.read_fields}
            self.engine.release(sid)
            for k, v in r["need"].items():
                self.used[k] -= v
            self.results.append(Result(req, r["admitted"], self.step_count, r["queue_s"], fields,
                                       admitted_s=r["admitted_s"], finished_s=self.clock() - self.t0))

    def poll(self) -> bool:
        """Harvest finished steps, admit, enqueue one global step if anything
        is resident, retire.  Returns False once nothing is waiting, resident
        or in flight."""
        now = self.clock() - self.t0
        self._harvest()
        self._blocked = False
        self._admit_ready(now)
        if self._blocked and not self.resident:
            # nothing resident: one step only compacts the pool (the released
            # scenes' particles leave it); the host's capacity count follows
            self.engine.step_async().ms()
            self._admit_ready(now)
        if self.resident:
            if len(self.inflight) >= self.max_inflight:
                pending, k = self.inflight.popleft()
                ms = pending.ms()
                self.busy_ms += ms
                self.latencies_ms.extend([ms] * k)
            self.inflight.append((self.engine.step_async(), len(self.resident)))
            self.step_count += 1
            for r in self.resident.values():
                r["left"] -= 1
                self.particle_steps += r["req"].scene.n
            self._retire_finished()
        if not (self.waiting or self.resident):
            self._harvest(wait=True)
        return bool(self.waiting or self.resident or self.inflight)

    def run(self, sleep: Callable[[float], None] = time.sleep):
        while self.poll():
            if not self.resident and self.waiting and not self.inflight:
                wait = self.waiting[0].arrival_s - (self.clock() - self.t0)
                if wait > 0:
                    sleep(min(wait, 0.01))
        return self.results

    def stats(self) -> dict:
        def pick(vals, q):
            v = sorted(vals)
            return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)] if v else None

        wall = self.clock() - self.t0
        e2e = [r.finished_s - r.request.arrival_s for r in self.results]
        per_step = [1e3 * (r.finished_s - r.admitted_s) / max(1, r.request.steps) for r in self.results]
        return {"p50_ms": pick(self.latencies_ms, 0.50), "p99_ms": pick(self.latencies_ms, 0.99),
                "scene_steps": len(self.latencies_ms),
                "global_steps": self.step_count, "scenes_finished": len(self.results),
                "aggregate_particle_steps_per_s": self.particle_steps / (self.busy_ms / 1e3) if self.busy_ms else None,
                "wall_particle_steps_per_s": self.particle_steps / wall if wall > 0 else None,
                "mean_queue_s": (sum(r.queue_s for r in self.results) / len(self.results)) if self.results else None,
                "request_latency_p50_s": pick(e2e, 0.50), "request_latency_p99_s": pick(e2e, 0.99),
                "resident_wall_ms_per_step_p50": pick(per_step, 0.50),
                "resident_wall_ms_per_step_p99": pick(per_step, 0.99)}
