"""Serving loop over a multi-scene CK-MPM context (continuous batching).

Requests (a scene and a number of steps) arrive over time.  All resident
scenes advance together: every global step is one launch per kernel over the
concatenated block lists of every scene in the context.  Between global steps
the loop retires finished scenes (reading back their final state) and admits
waiting requests, first come first served, as soon as the device-memory
budget they need is free.  Each scene-step's latency is the device time of the
global step it belonged to; p50 / p99 are reported beside the throughput.

The admission arithmetic is plain host code (``Budget``); the engine is any
object with the ``admit / release / step / read`` methods of ``EngineCK``.
"""
from __future__ import annotations

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

    def step(self) -> float:
        """One global step; returns its device time in ms."""
        a = self.torch.cuda.Event(enable_timing=True)
        b = self.torch.cuda.Event(enable_timing=True)
        a.record(self.stream)
        self.ck.ckmpm_step(self.ctx, 1)
        b.record(self.stream)
        b.synchronize()
        return a.elapsed_time(b)

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
    """Continuous-batching loop: FIFO admission under a resource budget."""

    def __init__(self, engine, budget: Budget, clock: Callable[[], float] = time.perf_counter):
        self.engine = engine
        self.budget = budget
        self.clock = clock
        self.waiting: List[Request] = []
        self.resident: Dict[int, dict] = {}
        self.used: Dict[str, int] = {}
        self.results: List[Result] = []
        self.latencies_ms: List[float] = []
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
                                  "queue_s": max(0.0, now - req.arrival_s)}
            self.waiting.pop(0)

    def _retire_finished(self):
        for sid in [s for s, r in self.resident.items() if r["left"] == 0]:
            r = self.resident.pop(sid)
            req = r["req"]
            fields = {f: self.engine.read(sid, f, req.scene.n) for f in req.read_fields}
            self.engine.release(sid)
            for k, v in r["need"].items():
                self.used[k] -= v
            self.results.append(Result(req, r["admitted"], self.step_count, r["queue_s"], fields))

    def poll(self) -> bool:
        """Admit, run one global step if anything is resident, retire.  Returns
        False once nothing is waiting or resident."""
        now = self.clock() - self.t0
        self._blocked = False
        self._admit_ready(now)
        if self._blocked and not self.resident:
            self.engine.step()  # nothing resident: this step only compacts the pool
            self._admit_ready(now)
        if self.resident:
            ms = self.engine.step()
            self.step_count += 1
            self.busy_ms += ms
            for r in self.resident.values():
                r["left"] -= 1
                self.latencies_ms.append(ms)
                self.particle_steps += r["req"].scene.n
            self._retire_finished()
        return bool(self.waiting or self.resident)

    def run(self, sleep: Callable[[float], None] = time.sleep):
        while self.poll():
            if not self.resident and self.waiting:
                wait = self.waiting[0].arrival_s - (self.clock() - self.t0)
                if wait > 0:
                    sleep(min(wait, 0.01))
        return self.results

    def stats(self) -> dict:
        lat = sorted(self.latencies_ms)
        pick = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)] if lat else None
        wall = self.clock() - self.t0
        return {"p50_ms": pick(0.50), "p99_ms": pick(0.99), "scene_steps": len(lat),
                "global_steps": self.step_count, "scenes_finished": len(self.results),
                "aggregate_particle_steps_per_s": self.particle_steps / (self.busy_ms / 1e3) if self.busy_ms else None,
                "wall_particle_steps_per_s": self.particle_steps / wall if wall > 0 else None,
                "mean_queue_s": (sum(r.queue_s for r in self.results) / len(self.results)) if self.results else None}
