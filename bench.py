#!/usr/bin/env python
"""Benchmark of the CK-MPM step on GB300 (prints one JSON line).

Workload: the 16,273,664-particle large-impact scene on a 512^3 virtual grid
(Drucker-Prager sand castle hit by four stiff fixed-corotated balls, dt 2e-5).
One step = binning + P2G + grid update + fused G2P/constitutive for every
particle.  Metric: particle-steps/s (whole job); the quadratic B-spline path
runs the same scene for comparison, and a short served mix reports p50/p99
step latency.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload.  With torchrun (N > 1) every rank runs its own
replica of the scene (weak scaling, no collective on the data path); rank 0
prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 16M particles vs quadratic B-spline; served step p50/p99"
UNIT = "particle-steps/s"
WORKLOAD = "large_impact: 512^3 virtual grid (dx 1/512), DP sand castle + 4 FC balls (E 1e7) at 20 m/s, 16,273,664 particles, 8 ppc, dt 2e-5"

# Algorithmic bytes per particle of each kernel (float32 state, one pass over each array):
#   P2G: read x 12 + v 12 + M 36 B, write 2 grids x 16 B per node at 1/8 node per particle = 4 B -> 64 B
#   G2P: read x 12 + F 36, gather 2 grids x 12 B / 8 = 3, write x 12 + v 12 + M 36 + F 36 -> 147 B
#   grid update: per node read 16 + write 12 B, 2 grids / 8 -> 7 B
ALGO_BYTES = {"p2g": 64.0, "g2p": 147.0, "grid_update": 7.0}
# whole-step algorithmic bytes per particle of the compact kernel under each
# transfer: PIC moves the same arrays; the kernel-gradient APIC adds its
# 36-byte stress term to P2G's reads and G2P's writes
STEP_BYTES = {"apic_mls": sum(ALGO_BYTES.values()), "pic": sum(ALGO_BYTES.values()),
              "apic_grad": sum(ALGO_BYTES.values()) + 72.0}
KERNEL_SLOT = {"bin": 0, "scatter": 1, "p2g": 2, "grid_update": 3, "g2p": 4, "grid_list": 5, "g2p_fp64": 6,
               "g2p2g": 7}
# The method's floor for one step: particle state x, v, B, F read and written
# once (192 B) plus the dual grid (14 B per particle at 8 per cell)
METHOD_FLOOR_BYTES = 206.0


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("common.cuh", "launch.h", "svd3.cuh", "transfer.cu")


def _source_hash():
    """Hash of the sources that define the P2G / grid / G2P kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2412_10399_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profile_value(kernel, field):
    """A figure from the committed ncu summary of a kernel, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", f"traffic_{kernel}_large_impact.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != _source_hash():
        return None
    try:
        return float(kv[field])
    except (KeyError, ValueError):
        return None


def _traffic(kernel):
    """DRAM bytes per launch of a kernel on the full scene (ncu, scaled)."""
    return _profile_value(kernel, "dram_bytes_per_launch_full_size")


def fp32_sgemm_tflops(n=8192, reps=3):
    """Measured FP32 ceiling of this GPU's CUDA cores: a cuBLAS SGEMM with
    TF32 off (the FP32 counterpart of the bf16 GEMM behind the HBM and tensor
    peaks), CUDA events around `reps` products after one warm-up."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        g = torch.Generator(device="cuda").manual_seed(0)
        a = torch.randn(n, n, device="cuda", generator=g)
        b = torch.randn(n, n, device="cuda", generator=g)
        torch.matmul(a, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            c = torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        del a, b, c
        torch.cuda.empty_cache()
        return 2.0 * n ** 3 * reps / (ms / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def aggregate_ranks(ms_local: float, particles_local: int, steps: int, dist=None, device="cpu"):
    """Whole-job throughput across ranks (weak scaling, one replica per rank):
    the slowest rank's time over the particles all ranks advanced.  Returns
    (value particle-steps/s, max ms).  With dist=None this is the one-rank case."""
    import torch
    if dist is None:
        return particles_local * steps / (ms_local / 1e3), ms_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([particles_local], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return float(n.item()) * steps / (ms / 1e3), ms


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()  # wait for the first sample so the timed region is covered
        while time.time() - t0 < 10 and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------- CPU leg

def _cpu_sample():
    """A bounded sample of the workload for the FP64 oracle: the castle base in
    a 64 x 32 x 64-cell window (cells [160,224) x [4,36) x [160,224) of the
    512^3 scene), shifted into its own 80^3 domain with the same dx, dt and
    material: 1,048,576 particles."""
    from paper_2412_10399_gb300 import scenes as S
    res = 512
    dx = 1.0 / res
    cells = S.filled_cells([S._box([160, 4, 160], [224, 36, 224])], res)
    x = S.sample_cells(cells, res, dx, seed=0)
    x = x - np.array([152, 0, 152]) * dx
    sc = S.Scene("large_impact_window", 80, dx, 2e-5, x, np.zeros_like(x), np.zeros(len(x), np.uint8),
                 [S.SAND], steps=2)
    return sc


def _cpu_model():
    """CPU model string of the host (from /proc/cpuinfo where present)."""
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu part", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(steps: int = 2):
    import torch
    from oracle import ckmpm_oracle as O
    sc = _cpu_sample()
    prm = O.params_from_scene(sc)
    st = O.state_from_scene(sc)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = O.step(st, prm)
    dt = time.perf_counter() - t0
    return {"value": sc.n * steps / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "host": f"{os.cpu_count()} logical CPUs, {_cpu_model()}",
            "sample": f"{sc.n} particles (castle-base window of the 16.27M scene, same dx/dt/material), "
                      f"{steps} FP64 steps, {dt:.1f} s"}


def run_reference(args):
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    warm = max(0, min(args.warmup, 1))
    if warm:
        cpu_baseline(steps=1)
    cb = cpu_baseline(steps=min(steps, 3))
    full_n = 16273664
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": min(steps, 3), "warmup": warm, "ms_per_step": full_n / cb["value"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"],
                       "ms_per_step": f"a step of the {full_n:,}-particle workload at the sample's rate"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- GPU leg

def _make_ctx(ck, scene, kernel, stream, timing=False):
    sc, keep = ck.scene_struct(scene)
    ctx = ck.ckmpm_create(sc, kernel, stream)
    if timing:
        ck.ckmpm_set_timing(ctx, True)
    return ctx, keep


def _kernel_breakdown(ck, scene, kernel, stream_ptr, warmup, steps):
    """Average device ms per launch of each kernel over the same W + K steps,
    from CUDA events recorded around every launch on the context's stream;
    also the largest per-step count of float64-pass particles seen."""
    ctx, keep = _make_ctx(ck, scene, kernel, stream_ptr)
    ck.ckmpm_step(ctx, warmup)
    ck.ckmpm_sync(ctx)
    ck.ckmpm_set_timing(ctx, True)
    ck.ckmpm_reset_timing(ctx)
    fp64_max = 0
    for _ in range(steps):
        ck.ckmpm_step(ctx, 1)
        if steps <= 400:
            fp64_max = max(fp64_max, int(ck.ckmpm_get_stats(ctx).fp64_particles))
    ck.ckmpm_sync(ctx)
    st = ck.ckmpm_get_stats(ctx)
    ck.ckmpm_destroy(ctx)
    return {k: st.ms_kernel[i] for k, i in KERNEL_SLOT.items()}, fp64_max


def _time_steps(ck, ctx, steps, stream_ptr):
    import torch
    stream = torch.cuda.ExternalStream(stream_ptr)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    ck.ckmpm_step(ctx, steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def end_to_end(ck, scene, stream_ptr, world, steps):
    """The headline metric through the public API from pinned host memory:
    admit the scene from host x/v/mat, then every step ckmpm_step and an
    asynchronous readback of all positions to pinned host memory; the host
    waits for step k's positions after enqueueing step k+1, so the copy of one
    step overlaps the next.  The timed region spans admission to the last
    position on the host.  The breakdown times admission alone and one
    gather + copy alone (after the loop, with the device idle)."""
    import torch
    n = scene.n
    xh = torch.from_numpy(scene.x32()).pin_memory()
    vh = torch.from_numpy(scene.v32()).pin_memory()
    mh = torch.from_numpy(scene.mat.copy()).pin_memory()
    outs = [torch.empty((n, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    nbytes = n * 12
    cfg = ck.ckmpm_config()
    cfg.kernel = ck.KERNEL_CK
    cfg.max_particles = n
    cfg.max_keys = 128 ** 3
    cfg.max_virtual_blocks = 129 ** 3
    cfg.max_grid_blocks = n // 64 + 4096
    cfg.max_scenes = 1
    cfg.max_materials = len(scene.materials)
    cfg.stream = stream_ptr
    srv = ck.ckmpm_create_server(cfg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sc, keep = ck.make_scene(scene.res, scene.dx, scene.dt, scene.materials, xh.numpy(), vh.numpy(),
                             mh.numpy(), gravity=scene.gravity, bc_cells=scene.bc_cells, ppc=scene.ppc)
    sid = ck.ckmpm_admit(srv, sc)
    prev = None
    for k in range(steps):
        ck.ckmpm_step(srv, 1)
        t = ck.ckmpm_readback_async(srv, sid, ck.FIELD_X, outs[k & 1].data_ptr(), nbytes)
        if prev is not None:
            ck.ckmpm_readback_wait(srv, prev)  # step k-1's positions are on the host
        prev = t
    ck.ckmpm_readback_wait(srv, prev)
    t_e2e = time.perf_counter() - t0
    # breakdown, outside the timed region
    ck.ckmpm_sync(srv)
    tc = time.perf_counter()
    for _ in range(3):
        ck.ckmpm_readback_wait(srv, ck.ckmpm_readback_async(srv, sid, ck.FIELD_X, outs[0].data_ptr(), nbytes))
    t_copy = (time.perf_counter() - tc) / 3
    ck.ckmpm_release(srv, sid)
    ck.ckmpm_step(srv, 1)
    ck.ckmpm_sync(srv)
    ta = time.perf_counter()
    sid = ck.ckmpm_admit(srv, sc)
    ck.ckmpm_sync(srv)
    t_admit = time.perf_counter() - ta
    ck.ckmpm_destroy(srv)
    del keep
    return {"value": world * n * steps / t_e2e, "unit": UNIT,
            "h2d_bytes_per_step": int((xh.numel() * 4 + vh.numel() * 4 + mh.numel()) / steps),
            "d2h_bytes_per_step": nbytes, "steps": steps, "wall_s": t_e2e,
            "admit_s": t_admit, "readback_s": t_copy, "readback_gbs": nbytes / t_copy / 1e9,
            "how": "admit from pinned host x/v/mat, then per step: ckmpm_step + ckmpm_readback_async of all "
                   "positions to pinned host (waited one step later, so the copy overlaps the next step); "
                   "admit_s and readback_s are each timed alone after the loop"}


def served_mix(ck, stream_ptr, n_scenes=64, steps=1000, n_max=2e6, seed=0, budget_bytes=24 << 30,
               max_scenes=16, compress=20.0):
    """Continuous batching of a Poisson stream of scenes (served-mix
    configuration: 64 scenes, N log-uniform in [1e4, 2e6], 1000 steps each)
    through the serving loop: admission by a device-memory budget, one launch
    per kernel per global step over every resident scene, steps enqueued
    without waiting, retirement with readback."""
    from paper_2412_10399_gb300 import scenes as S
    from paper_2412_10399_gb300 import serving as SV
    reqs = S.served_mix(n_scenes=n_scenes, seed=seed, n_max=n_max, steps=steps)
    budget = SV.Budget.from_bytes(budget_bytes, max_res=128, max_scenes=max_scenes)
    eng = SV.EngineCK(budget, stream=stream_ptr)
    srv = SV.Server(eng, budget)
    for r in reqs:
        srv.submit(SV.Request(r.scene, r.scene.steps, arrival_s=r.arrival_s / compress, read_fields=(ck.FIELD_X,)))
    srv.run()
    st = srv.stats()
    eng.close()
    st.update({"scenes": n_scenes, "steps_per_scene": steps, "budget_bytes": budget_bytes,
               "particles_total": int(sum(r.scene.n for r in reqs)),
               "mix": f"{n_scenes} scenes, N log-uniform in [1e4, {n_max:.0f}], box/sphere, elastic or sand, "
                      f"{steps} steps each, Poisson arrivals (20 ms mean, time-compressed x{compress:g}), admitted "
                      f"under a {budget_bytes >> 30} GiB device budget (at most {max_scenes} resident)",
               "latency": "p50_ms/p99_ms: device time of the global step a scene step belonged to; "
                          "request_latency_*: arrival to result (queue + admission + steps + readback); "
                          "resident_wall_ms_per_step_*: a request's wall time per step while resident"})
    return st


def impact_window(ck, scene, stream_ptr, start=75, steps=20):
    """Steps start..start+steps of the large-impact scene, after the balls
    reach the keep (about step 73): CK ms per step with no per-kernel events,
    then the same window again with events around each launch; the largest
    float64-pass count of a step in the window."""
    ctx, keep = _make_ctx(ck, scene, ck.KERNEL_CK, stream_ptr)
    ck.ckmpm_step(ctx, start)
    ck.ckmpm_sync(ctx)
    ms = _time_steps(ck, ctx, steps, stream_ptr)
    ck.ckmpm_sync(ctx)
    ck.ckmpm_destroy(ctx)
    per_kernel, fp64_max = _kernel_breakdown(ck, scene, ck.KERNEL_CK, stream_ptr, start, steps)
    return {"steps": f"{start}..{start + steps}", "ms_per_step": ms / steps, "value": scene.n * steps / (ms / 1e3),
            "per_kernel_ms": per_kernel, "fp64_particles_max_step": fp64_max}


def granular_column_lines(ck, stream_ptr, peak=None, steps=500):
    """Granular column collapse (346,112 Drucker-Prager particles, 128^3,
    dt 5e-5): all of its 500 steps, CK and the quadratic twin on identical
    inputs, split and fused steps, device-resident."""
    from paper_2412_10399_gb300 import scenes as S
    sc = S.granular_column()
    out = {}
    for name, kernel in (("ck", ck.KERNEL_CK), ("quadratic", ck.KERNEL_QUADRATIC),
                         ("ck_fused", ck.KERNEL_CK | ck.STEP_G2P2G),
                         ("quadratic_fused", ck.KERNEL_QUADRATIC | ck.STEP_G2P2G)):
        warm, keep = _make_ctx(ck, sc, kernel, stream_ptr)  # loads the kernels: the timed run starts at step 0
        ck.ckmpm_step(warm, 3)
        ck.ckmpm_destroy(warm)
        ctx, keep = _make_ctx(ck, sc, kernel, stream_ptr)
        ms = _time_steps(ck, ctx, steps, stream_ptr)
        ck.ckmpm_sync(ctx)
        ck.ckmpm_destroy(ctx)
        out[name] = {"ms_per_step": ms / steps, "value": sc.n * steps / (ms / 1e3)}
    out["ck_speedup"] = out["quadratic"]["ms_per_step"] / out["ck"]["ms_per_step"]
    if peak:
        out["ck"]["step_frac"] = _step_frac(STEP_BYTES["apic_mls"], sc.n, out["ck"]["ms_per_step"], peak)
    out["workload"] = (f"granular column: 128^3, column cells [51,77)x[4,68)x[51,77), {sc.n} particles at 8 per "
                       f"cell, DP sand E 3.5e5 nu 0.3 phi 30 rho 1600, dt 5e-5; steps 0..{steps}")
    return out


def fused_lines(ck, scene, stream_ptr, warmup, steps, peak=None):
    """The fused G2P2G step (CKMPM_STEP_G2P2G) on the headline scene and
    window, CK and quadratic, device-resident, with per-kernel times from a
    second run; with peak (GB/s), the CK step against the method floor."""
    out = {}
    for name, kernel in (("ck", ck.KERNEL_CK), ("quadratic", ck.KERNEL_QUADRATIC)):
        ctx, keep = _make_ctx(ck, scene, kernel | ck.STEP_G2P2G, stream_ptr)
        ck.ckmpm_step(ctx, warmup)
        ck.ckmpm_sync(ctx)
        ms = _time_steps(ck, ctx, steps, stream_ptr)
        ck.ckmpm_sync(ctx)
        lo = int(ck.ckmpm_get_stats(ctx).leftover_particles)
        ck.ckmpm_destroy(ctx)
        per_kernel, _ = _kernel_breakdown(ck, scene, kernel | ck.STEP_G2P2G, stream_ptr, warmup, steps)
        out[name] = {"ms_per_step": ms / steps, "value": scene.n * steps / (ms / 1e3), "per_kernel_ms": per_kernel,
                     "leftover_particles_last_step": lo}
    if peak:
        out["ck"]["method_floor_frac"] = _step_frac(METHOD_FLOOR_BYTES, scene.n, out["ck"]["ms_per_step"], peak)
    out["workload"] = f"{WORKLOAD}, steps {warmup}..{warmup + steps}"
    return out


def diff_lines(stream_ptr, steps=64, k=8):
    """Differentiable configuration (262,144 particles, 128^3, 64 steps,
    checkpoints every 8): forward ms per step, adjoint ms per step, and a
    whole rollout (forward, then backward with recomputation from the
    checkpoints) through torch.autograd."""
    import torch
    from paper_2412_10399_gb300 import diff as D
    from paper_2412_10399_gb300 import scenes as S
    sc = S.differentiable_cube()
    dev = torch.device("cuda")
    sim = D.DiffSim(sc, stream=stream_ptr)
    stream = torch.cuda.ExternalStream(stream_ptr)
    x0 = torch.from_numpy(sc.x32()).to(dev)
    v0 = torch.from_numpy(sc.v32()).to(dev)
    E = torch.full((sc.n,), float(sc.materials[0].E), dtype=torch.float32, device=dev)
    B0, F0 = D.initial_state(x0)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        s = (x0, v0, B0, F0)
        s = sim.step(*s, E)  # loads the kernels
        torch.cuda.synchronize()
        states = [(x0, v0, B0, F0)]
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(steps):
            states.append(sim.step(*states[-1], E))
        b.record(stream)
        torch.cuda.synchronize()
        fwd = a.elapsed_time(b) / steps
        gE = torch.zeros_like(E)
        adj = tuple(torch.zeros_like(t) for t in states[-1])
        adj = (torch.ones_like(adj[0]),) + adj[1:]
        a.record(stream)
        for j in reversed(range(steps)):
            adj = sim.step_backward(*states[j], E, *adj, gE)
        b.record(stream)
        torch.cuda.synchronize()
        bwd = a.elapsed_time(b) / steps
        roll = []
        for _ in range(2):  # the first rollout also pays one-off loading costs; the second is reported
            x0r, v0r = x0.clone().requires_grad_(True), v0.clone().requires_grad_(True)
            Er = E.clone().requires_grad_(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xT, vT = D.Rollout.apply(x0r, v0r, Er, sim, steps, k)
            loss = D.com_loss(xT, xT.detach().mean(0) + 0.01)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            loss.backward()
            torch.cuda.synchronize()
            roll.append((t1 - t0, time.perf_counter() - t1))
    sim.close()
    return {"forward_ms_per_step": fwd, "adjoint_ms_per_step": bwd, "adjoint_over_forward": bwd / fwd,
            "rollout_forward_s": roll[1][0], "rollout_backward_s": roll[1][1],
            "rollout_first_call_s": roll[0][0] + roll[0][1],
            "particles": sc.n, "steps": steps, "checkpoint_every": k,
            "workload": "differentiable cube: 128^3, cells [48,80)^3, 262,144 FC particles, dt 1e-4, v = (0.5,0,0) "
                        "+ N(0, 0.5^2); the rollout's backward replays each 8-step segment from its checkpoint"}


# The paper's G2P2G kernel times per substep for the dam-break scenes (its
# performance table; RTX 3090, CK and the quadratic kernel of Wang 2020), for
# context only: another machine and a fused kernel.
PAPER_DAM_BREAK_MS = {4175808: {"ck": 2.9, "quadratic": 3.7}, 8994048: {"ck": 5.7, "quadratic": 7.2}}


def _step_frac(bytes_per_particle, n, ms_per_step, peak_gbs):
    """Whole-step algorithmic bandwidth as a fraction of the HBM peak."""
    return bytes_per_particle * n / (ms_per_step / 1e3) / 1e9 / peak_gbs


def dam_break_lines(ck, stream_ptr, warmup, steps, sizes=(4175808, 8994048), peak=None):
    """The paper's dam-break workload (J-based fluid, 256^3): CK and quadratic
    ms per step over the same steps, device-resident, no per-kernel events;
    with peak (GB/s), the CK step's fraction of it."""
    from paper_2412_10399_gb300 import scenes as S
    out = {}
    for n in sizes:
        sc = S.dam_break(n)
        row = {}
        for name, kernel in (("ck", ck.KERNEL_CK), ("quadratic", ck.KERNEL_QUADRATIC)):
            ctx, keep = _make_ctx(ck, sc, kernel, stream_ptr)
            ck.ckmpm_step(ctx, warmup)
            ck.ckmpm_sync(ctx)
            ms = _time_steps(ck, ctx, steps, stream_ptr)
            ck.ckmpm_sync(ctx)
            ck.ckmpm_destroy(ctx)
            row[name] = {"ms_per_step": ms / steps, "value": n * steps / (ms / 1e3)}
        row["ck_speedup"] = row["quadratic"]["ms_per_step"] / row["ck"]["ms_per_step"]
        if peak:
            row["ck"]["step_frac"] = _step_frac(STEP_BYTES["apic_mls"], n, row["ck"]["ms_per_step"], peak)
        row["paper_g2p2g_ms_rtx3090"] = PAPER_DAM_BREAK_MS.get(n)
        out[str(n)] = row
    out["workload"] = ("J-based fluid (B = 10 Pa, gamma = 7.15, rho = 1000), uniform in a cuboid at 8 per cell, "
                       f"256^3, dt 1e-4; steps {warmup}..{warmup + steps}")
    return out


def transfer_lines(ck, scene, stream_ptr, warmup, steps, peak=None):
    """The kernel-gradient transfers on the headline scene and window: PIC
    (Sec. 4.3) and APIC with the kernel gradient (Sec. 4.4 with the force and
    grad v of Sec. 4.3); CK and quadratic ms per step, device-resident, no
    per-kernel events; with peak (GB/s), the CK step's fraction of it."""
    out = {}
    for tname, flag in (("pic", ck.TRANSFER_PIC), ("apic_grad", ck.TRANSFER_APIC_GRAD)):
        row = {}
        for name, kernel in (("ck", ck.KERNEL_CK), ("quadratic", ck.KERNEL_QUADRATIC)):
            ctx, keep = _make_ctx(ck, scene, kernel | flag, stream_ptr)
            ck.ckmpm_step(ctx, warmup)
            ck.ckmpm_sync(ctx)
            ms = _time_steps(ck, ctx, steps, stream_ptr)
            ck.ckmpm_sync(ctx)
            ck.ckmpm_destroy(ctx)
            row[name] = {"ms_per_step": ms / steps, "value": scene.n * steps / (ms / 1e3)}
        row["ck_speedup"] = row["quadratic"]["ms_per_step"] / row["ck"]["ms_per_step"]
        if peak:
            row["ck"]["step_frac"] = _step_frac(STEP_BYTES[tname], scene.n, row["ck"]["ms_per_step"], peak)
        out[tname] = row
    out["workload"] = f"{WORKLOAD}, steps {warmup}..{warmup + steps}"
    return out


def run_gpu(args):
    import torch
    rank, local_rank, world = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2412_10399_gb300 import ckmpm as ck
    from paper_2412_10399_gb300 import scenes as S

    stream_ptr = torch.cuda.Stream().cuda_stream
    scene = S.large_impact(seed=rank)
    if args.max_particles and args.max_particles < scene.n:
        k = args.max_particles
        scene.x, scene.v, scene.mat = scene.x[:k], scene.v[:k], scene.mat[:k]
    n = scene.n

    # ---------------- device-resident timing of the CK path: W untimed steps,
    # then K timed steps with no per-kernel events; the per-kernel breakdown
    # comes from a second run over the same steps with events around each launch
    ctx, keep = _make_ctx(ck, scene, ck.KERNEL_CK, stream_ptr)
    ck.ckmpm_step(ctx, args.warmup)
    ck.ckmpm_sync(ctx)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms = _time_steps(ck, ctx, args.steps, stream_ptr)
    clocks = sampler.stop()
    ck.ckmpm_sync(ctx)
    st = ck.ckmpm_get_stats(ctx)
    value, ms = aggregate_ranks(ms, n, args.steps, dist, device="cuda")
    if dist:
        dist.barrier()
    launches = int(st.launches_per_step) * args.steps
    fp64_frac = st.fp64_particles / max(1, n)
    n_pb, n_gb = int(st.n_particle_blocks), int(st.n_grid_blocks)
    ck.ckmpm_destroy(ctx)
    per_kernel, fp64_max = _kernel_breakdown(ck, scene, ck.KERNEL_CK, stream_ptr, args.warmup, args.steps)

    dominant = max(("p2g", "g2p"), key=lambda k: per_kernel[k])
    peak, peak_src = _peaks()
    achieved = ALGO_BYTES[dominant] * n / (per_kernel[dominant] / 1e3) / 1e9
    traffic = _traffic(dominant)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "frac_of_nominal_7900_gbs": achieved / 7900.0,
                "algorithmic_bytes_per_particle": ALGO_BYTES[dominant], "traffic": traffic,
                "per_kernel_ms": per_kernel,
                "step_algorithmic_bytes_per_particle": sum(ALGO_BYTES.values()),
                "step_frac": sum(ALGO_BYTES.values()) * n / (ms / args.steps / 1e3) / 1e9 / peak,
                "method_floor_bytes_per_particle": METHOD_FLOOR_BYTES,
                "step_frac_method_floor": METHOD_FLOOR_BYTES * n / (ms / args.steps / 1e3) / 1e9 / peak}
    # the dominant kernel's FP32 arithmetic against the CUDA cores' ceiling
    # (FLOP per particle from the same ncu capture as its traffic)
    flops_pp = _profile_value(dominant, "fp32_flops_per_particle")
    sgemm = fp32_sgemm_tflops()
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    max_mhz = float(clocks.get("sm_max_mhz") or 2070.0)
    nominal_fp32 = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12
    alu_tf = flops_pp * n / (per_kernel[dominant] / 1e3) / 1e12 if flops_pp else None
    roofline["alu"] = {"fp32_flops_per_particle": flops_pp, "achieved_tflops": alu_tf,
                       "sgemm_tflops": sgemm, "frac_of_sgemm": alu_tf / sgemm if alu_tf else None,
                       "nominal_tflops": nominal_fp32, "frac_of_nominal": alu_tf / nominal_fp32 if alu_tf else None,
                       "note": "FP32 FLOP of the dominant kernel (2 FFMA + FMUL + FADD per the ncu counts) per "
                               "CUDA-event launch time, against a cuBLAS SGEMM with TF32 off and against "
                               "SMs x 128 lanes x 2 x max SM clock"}

    # ---------------- quadratic B-spline twin on the same inputs and steps
    qsteps = args.steps
    ctxq, keepq = _make_ctx(ck, scene, ck.KERNEL_QUADRATIC, stream_ptr)
    ck.ckmpm_step(ctxq, args.warmup)
    ck.ckmpm_sync(ctxq)
    msq = _time_steps(ck, ctxq, qsteps, stream_ptr)
    ck.ckmpm_sync(ctxq)
    ck.ckmpm_destroy(ctxq)
    per_kernel_q, _ = _kernel_breakdown(ck, scene, ck.KERNEL_QUADRATIC, stream_ptr, args.warmup, qsteps)
    quad = {"value": n * qsteps / (msq / 1e3), "ms_per_step": msq / qsteps, "steps": qsteps,
            "ck_speedup": (msq / qsteps) / (ms / args.steps), "per_kernel_ms": per_kernel_q}

    # ---------------- end to end through the C ABI with pinned host buffers
    e2e = end_to_end(ck, scene, stream_ptr, world, max(2, min(args.steps, 50)))

    served = served_mix(ck, stream_ptr) if not args.no_served else None
    dam = dam_break_lines(ck, stream_ptr, args.warmup, args.steps, peak=peak) if not args.no_dam else None
    transfers = (transfer_lines(ck, scene, stream_ptr, args.warmup, args.steps, peak=peak)
                 if not args.no_transfers else None)
    extra = not args.no_extra and not args.max_particles
    impact = impact_window(ck, scene, stream_ptr) if extra else None
    column = granular_column_lines(ck, stream_ptr, peak=peak) if extra else None
    fused = fused_lines(ck, scene, stream_ptr, args.warmup, args.steps, peak=peak) if not args.no_extra else None
    diffl = diff_lines(stream_ptr) if extra else None
    cb = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu) else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "particles_per_gpu": n, "particle_blocks": n_pb,
                           "grid_blocks": n_gb, "l2": "inputs larger than L2 (about 3.7 GB of particle state)",
                           "parallelism": "replicas" if world > 1 else "single",
                           "fp64_fraction_last_step": fp64_frac, "fp64_particles_max_step": fp64_max,
                           "timed": f"steps {args.warmup}..{args.warmup + args.steps} of the scene (ball impact on "
                                    f"the keep from about step 73)",
                           "per_kernel_ms": "second run over the same steps with CUDA events around each launch"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "quadratic": quad, "served": served, "dam_break": dam, "transfers": transfers,
                "impact": impact, "granular_column": column, "fused": fused, "diff": diffl}
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--max-particles", type=int, default=0,
                    help="keep only the first N particles of the scene (a slab of the castle base; "
                         "for profiling a smaller case)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-dam", action="store_true", help="skip the dam-break lines")
    ap.add_argument("--no-transfers", action="store_true", help="skip the kernel-gradient transfer lines")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the impact window, granular column, fused-step and differentiation lines")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
