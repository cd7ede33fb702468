"""Command line: inspect or run a scene description.

    python -m paper_2412_10399_gb300 info SCENE.json
        particle count, grid, materials and the device memory the scene needs
        (no GPU).
    python -m paper_2412_10399_gb300 run SCENE.json --steps N [--every K]
            [--kernel ck|quadratic] [--transfer apic_mls|pic|apic_grad]
            [--out DIR] [--resume CHECKPOINT.npz]
        steps the scene on the current CUDA device and writes a checkpoint
        (x, v, F, B) to DIR/frame_NNNNN.npz every K steps and at the end.

The scene format is the one scenes.scene_from_spec documents.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

from . import scenes as S
from . import serving as SV


def _apply_overrides(sc, args):
    if getattr(args, "kernel", None):
        sc.kernel = S._KERNELS[args.kernel]
    if getattr(args, "transfer", None):
        sc.transfer = S._TRANSFERS[args.transfer]
    return sc


def cfl_number(sc) -> float:
    """dt (c + |v|max) / dx with c the largest dilatational wave speed of the
    scene's materials, sqrt((lam + 2 mu) / rho) for the solids and
    sqrt(gamma B / rho) for the J-based fluid at rest volume; explicit MPM
    wants this well below 1."""
    import math
    c = 0.0
    for m in sc.materials:
        if m.model == S.J_FLUID:
            k = m.gamma * m.E
        else:
            k = m.E * (1.0 - m.nu) / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu))
        c = max(c, math.sqrt(k / m.rho))
    vmax = float(abs(sc.v).max()) if sc.n else 0.0
    return sc.dt * (c + vmax) / sc.dx


def scene_info(sc) -> dict:
    """What a scene holds and the device memory a context for it takes."""
    from .ckmpm import kernel_code
    code = kernel_code(sc)
    res = SV.scene_resources(sc.n, sc.res)
    mem = (sc.n * SV.bytes_per_particle(code) + res["keys"] * SV.BYTES_PER_KEY
           + res["virtual_blocks"] * SV.BYTES_PER_VIRTUAL_BLOCK + min(res["virtual_blocks"], sc.n // 64 + 4096)
           * SV.bytes_per_pool_block(code))
    names = {v: k for k, v in S._MODELS.items()}
    return {"name": sc.name, "particles": sc.n, "res": sc.res, "dx": sc.dx, "dt": sc.dt, "steps": sc.steps,
            "kernel": {v: k for k, v in S._KERNELS.items()}[sc.kernel],
            "transfer": {v: k for k, v in S._TRANSFERS.items()}[sc.transfer],
            "materials": [dict(model=names[m.model], E=m.E, nu=m.nu, rho=m.rho) for m in sc.materials],
            "device_bytes": int(mem), "cfl": cfl_number(sc)}


def run(sc, steps: int, every: int, out: str, resume: str | None = None, sim_cls=None, log=print) -> list:
    """Step a scene, checkpointing every `every` steps into `out`; returns the
    checkpoint paths written."""
    if sim_cls is None:
        from . import build as _build
        _build.build()  # compiles the library in-tree if it is missing or out of date
        from .ckmpm import Simulation as sim_cls
    from .ckmpm import kernel_code
    os.makedirs(out, exist_ok=True)
    cfl = cfl_number(sc)
    if cfl > 1.0:
        log(f"warning: dt (c + |v|) / dx = {cfl:.2f} > 1; the explicit step is likely unstable")
    sim = sim_cls(sc, kernel_code(sc))
    written = []
    try:
        if resume:
            sim.load(resume)
        done = 0
        t0 = time.perf_counter()
        while done < steps:
            k = min(every, steps - done)
            sim.step(k)
            done += k
            sim.sync()
            path = os.path.join(out, f"frame_{done:05d}.npz")
            sim.save(path)
            written.append(path)
            log(f"step {done}/{steps}  {time.perf_counter() - t0:.2f} s")
    finally:
        sim.close()
    return written


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2412_10399_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    p_info = sub.add_parser("info", help="describe a scene file (no GPU)")
    p_info.add_argument("scene")
    p_run = sub.add_parser("run", help="step a scene file on the GPU")
    p_run.add_argument("scene")
    p_run.add_argument("--steps", type=int, default=None, help="default: the scene's own step count")
    p_run.add_argument("--every", type=int, default=None, help="checkpoint interval (default: only at the end)")
    p_run.add_argument("--kernel", choices=sorted(S._KERNELS))
    p_run.add_argument("--transfer", choices=sorted(S._TRANSFERS))
    p_run.add_argument("--out", default="ckmpm_out")
    p_run.add_argument("--resume", default=None, help="a checkpoint of the same scene to start from")
    p_run.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    if args.cmd == "info":
        print(json.dumps(scene_info(S.load_scene(args.scene)), indent=1))
        return 0
    sc = _apply_overrides(S.load_scene(args.scene, args.seed), args)
    steps = sc.steps if args.steps is None else args.steps
    if steps < 1:
        ap.error("--steps must be >= 1")
    every = steps if args.every is None else args.every
    if every < 1:
        ap.error("--every must be >= 1")
    run(sc, steps, every, args.out, args.resume)
    return 0


if __name__ == "__main__":
    sys.exit(main())
