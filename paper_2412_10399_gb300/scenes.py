"""Seeded synthetic scene generators (input only: no method arithmetic).

Every particle position, velocity and material tag used by the CUDA path, the
FP64 oracle, the tests and the benchmark comes from here.  Nothing in this file
computes a kernel weight, a transfer, a stress or a time step.

Sampling rule (shared by all scenes):
  * the domain is [0, res*dx]^3, y up;
  * a cell is *filled* when its centre lies inside the union of the scene's
    shapes (strict inequalities; half-integer cell centres never sit exactly
    on a sphere or cylinder surface centred on an integer lattice point);
  * each filled cell receives 8 particles, one uniform point in each of its
    2x2x2 sub-cells (stratified jitter);
  * uniforms come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
    pseudorandom number generators", OOPSLA 2014) evaluated on the counter
    ((cell_linear * 8 + sub) * 4 + component), keyed by the seed.

The paper's own benchmark scenes are meshes (dragons, armadillos, a sand castle,
...) that are not available; these boxes, cylinders and spheres stand in for
them with the same workload shape (8 particles per cell, 1e4..1e7 particles,
mixed elastic and granular material).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Material models understood by both the CUDA path and the oracle.
FIXED_COROTATED = 0
DRUCKER_PRAGER = 1
J_FLUID = 2

# Transfer kernels.
KERNEL_CK = 0          # the paper's compact kernel on the dual staggered grid
KERNEL_QUADRATIC = 1   # quadratic B-spline MLS-MPM on one grid (comparison path)

# Transfer schemes.
TRANSFER_APIC_MLS = 0  # APIC momentum with the MLS force (Sec. 4.4, 4.5)
TRANSFER_PIC = 1       # PIC of Sec. 4.3 with the kernel gradient
TRANSFER_APIC_GRAD = 2  # APIC momentum (Sec. 4.4) with the kernel-gradient force and grad v


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for each uint64 counter (vectorised, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) * _M2 + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(counter: np.ndarray, seed: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(counter, seed)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(counter: np.ndarray, seed: int) -> np.ndarray:
    """Standard normals by Box-Muller on two SplitMix64 streams."""
    c = counter.astype(np.uint64) * np.uint64(2)
    u1 = uniform01(c, seed)
    u2 = uniform01(c + np.uint64(1), seed)
    u1 = np.maximum(u1, 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass
class Material:
    """Constitutive parameters of one material (SI units)."""
    model: int               # FIXED_COROTATED, DRUCKER_PRAGER or J_FLUID
    E: float                 # Young's modulus [Pa]; for the fluid the equation-of-state constant B [Pa]
    nu: float                # Poisson ratio
    rho: float               # density [kg/m^3]
    friction_deg: float = 0.0  # Drucker-Prager friction angle [deg]
    gamma: float = 7.15      # fluid equation-of-state exponent


@dataclasses.dataclass
class Scene:
    """A particle set plus the grid and integration parameters of one simulation."""
    name: str
    res: int                   # cells per axis; domain is [0, res*dx]^3
    dx: float
    dt: float
    x: np.ndarray              # (N, 3) float64 positions
    v: np.ndarray              # (N, 3) float64 velocities
    mat: np.ndarray            # (N,) uint8 material index into `materials`
    materials: List[Material]
    gravity: Tuple[float, float, float] = (0.0, -9.8, 0.0)
    bc_cells: int = 3          # sticky wall thickness in cells
    ppc: int = 8               # particles per filled cell (sets V0 = dx^3/ppc)
    steps: int = 100
    kernel: int = KERNEL_CK
    transfer: int = TRANSFER_APIC_MLS

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def x32(self) -> np.ndarray:
        return np.ascontiguousarray(self.x, dtype=np.float32)

    def v32(self) -> np.ndarray:
        return np.ascontiguousarray(self.v, dtype=np.float32)


# ----------------------------------------------------------------------------
# shapes: predicates on cell-centre coordinates measured in cells
# ----------------------------------------------------------------------------

def _box(lo: Sequence[float], hi: Sequence[float]):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)

    def inside(c):
        return np.all((c >= lo) & (c < hi), axis=-1)
    bb = (np.floor(lo).astype(int), np.ceil(hi).astype(int))
    return inside, bb


def _sphere(centre: Sequence[float], r: float):
    centre = np.asarray(centre, np.float64)

    def inside(c):
        d = c - centre
        return np.einsum("...i,...i->...", d, d) < r * r
    lo = np.floor(centre - r).astype(int)
    hi = np.ceil(centre + r).astype(int) + 1
    return inside, (lo, hi)


def _cylinder_y(cx: float, cz: float, r: float, y0: float, y1: float):
    def inside(c):
        dx = c[..., 0] - cx
        dz = c[..., 2] - cz
        return (dx * dx + dz * dz < r * r) & (c[..., 1] >= y0) & (c[..., 1] < y1)
    lo = np.array([math.floor(cx - r), math.floor(y0), math.floor(cz - r)])
    hi = np.array([math.ceil(cx + r) + 1, math.ceil(y1), math.ceil(cz + r) + 1])
    return inside, (lo, hi)


def filled_cells(shapes, res: int) -> np.ndarray:
    """Sorted unique linear indices (z-major: (cz*res + cy)*res + cx) of cells
    whose centre lies in the union of `shapes`."""
    out = []
    for inside, (lo, hi) in shapes:
        lo = np.clip(lo, 0, res)
        hi = np.clip(hi, 0, res)
        if np.any(hi <= lo):
            continue
        gx = np.arange(lo[0], hi[0])
        gy = np.arange(lo[1], hi[1])
        gz = np.arange(lo[2], hi[2])
        cz, cy, cx = np.meshgrid(gz, gy, gx, indexing="ij")
        cen = np.stack([cx, cy, cz], axis=-1).astype(np.float64) + 0.5
        m = inside(cen)
        lin = (cz[m].astype(np.int64) * res + cy[m]) * res + cx[m]
        out.append(lin)
    if not out:
        return np.zeros(0, np.int64)
    return np.unique(np.concatenate(out))


def sample_cells(cells: np.ndarray, res: int, dx: float, seed: int) -> np.ndarray:
    """8 stratified-jitter particles per cell; returns (8*len(cells), 3) float64."""
    cells = np.asarray(cells, np.int64)
    cx = cells % res
    cy = (cells // res) % res
    cz = cells // (res * res)
    sub = np.arange(8, dtype=np.int64)
    sx, sy, sz = sub & 1, (sub >> 1) & 1, (sub >> 2) & 1
    base = (cells[:, None] * 8 + sub[None, :]) * 4
    ux = uniform01(base.astype(np.uint64), seed)
    uy = uniform01((base + 1).astype(np.uint64), seed)
    uz = uniform01((base + 2).astype(np.uint64), seed)
    x = (cx[:, None] + (sx[None, :] + ux) * 0.5) * dx
    y = (cy[:, None] + (sy[None, :] + uy) * 0.5) * dx
    z = (cz[:, None] + (sz[None, :] + uz) * 0.5) * dx
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

ELASTIC = Material(FIXED_COROTATED, 1e5, 0.3, 1000.0)
SAND = Material(DRUCKER_PRAGER, 3.5e5, 0.3, 1600.0, 30.0)
STIFF_BALL = Material(FIXED_COROTATED, 1e7, 0.3, 1e4)
# J-based fluid of the dam-break scenes: B = 10 Pa, gamma = 7.15 (the paper's
# parameters; its density is not stated, water's is used)
FLUID = Material(J_FLUID, 10.0, 0.0, 1000.0, 0.0, 7.15)


def elastic_cube(seed: int = 0, res: int = 64) -> Scene:
    """Elastic cube of side 0.25 centred at the top of a 64^3 grid: cells
    [24,40) x [40,56) x [24,40), 8 ppc -> 32,768 particles."""
    s = res // 64
    shapes = [_box([24 * s, 40 * s, 24 * s], [40 * s, 56 * s, 40 * s])]
    dx = 1.0 / res
    x = sample_cells(filled_cells(shapes, res), res, dx, seed)
    return Scene("elastic_cube", res, dx, 1e-4, x, np.zeros_like(x),
                 np.zeros(len(x), np.uint8), [ELASTIC], steps=100)


def granular_column(seed: int = 0) -> Scene:
    """Drucker-Prager sand column 0.203 x 0.5 x 0.203 on a 128^3 grid: cells
    [51,77) x [4,68) x [51,77), 8 ppc -> 346,112 particles."""
    res = 128
    shapes = [_box([51, 4, 51], [77, 68, 77])]
    dx = 1.0 / res
    x = sample_cells(filled_cells(shapes, res), res, dx, seed)
    return Scene("granular_column", res, dx, 5e-5, x, np.zeros_like(x),
                 np.zeros(len(x), np.uint8), [SAND], steps=500)


def large_impact(seed: int = 0) -> Scene:
    """512^3 virtual grid: a castle of Drucker-Prager sand (base box, four
    cylindrical towers, a keep) hit by four stiff fixed-corotated balls at
    20 m/s; 16,138,496 sand + 135,168 ball particles = 16,273,664.  The balls
    start 15 cells from the keep's four faces at mid-height (0.2 cells per
    step), so they strike it at about step 73 of the 200."""
    res = 512
    dx = 1.0 / res
    sand = [_box([154, 4, 154], [358, 36, 358]),
            _box([226, 36, 226], [286, 86, 286])]
    for tx in (174, 338):
        for tz in (174, 338):
            sand.append(_cylinder_y(tx, tz, 20.0, 36, 136))
    sand_cells = filled_cells(sand, res)
    centres = [(201, 60, 256), (311, 60, 256), (256, 60, 201), (256, 60, 311)]
    xs = [sample_cells(sand_cells, res, dx, seed)]
    vs = [np.zeros_like(xs[0])]
    ms = [np.zeros(len(xs[0]), np.uint8)]
    for c in centres:
        cells = filled_cells([_sphere(c, 10.0)], res)
        xb = sample_cells(cells, res, dx, seed)
        d = np.array([256.0 - c[0], 0.0, 256.0 - c[2]])
        d /= np.linalg.norm(d)
        xs.append(xb)
        vs.append(np.tile(20.0 * d, (len(xb), 1)))
        ms.append(np.ones(len(xb), np.uint8))
    x = np.concatenate(xs)
    return Scene("large_impact", res, dx, 2e-5, x, np.concatenate(vs),
                 np.concatenate(ms), [SAND, STIFF_BALL], steps=200)


def dam_break(n: int = 4175808, seed: int = 0, res: int = 256) -> Scene:
    """A single dam break: n particles of J-based fluid uniform at random in a
    cuboid against the x = 0 and z = 0 walls of a res^3 grid (dx = 1/res), at 8
    particles per cell on average (width 96 cells for n <= 5e6, else 128; the
    height follows from n).  The paper's performance section runs 4,175,808 and
    8,994,048 particles on 256^3; dt 1e-4."""
    dx = 1.0 / res
    w = 96.0 if n <= 5_000_000 else 128.0
    h = n / 8.0 / (w * w)
    lo = 4.0
    if lo + max(w, h) > res - 4:
        raise ValueError("dam-break cuboid does not fit the grid")
    ctr = np.arange(3 * n, dtype=np.uint64) + np.uint64(1 << 50)
    u = uniform01(ctr, seed).reshape(n, 3)
    x = (lo + u * np.array([w, h, w])) * dx
    return Scene(f"dam_break_{n}", res, dx, 1e-4, x, np.zeros_like(x), np.zeros(n, np.uint8), [FLUID],
                 steps=200)


def diffusion_bar(seed: int = 0, res: int = 256) -> Scene:
    """The numerical-diffusion scene of the paper's comparisons: a 20 x 10 x
    140-cell cuboid (dx = 1/256) with the high-frequency initial velocity
    v_y = 0.2 sin(500 z), no gravity, dt 2e-5, 500 steps (100 frames at 10 kHz).
    The paper does not give the material; the elastic cube's is used."""
    dx = 1.0 / res
    lo = np.array([118, 123, 58])
    cells = filled_cells([_box(lo.tolist(), (lo + np.array([20, 10, 140])).tolist())], res)
    x = sample_cells(cells, res, dx, seed)
    v = np.zeros_like(x)
    v[:, 1] = 0.2 * np.sin(500.0 * x[:, 2])
    return Scene("diffusion_bar", res, dx, 2e-5, x, v, np.zeros(len(x), np.uint8), [ELASTIC],
                 gravity=(0.0, 0.0, 0.0), steps=500)


def differentiable_cube(seed: int = 0, res: int = 128, lo: int = 48, hi: int = 80) -> Scene:
    """Elastic cube cells [48,80)^3 on 128^3 (262,144 particles) with initial
    velocity (0.5, 0, 0) + N(0, 0.5^2) per component."""
    dx = 1.0 / res
    x = sample_cells(filled_cells([_box([lo] * 3, [hi] * 3)], res), res, dx, seed)
    n = len(x)
    ctr = np.arange(3 * n, dtype=np.uint64) + np.uint64(1 << 40)
    v = 0.5 * normal(ctr, seed).reshape(n, 3)
    v[:, 0] += 0.5
    return Scene("differentiable_cube", res, dx, 1e-4, x, v,
                 np.zeros(n, np.uint8), [ELASTIC], steps=64)


@dataclasses.dataclass
class ServedRequest:
    scene: Scene
    arrival_s: float


def served_mix(n_scenes: int = 64, seed: int = 0, mean_interarrival_s: float = 0.02,
               n_min: float = 1e4, n_max: float = 2e6, steps: int = 1000,
               res: int = 128) -> List[ServedRequest]:
    """Poisson stream of independent scenes: particle counts log-uniform in
    [n_min, n_max], box or sphere, elastic (dt 1e-4) or sand (dt 5e-5), each in
    its own res^3 domain."""
    ctr = np.arange(8 * n_scenes, dtype=np.uint64) + np.uint64(1 << 44)
    u = uniform01(ctr, seed).reshape(n_scenes, 8)
    out: List[ServedRequest] = []
    t = 0.0
    dx = 1.0 / res
    for s in range(n_scenes):
        t += -mean_interarrival_s * math.log(max(u[s, 0], 1e-300))
        n_target = math.exp(math.log(n_min) + u[s, 1] * (math.log(n_max) - math.log(n_min)))
        ncells = n_target / 8.0
        is_sphere = u[s, 2] < 0.5
        is_sand = u[s, 3] < 0.5
        cx = res / 2 + (u[s, 4] - 0.5) * 8
        cz = res / 2 + (u[s, 5] - 0.5) * 8
        if is_sphere:
            r = (3.0 * ncells / (4.0 * math.pi)) ** (1.0 / 3.0)
            cy = 6 + r + u[s, 6] * 8
            shapes = [_sphere((cx, cy, cz), r)]
        else:
            a = ncells ** (1.0 / 3.0)
            y0 = 6 + u[s, 6] * 8
            shapes = [_box([cx - a / 2, y0, cz - a / 2], [cx + a / 2, y0 + a, cz + a / 2])]
        cells = filled_cells(shapes, res)
        x = sample_cells(cells, res, dx, seed + 1 + s)
        mat = SAND if is_sand else ELASTIC
        sc = Scene(f"served_{s}", res, dx, 5e-5 if is_sand else 1e-4, x, np.zeros_like(x),
                   np.zeros(len(x), np.uint8), [mat], steps=steps)
        out.append(ServedRequest(sc, t))
    return out


def random_state(n: int, res: int, seed: int, margin_cells: float = 4.0,
                 v_scale: float = 1.0, b_scale: float = 1.0, f_scale: float = 0.05,
                 box: Optional[Tuple[float, float]] = None):
    """Random particle state (x, v, B, F) for transfer-level parity tests.

    Positions uniform in the interior (or in `box`, given in cells), velocities
    uniform in [-v_scale, v_scale], B uniform in [-b_scale, b_scale]*dx,
    F = I + uniform[-f_scale, f_scale].  All float64; callers round to float32
    before handing the same values to both implementations."""
    dx = 1.0 / res
    c = np.arange(n * 32, dtype=np.uint64).reshape(n, 32) + np.uint64(1 << 48)
    u = uniform01(c, seed)
    lo, hi = (margin_cells, res - margin_cells) if box is None else box
    x = (lo + (hi - lo) * u[:, 0:3]) * dx
    v = v_scale * (2.0 * u[:, 3:6] - 1.0)
    B = b_scale * dx * (2.0 * u[:, 6:15] - 1.0)
    F = np.eye(3)[None].repeat(n, 0).reshape(n, 9) + f_scale * (2.0 * u[:, 15:24] - 1.0)
    return x, v, B.reshape(n, 3, 3), F.reshape(n, 3, 3)


# ----------------------------------------------------------------------------
# declarative scenes (a JSON-friendly description of the same shapes)
# ----------------------------------------------------------------------------

_MODELS = {"fixed_corotated": FIXED_COROTATED, "drucker_prager": DRUCKER_PRAGER, "j_fluid": J_FLUID}
_KERNELS = {"ck": KERNEL_CK, "quadratic": KERNEL_QUADRATIC}
_TRANSFERS = {"apic_mls": TRANSFER_APIC_MLS, "pic": TRANSFER_PIC, "apic_grad": TRANSFER_APIC_GRAD}


def _shape_of(d: dict, res: int):
    if len(d) != 1:
        raise ValueError(f"a shape has exactly one kind: {d!r}")
    (kind, p), = d.items()
    if kind == "box":
        return _box(p["lo"], p["hi"])
    if kind == "sphere":
        return _sphere(p["centre"], float(p["r"]))
    if kind == "cylinder_y":
        return _cylinder_y(float(p["cx"]), float(p["cz"]), float(p["r"]), float(p["y0"]), float(p["y1"]))
    raise ValueError(f"unknown shape {kind!r} (box, sphere, cylinder_y)")


def scene_from_spec(spec: dict, seed: int = 0) -> Scene:
    """A Scene from a plain description (the form a JSON file holds), sampled
    by the rule of this module.  Coordinates are in cells.

        {"name": "...", "res": 128, "dt": 1e-4,             # required
         "dx": 1/res, "gravity": [0, -9.8, 0], "bc_cells": 3, "steps": 100,
         "kernel": "ck" | "quadratic", "transfer": "apic_mls" | "pic" | "apic_grad",
         "materials": [{"model": "fixed_corotated" | "drucker_prager" | "j_fluid",
                        "E": ..., "nu": ..., "rho": ..., "friction_deg": 0, "gamma": 7.15}],
         "bodies": [{"material": 0, "velocity": [vx, vy, vz],
                     "shapes": [{"box": {"lo": [x, y, z], "hi": [x, y, z]}},
                                {"sphere": {"centre": [x, y, z], "r": r}},
                                {"cylinder_y": {"cx": x, "cz": z, "r": r, "y0": y, "y1": y}}]}]}

    A body fills the cells whose centres lie in the union of its shapes, less
    the cells an earlier body filled; bodies are concatenated in order."""
    res = int(spec["res"])
    dx = float(spec.get("dx", 1.0 / res))
    mats = []
    for m in spec["materials"]:
        if m["model"] not in _MODELS:
            raise ValueError(f"unknown material model {m['model']!r}")
        mats.append(Material(_MODELS[m["model"]], float(m["E"]), float(m["nu"]), float(m["rho"]),
                             float(m.get("friction_deg", 0.0)), float(m.get("gamma", 7.15))))
    if not mats or len(mats) > 255:
        raise ValueError("a scene has 1..255 materials")
    xs, vs, ms = [], [], []
    taken = np.zeros(0, np.int64)
    for b in spec["bodies"]:
        k = int(b.get("material", 0))
        if not 0 <= k < len(mats):
            raise ValueError(f"body material {k} out of range")
        cells = filled_cells([_shape_of(s, res) for s in b["shapes"]], res)
        cells = np.setdiff1d(cells, taken, assume_unique=True)
        taken = np.union1d(taken, cells)
        x = sample_cells(cells, res, dx, seed)
        xs.append(x)
        vs.append(np.tile(np.asarray(b.get("velocity", (0.0, 0.0, 0.0)), np.float64), (len(x), 1)))
        ms.append(np.full(len(x), k, np.uint8))
    if not xs or sum(len(x) for x in xs) == 0:
        raise ValueError("the scene's bodies fill no cell")
    kernel = spec.get("kernel", "ck")
    transfer = spec.get("transfer", "apic_mls")
    if kernel not in _KERNELS or transfer not in _TRANSFERS:
        raise ValueError(f"unknown kernel {kernel!r} or transfer {transfer!r}")
    return Scene(str(spec.get("name", "scene")), res, dx, float(spec["dt"]), np.concatenate(xs),
                 np.concatenate(vs), np.concatenate(ms), mats,
                 gravity=tuple(float(g) for g in spec.get("gravity", (0.0, -9.8, 0.0))),
                 bc_cells=spec.get("bc_cells", 3), steps=int(spec.get("steps", 100)),
                 kernel=_KERNELS[kernel], transfer=_TRANSFERS[transfer])


def load_scene(path: str, seed: int = 0) -> Scene:
    """scene_from_spec of a JSON file."""
    import json
    with open(path) as f:
        return scene_from_spec(json.load(f), seed)
