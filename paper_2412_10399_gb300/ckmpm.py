"""Python binding of the CK-MPM C ABI (include/ckmpm.h).

Argument marshalling only: every computation runs in libckmpm.so.  The
functions keep the C names; ``Simulation`` and ``Server`` are small
conveniences over them.  PyTorch is used only to supply the CUDA stream and,
optionally, device memory (``torch_allocator``).  If the shared library is
missing, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libckmpm.so")

OK, EINVAL, ENOMEM, ECUDA, EDOMAIN, ENONFINITE, ETIMEOUT, EBUSY, ENOTFOUND = range(9)
KERNEL_CK, KERNEL_QUADRATIC = 0, 1
TRANSFER_APIC_MLS, TRANSFER_PIC, TRANSFER_APIC_GRAD = 0, 2, 4  # OR-ed into a kernel argument
STEP_SPLIT, STEP_G2P2G = 0, 8  # step structure, OR-ed into a kernel argument
FIXED_COROTATED, DRUCKER_PRAGER, J_FLUID = 0, 1, 2
FIELD_X, FIELD_V, FIELD_B, FIELD_C, FIELD_F, FIELD_E = 0, 1, 2, 3, 4, 5
FIELD_GRID_M, FIELD_GRID_P, FIELD_GRID_V = 16, 17, 18
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EDOMAIN", "ENONFINITE", "ETIMEOUT", "EBUSY", "ENOTFOUND"]


class ckmpm_material(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho", ctypes.c_double), ("friction_deg", ctypes.c_double), ("gamma", ctypes.c_double)]


class ckmpm_scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("mat", ctypes.c_void_p), ("is_device", ctypes.c_int), ("res", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3),
                ("bc_cells", ctypes.c_double), ("ppc", ctypes.c_int),
                ("materials", ctypes.POINTER(ckmpm_material)), ("n_materials", ctypes.c_int),
                ("fp64_j_tol", ctypes.c_double), ("fp64_cond_tol", ctypes.c_double),
                ("fp64_gap_tol", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class ckmpm_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class ckmpm_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("max_particles", ctypes.c_int64), ("max_keys", ctypes.c_int64),
                ("max_grid_blocks", ctypes.c_int64), ("max_virtual_blocks", ctypes.c_int64),
                ("max_scenes", ctypes.c_int),
                ("max_materials", ctypes.c_int), ("per_particle_E", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("allocator", ctypes.POINTER(ckmpm_allocator))]


class ckmpm_stats(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_particle_blocks", ctypes.c_int64),
                ("n_grid_blocks", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("fp64_particles", ctypes.c_int64), ("ms_last_step", ctypes.c_double),
                ("ms_kernel", ctypes.c_double * 8), ("launches_kernel", ctypes.c_int64 * 8),
                ("launches_per_step", ctypes.c_int64), ("leftover_particles", ctypes.c_int64),
                ("graph_steps", ctypes.c_int64)]


# Every symbol the header declares, with its signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "ckmpm_create": (ctypes.c_int, [ctypes.POINTER(ckmpm_scene), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "ckmpm_create_server": (ctypes.c_int, [ctypes.POINTER(ckmpm_config), ctypes.POINTER(_P)]),
    "ckmpm_admit": (ctypes.c_int, [_P, ctypes.POINTER(ckmpm_scene), ctypes.POINTER(ctypes.c_int)]),
    "ckmpm_release": (ctypes.c_int, [_P, ctypes.c_int]),
    "ckmpm_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "ckmpm_sync": (ctypes.c_int, [_P]),
    "ckmpm_probe_grids": (ctypes.c_int, [_P]),
    "ckmpm_readback": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int]),
    "ckmpm_readback_async": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_int64)]),
    "ckmpm_readback_wait": (ctypes.c_int, [_P, ctypes.c_int64]),
    "ckmpm_upload": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int]),
    "ckmpm_scene_particles": (ctypes.c_int64, [_P, ctypes.c_int]),
    "ckmpm_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ckmpm_stats)]),
    "ckmpm_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "ckmpm_reset_timing": (ctypes.c_int, [_P]),
    "ckmpm_destroy": (ctypes.c_int, [_P]),
    "ckmpm_last_error": (ctypes.c_char_p, [_P]),
    "ckmpm_version": (ctypes.c_char_p, []),
    "ckmpm_p2g_grids_static": (ctypes.c_int, [ctypes.POINTER(ckmpm_scene), ctypes.c_int, _P, _P, _P, _P, _P]),
    "ckmpm_diff_create": (ctypes.c_int, [ctypes.POINTER(ckmpm_scene), _P, ctypes.POINTER(_P)]),
    "ckmpm_diff_step": (ctypes.c_int, [_P] + [_P] * 9),
    "ckmpm_diff_step_backward": (ctypes.c_int, [_P] + [_P] * 14),
    "ckmpm_diff_sync": (ctypes.c_int, [_P]),
    "ckmpm_diff_destroy": (ctypes.c_int, [_P]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libckmpm.so (built by paper_2412_10399_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2412_10399_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class CKMPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _check(st: int, ctx=None):
    if st != OK:
        msg = load().ckmpm_last_error(ctx).decode() if ctx else ""
        raise CKMPMError(st, msg)


# ------------------------------------------------------------ same-name wrappers

def ckmpm_version() -> str:
    return load().ckmpm_version().decode()


def ckmpm_create(scene: ckmpm_scene, kernel: int, stream: int = 0):
    out = _P()
    st = load().ckmpm_create(ctypes.byref(scene), kernel, _P(stream or None), ctypes.byref(out))
    _check(st)
    return out


def ckmpm_create_server(cfg: ckmpm_config):
    out = _P()
    _check(load().ckmpm_create_server(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def ckmpm_admit(ctx, scene: ckmpm_scene) -> int:
    sid = ctypes.c_int(-1)
    _check(load().ckmpm_admit(ctx, ctypes.byref(scene), ctypes.byref(sid)), ctx)
    return sid.value


def ckmpm_release(ctx, scene_id: int):
    _check(load().ckmpm_release(ctx, scene_id), ctx)


def ckmpm_step(ctx, n: int = 1):
    _check(load().ckmpm_step(ctx, n), ctx)


def ckmpm_sync(ctx):
    _check(load().ckmpm_sync(ctx), ctx)


def ckmpm_probe_grids(ctx):
    _check(load().ckmpm_probe_grids(ctx), ctx)


def ckmpm_readback(ctx, scene_id: int, field: int, dst_ptr: int, nbytes: int, dst_is_device: bool):
    _check(load().ckmpm_readback(ctx, scene_id, field, _P(dst_ptr), nbytes, int(dst_is_device)), ctx)


def ckmpm_readback_async(ctx, scene_id: int, field: int, host_ptr: int, nbytes: int) -> int:
    t = ctypes.c_int64(-1)
    _check(load().ckmpm_readback_async(ctx, scene_id, field, _P(host_ptr), nbytes, ctypes.byref(t)), ctx)
    return t.value


def ckmpm_readback_wait(ctx, ticket: int):
    _check(load().ckmpm_readback_wait(ctx, ticket), ctx)


def ckmpm_upload(ctx, scene_id: int, field: int, src_ptr: int, nbytes: int, src_is_device: bool):
    _check(load().ckmpm_upload(ctx, scene_id, field, _P(src_ptr), nbytes, int(src_is_device)), ctx)


def ckmpm_scene_particles(ctx, scene_id: int) -> int:
    return int(load().ckmpm_scene_particles(ctx, scene_id))


def ckmpm_get_stats(ctx) -> ckmpm_stats:
    s = ckmpm_stats()
    _check(load().ckmpm_get_stats(ctx, ctypes.byref(s)), ctx)
    return s


def ckmpm_set_timing(ctx, on: bool):
    _check(load().ckmpm_set_timing(ctx, int(on)), ctx)


def ckmpm_reset_timing(ctx):
    _check(load().ckmpm_reset_timing(ctx), ctx)


def ckmpm_destroy(ctx):
    load().ckmpm_destroy(ctx)


def ckmpm_last_error(ctx) -> str:
    return load().ckmpm_last_error(ctx).decode()


def ckmpm_p2g_grids_static(scene: ckmpm_scene, kernel: int, B_ptr: int, F_ptr: int, grid_m_ptr: int,
                           grid_p_ptr: int, stream: int = 0):
    """Allocation-free P2G into caller-provided device grids (see the C header)."""
    _check(load().ckmpm_p2g_grids_static(ctypes.byref(scene), kernel, _P(B_ptr or None), _P(F_ptr or None),
                                         _P(grid_m_ptr), _P(grid_p_ptr), _P(stream or None)))


# ------------------------------------------------------------ marshalling helpers

def make_scene(res: int, dx: float, dt: float, materials, x, v=None, mat=None, gravity=(0.0, -9.8, 0.0),
               bc_cells: float = 3.0, ppc: int = 8, fp64_j_tol: float = 1e-2, fp64_cond_tol: float = 1e-2,
               fp64_gap_tol: float = 0.0):
    """Build a ckmpm_scene from numpy arrays (host) or CUDA torch tensors:
    x (n, 3), v (n, 3) or None, mat (n,) or None; converted to float32 /
    uint8 and made contiguous here (the library reads them as such).

    Returns (scene, keepalive) where keepalive must outlive the C call."""
    keep = []
    n = (x.shape[0] if hasattr(x, "shape") else len(x))

    def ptr(a, dtype, name, shape):
        if a is None:
            return None, False
        got = tuple(a.shape) if hasattr(a, "shape") else np.shape(a)
        if got != shape:
            raise ValueError(f"{name} has shape {got}, expected {shape}")
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            t = a.to(torch.float32 if dtype == np.float32 else torch.uint8).contiguous()
            keep.append(t)
            return t.data_ptr(), True
        arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
        keep.append(arr)
        return arr.ctypes.data, False

    px, dev = ptr(x, np.float32, "x", (n, 3))
    pv, dv = ptr(v, np.float32, "v", (n, 3))
    pm, dm = ptr(mat, np.uint8, "mat", (n,))
    if (pv is not None and dv != dev) or (pm is not None and dm != dev):
        raise ValueError("x, v and mat must all be host arrays or all CUDA tensors")
    mats = (ckmpm_material * len(materials))()
    for i, m in enumerate(materials):
        mats[i] = ckmpm_material(int(m.model), float(m.E), float(m.nu), float(m.rho), float(m.friction_deg),
                                 float(getattr(m, "gamma", 7.15)))
    keep.append(mats)
    sc = ckmpm_scene()
    sc.n = int(n)
    sc.x = px
    sc.v = pv
    sc.mat = pm
    sc.is_device = int(dev)
    sc.res = int(res)
    sc.dx = float(dx)
    sc.dt = float(dt)
    sc.gravity = (ctypes.c_double * 3)(*gravity)
    sc.bc_cells = float(bc_cells)
    sc.ppc = int(ppc)
    sc.materials = ctypes.cast(mats, ctypes.POINTER(ckmpm_material))
    sc.n_materials = len(materials)
    sc.fp64_j_tol = float(fp64_j_tol)
    sc.fp64_cond_tol = float(fp64_cond_tol)
    sc.fp64_gap_tol = float(fp64_gap_tol)
    return sc, keep


def scene_struct(sc, x=None, v=None, **kw):
    """ckmpm_scene from a paper_2412_10399_gb300.scenes.Scene (positions rounded to float32)."""
    return make_scene(sc.res, sc.dx, sc.dt, sc.materials, sc.x32() if x is None else x,
                      sc.v32() if v is None else v, sc.mat, gravity=sc.gravity, bc_cells=sc.bc_cells,
                      ppc=sc.ppc, **kw)


def torch_allocator():
    """A ckmpm_allocator backed by torch's CUDA caching allocator (kept alive by the caller)."""
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
        except Exception:
            return None

    def _free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = ckmpm_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


_FIELD_SHAPE = {FIELD_X: (3,), FIELD_V: (3,), FIELD_B: (3, 3), FIELD_C: (3, 3), FIELD_F: (3, 3), FIELD_E: ()}


def kernel_code(scene) -> int:
    """The C ABI's kernel argument for a scene: its kernel, with the transfer
    flag of scene.transfer (0 APIC + MLS, 1 PIC, 2 APIC with the kernel gradient)."""
    flag = {0: TRANSFER_APIC_MLS, 1: TRANSFER_PIC, 2: TRANSFER_APIC_GRAD}[int(getattr(scene, "transfer", 0))]
    return int(scene.kernel) | flag


class Simulation:
    """One scene in its own context (thin wrapper over the C calls)."""

    def __init__(self, scene, kernel: Optional[int] = None, stream: Optional[int] = None, **kw):
        """kernel: the C ABI's kernel argument (ckmpm_kernel | ckmpm_transfer);
        None takes the scene's own (kernel_code(scene))."""
        if kernel is None:
            kernel = kernel_code(scene)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.scene = scene
        self.kernel = kernel
        sc, self._keep = scene_struct(scene, **kw)
        self.ctx = ckmpm_create(sc, kernel, stream)
        self.n = scene.n
        self.res = scene.res

    def close(self):
        if self.ctx:
            ckmpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        ckmpm_step(self.ctx, n)

    def sync(self):
        ckmpm_sync(self.ctx)

    def probe_grids(self):
        ckmpm_probe_grids(self.ctx)

    def read(self, field: int, scene_id: int = 0) -> np.ndarray:
        if field >= FIELD_GRID_M:
            ng = 2 if (self.kernel & 1) == KERNEL_CK else 1
            nn = self.res + 1
            shape = (ng, nn, nn, nn) if field == FIELD_GRID_M else (ng, nn, nn, nn, 3)
        else:
            shape = (self.n,) + _FIELD_SHAPE[field]
        out = np.empty(shape, np.float32)
        ckmpm_readback(self.ctx, scene_id, field, out.ctypes.data, out.nbytes, False)
        return out

    def write(self, field: int, arr, scene_id: int = 0):
        a = np.ascontiguousarray(arr, dtype=np.float32)
        ckmpm_upload(self.ctx, scene_id, field, a.ctypes.data, a.nbytes, False)

    def stats(self) -> ckmpm_stats:
        return ckmpm_get_stats(self.ctx)

    def diagnostics(self) -> dict:
        """Total mass, momentum, angular momentum (with APIC's particle spin
        where the transfer keeps B) and kinetic energy of the current state."""
        from .diagnostics import conserved
        B = None if self.kernel & TRANSFER_PIC else self.read(FIELD_B)
        sc = self.scene
        return conserved(self.read(FIELD_X), self.read(FIELD_V), sc.mat, sc.materials, sc.dx, sc.ppc, B)

    def save(self, path: str):
        """Checkpoint the particle state (x, v, F and, except under the PIC
        transfer, B; original particle order) to an .npz file."""
        fields = {"x": self.read(FIELD_X), "v": self.read(FIELD_V), "F": self.read(FIELD_F)}
        if not self.kernel & TRANSFER_PIC:
            fields["B"] = self.read(FIELD_B)
        np.savez(path, kernel=np.int64(self.kernel), **fields)

    def load(self, path: str):
        """Restore a checkpoint written by save() for the same scene and kernel
        argument.  Order matters: positions (re-binning), velocities, F, and B
        last, since an upload of B stores m B - dt V0 tau(F) with the F already
        there."""
        d = np.load(path)
        if int(d["kernel"]) != self.kernel or d["x"].shape != (self.n, 3):
            raise ValueError("checkpoint of another kernel argument or particle count")
        self.write(FIELD_X, d["x"])
        self.write(FIELD_V, d["v"])
        self.write(FIELD_F, d["F"])
        if "B" in d.files:
            self.write(FIELD_B, d["B"])
