"""Differentiable CK-MPM rollouts: torch.autograd over the hand-written adjoint
kernels of libckmpm (ckmpm_diff_*), with checkpointing every k steps and
recomputation in the backward pass.

Only argument marshalling happens here; the forward step and its
vector-Jacobian product run in CUDA.  PyTorch provides the device memory, the
stream and the autograd plumbing.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import torch

from . import ckmpm as ck


class DiffSim:
    """One differentiable scene (fixed-corotated, CK dual grid, dense grid)."""

    def __init__(self, scene, stream: Optional[int] = None):
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        sc, self._keep = ck.make_scene(scene.res, scene.dx, scene.dt, scene.materials, scene.x32()[:1],
                                       gravity=scene.gravity, bc_cells=scene.bc_cells, ppc=scene.ppc)
        sc.n = scene.n
        out = ctypes.c_void_p()
        st = ck.load().ckmpm_diff_create(ctypes.byref(sc), ctypes.c_void_p(stream or None), ctypes.byref(out))
        if st != ck.OK:
            raise ck.CKMPMError(st, "ckmpm_diff_create failed")
        self.h = out
        self.n = scene.n

    def close(self):
        if self.h:
            ck.load().ckmpm_diff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    def _check(self, **arrays):
        """The library reads and writes these through raw device pointers:
        every array must be a contiguous float32 CUDA tensor of its state's
        shape (x, v: n x 3; B, F: n x 3 x 3; E: n)."""
        want = {"x": (self.n, 3), "v": (self.n, 3), "B": (self.n, 3, 3), "F": (self.n, 3, 3), "E": (self.n,)}
        for name, t in arrays.items():
            shape = want[name.lstrip("g").rstrip("1")]
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda \
                    or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"{name}: need a contiguous float32 CUDA tensor of shape {shape}")

    def _chk(self, st):
        if st != ck.OK:
            raise ck.CKMPMError(st, "differentiable step failed")

    def step(self, x, v, B, F, E) -> Tuple[torch.Tensor, ...]:
        self._check(x=x, v=v, B=B, F=F, E=E)
        x1, v1, B1, F1 = (torch.empty_like(x), torch.empty_like(v), torch.empty_like(B), torch.empty_like(F))
        self._chk(ck.load().ckmpm_diff_step(self.h, *map(self._p, (x, v, B, F, E, x1, v1, B1, F1))))
        return x1, v1, B1, F1

    def step_backward(self, x, v, B, F, E, gx1, gv1, gB1, gF1, gE):
        self._check(x=x, v=v, B=B, F=F, E=E, gx1=gx1, gv1=gv1, gB1=gB1, gF1=gF1, gE=gE)
        gx, gv, gB, gF = (torch.empty_like(x), torch.empty_like(v), torch.empty_like(B), torch.empty_like(F))
        self._chk(ck.load().ckmpm_diff_step_backward(
            self.h, *map(self._p, (x, v, B, F, E, gx1, gv1, gB1, gF1, gx, gv, gB, gF, gE))))
        return gx, gv, gB, gF

    def sync(self):
        self._chk(ck.load().ckmpm_diff_sync(self.h))


def initial_state(x0: torch.Tensor):
    n = x0.shape[0]
    B0 = torch.zeros(n, 3, 3, dtype=torch.float32, device=x0.device)
    F0 = torch.eye(3, dtype=torch.float32, device=x0.device).expand(n, 3, 3).contiguous()
    return B0, F0


class Rollout(torch.autograd.Function):
    """(x0, v0, E) -> (x_T, v_T) after `steps` steps from B = 0, F = I.

    Forward keeps the state every `k` steps; backward replays each segment
    from its checkpoint (keeping the k states of that segment) and runs the
    per-step adjoints in reverse, accumulating dL/dE over all steps."""

    @staticmethod
    def forward(ctx, x0, v0, E, sim: DiffSim, steps: int, k: int):
        B0, F0 = initial_state(x0)
        s = (x0.contiguous(), v0.contiguous(), B0, F0)
        ckpts = []
        for t in range(steps):
            if t % k == 0:
                ckpts.append(s)
            s = sim.step(*s, E)
        ctx.sim, ctx.steps, ctx.k = sim, steps, k
        ctx.ckpts = ckpts
        ctx.save_for_backward(E)
        return s[0], s[1]

    @staticmethod
    def backward(ctx, gx, gv):
        (E,) = ctx.saved_tensors
        sim, steps, k = ctx.sim, ctx.steps, ctx.k
        x0 = ctx.ckpts[0][0]
        n = x0.shape[0]
        gx = torch.zeros_like(x0) if gx is None else gx.contiguous()
        gv = torch.zeros_like(x0) if gv is None else gv.contiguous()
        gB = torch.zeros(n, 3, 3, dtype=torch.float32, device=x0.device)
        gF = torch.zeros_like(gB)
        gE = torch.zeros_like(E)
        adj = (gx, gv, gB, gF)
        for seg in reversed(range(len(ctx.ckpts))):
            t0 = seg * k
            t1 = min(steps, t0 + k)
            states = [ctx.ckpts[seg]]
            for _ in range(t0, t1 - 1):
                states.append(sim.step(*states[-1], E))
            for j in reversed(range(t1 - t0)):
                adj = sim.step_backward(*states[j], E, *adj, gE)
        ctx.ckpts = None
        return adj[0], adj[1], gE, None, None, None


def com_loss(x: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Distance of the centre of mass (uniform particle mass) to the target."""
    return torch.linalg.vector_norm(x.mean(0) - target)
