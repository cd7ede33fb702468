"""Steady steps replayed as CUDA graphs give the trajectory of direct launches.

A context created with CKMPM_GRAPHS=0 launches every kernel directly; one
created without it captures each parity of its double-buffered state once and
replays it.  Both run the same scene on a non-default stream (the legacy
stream cannot be captured); results agree within the run-to-run rounding of
the float atomics that meet between blocks (the tolerance of the probe/upload
test).  The graphs must be dropped and re-captured across an upload, so the
same comparison runs through one."""
import os

import numpy as np
import pytest
import torch

from gpu_helpers import need_gpu, random_scene, rel
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _run(ck, sc, B, F, kernel, graphs, stream):
    if graphs:
        os.environ.pop("CKMPM_GRAPHS", None)
    else:
        os.environ["CKMPM_GRAPHS"] = "0"
    try:
        sim = ck.Simulation(sc, kernel, stream=stream.cuda_stream)
    finally:
        os.environ.pop("CKMPM_GRAPHS", None)
    sim.write(ck.FIELD_F, F)
    sim.write(ck.FIELD_B, B)
    sim.step(6)
    v = sim.read(ck.FIELD_V)
    sim.write(ck.FIELD_V, v)  # an upload between steps drops the graphs
    sim.step(6)
    sim.sync()
    out = [sim.read(f) for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F)]
    st = sim.stats()
    sim.close()
    return out, int(st.graph_steps)


@pytest.mark.parametrize("kernel", [S.KERNEL_CK, S.KERNEL_QUADRATIC])
@pytest.mark.parametrize("fused", [False, True])
def test_graph_steps_match_direct_launches(kernel, fused):
    ck = need_gpu()
    sc, B, F = random_scene(6000, 32, 91, kernel=kernel, f_scale=0.05, v_scale=20.0)
    k = kernel | (ck.STEP_G2P2G if fused else 0)
    stream = torch.cuda.Stream()
    want, n0 = _run(ck, sc, B, F, k, False, stream)
    got, n1 = _run(ck, sc, B, F, k, True, stream)
    assert n0 == 0
    assert n1 >= 8  # all but the first step after creation and after the upload (fused: also the prologues)
    assert np.abs(got[0] - want[0]).max() <= 1e-6 * sc.dx + 2e-7
    assert rel(got[1], want[1]) <= 1e-5
    # F integrates the gradients of the same grid velocities (1.4e-6 seen
    # for the fused step, whose leftover list order varies between runs)
    assert rel(got[2], want[2]) <= 1e-5


def test_graph_steps_across_admission_and_release():
    """A served context (split step, graphs on): two scenes admitted, steps,
    one released, steps (the first step after a release drops its particles
    from the pool, which changes the count the graphs were captured with),
    a third admitted, steps; every scene's positions match the scene stepped
    alone with graphs off."""
    ck = need_gpu()
    scenes = [random_scene(3000, 32, 92, f_scale=0.05, v_scale=10.0),
              random_scene(2000, 16, 93, model=S.DRUCKER_PRAGER, f_scale=0.05, v_scale=10.0),
              random_scene(1500, 32, 94, f_scale=0.05, v_scale=10.0)]
    stream = torch.cuda.Stream()
    cfg = ck.ckmpm_config()
    cfg.kernel = ck.KERNEL_CK
    cfg.max_particles = sum(sc.n for sc, _, _ in scenes)
    cfg.max_keys = 3 * 8 ** 3
    cfg.max_virtual_blocks = 3 * 9 ** 3
    cfg.max_grid_blocks = 3 * 9 ** 3
    cfg.max_scenes = 3
    cfg.max_materials = 3
    cfg.stream = stream.cuda_stream
    srv = ck.ckmpm_create_server(cfg)
    keep = []

    def admit(sc, B, F):
        s, k = ck.scene_struct(sc)
        keep.append(k)
        sid = ck.ckmpm_admit(srv, s)
        for fld, arr in ((ck.FIELD_F, F), (ck.FIELD_B, B)):
            x = np.ascontiguousarray(arr, np.float32)
            ck.ckmpm_upload(srv, sid, fld, x.ctypes.data, x.nbytes, False)
        return sid

    def read(sid, n):
        out = np.empty((n, 3), np.float32)
        ck.ckmpm_readback(srv, sid, ck.FIELD_X, out.ctypes.data, out.nbytes, False)
        return out

    i0, i1 = admit(*scenes[0]), admit(*scenes[1])
    ck.ckmpm_step(srv, 5)
    x1 = read(i1, scenes[1][0].n)
    ck.ckmpm_release(srv, i1)
    ck.ckmpm_step(srv, 5)
    i2 = admit(*scenes[2])
    ck.ckmpm_step(srv, 5)
    x0, x2 = read(i0, scenes[0][0].n), read(i2, scenes[2][0].n)
    assert int(ck.ckmpm_get_stats(srv).graph_steps) >= 8
    ck.ckmpm_destroy(srv)
    os.environ["CKMPM_GRAPHS"] = "0"
    try:
        for (sc, B, F), steps, got in ((scenes[0], 15, x0), (scenes[1], 5, x1), (scenes[2], 5, x2)):
            alone = ck.Simulation(sc, sc.kernel, stream=stream.cuda_stream)
            alone.write(ck.FIELD_F, F)
            alone.write(ck.FIELD_B, B)
            alone.step(steps)
            want = alone.read(ck.FIELD_X)
            alone.close()
            assert np.abs(got - want).max() <= 1e-6 * sc.dx + 2e-7
    finally:
        os.environ.pop("CKMPM_GRAPHS", None)
