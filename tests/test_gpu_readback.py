"""Asynchronous host readback (ckmpm_readback_async / ckmpm_readback_wait).

Positions gathered after each step and copied on the context's second stream
while later steps run equal the synchronous readback of the same steps (a
second context, same scene, graphs on in both; cross-block float atomics
leave run-to-run rounding, the tolerance of the graph test).  Tickets
alternate between two staging slots, so a third readback waits on the device
for the first slot's copy; waiting on an old ticket, a grid field, pageable
host memory, the error of a step surfacing at the wait, and the argument
errors are covered too."""
import numpy as np
import pytest
import torch

from gpu_helpers import need_gpu, random_scene

pytestmark = pytest.mark.gpu


def _pinned(shape):
    return torch.empty(shape, dtype=torch.float32).pin_memory()


def test_async_readback_matches_synchronous_readback():
    ck = need_gpu()
    sc, B, F = random_scene(20000, 32, 301, f_scale=0.05, v_scale=20.0)
    stream = torch.cuda.Stream()
    a = ck.Simulation(sc, sc.kernel, stream=stream.cuda_stream)
    b = ck.Simulation(sc, sc.kernel, stream=stream.cuda_stream)
    for sim in (a, b):
        sim.write(ck.FIELD_F, F)
        sim.write(ck.FIELD_B, B)
    steps = 7
    bufs = [_pinned((sc.n, 3)) for _ in range(steps)]
    tickets = []
    for k in range(steps):
        a.step(1)
        tickets.append(ck.ckmpm_readback_async(a.ctx, 0, ck.FIELD_X, bufs[k].data_ptr(), sc.n * 12))
    assert tickets == list(range(steps))
    want = []
    for k in range(steps):
        b.step(1)
        want.append(b.read(ck.FIELD_X))
    # the last two tickets own the slots; older ones completed before their
    # slot was reused, and waiting on them waits for the slot's newest copy
    for t in reversed(tickets):
        ck.ckmpm_readback_wait(a.ctx, t)
    for k in range(steps):
        got = bufs[k].numpy()
        assert np.abs(got - want[k]).max() <= 1e-6 * sc.dx + 2e-7, k
    # velocities and F of the final state through the same slots
    v = _pinned((sc.n, 3))
    f = _pinned((sc.n, 3, 3))
    tv = ck.ckmpm_readback_async(a.ctx, 0, ck.FIELD_V, v.data_ptr(), sc.n * 12)
    tf = ck.ckmpm_readback_async(a.ctx, 0, ck.FIELD_F, f.data_ptr(), sc.n * 36)
    ck.ckmpm_readback_wait(a.ctx, tf)
    ck.ckmpm_readback_wait(a.ctx, tv)
    vw, fw = b.read(ck.FIELD_V), b.read(ck.FIELD_F)
    assert np.abs(v.numpy() - vw).max() <= 1e-5 * (np.abs(vw).max() + 1.0)
    assert np.abs(f.numpy() - fw).max() <= 1e-6 * (np.abs(fw).max() + 1.0)
    a.close()
    b.close()


def test_async_readback_of_a_grid_field_and_into_pageable_memory():
    ck = need_gpu()
    sc, B, F = random_scene(5000, 16, 302, f_scale=0.05, v_scale=5.0)
    sim = ck.Simulation(sc, sc.kernel)
    sim.write(ck.FIELD_F, F)
    sim.write(ck.FIELD_B, B)
    sim.step(3)
    sim.probe_grids()
    want = sim.read(ck.FIELD_GRID_M)
    got = np.empty_like(want)  # pageable: the copy completes within the call's stream order
    t = ck.ckmpm_readback_async(sim.ctx, 0, ck.FIELD_GRID_M, got.ctypes.data, got.nbytes)
    ck.ckmpm_readback_wait(sim.ctx, t)
    assert np.array_equal(got, want)
    sim.close()


def test_async_readback_argument_errors():
    ck = need_gpu()
    sc, B, F = random_scene(1000, 16, 303, f_scale=0.05)
    sim = ck.Simulation(sc, sc.kernel)
    buf = _pinned((sc.n, 3))
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_readback_async(sim.ctx, 0, ck.FIELD_X, buf.data_ptr(), sc.n * 12 - 4)
    assert ei.value.status == ck.EINVAL
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_readback_async(sim.ctx, 5, ck.FIELD_X, buf.data_ptr(), sc.n * 12)
    assert ei.value.status == ck.ENOTFOUND
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_readback_wait(sim.ctx, 0)  # no ticket issued yet
    assert ei.value.status == ck.EINVAL
    t = ck.ckmpm_readback_async(sim.ctx, 0, ck.FIELD_X, buf.data_ptr(), sc.n * 12)
    ck.ckmpm_readback_wait(sim.ctx, t)
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_readback_wait(sim.ctx, t + 1)
    assert ei.value.status == ck.EINVAL
    sim.close()


def test_device_error_surfaces_at_the_wait():
    """A particle driven out of the domain: the step flags EDOMAIN on the
    device, and the wait on a readback gathered after that step reports it."""
    ck = need_gpu()
    from paper_2412_10399_gb300 import scenes as S
    x0 = np.array([[0.52 / 16, 0.5, 0.5]], np.float64)
    v0 = np.array([[-100.0, 0.0, 0.0]], np.float64)
    sc = S.Scene("out", 16, 1 / 16, 1e-3, x0, v0, np.zeros(1, np.uint8), [S.ELASTIC], bc_cells=0.0,
                 gravity=(0.0, 0.0, 0.0))
    sim = ck.Simulation(sc, ck.KERNEL_CK)
    buf = _pinned((1, 3))
    sim.step(1)
    t = ck.ckmpm_readback_async(sim.ctx, 0, ck.FIELD_X, buf.data_ptr(), 12)
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_readback_wait(sim.ctx, t)
    assert ei.value.status == ck.EDOMAIN
    sim.close()


def test_admission_from_page_locked_host_arrays():
    """Page-locked x, v, mat are copied asynchronously in stream order,
    pageable ones before the call returns.  All admissions give the same
    state, bit for bit, and so the same first step; the third case passes
    arrays that start inside a larger page-locked allocation."""
    ck = need_gpu()
    from paper_2412_10399_gb300 import scenes as S
    sc, B, F = random_scene(7000, 32, 304, f_scale=0.05, v_scale=5.0)
    mats = [S.ELASTIC, S.SAND]
    g = np.random.default_rng(304)
    mat = (g.random(sc.n) < 0.3).astype(np.uint8)
    x32, v32 = sc.x32(), sc.v32()
    out = {}
    for case in ("pageable", "pinned", "interior"):
        if case == "pinned":
            xh = torch.from_numpy(x32.copy()).pin_memory()
            vh = torch.from_numpy(v32.copy()).pin_memory()
            mh = torch.from_numpy(mat.copy()).pin_memory()
            xa, va, ma = xh.numpy(), vh.numpy(), mh.numpy()
        elif case == "interior":
            xh = torch.zeros((sc.n + 3, 3), dtype=torch.float32).pin_memory()
            vh = torch.zeros((sc.n + 5, 3), dtype=torch.float32).pin_memory()
            mh = torch.zeros(sc.n + 16, dtype=torch.uint8).pin_memory()
            xh[3:] = torch.from_numpy(x32)
            vh[5:] = torch.from_numpy(v32)
            mh[16:] = torch.from_numpy(mat)
            xa, va, ma = xh.numpy()[3:], vh.numpy()[5:], mh.numpy()[16:]
        else:
            xa, va, ma = x32.copy(), v32.copy(), mat.copy()
        s, keep = ck.make_scene(sc.res, sc.dx, sc.dt, mats, xa, va, ma, gravity=sc.gravity, bc_cells=sc.bc_cells,
                                ppc=sc.ppc)
        ctx = ck.ckmpm_create(s, ck.KERNEL_CK, torch.cuda.current_stream().cuda_stream)
        ck.ckmpm_sync(ctx)  # the pinned arrays are read in stream order
        got = []
        for f, shape in ((ck.FIELD_X, (sc.n, 3)), (ck.FIELD_V, (sc.n, 3))):
            a = np.empty(shape, np.float32)
            ck.ckmpm_readback(ctx, 0, f, a.ctypes.data, a.nbytes, False)
            got.append(a)
        ck.ckmpm_step(ctx, 1)
        a = np.empty((sc.n, 3), np.float32)
        ck.ckmpm_readback(ctx, 0, ck.FIELD_X, a.ctypes.data, a.nbytes, False)
        got.append(a)
        ck.ckmpm_destroy(ctx)
        out[case] = got
        del keep
    for case in ("pinned", "interior"):
        assert np.array_equal(out[case][0], x32), case
        assert np.array_equal(out[case][0], out["pageable"][0]), case
        assert np.array_equal(out[case][1], out["pageable"][1]), case
        assert np.abs(out[case][2] - out["pageable"][2]).max() <= 1e-6 * sc.dx + 2e-7, case
