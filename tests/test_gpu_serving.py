"""Serving extension: scenes run in one continuously batched context give the
same result as each scene run alone (positions within 1e-3 dx, the position
tolerance of the parity tests), while arriving at different times and with
different sizes and materials."""
import numpy as np
import pytest

from gpu_helpers import need_gpu
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


class StepClock:
    """Deterministic clock: 10 ms per poll, so arrivals map to global steps."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.01
        return self.t


def test_each_scene_alone_equals_in_the_mix():
    ck = need_gpu()
    from paper_2412_10399_gb300 import serving as SV
    reqs = S.served_mix(n_scenes=5, seed=7, n_max=3e5, steps=30)
    # stagger arrivals by global steps: 0, 0, 4, 9, 15 polls
    arrivals = [0.0, 0.0, 0.045, 0.095, 0.155]
    budget = SV.Budget.from_bytes(2 << 30, max_res=128, max_scenes=3)  # at most 3 resident at once
    eng = SV.EngineCK(budget)
    srv = SV.Server(eng, budget, clock=StepClock())
    for r, t in zip(reqs, arrivals):
        srv.submit(SV.Request(r.scene, r.scene.steps, arrival_s=t, read_fields=(ck.FIELD_X, ck.FIELD_F)))
    results = srv.run(sleep=lambda s: None)
    eng.close()
    assert len(results) == 5
    assert any(r.admitted_at_step > 0 for r in results)
    st = srv.stats()
    assert st["p99_ms"] is not None and st["p50_ms"] <= st["p99_ms"]
    for res in results:
        sc = res.request.scene
        sim = ck.Simulation(sc, ck.KERNEL_CK)
        sim.step(sc.steps)
        sim.sync()
        x = sim.read(ck.FIELD_X)
        F = sim.read(ck.FIELD_F)
        sim.close()
        assert np.abs(res.fields[ck.FIELD_X] - x).max() <= 1e-3 * sc.dx, sc.name
        assert np.abs(res.fields[ck.FIELD_F] - F).max() <= 1e-4, sc.name


def test_scenes_in_a_mixed_batch_match_the_oracle():
    """Three scenes with different cell sizes, time steps and materials share
    one context (one launch per kernel for all of them): a fixed-corotated
    scene on 32^3 (dt 1e-4), a Drucker-Prager scene on 64^3 (dt 5e-5) and a
    J-fluid scene on 16^3 (dt 2e-4), admitted at different global steps, one
    released before the end.  Each scene's positions match the FP64 oracle
    run of that scene alone within 1e-3 dx (the position tolerance of the
    parity tests) and its F within float32 rounding; key bases, block-table
    bases and material ranges of different scenes cannot cross."""
    import torch
    from gpu_helpers import oracle_state, random_scene, rel
    from oracle import ckmpm_oracle as O
    ck = need_gpu()
    a = random_scene(2000, 32, 61, model=S.FIXED_COROTATED, dt=1e-4, f_scale=0.05)
    b = random_scene(3000, 64, 62, model=S.DRUCKER_PRAGER, dt=5e-5, E=3.5e5, f_scale=0.05)
    c = random_scene(1500, 16, 63, model=S.J_FLUID, dt=2e-4, E=1e4, f_scale=0.05)
    scenes = [a, b, c]
    cfg = ck.ckmpm_config()
    cfg.kernel = ck.KERNEL_CK
    cfg.max_particles = sum(sc.n for sc, _, _ in scenes)
    cfg.max_keys = sum(((sc.res + 3) // 4) ** 3 for sc, _, _ in scenes)
    cfg.max_virtual_blocks = sum(((sc.res + 3) // 4 + 1) ** 3 for sc, _, _ in scenes)
    cfg.max_grid_blocks = cfg.max_virtual_blocks
    cfg.max_scenes = 3
    cfg.max_materials = 3
    cfg.stream = torch.cuda.current_stream().cuda_stream
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

    def read(sid, n, fld, shape):
        out = np.empty((n,) + shape, np.float32)
        ck.ckmpm_readback(srv, sid, fld, out.ctypes.data, out.nbytes, False)
        return out

    ia = admit(*a)
    ib = admit(*b)
    ck.ckmpm_step(srv, 3)
    ic = admit(*c)
    ck.ckmpm_step(srv, 5)
    got_a = (read(ia, a[0].n, ck.FIELD_X, (3,)), read(ia, a[0].n, ck.FIELD_F, (3, 3)))
    ck.ckmpm_release(srv, ia)
    ck.ckmpm_step(srv, 2)
    got_b = (read(ib, b[0].n, ck.FIELD_X, (3,)), read(ib, b[0].n, ck.FIELD_F, (3, 3)))
    got_c = (read(ic, c[0].n, ck.FIELD_X, (3,)), read(ic, c[0].n, ck.FIELD_F, (3, 3)))
    ck.ckmpm_destroy(srv)
    for (sc, B, F), steps, (x, Fg) in ((a, 8, got_a), (b, 10, got_b), (c, 7, got_c)):
        st = O.run(oracle_state(sc, B, F), O.params_from_scene(sc), steps)
        assert np.abs(x - st.x.numpy()).max() <= 1e-3 * sc.dx, sc.res
        assert rel(Fg, st.F.numpy()) <= 1e-4, sc.res
