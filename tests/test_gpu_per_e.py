"""Per-particle Young's modulus in a context (ckmpm_config.per_particle_E,
CKMPM_FIELD_E): upload E per particle, step once, compare every particle field
with the FP64 oracle given the same per-particle E.  Tolerances as for the
one-step parity tests (x within 1e-6 dx, v 2e-5, F 2e-6, B 5e-5 relative)."""
import numpy as np
import pytest
import torch

from gpu_helpers import need_gpu, oracle_state, random_scene, rel
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_per_particle_E_one_step_parity():
    ck = need_gpu()
    sc, B, F = random_scene(3000, 32, 71, model=S.FIXED_COROTATED, f_scale=0.08)
    n = sc.n
    E = (1e5 * np.random.default_rng(71).uniform(0.5, 1.5, n)).astype(np.float32)
    cfg = ck.ckmpm_config()
    cfg.kernel = ck.KERNEL_CK
    cfg.max_particles = n
    cfg.max_keys = 8 ** 3
    cfg.max_virtual_blocks = 9 ** 3
    cfg.max_grid_blocks = 9 ** 3
    cfg.max_scenes = 1
    cfg.max_materials = 1
    cfg.per_particle_E = 1
    cfg.stream = torch.cuda.current_stream().cuda_stream
    ctx = ck.ckmpm_create_server(cfg)
    scs, keep = ck.scene_struct(sc)
    sid = ck.ckmpm_admit(ctx, scs)

    def put(field, a):
        a = np.ascontiguousarray(a, np.float32)
        ck.ckmpm_upload(ctx, sid, field, a.ctypes.data, a.nbytes, False)

    def get(field, shape):
        out = np.empty(shape, np.float32)
        ck.ckmpm_readback(ctx, sid, field, out.ctypes.data, out.nbytes, False)
        return out

    put(ck.FIELD_E, E)
    put(ck.FIELD_F, F)
    put(ck.FIELD_B, B)
    assert np.array_equal(get(ck.FIELD_E, (n,)), E)
    ck.ckmpm_step(ctx, 1)
    ck.ckmpm_sync(ctx)
    got = {f: get(f, (n, 3) if f in (ck.FIELD_X, ck.FIELD_V) else (n, 3, 3))
           for f in (ck.FIELD_X, ck.FIELD_V, ck.FIELD_F, ck.FIELD_B)}
    ck.ckmpm_destroy(ctx)
    prm = O.params_from_scene(sc)
    st = oracle_state(sc, B, F)
    st.E = torch.from_numpy(E.astype(np.float64))
    new = O.step(st, prm)
    assert np.abs(got[ck.FIELD_X] - new.x.numpy()).max() <= 1e-6 * sc.dx + 2e-7
    assert rel(got[ck.FIELD_V], new.v.numpy()) <= 2e-5
    assert rel(got[ck.FIELD_F], new.F.numpy()) <= 2e-6
    assert rel(got[ck.FIELD_B], new.B.numpy()) <= 5e-5
    # the per-particle moduli matter: the material's single E gives another step
    plain = O.step(oracle_state(sc, B, F), prm)
    assert rel(plain.v.numpy(), new.v.numpy()) > 1e-3
