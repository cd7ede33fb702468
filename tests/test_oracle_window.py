"""The local-window oracle step the full-size GPU parity test relies on: one
particle's step computed from only the particles within 3 cells of it,
shifted by whole cells into a 14^3 domain without walls, equals the same
particle's step in the whole domain (to float64 rounding), for both kernels,
for elastic and plastic particles with stress, when the whole domain's walls
touch none of its nodes.  A window of 1 cell (missing neighbours) must not."""
import numpy as np
import pytest
import torch

from gpu_helpers import window_step
from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S


@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_window_step_equals_whole_domain_step(kernel):
    res = 32
    x, v, B, F = S.random_state(4000, res, 61, margin_cells=4.0, f_scale=0.1)
    mat = (np.arange(4000) % 2).astype(np.uint8)
    mats = [O.Mat(O.FIXED_COROTATED, 1e5, 0.3, 1000.0), O.Mat(O.DRUCKER_PRAGER, 1e5, 0.3, 1600.0, 30.0)]
    prm = O.Params(res=res, dx=1.0 / res, dt=1e-4, materials=mats, kernel=kernel)
    whole = O.step(O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.from_numpy(B),
                                torch.from_numpy(F), mat=torch.from_numpy(mat.astype(np.int64))), prm)
    local = O.Params(res=14, dx=prm.dx, dt=prm.dt, materials=mats, kernel=kernel, bc_cells=0.0)
    cell = np.floor(x / prm.dx).astype(np.int32)
    inner = np.flatnonzero(np.all((cell >= 8) & (cell < res - 8), axis=1))
    rng = np.random.default_rng(0)
    for p in rng.choice(inner, 12, replace=False):
        (wx, wv, wF, wB), near, _, _ = window_step(x, v, B, F, mat, cell, p, local, prm.dx)
        assert np.abs(wx - whole.x[p].numpy()).max() <= 1e-15
        assert np.abs(wv - whole.v[p].numpy()).max() <= 1e-12
        assert np.abs(wF - whole.F[p].numpy()).max() <= 1e-12
        assert np.abs(wB - whole.B[p].numpy()).max() <= 1e-12
    # too small a window misses particles that reach p's nodes
    diffs = [np.abs(window_step(x, v, B, F, mat, cell, p, local, prm.dx, halo=1)[0][1] - whole.v[p].numpy()).max()
             for p in inner[:12]]
    assert max(diffs) > 1e-6
