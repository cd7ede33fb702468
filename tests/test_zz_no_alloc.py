"""The allocation-free P2G entry point (ckmpm_p2g_grids_static) against the
regular context path.

Callers that may not allocate device memory at call time (an application
whose own arena owns the GPU memory, a real-time loop that cannot take
cudaMalloc's implicit synchronisation, a plug-in that must keep its footprint
fixed) use ckmpm_p2g_grids_static, which works in a fixed array inside the
library.  This test calls it through the C ABI twice in a row, with different
particle sets, and checks both results against ckmpm_create + ckmpm_upload +
ckmpm_probe_grids + ckmpm_readback, within the 1e-5 relative grid tolerance
the other parity tests use.  The second call checks that what the first call
left in the shared array does not leak into the next result.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import f32, need_gpu, random_scene, rel
from paper_2412_10399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _context_grids(ck, sc, B, F):
    sim = ck.Simulation(sc, sc.kernel)
    sim.write(ck.FIELD_F, F)
    sim.write(ck.FIELD_B, B)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    return gm, gp


def _static_grids(ck, sc, B, F):
    dev = torch.device("cuda")
    x = torch.from_numpy(f32(sc.x)).to(dev)
    v = torch.from_numpy(f32(sc.v)).to(dev)
    mat = torch.from_numpy(sc.mat.copy()).to(dev)
    Bd = torch.from_numpy(B.reshape(-1, 9).copy()).to(dev)
    Fd = torch.from_numpy(F.reshape(-1, 9).copy()).to(dev)
    ng = 2 if sc.kernel == S.KERNEL_CK else 1
    nn = sc.res + 1
    gm = torch.empty((ng, nn, nn, nn), dtype=torch.float32, device=dev)
    gp = torch.empty((ng, nn, nn, nn, 3), dtype=torch.float32, device=dev)
    scs, keep = ck.make_scene(sc.res, sc.dx, sc.dt, sc.materials, x, v, mat, gravity=sc.gravity,
                              bc_cells=sc.bc_cells, ppc=sc.ppc)
    stream = torch.cuda.current_stream().cuda_stream
    ck.ckmpm_p2g_grids_static(scs, sc.kernel, Bd.data_ptr(), Fd.data_ptr(), gm.data_ptr(), gp.data_ptr(), stream)
    return gm.cpu().numpy(), gp.cpu().numpy()


@pytest.mark.parametrize("kernel", [S.KERNEL_CK, S.KERNEL_QUADRATIC])
def test_static_p2g_matches_context_path_on_two_calls(kernel):
    ck = need_gpu()
    for n, res, seed in ((20000, 48, 21), (7000, 32, 22)):
        sc, B, F = random_scene(n, res, seed, model=S.DRUCKER_PRAGER if seed % 2 else S.FIXED_COROTATED,
                                kernel=kernel, f_scale=0.08)
        gm_ref, gp_ref = _context_grids(ck, sc, B, F)
        gm, gp = _static_grids(ck, sc, B, F)
        for g in range(gm.shape[0]):
            assert rel(gm[g], gm_ref[g]) <= 1e-5
            assert np.abs(gp[g] - gp_ref[g]).max() <= 1e-5 * np.abs(gp_ref[g]).max()


def test_static_p2g_rejects_sizes_beyond_its_limits():
    ck = need_gpu()
    sc, B, F = random_scene(100, 80, 23)  # res 80 > 64
    dev = torch.device("cuda")
    x = torch.from_numpy(f32(sc.x)).to(dev)
    scs, keep = ck.make_scene(sc.res, sc.dx, sc.dt, sc.materials, x)
    out = torch.empty(8, device=dev)
    with pytest.raises(ck.CKMPMError) as ei:
        ck.ckmpm_p2g_grids_static(scs, 0, 0, 0, out.data_ptr(), out.data_ptr(), 0)
    assert ei.value.status == ck.EINVAL
