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


def _context_grids(ck, sc, B, F, transfer=0):
    sim = ck.Simulation(sc, sc.kernel | transfer)
    sim.write(ck.FIELD_F, F)
    if B is not None:
        sim.write(ck.FIELD_B, B)
    sim.probe_grids()
    gm = sim.read(ck.FIELD_GRID_M)
    gp = sim.read(ck.FIELD_GRID_P)
    sim.close()
    return gm, gp


class _StaticCall:
    """Device inputs and outputs of one scene, allocated up front, so that a
    call of the entry point itself needs no memory from anyone."""

    def __init__(self, ck, sc, B, F, transfer=0):
        dev = torch.device("cuda")
        self.ck, self.kernel = ck, sc.kernel | transfer
        self.x = torch.from_numpy(f32(sc.x)).to(dev)
        self.v = torch.from_numpy(f32(sc.v)).to(dev)
        self.mat = torch.from_numpy(sc.mat.copy()).to(dev)
        self.B = None if B is None else torch.from_numpy(B.reshape(-1, 9).copy()).to(dev)
        self.F = torch.from_numpy(F.reshape(-1, 9).copy()).to(dev)
        ng = 2 if sc.kernel == S.KERNEL_CK else 1
        nn = sc.res + 1
        self.gm = torch.empty((ng, nn, nn, nn), dtype=torch.float32, device=dev)
        self.gp = torch.empty((ng, nn, nn, nn, 3), dtype=torch.float32, device=dev)
        self.scs, self.keep = ck.make_scene(sc.res, sc.dx, sc.dt, sc.materials, self.x, self.v, self.mat,
                                            gravity=sc.gravity, bc_cells=sc.bc_cells, ppc=sc.ppc)
        self.stream = torch.cuda.current_stream().cuda_stream

    def __call__(self):
        self.ck.ckmpm_p2g_grids_static(self.scs, self.kernel, 0 if self.B is None else self.B.data_ptr(),
                                       self.F.data_ptr(), self.gm.data_ptr(), self.gp.data_ptr(), self.stream)
        return self.gm.cpu().numpy(), self.gp.cpu().numpy()


def _static_grids(ck, sc, B, F, transfer=0):
    return _StaticCall(ck, sc, B, F, transfer)()


def _check(gm, gp, gm_ref, gp_ref):
    for g in range(gm.shape[0]):
        assert rel(gm[g], gm_ref[g]) <= 1e-5
        assert np.abs(gp[g] - gp_ref[g]).max() <= 1e-5 * np.abs(gp_ref[g]).max()


@pytest.mark.parametrize("kernel", [S.KERNEL_CK, S.KERNEL_QUADRATIC])
def test_static_p2g_matches_context_path_on_two_calls(kernel):
    ck = need_gpu()
    for n, res, seed in ((20000, 48, 21), (7000, 32, 22)):
        sc, B, F = random_scene(n, res, seed, model=S.DRUCKER_PRAGER if seed % 2 else S.FIXED_COROTATED,
                                kernel=kernel, f_scale=0.08)
        gm_ref, gp_ref = _context_grids(ck, sc, B, F)
        gm, gp = _static_grids(ck, sc, B, F)
        _check(gm, gp, gm_ref, gp_ref)


def test_static_p2g_pic_matches_a_pic_context_on_two_calls():
    """The PIC transfer (no B; force from the kernel gradient) on the same
    fixed array, against a context created with CKMPM_TRANSFER_PIC."""
    ck = need_gpu()
    for n, res, seed in ((9000, 32, 24), (3000, 24, 25)):
        sc, _, F = random_scene(n, res, seed, model=S.FIXED_COROTATED, f_scale=0.08)
        gm_ref, gp_ref = _context_grids(ck, sc, None, F, transfer=ck.TRANSFER_PIC)
        gm, gp = _static_grids(ck, sc, None, F, transfer=ck.TRANSFER_PIC)
        _check(gm, gp, gm_ref, gp_ref)


def test_static_p2g_at_its_limits_takes_no_device_memory():
    """At the stated limits (65,536 particles on a 64^3 grid) the fixed array
    is large enough, and a call takes no device memory: with the inputs and
    outputs allocated beforehand and one warm-up call made (the first call on
    a GPU reserves the array and loads the kernels), the device's free memory
    is the same before and after a second call."""
    ck = need_gpu()
    sc, B, F = random_scene(65536, 64, 26, model=S.DRUCKER_PRAGER, f_scale=0.08)
    gm_ref, gp_ref = _context_grids(ck, sc, B, F)
    call = _StaticCall(ck, sc, B, F)
    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    gm, gp = call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check(gm, gp, gm_ref, gp_ref)


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
