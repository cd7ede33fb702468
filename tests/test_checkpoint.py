"""Checkpoints of a Simulation (save / load through readback and upload): the
file holds the fields the transfer keeps, and load uploads them in the order
the state needs (x, v, F, then B).  Runs on CPU against an in-memory stand-in
for the context's readback and upload."""
import numpy as np
import pytest

from paper_2412_10399_gb300 import ckmpm as ck


class _Fake:
    def __init__(self, n, kernel, seed):
        self.sim = object.__new__(ck.Simulation)
        self.sim.n, self.sim.kernel, self.sim.res = n, kernel, 16
        rng = np.random.default_rng(seed)
        self.state = {ck.FIELD_X: rng.random((n, 3)), ck.FIELD_V: rng.random((n, 3)),
                      ck.FIELD_F: rng.random((n, 3, 3)), ck.FIELD_B: rng.random((n, 3, 3))}
        self.state = {k: v.astype(np.float32) for k, v in self.state.items()}
        self.writes = []
        self.sim.read = lambda f, scene_id=0: self.state[f].copy()
        self.sim.write = self._write

    def _write(self, f, a, scene_id=0):
        self.writes.append(f)
        self.state[f] = np.asarray(a, np.float32).copy()


@pytest.mark.parametrize("kernel", [ck.KERNEL_CK, ck.KERNEL_QUADRATIC, ck.KERNEL_CK | ck.TRANSFER_APIC_GRAD])
def test_checkpoint_round_trip_and_upload_order(tmp_path, kernel):
    a, b = _Fake(50, kernel, 1), _Fake(50, kernel, 2)
    a.sim.save(str(tmp_path / "c.npz"))
    b.sim.load(str(tmp_path / "c.npz"))
    assert b.writes == [ck.FIELD_X, ck.FIELD_V, ck.FIELD_F, ck.FIELD_B]
    for f in a.state:
        assert np.array_equal(a.state[f], b.state[f])


def test_pic_checkpoint_has_no_B(tmp_path):
    a, b = _Fake(20, ck.KERNEL_CK | ck.TRANSFER_PIC, 1), _Fake(20, ck.KERNEL_CK | ck.TRANSFER_PIC, 2)
    a.sim.save(str(tmp_path / "c.npz"))
    assert "B" not in np.load(str(tmp_path / "c.npz")).files
    b.sim.load(str(tmp_path / "c.npz"))
    assert b.writes == [ck.FIELD_X, ck.FIELD_V, ck.FIELD_F]


def test_checkpoint_of_another_scene_is_refused(tmp_path):
    a = _Fake(20, ck.KERNEL_CK, 1)
    a.sim.save(str(tmp_path / "c.npz"))
    with pytest.raises(ValueError):
        _Fake(21, ck.KERNEL_CK, 2).sim.load(str(tmp_path / "c.npz"))
    with pytest.raises(ValueError):
        _Fake(20, ck.KERNEL_QUADRATIC, 2).sim.load(str(tmp_path / "c.npz"))
