"""Argument checks of the differentiable stepper's Python side: the library
reads and writes its arrays through raw device pointers, so anything but a
contiguous float32 CUDA tensor of the state's shape is refused before any
call into the library (no GPU needed)."""
from unittest import mock

import pytest
import torch

from paper_2412_10399_gb300 import diff


def _sim(n):
    s = object.__new__(diff.DiffSim)
    s.n, s.h = n, None
    return s


def _state(n):
    return (torch.zeros(n, 3), torch.zeros(n, 3), torch.zeros(n, 3, 3), torch.zeros(n, 3, 3), torch.zeros(n))


def test_cpu_tensors_are_refused_before_the_library_is_called():
    s = _sim(5)
    with mock.patch.object(diff.ck, "load", side_effect=AssertionError("library called")):
        with pytest.raises(ValueError, match="CUDA"):
            s.step(*_state(5))
        with pytest.raises(ValueError):
            s.step_backward(*_state(5), *_state(5)[:4], torch.zeros(5))


def test_shapes_dtypes_and_layout_are_checked():
    s = _sim(4)
    good = dict(zip(("x", "v", "B", "F", "E"), _state(4)))
    with mock.patch.object(torch.Tensor, "is_cuda", new_callable=mock.PropertyMock, return_value=True):
        s._check(**good)  # passes
        s._check(gx1=good["x"], gv1=good["v"], gB1=good["B"], gF1=good["F"], gE=good["E"])
        for name, bad in (("x", torch.zeros(4, 4)), ("B", torch.zeros(4, 9)), ("E", torch.zeros(4, 1)),
                          ("v", torch.zeros(4, 3, dtype=torch.float64)), ("F", torch.zeros(4, 3, 3).transpose(1, 2)),
                          ("gB1", torch.zeros(3, 3, 3))):
            with pytest.raises(ValueError, match=name):
                s._check(**{name: bad})
