"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"^CKMPM_API\s+[\w\s\*]+?\b(ckmpm_\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("ckmpm_create", "ckmpm_step", "ckmpm_readback", "ckmpm_upload", "ckmpm_destroy",
              "ckmpm_last_error", "ckmpm_admit", "ckmpm_release", "ckmpm_sync"):
        assert n in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_2412_10399_gb300 import ckmpm
    lib = ckmpm.load()
    for n in _declared():
        assert hasattr(lib, n), n
        assert n in ckmpm.SIGNATURES, f"binding lacks {n}"
    assert ckmpm.ckmpm_version().startswith("ckmpm")


def test_null_arguments_are_rejected_without_a_gpu():
    from paper_2412_10399_gb300 import ckmpm
    lib = ckmpm.load()
    assert lib.ckmpm_destroy(None) == ckmpm.OK
    assert lib.ckmpm_step(None, 1) == ckmpm.EINVAL
    assert lib.ckmpm_sync(None) == ckmpm.EINVAL
    assert lib.ckmpm_last_error(None) == b"no context"
    assert lib.ckmpm_scene_particles(None, 0) == -1
    out = ctypes.c_void_p()
    assert lib.ckmpm_create(None, 0, None, ctypes.byref(out)) == ckmpm.EINVAL
    assert out.value is None


def test_invalid_scene_is_rejected_before_any_device_work():
    import numpy as np
    from paper_2412_10399_gb300 import ckmpm, scenes
    x = np.full((4, 3), 0.5, np.float32)
    sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, [scenes.ELASTIC], x)
    sc.res = 2  # below the minimum
    out = ctypes.c_void_p()
    assert ckmpm.load().ckmpm_create(ctypes.byref(sc), 0, None, ctypes.byref(out)) == ckmpm.EINVAL
    sc.res = 16
    sc.dt = -1.0
    assert ckmpm.load().ckmpm_create(ctypes.byref(sc), 0, None, ctypes.byref(out)) == ckmpm.EINVAL
