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
    assert lib.ckmpm_readback_wait(None, 0) == ckmpm.EINVAL
    t = ctypes.c_int64(7)
    assert lib.ckmpm_readback_async(None, 0, ckmpm.FIELD_X, None, 0, ctypes.byref(t)) == ckmpm.EINVAL
    assert t.value == -1
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


def _header_text():
    return "\n".join(open(h).read() for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))


def _strip_comments(txt):
    return re.sub(r"/\*.*?\*/", "", txt, flags=re.S)


def test_binding_constants_match_the_header_enums():
    """Every CKMPM_* enumerator of the header has the value the Python binding uses."""
    from paper_2412_10399_gb300 import ckmpm
    txt = _strip_comments(_header_text())
    enums = {}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", txt, flags=re.S):
        for name, val in re.findall(r"(CKMPM_\w+)\s*=\s*(\d+)", body):
            enums[name] = int(val)
    assert len(enums) >= 25
    for name, val in enums.items():
        py = name[len("CKMPM_"):]
        if py.startswith("FIELD_") or py.startswith("KERNEL_") or py.startswith("TRANSFER_") or \
                py in ckmpm.STATUS_NAMES or py in ("FIXED_COROTATED", "DRUCKER_PRAGER", "J_FLUID"):
            assert getattr(ckmpm, py) == val, name


def test_binding_structs_match_the_header_field_order():
    """The ctypes structures list the header's struct members in the same order
    (the C ABI passes them by layout)."""
    from paper_2412_10399_gb300 import ckmpm
    txt = _strip_comments(_header_text())
    structs = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(ckmpm_\w+)\s*;", txt, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.search(r"\(\s*\*\s*(\w+)\s*\)", decl)  # function pointer
            if m is None:
                m = re.search(r"(\w+)\s*(\[[^\]]*\])?\s*$", decl)
            fields.append(m.group(1))
        structs[name] = fields
    for name in ("ckmpm_material", "ckmpm_scene", "ckmpm_allocator", "ckmpm_config", "ckmpm_stats"):
        py = [f[0] for f in getattr(ckmpm, name)._fields_]
        assert py == structs[name], name


def test_header_is_plain_c_and_a_c_program_links_and_calls(tmp_path):
    """include/ckmpm.h compiles as C99 with warnings as errors, and a C program
    linked against the library calls it (argument checks only, no GPU)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    import __graft_entry__ as g
    g.build()
    lib = os.path.join(ROOT, "paper_2412_10399_gb300")
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "ckmpm.h"
int main(void) {
  ckmpm_ctx* ctx = NULL;
  ckmpm_scene sc;
  memset(&sc, 0, sizeof sc);
  if (ckmpm_create(NULL, CKMPM_KERNEL_CK | CKMPM_TRANSFER_PIC, NULL, &ctx) != CKMPM_EINVAL || ctx) return 1;
  if (ckmpm_create(&sc, CKMPM_KERNEL_CK, NULL, &ctx) != CKMPM_EINVAL || ctx) return 2;
  if (ckmpm_step(NULL, 1) != CKMPM_EINVAL) return 3;
  if (ckmpm_destroy(NULL) != CKMPM_OK) return 4;
  if (strncmp(ckmpm_version(), "ckmpm", 5) != 0) return 5;
  printf("%s\n", ckmpm_version());
  return 0;
}
''')
    exe = tmp_path / "use"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", lib, "-lckmpm", f"-Wl,-rpath,{lib}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("ckmpm")


def test_make_scene_checks_shapes_and_converts_types():
    import numpy as np
    from unittest import mock

    import torch

    from paper_2412_10399_gb300 import ckmpm, scenes
    x = np.full((4, 3), 0.5)
    for kw in ({"v": np.zeros((3, 3))}, {"v": np.zeros(12)}, {"mat": np.zeros(5, np.uint8)}):
        with pytest.raises(ValueError):
            ckmpm.make_scene(16, 1 / 16, 1e-4, [scenes.ELASTIC], x, **kw)
    with pytest.raises(ValueError):
        ckmpm.make_scene(16, 1 / 16, 1e-4, [scenes.ELASTIC], np.zeros((4, 2)))
    sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, [scenes.ELASTIC], x, np.zeros((4, 3)), [0, 0, 0, 0])
    assert sc.n == 4 and keep[0].dtype == np.float32 and keep[2].dtype == np.uint8
    # device tensors are converted on their device, not reinterpreted
    with mock.patch.object(torch.Tensor, "is_cuda", new_callable=mock.PropertyMock, return_value=True):
        sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, [scenes.ELASTIC], torch.full((4, 3), 0.5, dtype=torch.float64),
                                    torch.zeros(4, 3).t().contiguous().t(), torch.zeros(4, dtype=torch.int64))
    assert sc.is_device == 1
    assert keep[0].dtype == torch.float32 and keep[1].is_contiguous() and keep[2].dtype == torch.uint8


@pytest.mark.parametrize("field,value", [
    ("dx", float("inf")), ("dt", float("nan")), ("dt", float("inf")), ("bc_cells", float("inf")),
    ("fp64_j_tol", -1.0), ("fp64_gap_tol", float("nan")), ("gravity", (0.0, float("nan"), 0.0)),
    ("E", float("inf")), ("rho", float("inf")), ("friction_deg", float("nan")), ("nu", 0.5), ("E", -1.0),
])
def test_non_finite_or_out_of_range_parameters_are_rejected(field, value):
    """Scene and material parameters that would turn into non-finite state on
    the device are refused with EINVAL at creation (no device work, no GPU)."""
    import numpy as np
    from paper_2412_10399_gb300 import ckmpm, scenes
    mat = scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3, 1000.0, 30.0)
    if field in ("E", "rho", "friction_deg", "nu"):
        mat = scenes.Material(**{**mat.__dict__, field: value})
    sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, [mat], np.full((4, 3), 0.5, np.float32))
    if field == "gravity":
        sc.gravity = (ctypes.c_double * 3)(*value)
    elif field not in ("E", "rho", "friction_deg", "nu"):
        setattr(sc, field, value)
    out = ctypes.c_void_p()
    assert ckmpm.load().ckmpm_create(ctypes.byref(sc), 0, None, ctypes.byref(out)) == ckmpm.EINVAL
    assert out.value is None


def test_material_index_and_friction_angle_are_checked_before_any_device_work():
    """A host material byte at or above n_materials, and a Drucker-Prager
    friction angle outside [0, 90) degrees, are EINVAL before the library
    touches the GPU (so this runs without one)."""
    import numpy as np
    from paper_2412_10399_gb300 import ckmpm, scenes
    x = np.full((6, 3), 0.5, np.float32)
    mat = np.array([0, 1, 1, 0, 2, 1], np.uint8)
    sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, [scenes.ELASTIC, scenes.SAND], x, mat=mat)
    out = ctypes.c_void_p()
    lib = ckmpm.load()
    assert lib.ckmpm_create(ctypes.byref(sc), 0, None, ctypes.byref(out)) == ckmpm.EINVAL
    assert out.value is None
    bad = scenes.Material(scenes.DRUCKER_PRAGER, 3.5e5, 0.3, 1600.0, -5.0)
    sc2, keep2 = ckmpm.make_scene(16, 1 / 16, 1e-4, [bad], x)
    assert lib.ckmpm_create(ctypes.byref(sc2), 0, None, ctypes.byref(out)) == ckmpm.EINVAL


def test_material_index_check_at_every_position_and_table_size():
    """The host check of material indices tests eight bytes per step for
    tables of up to 128 materials and one byte at a time for larger ones
    and for the tail: an index equal to n_materials (or 255) is EINVAL at
    any position, and arrays whose largest index is n_materials - 1 pass the
    check (without a GPU, creation then fails later, but not with EINVAL)."""
    import numpy as np
    from paper_2412_10399_gb300 import ckmpm, scenes
    lib = ckmpm.load()
    n = 37  # four words and a five-byte tail
    x = np.full((n, 3), 0.5, np.float32)
    g = np.random.default_rng(7)
    for nm in (1, 2, 3, 127, 128, 129, 200, 255):
        mats = [scenes.ELASTIC] * nm
        for fill in ("max", "random"):
            mat = np.full(n, nm - 1, np.uint8) if fill == "max" else g.integers(0, nm, n).astype(np.uint8)
            sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, mats, x, mat=mat)
            out = ctypes.c_void_p()
            st = lib.ckmpm_create(ctypes.byref(sc), 0, None, ctypes.byref(out))
            assert st != ckmpm.EINVAL, (nm, fill)
            if st == ckmpm.OK:
                lib.ckmpm_destroy(out)
        if nm == 255:
            continue  # every byte value is a valid index
        for pos in (0, 7, 8, 15, 31, 32, 36):
            for badv in (nm, 255):
                mat = np.zeros(n, np.uint8)
                mat[pos] = badv
                sc, keep = ckmpm.make_scene(16, 1 / 16, 1e-4, mats, x, mat=mat)
                out = ctypes.c_void_p()
                assert lib.ckmpm_create(ctypes.byref(sc), 0, None, ctypes.byref(out)) == ckmpm.EINVAL, (nm, pos, badv)
