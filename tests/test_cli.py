"""The command line (python -m paper_2412_10399_gb300): scene info without a
GPU, and the run loop's stepping and checkpoint schedule against a stand-in
for the Simulation class."""
import json

import pytest

from paper_2412_10399_gb300 import __main__ as cli
from paper_2412_10399_gb300 import scenes as S

SPEC = {"name": "two_bodies", "res": 32, "dt": 1e-4, "steps": 7,
        "materials": [{"model": "fixed_corotated", "E": 1e5, "nu": 0.3, "rho": 1000.0},
                      {"model": "drucker_prager", "E": 3.5e5, "nu": 0.3, "rho": 1600.0, "friction_deg": 30.0}],
        "bodies": [{"material": 0, "shapes": [{"box": {"lo": [8, 8, 8], "hi": [12, 12, 12]}}]},
                   {"material": 1, "velocity": [1, 0, 0], "shapes": [{"sphere": {"centre": [20, 20, 20], "r": 3}}]}]}


@pytest.fixture
def spec_file(tmp_path):
    p = tmp_path / "scene.json"
    p.write_text(json.dumps(SPEC))
    return str(p)


def test_info(spec_file, capsys):
    assert cli.main(["info", spec_file]) == 0
    info = json.loads(capsys.readouterr().out)
    sc = S.load_scene(spec_file)
    assert info["particles"] == sc.n == 8 * (4 ** 3 + len(S.filled_cells([S._sphere((20, 20, 20), 3.0)], 32)))
    assert info["kernel"] == "ck" and info["transfer"] == "apic_mls"
    assert [m["model"] for m in info["materials"]] == ["fixed_corotated", "drucker_prager"]
    assert info["device_bytes"] > sc.n * 200


class _FakeSim:
    log = []

    def __init__(self, sc, kernel):
        _FakeSim.log.append(("create", sc.n, kernel))

    def load(self, p):
        _FakeSim.log.append(("load", p))

    def step(self, k):
        _FakeSim.log.append(("step", k))

    def sync(self):
        pass

    def save(self, p):
        _FakeSim.log.append(("save", p))
        open(p, "w").close()

    def close(self):
        _FakeSim.log.append(("close",))


def test_run_schedule(spec_file, tmp_path):
    _FakeSim.log = []
    sc = cli._apply_overrides(S.load_scene(spec_file), type("A", (), {"kernel": "quadratic", "transfer": "pic"}))
    out = str(tmp_path / "frames")
    paths = cli.run(sc, 7, 3, out, resume="r.npz", sim_cls=_FakeSim, log=lambda *a: None)
    assert [p.rsplit("/", 1)[1] for p in paths] == ["frame_00003.npz", "frame_00006.npz", "frame_00007.npz"]
    assert _FakeSim.log[0] == ("create", sc.n, S.KERNEL_QUADRATIC | 2)
    assert _FakeSim.log[1] == ("load", "r.npz")
    assert [e[1] for e in _FakeSim.log if e[0] == "step"] == [3, 3, 1]
    assert _FakeSim.log[-1] == ("close",)


def test_run_rejects_bad_counts(spec_file):
    for bad in (["--steps", "0"], ["--every", "0"]):
        with pytest.raises(SystemExit):
            cli.main(["run", spec_file, *bad])


def test_cfl_number_of_the_built_in_scenes():
    import math
    sc = S.elastic_cube()  # E 1e5, nu 0.3, rho 1000, at rest, dt 1e-4, dx 1/64
    c = math.sqrt(1e5 * 0.7 / (1.3 * 0.4) / 1000.0)
    assert cli.cfl_number(sc) == pytest.approx(1e-4 * c * 64)
    impact = S.large_impact()  # stiff balls at 20 m/s
    assert 0.3 < cli.cfl_number(impact) < 1.0
    dam = S.dam_break(20000)  # fluid: sqrt(gamma B / rho)
    assert cli.cfl_number(dam) == pytest.approx(1e-4 * math.sqrt(7.15 * 10.0 / 1000.0) * 256)


def test_run_warns_when_dt_is_too_large(spec_file):
    _FakeSim.log = []
    sc = S.load_scene(spec_file)
    sc.dt = 1.0
    msgs = []
    cli.run(sc, 1, 1, spec_file + "_out", sim_cls=_FakeSim, log=msgs.append)
    assert msgs and msgs[0].startswith("warning")
