"""Seeded scene generators: exact particle counts, determinism, and the declarative scene specs."""
import numpy as np
import pytest

from paper_2412_10399_gb300 import scenes as S


def test_splitmix64_reference_values():
    # SplitMix64 (Steele, Lea, Flood 2014) with state 0 advanced once by the
    # golden gamma yields 0xE220A8397B1DCDAF (published first output for seed 0).
    z = S.splitmix64(np.array([0], np.uint64), 0)
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_config_particle_counts():
    assert S.elastic_cube().n == 32768
    assert S.granular_column().n == 346112
    assert S.differentiable_cube().n == 262144


def test_large_impact_counts():
    sc = S.large_impact()
    assert sc.n == 16273664
    assert int((sc.mat == 0).sum()) == 16138496
    assert int((sc.mat == 1).sum()) == 135168
    u = sc.x / sc.dx
    assert u.min() > 3.0 and u.max() < sc.res - 3.0


def test_generators_are_deterministic_and_stratified():
    a, b = S.elastic_cube(seed=3), S.elastic_cube(seed=3)
    assert np.array_equal(a.x, b.x)
    c = S.elastic_cube(seed=4)
    assert not np.array_equal(a.x, c.x)
    # one particle per sub-cell: 2*frac(x/dx) floors to the sub-cell index
    sub = np.floor(2 * (a.x / a.dx - np.floor(a.x / a.dx))).astype(int)
    code = sub[:, 0] + 2 * sub[:, 1] + 4 * sub[:, 2]
    assert np.array_equal(code.reshape(-1, 8), np.tile(np.arange(8), (a.n // 8, 1)))


def test_served_mix_shapes():
    reqs = S.served_mix(n_scenes=16)
    assert len(reqs) == 16
    t = [r.arrival_s for r in reqs]
    assert all(t1 > t0 for t0, t1 in zip(t, t[1:]))
    for r in reqs:
        assert 5e3 < r.scene.n < 2.2e6
        u = r.scene.x / r.scene.dx
        assert u.min() > 3.0 and u.max() < r.scene.res - 3.0


def test_dam_break_counts_and_bounds():
    for n in (4175808, 8994048):
        sc = S.dam_break(n)
        assert sc.n == n and sc.res == 256
        u = sc.x / sc.dx
        assert u.min() >= 4.0 and u[:, 1].max() < 4.0 + n / 8.0 / (96.0 if n <= 5_000_000 else 128.0) ** 2
        assert sc.materials[0].model == S.J_FLUID


def _impact_spec():
    sand = [{"box": {"lo": [154, 4, 154], "hi": [358, 36, 358]}},
            {"box": {"lo": [226, 36, 226], "hi": [286, 86, 286]}}]
    for tx in (174, 338):
        for tz in (174, 338):
            sand.append({"cylinder_y": {"cx": tx, "cz": tz, "r": 20.0, "y0": 36, "y1": 136}})
    bodies = [{"material": 0, "shapes": sand}]
    for c in ((201, 60, 256), (311, 60, 256), (256, 60, 201), (256, 60, 311)):
        d = np.array([256.0 - c[0], 0.0, 256.0 - c[2]])
        d /= np.linalg.norm(d)
        bodies.append({"material": 1, "velocity": (20.0 * d).tolist(), "shapes": [{"sphere": {"centre": list(c), "r": 10.0}}]})
    return {"name": "large_impact", "res": 512, "dt": 2e-5, "steps": 200,
            "materials": [{"model": "drucker_prager", "E": 3.5e5, "nu": 0.3, "rho": 1600.0, "friction_deg": 30.0},
                          {"model": "fixed_corotated", "E": 1e7, "nu": 0.3, "rho": 1e4}],
            "bodies": bodies}


def test_spec_reproduces_the_built_in_scenes():
    cube = {"name": "elastic_cube", "res": 64, "dt": 1e-4,
            "materials": [{"model": "fixed_corotated", "E": 1e5, "nu": 0.3, "rho": 1000.0}],
            "bodies": [{"shapes": [{"box": {"lo": [24, 40, 24], "hi": [40, 56, 40]}}]}]}
    for spec, ref in ((cube, S.elastic_cube()), (_impact_spec(), S.large_impact())):
        sc = S.scene_from_spec(spec)
        assert sc.n == ref.n
        assert np.array_equal(sc.x, ref.x) and np.array_equal(sc.v, ref.v) and np.array_equal(sc.mat, ref.mat)
        assert (sc.res, sc.dx, sc.dt, sc.gravity, sc.materials) == (ref.res, ref.dx, ref.dt, ref.gravity, ref.materials)


def test_spec_bodies_do_not_overlap_and_json_round_trip(tmp_path):
    import json
    spec = {"res": 32, "dt": 1e-4, "kernel": "quadratic", "transfer": "pic",
            "materials": [{"model": "fixed_corotated", "E": 1e5, "nu": 0.3, "rho": 1000.0},
                          {"model": "j_fluid", "E": 10.0, "nu": 0.0, "rho": 1000.0, "gamma": 7.0}],
            "bodies": [{"material": 0, "shapes": [{"box": {"lo": [8, 8, 8], "hi": [16, 16, 16]}}]},
                       {"material": 1, "velocity": [0, -1, 0], "shapes": [{"box": {"lo": [12, 12, 12], "hi": [20, 20, 20]}}]}]}
    p = tmp_path / "s.json"
    p.write_text(json.dumps(spec))
    sc = S.load_scene(str(p))
    assert sc.n == 8 * (2 * 8 ** 3 - 4 ** 3)  # the second body skips the 4^3 cells the first one filled
    cells = np.unique(np.floor(sc.x / sc.dx).astype(np.int64) @ np.array([1, 32, 32 * 32]))
    assert len(cells) * 8 == sc.n
    assert sc.kernel == S.KERNEL_QUADRATIC and sc.transfer == S.TRANSFER_PIC
    assert sc.materials[1].model == S.J_FLUID and sc.materials[1].gamma == 7.0
    assert np.all(sc.v[sc.mat == 1] == [0, -1, 0]) and np.all(sc.v[sc.mat == 0] == 0)


@pytest.mark.parametrize("bad", [
    {"bodies": [{"shapes": [{"cone": {}}]}]},
    {"materials": [{"model": "nacc", "E": 1.0, "nu": 0.3, "rho": 1.0}]},
    {"bodies": [{"material": 3, "shapes": [{"box": {"lo": [8, 8, 8], "hi": [9, 9, 9]}}]}]},
    {"bodies": [{"shapes": [{"box": {"lo": [8, 8, 8], "hi": [8, 8, 8]}}]}]},
    {"kernel": "cubic"},
])
def test_spec_errors(bad):
    spec = {"res": 32, "dt": 1e-4, "materials": [{"model": "fixed_corotated", "E": 1e5, "nu": 0.3, "rho": 1000.0}],
            "bodies": [{"shapes": [{"box": {"lo": [8, 8, 8], "hi": [12, 12, 12]}}]}]}
    spec.update(bad)
    with pytest.raises(ValueError):
        S.scene_from_spec(spec)
