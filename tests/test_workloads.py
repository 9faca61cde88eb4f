"""The seeded input generator: determinism and the scales the recipe fixes."""
import numpy as np

from workloads import lunar_tile, make_instance, random_origins, bump_target, sun_list
from workloads.terrain import crater_radii


def test_tile_is_deterministic_and_float32():
    a = lunar_tile(64, 20.0, seed=3)
    b = lunar_tile(64, 20.0, seed=3)
    c = lunar_tile(64, 20.0, seed=4)
    assert a.dtype == np.float32 and a.shape == (64, 64)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_fbm_amplitude_and_crater_sizes():
    from workloads.terrain import fbm
    h = fbm(128, 96, np.random.default_rng(0), amplitude=1500.0)
    assert abs(np.abs(h).max() - 1500.0) < 1e-9
    assert abs(h.mean()) < 1e-9
    r = crater_radii(100000, np.random.default_rng(1))
    assert r.min() >= 200.0 and r.max() <= 2000.0
    # N(>r) ~ r^-2: the fraction above 400 m is (400^-2 - 2000^-2)/(200^-2 - 2000^-2)
    frac = np.mean(r > 400.0)
    expect = (400.0 ** -2 - 2000.0 ** -2) / (200.0 ** -2 - 2000.0 ** -2)
    assert abs(frac - expect) < 0.01


def test_named_instances():
    tiny = make_instance("tiny")
    assert tiny["h"].shape == (256, 256) and tiny["g"] == 20.0 and tiny["lmax"] == 20e3
    diff = make_instance("diff", n=128)
    assert diff["h"].shape == (128, 128) and len(diff["suns"]) == 4
    t = bump_target(diff["h"], diff["g"], diff["seed"])
    assert t.shape == diff["h"].shape and np.abs(t - diff["h"]).max() > 1.0
    uv = random_origins(10, 32, 16, seed=1)
    assert uv.dtype == np.float32 and uv[:, 0].max() <= 31 and uv[:, 1].max() <= 15
    suns = sun_list(64, 5)
    e = np.degrees([s[0] for s in suns])
    assert e.min() >= 0.2 and e.max() <= 3.0
