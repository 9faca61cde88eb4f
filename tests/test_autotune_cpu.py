"""Host logic of the autotuner (no GPU): size classes, table persistence, validity,
and the coordinate descent of the shape search (paper_2005_06671_gb300/autotune.py)."""
from paper_2005_06671_gb300 import autotune


def test_size_classes_and_validity(tmp_path):
    assert autotune.size_class(512, 512) == "512"
    assert autotune.size_class(4096, 4096) == "4096"
    assert autotune.size_class(1000, 1100) == "1024"
    assert autotune._valid(dict(autotune.DEFAULT))
    assert not autotune._valid(dict(autotune.DEFAULT, rays_per_thread=4, ray_tile_w=48))
    p = str(tmp_path / "t.json")
    autotune.save_table({"x|512": {"params": {"block_threads": 128}}}, p)
    assert autotune.load_table(p)["x|512"]["params"]["block_threads"] == 128
    assert autotune.load_table(str(tmp_path / "missing.json")) == {}


def test_default_is_a_point_of_the_space():
    d = autotune.DEFAULT
    assert set(d) == set(autotune.SPACE)
    for name, v in d.items():
        assert v in autotune.SPACE[name], name


def test_coordinate_descent_finds_the_minimum_of_a_separable_cost(monkeypatch):
    """A cost that grows with each parameter's distance (in steps of the space) from
    a target shape: the descent from the default reaches the target, times only
    valid shapes (the batch call rejects the others), and times each shape once."""
    target = {"block_threads": 128, "rays_per_thread": 64, "ray_tile_w": 32, "refill_min": 10,
              "leaf_level": 2, "strip_len": 0}
    timed = []

    def fake_time(hfs, suns, lmax, p, reps, step):
        assert autotune._valid(p), p
        timed.append(tuple(sorted(p.items())))
        return 100.0 + sum(abs(autotune.SPACE[k].index(p[k]) - autotune.SPACE[k].index(target[k]))
                           for k in p)

    monkeypatch.setattr(autotune, "time_batch", fake_time)
    best, seen = autotune.tune([], [], 50e3, reps=1, rounds=3)
    assert best == target
    assert len(timed) == len(set(timed)) == len(seen)
