"""Host logic of the autotuner (no GPU): size classes, table persistence, validity."""
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
