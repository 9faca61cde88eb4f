"""Batched persistent forward (ss_batch_submit / plans) on the GPU.

Each instance of a batch must give exactly the outputs of ss_shadow_forward on
that instance alone (same descent, same sample values), whatever the chunk
shape; graph replays must repeat them; a sample of rays is checked against the
FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

from workloads import lunar_tile, batched_instances, MOON_RADIUS_M, SUN_ANGULAR_RADIUS_RAD

import paper_2005_06671_gb300 as ss
from _parity import compare_to_oracle, random_ids

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M
ALPHA = SUN_ANGULAR_RADIUS_RAD


def _instances():
    shapes = [(96, 96), (70, 130), (256, 256), (64, 64), (200, 200), (33, 47)]
    suns = [(1.2, 30.0), (0.4, 200.0), (2.5, 95.0), (0.9, 310.0), (1.7, 150.0), (-0.2, 10.0)]
    out = []
    for i, ((ny, nx), (e, a)) in enumerate(zip(shapes, suns)):
        h = lunar_tile(nx, 12.0, seed=300 + i, amplitude=600.0, n_craters=5, ny=ny)
        out.append((h, 12.0, (math.radians(e), math.radians(a), ALPHA)))
    return out


def _single(h, g, sun, lmax, **kw):
    hf = ss.Heightfield(torch.from_numpy(h).cuda(), g, R)
    mip = ss.ss_build_maxmip(hf)
    r = ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), lmax, **kw)
    return {k: (None if v is None else v.cpu().numpy()) for k, v in r.items()}


def _batch(insts, lmax, plan=False, replays=1, **kw):
    hfs = [ss.Heightfield(torch.from_numpy(h).cuda(), g, R) for h, g, _ in insts]
    suns = [ss.Sun(*s) for _, _, s in insts]
    b = ss.Batch(hfs, suns, lmax, want_cost=True, **kw)
    results = []
    for _ in range(replays):
        for o in b.outs:
            o["light"].fill_(-1.0)
            o["argmin"].fill_(-7)
        outs = b.launch() if plan else b.submit()
        torch.cuda.synchronize()
        results.append([{k: (None if v is None else v.cpu().numpy()) for k, v in o.items()}
                        for o in outs])
    b.close()
    return results


def _same(a, b):
    assert np.array_equal(a["argmin"], b["argmin"])
    assert np.array_equal(a["cost"].view(np.uint32), b["cost"].view(np.uint32))
    assert np.array_equal(a["light"].view(np.uint32), b["light"].view(np.uint32))


@pytest.mark.parametrize("kw", [dict(), dict(rays_per_thread=4, ray_tile_w=32),
                                dict(rays_per_thread=2, ray_tile_w=8, refill_min=4),
                                dict(block_threads=128, leaf_level=3),
                                dict(strip_len=1), dict(strip_len=7, ray_tile_w=16),
                                dict(strip_len=64, rays_per_thread=8, ray_tile_w=32),
                                dict(lane_leaves=True), dict(lane_leaves=True, refill_min=3),
                                dict(leaf_level=0, rays_per_thread=6, ray_tile_w=64)])
def test_batch_equals_single_forward(kw):
    """Every instance of a batch gives exactly the single-tile forward's outputs,
    with leaf samples as warp tasks (default) or in the walking lane."""
    insts = _instances()
    lmax = 2500.0
    res = _batch(insts, lmax, **kw)[0]
    for (h, g, sun), got in zip(insts, res):
        _same(got, _single(h, g, sun, lmax))


@pytest.mark.parametrize("kw", [dict(rays_per_thread=1, refill_min=1, strip_len=1),
                                dict(rays_per_thread=1, refill_min=2, ray_tile_w=8),
                                dict(rays_per_thread=1, refill_min=2, ray_tile_w=8,
                                     lane_leaves=True),
                                dict(rays_per_thread=3, refill_min=1, strip_len=5, ray_tile_w=32)])
def test_batch_chunk_switches_keep_every_ray(kw):
    """Tiny chunks and eager refills: warps move to their next chunk while other
    lanes still walk rays of the previous one; every ray must still be written
    with its own result (outputs are pre-filled with sentinels)."""
    h = lunar_tile(300, 12.0, seed=77, amplitude=700.0, n_craters=6, ny=260)
    insts = [(h, 12.0, (math.radians(1.1), math.radians(60.0), ALPHA)),
             (h[:100, :130].copy(), 12.0, (math.radians(0.7), math.radians(250.0), ALPHA))]
    res = _batch(insts, 3000.0, **kw)[0]
    for (hh, g, sun), got in zip(insts, res):
        assert np.all(got["argmin"] != -7) and np.all(got["light"] >= 0.0)
        _same(got, _single(hh, g, sun, 3000.0))


def test_plan_replays_repeat_results_and_count_probes():
    insts = _instances()
    lmax = 2500.0
    # without seeded strips every ray is walked from scratch in both kernels, so
    # the probe counts match too
    runs = _batch(insts, lmax, plan=True, replays=3, count_samples=True, strip_len=1,
                  lane_leaves=True)
    for (h, g, sun), a, b, c in zip(insts, *runs):
        ref = _single(h, g, sun, lmax, count_samples=True, strip_len=1, lane_leaves=True)
        _same(a, ref)
        _same(b, ref)
        _same(c, ref)
        assert np.array_equal(a["counters"], ref["counters"])


def test_batch_sample_vs_oracle():
    insts = _instances()
    lmax = 2500.0
    res = _batch(insts, lmax)[0]
    for k, ((h, g, sun), got) in enumerate(zip(insts, res)):
        ids = random_ids(h.size, 400, seed=900 + k)
        compare_to_oracle(h, g, R, sun, lmax, 0.5, got["light"][ids], got["argmin"][ids],
                          got["cost"][ids], ray_ids=ids)


def test_batched_recipe_small():
    """The 'batched' workload recipe (uneven tile sizes, a sun each over a lunar
    day, 50 km rays) at reduced sizes: every instance equals its single run."""
    insts = [(d["h"], d["g"], (d["suns"][0][0], d["suns"][0][1], d["alpha"]))
             for d in batched_instances(n_instances=8, sizes=(64, 128, 256, 512))]
    res = _batch(insts, 50e3, plan=True)[0]
    for (h, g, sun), got in zip(insts, res):
        _same(got, _single(h, g, sun, 50e3))


def test_autotuner_picks_a_valid_shape_and_persists(tmp_path):
    from paper_2005_06671_gb300 import autotune
    insts = _instances()[:4]
    hfs = [ss.Heightfield(torch.from_numpy(h).cuda(), g, R) for h, g, _ in insts]
    suns = [ss.Sun(*s) for _, _, s in insts]
    path = str(tmp_path / "table.json")
    best = autotune.tune_and_store(hfs, suns, 2500.0, path=path, reps=1, rounds=1)
    assert autotune._valid(best)
    assert autotune.lookup(hfs, autotune.load_table(path)) == best
    res = _batch(insts, 2500.0, **best)[0]
    for (h, g, sun), got in zip(insts, res):
        _same(got, _single(h, g, sun, 2500.0))
