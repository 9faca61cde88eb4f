"""Polar stereographic tiles: CUDA path (through the C ABI) against the FP64 oracle.

The tile is centred on the pole and mapped by stereographic projection from the
antipode, so a shadow ray's texel image is a circular arc instead of the
gnomonic straight line (Sec. 3.2 states the method for any mapping whose
inverse is available; the lunar polar scenes are the paper's setting).  Same
bars as the gnomonic parity tests: light within 1e-5, argmin equal except at
ties within 1e-6 rad, descent and uniform stepping bit-identical.  Besides the
polar scene recipe at reduced size, wide tiles (hundreds of km across, texels
of 300-1000 m) make the arcs bend by several texels over a block, which is
what the footprint boxes' sagitta margin has to cover.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import make_instance, lunar_tile, random_origins, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss
from _parity import compare_to_oracle, random_ids, grad_weights_mask, assert_grad_close

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M
PROJ = "polar_stereo"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(h, g, sun, lmax, method="dp", uv=None, lift=None, light_only=False, step=0.5):
    hf = ss.Heightfield(_dev(h), g, R, projection=PROJ)
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    uvt = None if uv is None else _dev(uv)
    lt = None if lift is None else _dev(lift)
    fn = ss.ss_shadow_forward if method == "dp" else ss.ss_shadow_uniform
    res = fn(hf, mip, s, lmax, step, uv=uvt, lift=lt, light_only=light_only)
    torch.cuda.synchronize()
    return {k: (None if v is None else v.cpu().numpy()) for k, v in res.items()}


def _same(a, b):
    assert np.array_equal(a["argmin"], b["argmin"])
    assert np.array_equal(a["cost"].view(np.uint32), b["cost"].view(np.uint32))
    assert np.array_equal(a["light"].view(np.uint32), b["light"].view(np.uint32))


def _wide(n, g, seed, amplitude=3000.0):
    return lunar_tile(n, g, seed=seed, amplitude=amplitude, n_craters=40)


def test_polar_scene_reduced_vs_oracle_and_uniform():
    inst = make_instance("polar", n=768)
    assert inst["proj"] == PROJ
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    sun = (elev, az, inst["alpha"])
    a = _run(h, g, sun, inst["lmax"])
    b = _run(h, g, sun, inst["lmax"], method="uniform")
    _same(a, b)
    # every ray of the tile (the oracle takes a few seconds here)
    st = compare_to_oracle(h, g, R, sun, inst["lmax"], 0.5, a["light"], a["argmin"], a["cost"],
                           ray_ids=np.arange(h.size), proj=PROJ)
    assert st["penumbra"] > 200


@pytest.mark.parametrize("n,g,lmax,elev,az", [
    (512, 300.0, 200e3, 1.0, 30.0),
    (384, 1000.0, 400e3, 2.5, 200.0),
    (300, 600.0, 250e3, -0.3, 115.0),     # sun below the pole's horizon: lit far from the pole
])
def test_wide_polar_tiles_vs_oracle_and_uniform(n, g, lmax, elev, az):
    h = _wide(n, g, seed=int(g) + n)
    sun = (math.radians(elev), math.radians(az), math.radians(0.2665))
    a = _run(h, g, sun, lmax)
    b = _run(h, g, sun, lmax, method="uniform")
    _same(a, b)
    ids = random_ids(h.size, 2500, seed=n)
    compare_to_oracle(h, g, R, sun, lmax, 0.5, a["light"][ids], a["argmin"][ids],
                      a["cost"][ids], ray_ids=ids, proj=PROJ)


@pytest.mark.parametrize("n,g,lmax,elev,az,kw", [
    (512, 300.0, 200e3, 1.0, 30.0, dict()),
    (384, 1000.0, 400e3, 2.5, 200.0, dict(refill_min=1, leaf_level=0)),
    (300, 600.0, 250e3, -0.3, 115.0, dict(refill_min=32, rays_per_thread=7, ray_tile_w=32)),
    (257, 400.0, 150e3, 1.2, 250.0, dict(block_threads=96, rays_per_thread=3, ray_tile_w=16)),
    (200, 500.0, 200e3, 0.7, 330.0, dict(leaf_level=2, count_samples=True)),
])
def test_polar_task_descent_equals_lane_descent(n, g, lmax, elev, az, kw):
    """The default exact descent on stereographic tiles (leaf samples as
    warp-wide tasks) against the single-lane walk (SS_FLAG_LANE_LEAVES) and
    uniform stepping, bit for bit: grid rays over launch shapes (leaf blocks of
    1, 4 and 8 samples, eager and lazy refills, partial warps, narrow and wide
    ray rectangles) and listed rays inside and outside the tile, with lifts."""
    h = _wide(n, g, seed=int(g) + 3 * n)
    hf = ss.Heightfield(_dev(h), g, R, projection=PROJ)
    mip = ss.ss_build_maxmip(hf)
    sun = ss.Sun(math.radians(elev), math.radians(az), math.radians(0.2665))
    rng = np.random.default_rng(n)
    uv = np.concatenate([random_origins(3000, n, n, seed=n + 1),
                         rng.uniform(-40, n + 40, (600, 2))]).astype(np.float32)
    lift = rng.uniform(0, 200, uv.shape[0]).astype(np.float32)
    lift[:1000] = 0.0
    for rays in (dict(), dict(uv=_dev(uv), lift=_dev(lift))):
        a = ss.ss_shadow_forward(hf, mip, sun, lmax, **rays, **kw)
        b = ss.ss_shadow_forward(hf, mip, sun, lmax, lane_leaves=True, **rays, **kw)
        u = ss.ss_shadow_uniform(hf, mip, sun, lmax, **rays)
        torch.cuda.synchronize()
        for x in (b, u):
            assert torch.equal(a["argmin"], x["argmin"])
            assert torch.equal(a["cost"].view(torch.int32), x["cost"].view(torch.int32))
            assert torch.equal(a["light"].view(torch.int32), x["light"].view(torch.int32))
        pen = ((a["light"] > 0) & (a["light"] < 1)).sum().item()
        assert pen > 20
        if kw.get("count_samples"):
            ca = a["counters"].sum(0).cpu().numpy()
            assert ca[0] > 0 and ca[1] > 0


def test_polar_list_mode_inside_and_outside_origins():
    n, g, lmax = 257, 400.0, 150e3
    h = _wide(n, g, seed=91)
    rng = np.random.default_rng(92)
    uv_in = random_origins(1500, n, n, seed=93)
    uv_out = np.concatenate([
        np.stack([rng.uniform(-120, -1, 300), rng.uniform(0, n - 1, 300)], 1),
        np.stack([rng.uniform(n, n + 120, 300), rng.uniform(0, n - 1, 300)], 1),
        np.stack([rng.uniform(0, n - 1, 300), rng.uniform(-120, -0.5, 300)], 1),
        np.stack([rng.uniform(-60, -1, 300), rng.uniform(-60, -1, 300)], 1),
    ]).astype(np.float32)
    uv = np.concatenate([uv_in, uv_out]).astype(np.float32)
    lift = rng.uniform(0, 300, uv.shape[0]).astype(np.float32)
    lift[:500] = 0.0
    for az in (20.0, 135.0, 250.0, 330.0):
        sun = (math.radians(1.2), math.radians(az), math.radians(0.2665))
        a = _run(h, g, sun, lmax, uv=uv, lift=lift)
        b = _run(h, g, sun, lmax, method="uniform", uv=uv, lift=lift)
        _same(a, b)
        compare_to_oracle(h, g, R, sun, lmax, 0.5, a["light"], a["argmin"], a["cost"],
                          uv=uv, lift=lift, proj=PROJ)


def test_polar_light_only_vs_exact():
    h = _wide(320, 500.0, seed=7)
    sun = (math.radians(1.5), math.radians(75.0), math.radians(0.2665))
    exact = _run(h, 500.0, sun, 200e3)
    for method in ("dp", "uniform"):
        lo = _run(h, 500.0, sun, 200e3, method=method, light_only=True)
        assert np.abs(lo["light"] - exact["light"]).max() <= 1e-5
        pen = (exact["light"] > 0) & (exact["light"] < 1)
        assert pen.sum() > 50
        assert np.array_equal(lo["argmin"][pen], exact["argmin"][pen])


def test_polar_backward_vs_oracle_gradient():
    n, g, lmax = 96, 400.0, 60e3
    h = _wide(n, g, seed=5, amplitude=2000.0)
    sun = (math.radians(1.1), math.radians(150.0), math.radians(1.5))
    hf = ss.Heightfield(_dev(h), g, R, projection=PROJ)
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    res = ss.ss_shadow_forward(hf, mip, s, lmax)
    am_gpu = res["argmin"].cpu().numpy().astype(np.int64)
    ol, oa, oc = oracle.shadow(h, g, R, sun[0], sun[1], sun[2], lmax, proj=PROJ)
    assert np.sum((ol > 0) & (ol < 1)) > 100
    sinp = oracle.sin_elev(h, g, R, sun[0], sun[1], proj=PROJ)
    gl = np.random.default_rng(8).normal(size=h.size)
    gl[~grad_weights_mask(ol, oc, sinp, sun[2], am_gpu, oa)] = 0.0
    gh_gpu, gs_gpu = ss.ss_shadow_backward(hf, s, lmax, res["argmin"],
                                           torch.from_numpy(gl.astype(np.float32)).cuda(),
                                           cost=res["cost"])
    torch.cuda.synchronize()
    gh_o, gs_o, ah, ch = oracle.grad(h, g, R, sun[0], sun[1], sun[2], oa,
                                     gl.astype(np.float32).astype(np.float64), proj=PROJ,
                                     with_abs=True)
    st = assert_grad_close(gh_gpu.cpu().numpy(), gh_o, ah, ch)
    assert st["texels"] > 100
    np.testing.assert_allclose(gs_gpu.cpu().numpy(), gs_o, rtol=1e-4,
                               atol=1e-6 * np.abs(gs_o).max())
