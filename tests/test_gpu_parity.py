"""CUDA path (through the C ABI) against the FP64 oracle, on the same seeded inputs.

Bars: light within 1e-5 absolute; argmin equal except at ties within 1e-6 rad;
mipmap levels bit-exact; descent and uniform stepping bit-identical (same
argmin and same float32 cost on every ray).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import make_instance, lunar_tile, random_origins, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss
from _parity import (compare_to_oracle, random_ids, LIGHT_TOL, grad_weights_mask,
                     assert_grad_close)

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M
ALPHA = math.radians(0.2665)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(h, g, sun, lmax, step=0.5, method="dp", uv=None, lift=None, count=False,
         early_exit=True, hpad=0, leaf_level=-1, block_threads=0, light_only=False):
    ny, nx = h.shape
    if hpad:
        store = torch.full((ny, nx + hpad), float("nan"), device="cuda")
        store[:, :nx] = _dev(h)
        ht = store[:, :nx]
    else:
        ht = _dev(h)
    hf = ss.Heightfield(ht, g, R)
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    uvt = None if uv is None else _dev(uv)
    lt = None if lift is None else _dev(lift)
    if method == "dp":
        res = ss.ss_shadow_forward(hf, mip, s, lmax, step, uv=uvt, lift=lt, count_samples=count,
                                   leaf_level=leaf_level, block_threads=block_threads,
                                   light_only=light_only)
    else:
        res = ss.ss_shadow_uniform(hf, mip, s, lmax, step, uv=uvt, lift=lt, count_samples=count,
                                   early_exit=early_exit, block_threads=block_threads,
                                   light_only=light_only)
    torch.cuda.synchronize()
    return {k: (None if v is None else v.cpu().numpy()) for k, v in res.items()}


# --------------------------------------------------------------- mipmap
@pytest.mark.parametrize("shape,pad", [((256, 256), 0), ((4096, 4096), 0), ((777, 1000), 0),
                                       ((31, 65), 3), ((2, 2), 0), ((1, 9), 0), ((130, 67), 1)])
def test_maxmip_bit_exact(shape, pad):
    ny, nx = shape
    rng = np.random.default_rng(nx * 7 + ny)
    h = (rng.normal(size=shape) * 900).astype(np.float32)
    ref = oracle.maxmip(h)
    if pad:
        store = torch.zeros((ny, nx + pad), device="cuda")
        store[:, :nx] = _dev(h)
        ht = store[:, :nx]
    else:
        ht = _dev(h)
    hf = ss.Heightfield(ht, 10.0, R)
    mip = ss.ss_build_maxmip(hf)
    torch.cuda.synchronize()
    views = ss.maxmip_views(mip, nx, ny)
    assert len(views) == len(ref) - 1
    for lvl, v in enumerate(views, start=1):
        assert np.array_equal(v.cpu().numpy(), ref[lvl]), lvl
    st = ss.maxmip_stats(mip, nx, ny).cpu().numpy()
    assert st[0] == h.max() and st[1] == h.min()


# ------------------------------------------------------- tiny, full grid
@pytest.mark.parametrize("method", ["dp", "uniform"])
def test_tiny_full_grid_vs_oracle(method):
    inst = make_instance("tiny")
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    sun = (elev, az, inst["alpha"])
    out = _run(h, g, sun, inst["lmax"], method=method)
    ids = np.arange(h.size)
    st = compare_to_oracle(h, g, R, sun, inst["lmax"], 0.5, out["light"], out["argmin"],
                           out["cost"], ray_ids=ids)
    assert st["penumbra"] > 100


def _pair(h, g, sun, lmax, step=0.5, **kw):
    a = _run(h, g, sun, lmax, step, method="dp", **kw)
    b = _run(h, g, sun, lmax, step, method="uniform", **kw)
    return a, b


@pytest.mark.parametrize("name,n", [("tiny", None), ("diff", 384), ("mid", 512)])
def test_descent_equals_uniform_bitwise(name, n):
    inst = make_instance(name, n=n)
    h, g = inst["h"], inst["g"]
    for (elev, az) in inst["suns"]:
        sun = (elev, az, inst["alpha"])
        a, b = _pair(h, g, sun, inst["lmax"])
        c = _run(h, g, sun, inst["lmax"], method="uniform", early_exit=False)
        assert np.array_equal(a["argmin"], b["argmin"])
        assert np.array_equal(a["cost"].view(np.uint32), b["cost"].view(np.uint32))
        assert np.array_equal(a["light"].view(np.uint32), b["light"].view(np.uint32))
        assert np.array_equal(b["argmin"], c["argmin"])
        assert np.array_equal(b["cost"].view(np.uint32), c["cost"].view(np.uint32))


@pytest.mark.parametrize("leaf_level,block", [(0, 64), (1, 128), (5, 256), (8, 96)])
def test_descent_tuning_knobs_do_not_change_results(leaf_level, block):
    inst = make_instance("diff", n=256)
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][2]
    sun = (elev, az, inst["alpha"])
    ref = _run(h, g, sun, inst["lmax"], method="uniform")
    out = _run(h, g, sun, inst["lmax"], leaf_level=leaf_level, block_threads=block)
    assert np.array_equal(out["argmin"], ref["argmin"])
    assert np.array_equal(out["cost"].view(np.uint32), ref["cost"].view(np.uint32))


@pytest.mark.parametrize("strip,tile_w,rpt,sw", [(0, 0, 0, 0), (0, 32, 3, 0), (0, 0, 7, 0),
                                                  (1, 0, 0, 0), (3, 0, 0, 0), (10, 32, 32, 0),
                                                  (33, 16, 8, 0), (10, 64, 1, 0),
                                                  (256, 32, 64, 0), (7, 0, 5, 0), (0, 0, 0, 1),
                                                  (0, 0, 0, 16), (4, 0, 0, 5)])
def test_seeded_strips_do_not_change_results(strip, tile_w, rpt, sw):
    """Seeded walks (column seeds by default, strip_len 0; strips of S rays;
    none; seed windows of several widths; sparse-sample seeds for rays with
    no finished neighbour) in grid and list mode, strips longer than a
    rectangle column, odd and partial chunks: the same argmin and cost bits as
    uniform stepping."""
    inst = make_instance("diff", n=320)
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][1]
    sun = (elev, az, inst["alpha"])
    ref = _run(h, g, sun, inst["lmax"], method="uniform")
    hf = ss.Heightfield(_dev(h), g, R)
    mip = ss.ss_build_maxmip(hf)
    res = ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), inst["lmax"], strip_len=strip,
                               ray_tile_w=tile_w, rays_per_thread=rpt, seed_width=sw)
    assert np.array_equal(res["argmin"].cpu().numpy(), ref["argmin"])
    assert np.array_equal(res["cost"].cpu().numpy().view(np.uint32), ref["cost"].view(np.uint32))
    uv = random_origins(5000, 320, 320, seed=strip)
    uv = uv[np.argsort(uv[:, 1] * 400 + uv[:, 0])]          # neighbours next to each other
    a = ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), inst["lmax"], uv=_dev(uv), strip_len=strip,
                             rays_per_thread=rpt, seed_width=sw)
    b = ss.ss_shadow_uniform(hf, mip, ss.Sun(*sun), inst["lmax"], uv=_dev(uv))
    assert torch.equal(a["argmin"], b["argmin"])
    assert torch.equal(a["cost"].view(torch.int32), b["cost"].view(torch.int32))


@pytest.mark.parametrize("name,n,kw", [
    ("tiny", None, dict()), ("diff", 384, dict()), ("mid", 600, dict()),
    ("diff", 333, dict(leaf_level=0)), ("diff", 257, dict(refill_min=1)),
    ("diff", 300, dict(refill_min=32, rays_per_thread=7, ray_tile_w=32)),
    ("tiny", 190, dict(block_threads=96, rays_per_thread=3, ray_tile_w=16)),
    ("diff", 200, dict(block_threads=64, seed_width=1, rays_per_thread=64, ray_tile_w=512)),
    ("tiny", 150, dict(count_samples=True)),
])
def test_task_descent_equals_lane_descent_and_uniform(name, n, kw):
    """The default descent for grid rays on gnomonic tiles (leaf samples as
    warp-wide tasks) against the single-lane walk (SS_FLAG_LANE_LEAVES) and
    uniform stepping, bit for bit, over launch shapes: leaf blocks of 2 and 4
    samples, eager and lazy refills, partial warps, narrow and wide ray
    rectangles, ragged tile edges."""
    inst = make_instance(name, n=n)
    h, g = inst["h"], inst["g"]
    hf = ss.Heightfield(_dev(h), g, R)
    mip = ss.ss_build_maxmip(hf)
    for (elev, az) in inst["suns"][:2]:
        sun = ss.Sun(elev, az, inst["alpha"])
        a = ss.ss_shadow_forward(hf, mip, sun, inst["lmax"], **kw)
        b = ss.ss_shadow_forward(hf, mip, sun, inst["lmax"], lane_leaves=True, **kw)
        u = ss.ss_shadow_uniform(hf, mip, sun, inst["lmax"])
        torch.cuda.synchronize()
        for x in (b, u):
            assert torch.equal(a["argmin"], x["argmin"])
            assert torch.equal(a["cost"].view(torch.int32), x["cost"].view(torch.int32))
            assert torch.equal(a["light"].view(torch.int32), x["light"].view(torch.int32))
        if kw.get("count_samples"):
            ca, cb = a["counters"].sum(0).cpu().numpy(), b["counters"].sum(0).cpu().numpy()
            assert ca[0] > 0 and ca[1] > 0 and cb[0] > 0
            assert (a["counters"][:, 1] >= 1).float().mean() > 0.9


# ------------------------------------------------------------- list mode
@pytest.mark.parametrize("method", ["dp", "uniform"])
def test_list_mode_with_lift_vs_oracle(method):
    inst = make_instance("tiny")
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    sun = (elev, az, inst["alpha"])
    n = 3000
    uv = random_origins(n, 256, 256, seed=77)
    lift = np.random.default_rng(78).uniform(0, 40, n).astype(np.float32)
    lift[:500] = 0.0
    out = _run(h, g, sun, inst["lmax"], method=method, uv=uv, lift=lift)
    compare_to_oracle(h, g, R, sun, inst["lmax"], 0.5, out["light"], out["argmin"],
                      out["cost"], uv=uv, lift=lift)


# ---------------------------------------------- differentiable config, 4 suns
def test_diff_config_sampled_vs_oracle():
    inst = make_instance("diff")
    h, g = inst["h"], inst["g"]
    for k, (elev, az) in enumerate(inst["suns"]):
        sun = (elev, az, inst["alpha"])
        out = _run(h, g, sun, inst["lmax"])
        ids = random_ids(h.size, 2500, seed=100 + k)
        compare_to_oracle(h, g, R, sun, inst["lmax"], 0.5, out["light"][ids],
                          out["argmin"][ids], out["cost"][ids], ray_ids=ids)


# ------------------------------------- mid config at full size (bench launch)
def test_mid_full_size_sampled_vs_oracle_and_uniform():
    inst = make_instance("mid")
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    sun = (elev, az, inst["alpha"])
    a = _run(h, g, sun, inst["lmax"], count=True)
    ids = random_ids(h.size, 4000, seed=4096)
    st = compare_to_oracle(h, g, R, sun, inst["lmax"], 0.5, a["light"][ids], a["argmin"][ids],
                           a["cost"][ids], ray_ids=ids)
    b = _run(h, g, sun, inst["lmax"], method="uniform", count=True)
    assert np.array_equal(a["argmin"], b["argmin"])
    assert np.array_equal(a["cost"].view(np.uint32), b["cost"].view(np.uint32))
    # the descent evaluates far fewer leaf samples than uniform stepping
    assert a["counters"][:, 1].sum() * 5 < b["counters"][:, 1].sum()
    print("mid parity", st, "mean bound probes", a["counters"][:, 0].mean(),
          "mean leaf samples dp/uniform", a["counters"][:, 1].mean(), b["counters"][:, 1].mean())


# ------------------------------------------------------------- edge cases
def test_edge_cases():
    h = lunar_tile(97, 15.0, seed=9, amplitude=400.0, n_craters=6, ny=61)
    sun = (math.radians(1.3), math.radians(211.0), ALPHA)
    # odd non-square tile, padded rows, non-default step
    for method in ("dp", "uniform"):
        out = _run(h, 15.0, sun, 3000.0, step=0.37, method=method, hpad=5)
        compare_to_oracle(h, 15.0, R, sun, 3000.0, 0.37, out["light"], out["argmin"],
                          out["cost"], ray_ids=np.arange(h.size))
    # max_len shorter than one step: no sample at all
    out = _run(h, 15.0, sun, 5.0)
    assert np.all(out["light"] == 1.0) and np.all(out["argmin"] == -1)
    assert np.all(np.isinf(out["cost"]))
    # sun below the horizon
    low = (math.radians(-1.0), 0.4, ALPHA)
    out = _run(h, 15.0, low, 2000.0)
    compare_to_oracle(h, 15.0, R, low, 2000.0, 0.5, out["light"], out["argmin"], out["cost"],
                      ray_ids=np.arange(h.size))
    # the longest ray the ABI allows (65535 samples) on a small tile
    out = _run(h, 15.0, sun, 65535 * 7.5, step=0.5)
    ids = random_ids(h.size, 300, seed=5)
    compare_to_oracle(h, 15.0, R, sun, 65535 * 7.5, 0.5, out["light"][ids], out["argmin"][ids],
                      out["cost"][ids], ray_ids=ids)
    # listed origins outside the tile: rays that enter it, rays that never do
    rng = np.random.default_rng(17)
    uv_out = np.concatenate([
        np.stack([rng.uniform(-40, -1, 200), rng.uniform(0, 60, 200)], 1),
        np.stack([rng.uniform(97, 140, 200), rng.uniform(0, 60, 200)], 1),
        np.stack([rng.uniform(0, 96, 200), rng.uniform(-30, -0.5, 200)], 1),
    ]).astype(np.float32)
    lift_out = rng.uniform(0, 200, uv_out.shape[0]).astype(np.float32)
    for az in (211.0, 60.0, 300.0):
        sun_o = (math.radians(1.3), math.radians(az), ALPHA)
        for method in ("dp", "uniform"):
            out = _run(h, 15.0, sun_o, 3000.0, method=method, uv=uv_out, lift=lift_out)
            compare_to_oracle(h, 15.0, R, sun_o, 3000.0, 0.5, out["light"], out["argmin"],
                              out["cost"], uv=uv_out, lift=lift_out)
    # empty ray list
    hf = ss.Heightfield(_dev(h), 15.0, R)
    mip = ss.ss_build_maxmip(hf)
    res = ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), 2000.0,
                               uv=torch.zeros((0, 2), device="cuda"))
    assert res["light"].numel() == 0


def test_flat_terrain_closed_form_on_gpu():
    nx, ny, g, h0 = 65, 48, 20.0, 123.25
    h = np.full((ny, nx), h0, np.float32)
    for e in (-0.4, -0.2, -0.1, 0.0, 0.1, 0.2, 0.3, 1.0):
        sun = (math.radians(e), math.radians(37.0), ALPHA)
        out = _run(h, g, sun, 2000.0)
        sinp = oracle.sin_elev(h, g, R, sun[0], sun[1])
        rho, dl = R + h0, 0.5 * g
        c = (2 * rho * sinp + dl) / (np.sqrt(rho * rho + 2 * dl * rho * sinp + dl * dl) + rho)
        d = np.clip(c * np.sqrt(1 - sinp ** 2) / ALPHA, -1, 1)
        f = (np.pi - np.arccos(d) + d * np.sqrt(1 - d * d)) / np.pi
        inner = np.zeros((ny, nx), bool)
        inner[1:-1, 1:-1] = True
        inner = inner.ravel()
        assert np.all(out["argmin"][inner] == 1)
        assert np.abs(out["light"][inner] - f[inner]).max() <= LIGHT_TOL


# --------------------------------------------------------------- backward
def _grad_case(n=96, k_sun=1):
    inst = make_instance("diff", n=n)
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][k_sun]
    alpha = math.radians(1.5)   # a wider disc puts more rays in the penumbra
    return h, g, (elev, az, alpha), 3000.0


@pytest.mark.parametrize("k_sun,pass_cost", [(0, False), (1, True), (2, False), (3, True)])
def test_backward_vs_oracle_gradient(k_sun, pass_cost):
    h, g, sun, lmax = _grad_case(k_sun=k_sun)
    ht = _dev(h)
    hf = ss.Heightfield(ht, g, R)
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    res = ss.ss_shadow_forward(hf, mip, s, lmax)
    am_gpu = res["argmin"].cpu().numpy().astype(np.int64)
    ol, oa, oc = oracle.shadow(h, g, R, sun[0], sun[1], sun[2], lmax)
    sinp = oracle.sin_elev(h, g, R, sun[0], sun[1])
    gl = np.random.default_rng(3 + k_sun).normal(size=h.size)
    gl[~grad_weights_mask(ol, oc, sinp, sun[2], am_gpu, oa)] = 0.0
    gh_gpu, gs_gpu = ss.ss_shadow_backward(hf, s, lmax, res["argmin"],
                                           torch.from_numpy(gl.astype(np.float32)).cuda(),
                                           cost=res["cost"] if pass_cost else None)
    torch.cuda.synchronize()
    gh_o, gs_o, ah, ch = oracle.grad(h, g, R, sun[0], sun[1], sun[2], oa,
                                     gl.astype(np.float32).astype(np.float64), with_abs=True)
    st = assert_grad_close(gh_gpu.cpu().numpy(), gh_o, ah, ch)
    assert st["texels"] > 50
    np.testing.assert_allclose(gs_gpu.cpu().numpy(), gs_o, rtol=1e-4, atol=1e-6 * np.abs(gs_o).max())


def test_autograd_function_matches_oracle():
    h, g, sun, lmax = _grad_case(n=80, k_sun=2)
    target = torch.rand(h.size, device="cuda", dtype=torch.float32)
    ht = _dev(h).requires_grad_(True)
    ang = torch.tensor([sun[0], sun[1]], dtype=torch.float64, requires_grad=True)
    light = ss.shadow(ht, ang, g, R, sun[2], lmax)
    loss = ((light - target) ** 2).mean()
    gh, gang = torch.autograd.grad(loss, [ht, ang])
    # dLoss/dlight as the GPU computed it (float32 light minus target, times 2/n)
    gl = (2.0 * (light.detach() - target) / h.size).cpu().numpy().astype(np.float64)
    hf = ss.Heightfield(_dev(h), g, R)
    fw = ss.ss_shadow_forward(hf, ss.ss_build_maxmip(hf), ss.Sun(*sun), lmax)
    am_gpu = fw["argmin"].cpu().numpy().astype(np.int64)
    assert np.array_equal(fw["light"].cpu().numpy(), light.detach().cpu().numpy())
    # every ray carries weight in the loss, so the GPU's subgradient is taken at
    # its own argmin, and where that differs from the oracle's the oracle's
    # gradient is evaluated at the GPU's argmin.  This 80 x 80 crop of the
    # +-1.5 km generator is far steeper than any config (adjacent texels differ
    # by up to ~200 m), so near the origin the float32 leaf cost carries up to
    # 2^-22 |dh| / t ~ 4e-6 rad of rounding (dh ~ 100 m, t = 5 m): a float32
    # argmin may then differ from the FP64 one by more than the 1e-6 tie bar
    # of the configs; the two samples' oracle costs must agree within that
    # rounding bound.
    ol, oa, oc = oracle.shadow(h, g, R, sun[0], sun[1], sun[2], lmax)
    for r in np.nonzero(am_gpu != oa)[0]:
        cs = oracle.ray_costs(h, g, R, sun[0], sun[1], lmax, r % h.shape[1], r // h.shape[1])
        assert abs(cs[am_gpu[r] - 1] - cs[oa[r] - 1]) <= 4e-6, r
    sinp = oracle.sin_elev(h, g, R, sun[0], sun[1])
    assert grad_weights_mask(ol, oc, sinp, sun[2], oa, oa).all()   # no ray at saturation
    gh_o, gs_o, ah, ch = oracle.grad(h, g, R, sun[0], sun[1], sun[2], am_gpu, gl, with_abs=True)
    assert np.abs(light.detach().cpu().numpy() - ol).max() <= LIGHT_TOL
    st = assert_grad_close(gh.cpu().numpy(), gh_o, ah, ch)
    assert st["texels"] > 20
    np.testing.assert_allclose(gang.numpy(), gs_o[:2], rtol=1e-4, atol=1e-7)


# ------------------------------------------------ light-only (saturation cutoffs)
@pytest.mark.parametrize("name,n", [("tiny", None), ("mid", 1024), ("diff", 512)])
def test_light_only_mode_vs_oracle(name, n):
    """Light-only mode: light exact (1e-5 of the oracle); in the penumbra the
    argmin and cost are the exact ones; fully lit rays report argmin -1; rays in
    umbra report a witness sample whose oracle cost proves the umbra."""
    import oracle as orc
    inst = make_instance(name, n=n)
    h, g = inst["h"], inst["g"]
    for (elev, az) in inst["suns"][:2]:
        sun = (elev, az, inst["alpha"])
        exact = _run(h, g, sun, inst["lmax"])
        for method in ("dp", "uniform"):
            lo = _run(h, g, sun, inst["lmax"], method=method, light_only=True)
            assert np.abs(lo["light"] - exact["light"]).max() <= LIGHT_TOL
            pen = (exact["light"] > 0) & (exact["light"] < 1)
            assert np.array_equal(lo["argmin"][pen], exact["argmin"][pen])
            lit = exact["light"] == 1
            assert np.all((lo["argmin"][lit] == -1) | (lo["argmin"][lit] == exact["argmin"][lit]))
        ids = random_ids(h.size, 1500, seed=55)
        compare_to_oracle(h, g, R, sun, inst["lmax"], 0.5, lo["light"][ids], exact["argmin"][ids],
                          exact["cost"][ids], ray_ids=ids)
        # umbra witnesses: the oracle's cost at the reported sample is below -alpha/cos(eps)
        dark = np.nonzero(exact["light"] == 0)[0][:40]
        sinp = orc.sin_elev(h, g, R, sun[0], sun[1])
        for r in dark:
            cs = orc.ray_costs(h, g, R, sun[0], sun[1], inst["lmax"], r % h.shape[1],
                               r // h.shape[1])
            j = lo["argmin"][r]
            assert j >= 1 and cs[j - 1] * math.sqrt(1 - sinp[r] ** 2) <= -inst["alpha"]


@pytest.mark.parametrize("kw", [dict(), dict(rays_per_thread=1, refill_min=1),
                                dict(rays_per_thread=3, refill_min=2, ray_tile_w=8),
                                dict(rays_per_thread=7, block_threads=64),
                                dict(rays_per_thread=5, block_threads=96, refill_min=32),
                                dict(strip_len=4), dict(seed_width=4, leaf_level=3)])
def test_light_only_descent_launch_shapes(kw):
    """The light-only descent (per-warp queues of parked rays) under odd launch
    shapes: tiny chunks, partial warps and blocks, eager and lazy refills,
    ragged rectangles, grid and listed rays.  Every ray is written (outputs are
    pre-filled with sentinels); the light equals the exact descent's bit for
    bit and so does the argmin of every penumbra ray."""
    h = lunar_tile(130, 12.0, seed=91, amplitude=700.0, n_craters=6, ny=77)
    hf = ss.Heightfield(_dev(h), 12.0, R)
    mip = ss.ss_build_maxmip(hf)
    # a 2 degree disc for wide penumbrae (the oracle finds 146 grid and 41 listed ones)
    sun = ss.Sun(math.radians(1.1), math.radians(140.0), math.radians(2.0))
    uv = random_origins(3001, 130, 77, seed=17)
    for uvt in (None, _dev(uv)):
        n = h.size if uvt is None else uv.shape[0]
        out = dict(light=torch.full((n,), -7.0, device="cuda"),
                   argmin=torch.full((n,), -7, dtype=torch.int32, device="cuda"))
        lo = ss.ss_shadow_forward(hf, mip, sun, 3000.0, uv=uvt, light_only=True, want_cost=False,
                                  out=out, **kw)
        ex = ss.ss_shadow_forward(hf, mip, sun, 3000.0, uv=uvt)
        torch.cuda.synchronize()
        light, arg = lo["light"].cpu().numpy(), lo["argmin"].cpu().numpy()
        el, ea = ex["light"].cpu().numpy(), ex["argmin"].cpu().numpy()
        assert np.all(light >= 0.0) and np.all(arg != -7)
        assert np.array_equal(light.view(np.uint32), el.view(np.uint32))
        pen = (el > 0) & (el < 1)
        assert pen.sum() > 30
        assert np.array_equal(arg[pen], ea[pen])
