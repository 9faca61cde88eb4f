"""The paper's greedy descent on the GPU (ss_shadow_greedy) against its FP64
oracle restatement, and its error against the exact minimum.

Both sides take the same discrete decisions in FP64, so the chosen tip t* must
agree; light, cost and t* are then compared at float32 output precision.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import make_instance, lunar_tile, random_origins, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu(h, g, sun, levels, proj="gnomonic", uv=None, lift=None):
    hf = ss.Heightfield(_dev(h), g, R, projection=proj)
    mip = ss.ss_build_maxmip(hf)
    res = ss.ss_shadow_greedy(hf, mip, ss.Sun(*sun), levels=levels,
                              uv=None if uv is None else _dev(uv),
                              lift=None if lift is None else _dev(lift))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in res.items()}


def _compare(got, light, cost, tstar):
    fin = np.isfinite(cost)
    assert np.array_equal(fin, np.isfinite(got["cost"]))
    assert np.array_equal(tstar < 0, got["t_star"] < 0)
    assert np.all(np.abs(got["t_star"] - tstar) <= 1e-6 * np.maximum(np.abs(tstar), 1.0))
    assert np.all(np.abs(got["cost"][fin] - cost[fin]) <= 1e-6 * np.abs(cost[fin]) + 1e-9)
    assert np.abs(got["light"] - light).max() <= 2e-6


@pytest.mark.parametrize("levels", [(5, 5, 5), (5, 5, 5, 3), (9,)])
def test_tiny_every_ray(levels):
    inst = make_instance("tiny")
    h, g = inst["h"], inst["g"]
    e, a = inst["suns"][0]
    sun = (e, a, inst["alpha"])
    got = _gpu(h, g, sun, levels)
    light, cost, tstar = oracle.greedy(h, g, R, e, a, inst["alpha"], levels=levels)
    _compare(got, light, cost, tstar)


def test_diff_config_four_suns_every_ray():
    inst = make_instance("diff")
    h, g = inst["h"], inst["g"]
    for e, a in inst["suns"]:
        sun = (e, a, inst["alpha"])
        got = _gpu(h, g, sun, (5, 5, 5))
        light, cost, tstar = oracle.greedy(h, g, R, e, a, inst["alpha"], levels=(5, 5, 5))
        _compare(got, light, cost, tstar)


def test_mid_full_size_sampled():
    inst = make_instance("mid")
    h, g = inst["h"], inst["g"]
    e, a = inst["suns"][0]
    sun = (e, a, inst["alpha"])
    got = _gpu(h, g, sun, (5, 5, 5))
    rng = np.random.default_rng(55)
    ids = np.sort(rng.choice(h.size, 20000, replace=False))
    uv = np.stack([ids % h.shape[1], ids // h.shape[1]], 1).astype(np.float32)
    light, cost, tstar = oracle.greedy(h, g, R, e, a, inst["alpha"], levels=(5, 5, 5), uv=uv)
    _compare({k: v[ids] for k, v in got.items()}, light, cost, tstar)


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_list_mode_with_lift(proj):
    n, g = 600, 30.0
    h = lunar_tile(n, g, seed=17, amplitude=1200.0, n_craters=12)
    uv = random_origins(4000, n, n, seed=18)
    lift = np.random.default_rng(19).uniform(0, 50, 4000).astype(np.float32)
    sun = (math.radians(1.3), math.radians(300.0), math.radians(0.2665))
    got = _gpu(h, g, sun, (6, 4), proj=proj, uv=uv, lift=lift)
    light, cost, tstar = oracle.greedy(h, g, R, sun[0], sun[1], sun[2], levels=(6, 4),
                                       proj=proj, uv=uv, lift=lift)
    _compare(got, light, cost, tstar)


@pytest.mark.parametrize("name,n,uv_n", [("tiny", None, 0), ("diff", None, 0), ("mid", 2048, 0),
                                         ("diff", None, 20000)])
def test_float32_build_against_fp64_build(name, n, uv_n):
    """ss_shadow_greedy_f32 (the paper's float32 arithmetic, run lengths of Eq.
    maxstep in float32 too) against the FP64 build, which is decision-identical
    to the oracle.  The tips of a run sit at fractions of its length T, which
    float32 computes to ~1e-3 relative (a cross product of nearly parallel
    vectors), so tip decisions can differ where tips nearly tie; nearly every
    ray's light must still agree, and the light's error against the exact
    descent must be that of the FP64 build.  Grid and listed rays."""
    inst = make_instance(name, n=n)
    h, g = inst["h"], inst["g"]
    uv = lift = None
    if uv_n:
        uv = random_origins(uv_n, h.shape[1], h.shape[0], seed=23)
        lift = np.random.default_rng(24).uniform(0, 20, uv_n).astype(np.float32)
    hf = ss.Heightfield(_dev(h), g, R)
    mip = ss.ss_build_maxmip(hf)
    for (e, a) in inst["suns"][:2]:
        s = ss.Sun(e, a, inst["alpha"])
        kw = dict(uv=None if uv is None else _dev(uv), lift=None if lift is None else _dev(lift))
        d = ss.ss_shadow_greedy(hf, mip, s, levels=(5, 5, 5), **kw)
        f = ss.ss_shadow_greedy(hf, mip, s, levels=(5, 5, 5), fp32=True, **kw)
        x = ss.ss_shadow_forward(hf, mip, s, inst["lmax"], **kw)
        torch.cuda.synchronize()
        d = {k: v.cpu().numpy().astype(np.float64) for k, v in d.items()}
        f = {k: v.cpu().numpy().astype(np.float64) for k, v in f.items()}
        exact = x["light"].cpu().numpy().astype(np.float64)
        assert np.all((f["light"] >= 0) & (f["light"] <= 1))
        agree = np.abs(f["light"] - d["light"]) <= 1e-4
        assert agree.mean() > 0.998, agree.mean()
        ed, ef = np.abs(d["light"] - exact).mean(), np.abs(f["light"] - exact).mean()
        assert abs(ef - ed) <= 0.05 * ed + 1e-3, (ed, ef)
        # inside the penumbra the light fixes the cost: where the lights agree
        # there, so do the costs.  Near either end of the penumbra the visible
        # disc fraction F(d) is flat (F'(d) = 2 sqrt(1 - d^2)/pi -> 0), so a light
        # agreement of 1e-4 says little about the cost; lights in (0.02, 0.98)
        # have F' > 0.1 and pin d to 1e-3, i.e. the cost to ~5e-6 rad.
        pen = (agree & (d["light"] > 0.02) & (d["light"] < 0.98) & (f["light"] > 0.02)
               & (f["light"] < 0.98) & (d["t_star"] > 0))
        assert pen.sum() > 20
        dc = np.abs(f["cost"][pen] - d["cost"][pen])
        bar = 2e-3 * np.abs(d["cost"][pen]) + 2e-5
        i = int(np.argmax(dc - bar))
        assert np.all(dc <= bar), (dc[i], bar[i], d["light"][pen][i], f["light"][pen][i])


def test_float32_build_rejects_stereographic_tiles():
    h = lunar_tile(64, 40.0, seed=3, amplitude=500.0, n_craters=4)
    hf = ss.Heightfield(_dev(h), 40.0, R, projection="polar_stereo")
    mip = ss.ss_build_maxmip(hf)
    with pytest.raises(RuntimeError):
        ss.ss_shadow_greedy(hf, mip, ss.Sun(0.02, 0.3, 0.005), fp32=True)
