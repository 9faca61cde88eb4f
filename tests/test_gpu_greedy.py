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
