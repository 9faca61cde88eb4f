"""Shading epilogue (ss_shade) against the FP64 shading oracle.

The lit fractions fed to both sides are seeded random numbers (or the oracle's
own shadow results), never GPU outputs; bar: irradiance within 2e-6 relative
+ 1e-7 absolute (float32 arithmetic on the GPU).  End to end (shadow pass per
light, then shading), GPU and oracle chains are independent and agree within
the light-fraction bar times the intensities.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import make_instance, lunar_tile, random_origins, MOON_RADIUS_M, EARTH_LIGHT

import paper_2005_06671_gb300 as ss

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _lights(n, seed):
    rng = np.random.default_rng(seed)
    return [(math.radians(1.5), math.radians(30.0), 1.0, rng.uniform(0, 1, n)),
            (math.radians(2.0), math.radians(200.0), 0.3, rng.uniform(0, 1, n)),
            (math.radians(-0.2), math.radians(95.0), 0.05, np.ones(n))]


def _check(E_gpu, E_ref):
    assert np.all(np.abs(E_gpu - E_ref) <= 2e-6 * np.abs(E_ref) + 1e-7), \
        np.abs(E_gpu - E_ref).max()


@pytest.mark.parametrize("proj,n,g", [("gnomonic", 256, 20.0), ("polar_stereo", 300, 400.0),
                                      ("gnomonic", 97, 1500.0)])
def test_grid_rays_every_texel(proj, n, g):
    h = lunar_tile(n, g, seed=n, amplitude=1500.0, n_craters=10, ny=n - 17)
    lights = _lights(h.size, 5)
    hf = ss.Heightfield(_dev(h), g, R, projection=proj)
    E = ss.ss_shade(hf, [(e, a, i, _dev(s.astype(np.float32))) for e, a, i, s in lights])
    E_ref = oracle.shade(h, g, R, [(e, a, i, s.astype(np.float32)) for e, a, i, s in lights],
                         proj=proj)
    _check(E.cpu().numpy().astype(np.float64), E_ref)


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_listed_origins(proj):
    n, g = 400, 60.0
    h = lunar_tile(n, g, seed=8, amplitude=2000.0, n_craters=10)
    uv = random_origins(5000, n, n, seed=9)
    lights = _lights(5000, 10)
    hf = ss.Heightfield(_dev(h), g, R, projection=proj)
    E = ss.ss_shade(hf, [(e, a, i, _dev(s.astype(np.float32))) for e, a, i, s in lights],
                    uv=_dev(uv))
    E_ref = oracle.shade(h, g, R, [(e, a, i, s.astype(np.float32)) for e, a, i, s in lights],
                         proj=proj, uv=uv)
    _check(E.cpu().numpy().astype(np.float64), E_ref)


def test_sun_and_earth_end_to_end_sampled():
    inst = make_instance("mid")
    h, g = inst["h"], inst["g"]
    rng = np.random.default_rng(77)
    ids = np.sort(rng.choice(h.size, 3000, replace=False))
    uv = np.stack([ids % h.shape[1], ids // h.shape[1]], 1).astype(np.float32)
    e_s, a_s = inst["suns"][0]
    earth = (math.radians(EARTH_LIGHT["elevation_deg"]), math.radians(EARTH_LIGHT["azimuth_deg"]),
             math.radians(EARTH_LIGHT["angular_radius_deg"]))
    hf = ss.Heightfield(_dev(h), g, R)
    mip = ss.ss_build_maxmip(hf)
    uvt = _dev(uv)
    lit_s = ss.ss_shadow_forward(hf, mip, ss.Sun(e_s, a_s, inst["alpha"]), inst["lmax"], uv=uvt)
    lit_e = ss.ss_shadow_forward(hf, mip, ss.Sun(*earth), inst["lmax"], uv=uvt)
    E = ss.ss_shade(hf, [(e_s, a_s, 1.0, lit_s["light"]),
                         (earth[0], earth[1], EARTH_LIGHT["intensity"], lit_e["light"])], uv=uvt)
    E = E.cpu().numpy().astype(np.float64)
    ol_s = oracle.shadow(h, g, R, e_s, a_s, inst["alpha"], inst["lmax"], uv=uv)[0]
    ol_e = oracle.shadow(h, g, R, earth[0], earth[1], earth[2], inst["lmax"], uv=uv)[0]
    E_ref = oracle.shade(h, g, R, [(e_s, a_s, 1.0, ol_s),
                                   (earth[0], earth[1], EARTH_LIGHT["intensity"], ol_e)], uv=uv)
    assert np.abs(E - E_ref).max() <= 1e-5 * (1.0 + EARTH_LIGHT["intensity"]) + 1e-6
    assert ((ol_s > 0) & (ol_s < 1)).sum() > 10
