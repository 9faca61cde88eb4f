"""The five synthetic workloads, as plain parameter records.

Sizes, scales and sun geometry follow the paper's lunar polar scenes (Sec. 1,
Sec. 3.1 Fig. 2: shadows tens of km long, penumbra ~1/7 of it, <=30 m/texel)
and the build's workload list.  Seeds are fixed: config k uses 20050667 + k.
Only parameters and seeded random draws live here; no shadow arithmetic.
"""
from __future__ import annotations

import math
import os

import numpy as np

from .terrain import lunar_tile, sun_list

MOON_RADIUS_M = 1737.4e3
SUN_ANGULAR_RADIUS_RAD = math.radians(0.2665)
SEED_BASE = 20050667

CONFIGS = {
    "tiny": dict(id=1, n=256, g=20.0, amplitude=1500.0, craters=20,
                 suns=[(1.5, 30.0)], lmax=20e3, proj="gnomonic"),
    "mid": dict(id=2, n=4096, g=10.0, amplitude=1500.0, craters=500,
                suns=[(1.0, 120.0)], lmax=60e3, proj="gnomonic"),
    "polar": dict(id=3, n=16384, g=5.0, amplitude=4000.0, craters=5000,
                  suns=[(0.5, 210.0)], lmax=100e3, proj="polar_stereo"),
    "batched": dict(id=4, n_instances=64, sizes=(512, 1024, 2048, 4096), g=10.0,
                    amplitude=1500.0, lmax=50e3, proj="gnomonic"),
    "diff": dict(id=5, n=1024, g=10.0, amplitude=1500.0, craters=32,
                 suns=[(0.8, 0.0), (1.2, 90.0), (1.6, 180.0), (2.0, 270.0)],
                 lmax=50e3, proj="gnomonic", bumps=64, bump_sigma=50.0, bump_amp=30.0),
}


def config(name):
    return dict(CONFIGS[name])


def _cache_dir():
    d = os.environ.get("SS_WORKLOAD_CACHE", "")
    if d:
        os.makedirs(d, exist_ok=True)
    return d


# The last few generated tiles, kept in memory (the 16384^2 polar tile takes
# about a minute to generate); callers get copies.
_MEMO = {}
_MEMO_MAX = 3


def _tile(n, g, seed, amplitude, craters):
    key = (n, g, seed, amplitude, craters)
    if key in _MEMO:
        return _MEMO[key].copy()
    h = _tile_uncached(n, g, seed, amplitude, craters)
    if len(_MEMO) >= _MEMO_MAX:
        _MEMO.pop(next(iter(_MEMO)))
    _MEMO[key] = h
    return h.copy()


def _tile_uncached(n, g, seed, amplitude, craters):
    cache = _cache_dir()
    path = os.path.join(cache, f"tile_{n}_{g:g}_{seed}_{amplitude:g}_{craters}.npy") if cache else ""
    if path and os.path.exists(path):
        return np.load(path)
    h = lunar_tile(n, g, seed, amplitude=amplitude, n_craters=craters)
    if path:
        np.save(path, h)
    return h


def make_instance(name, n=None, sun_index=None):
    """Heightfield + sun(s) for a named single-tile config.

    ``n`` overrides the tile size (same generator, crater count scaled by area)
    so that tests can run the same recipe at sizes the oracle finishes quickly.
    Returns a dict with keys h (float32 [n, n]), g, radius, suns [(elev, az) rad],
    alpha, lmax, proj, seed.
    """
    c = CONFIGS[name]
    seed = SEED_BASE + c["id"]
    size = c["n"] if n is None else int(n)
    craters = c["craters"]
    if n is not None and size != c["n"]:
        craters = max(4, int(round(craters * (size / c["n"]) ** 2)))
    h = _tile(size, c["g"], seed, c["amplitude"], craters)
    suns = [(math.radians(e), math.radians(a)) for e, a in c["suns"]]
    if sun_index is not None:
        suns = [suns[sun_index]]
    return dict(h=h, g=c["g"], radius=MOON_RADIUS_M, suns=suns,
                alpha=SUN_ANGULAR_RADIUS_RAD, lmax=c["lmax"], proj=c["proj"],
                seed=seed)


def batched_instances(n_instances=None, sizes=None, seed_offset=0):
    """Config 'batched': tiles with sizes drawn from {512..4096}^2, one sun each
    (elevation U(0.2, 3) deg, azimuth U(0, 360) deg), crater count 500*(N/4096)^2, min 8."""
    c = CONFIGS["batched"]
    k = c["n_instances"] if n_instances is None else n_instances
    sizes = c["sizes"] if sizes is None else sizes
    seed = SEED_BASE + c["id"] + seed_offset
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=k)
    suns = sun_list(k, seed + 1)
    out = []
    for i, (nn, sun) in enumerate(zip(ns, suns)):
        nn = int(nn)
        craters = max(8, int(round(500 * (nn / 4096) ** 2)))
        h = _tile(nn, c["g"], seed * 1000 + i, c["amplitude"], craters)
        out.append(dict(h=h, g=c["g"], radius=MOON_RADIUS_M, suns=[sun],
                        alpha=SUN_ANGULAR_RADIUS_RAD, lmax=c["lmax"], proj=c["proj"]))
    return out


def bump_target(h, g, seed, n_bumps=64, sigma=50.0, amp=30.0):
    """Config 'diff' target field: h + sum of seeded Gaussian bumps (sigma, amplitude in m)."""
    ny, nx = h.shape
    rng = np.random.default_rng(seed + 7)
    out = h.astype(np.float64).copy()
    xs = np.arange(nx) * g
    ys = np.arange(ny) * g
    for _ in range(n_bumps):
        cx = rng.uniform(0, (nx - 1) * g)
        cy = rng.uniform(0, (ny - 1) * g)
        s = rng.choice([-1.0, 1.0])
        out += s * amp * np.exp(-((ys[:, None] - cy) ** 2 + (xs[None, :] - cx) ** 2) / (2 * sigma * sigma))
    return out.astype(np.float32)


# Oblique view of the polar scene whose visible surface points are the polar
# config's shadow-ray origins: camera 10 km above the surface, 30 km from the
# pole toward grid -y, aimed at the pole, 40 deg vertical field of view,
# 3840 x 2160 pixels (smaller pixel grids keep the same frustum).
POLAR_CAMERA = dict(altitude=10e3, offset=30e3, fov_y_deg=40.0, width=3840, height=2160,
                    step_m=2.5, max_dist_m=150e3)


def camera(width=None, height=None, radius=MOON_RADIUS_M):
    """The polar view as plain numbers: centre ``pos`` (m, tile frame: z through
    the pole, grid +y = y), orthonormal ``forward``/``right``/``up`` (up in the
    plane of forward and the local vertical), ``tan_x``/``tan_y`` (half-angle
    tangents), ``width``/``height`` (pixel (i, j), row 0 at the top, looks along
    forward + a right + b up with a = (2(i+0.5)/W - 1) tan_x,
    b = (1 - 2(j+0.5)/H) tan_y), and the march parameters ``step_m``,
    ``max_dist_m``."""
    c = POLAR_CAMERA
    W = c["width"] if width is None else int(width)
    H = c["height"] if height is None else int(height)
    th = c["offset"] / radius
    vert = np.array([0.0, -math.sin(th), math.cos(th)])
    pos = (radius + c["altitude"]) * vert
    target = np.array([0.0, 0.0, radius])
    fwd = target - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, vert)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    tan_y = math.tan(math.radians(c["fov_y_deg"]) / 2.0)
    tan_x = tan_y * W / H
    return dict(pos=pos, forward=fwd, right=right, up=up, tan_x=tan_x, tan_y=tan_y,
                width=W, height=H, step_m=c["step_m"], max_dist_m=c["max_dist_m"])


# Lights of the shading epilogue (Sec. 3.4: Sun and Earth as discs).  Sun:
# the config's sun, unit intensity.  Earth as seen from a lunar pole: low over
# the horizon, apparent radius 0.95 deg (6371 km at 384,400 km), earthshine
# irradiance ~1/5000 of sunlight (proposed values).
EARTH_LIGHT = dict(elevation_deg=2.0, azimuth_deg=0.0, angular_radius_deg=0.95,
                   intensity=2e-4)
