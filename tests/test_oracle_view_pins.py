"""Pins of the view-ray oracle (first terrain hit of each pixel's view ray).

Checked against what the geometry fixes, not against the oracle's own code:
  * flat terrain h = h0: the hit is the ray's intersection with the sphere of
    radius R + h0 (closed-form quadratic); compared in 3-D after mapping the
    oracle's texel coordinates back to a direction with the INVERSE mapping;
  * a 1 x 1 camera looks along `forward`: aimed at the pole over flat ground it
    hits the tile centre;
  * brute force on small tiles: a NumPy evaluation of every sample tau_k = k*step
    finds the same first sample below the terrain, and the refined hit lies in
    [tau_{k-1}, tau_k] with the terrain clearance ~0 there;
  * rays above the horizon hit nothing.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import camera, lunar_tile, MOON_RADIUS_M

R = MOON_RADIUS_M


def _inv_map(u, v, nx, ny, g, proj):
    """texel -> unit direction (inverse of the tile mapping)."""
    X = (u - (nx - 1) / 2.0) * g
    Y = (v - (ny - 1) / 2.0) * g
    if proj == "gnomonic":
        d = np.stack([X, Y, np.full_like(X, R)], -1)
        return d / np.linalg.norm(d, axis=-1, keepdims=True)
    r2 = X * X + Y * Y
    return np.stack([4 * R * X, 4 * R * Y, 4 * R * R - r2], -1) / (4 * R * R + r2)[..., None]


def _dirs(cam, pixels):
    i = pixels % cam["width"]
    j = pixels // cam["width"]
    a = (2 * (i + 0.5) / cam["width"] - 1) * cam["tan_x"]
    b = (1 - 2 * (j + 0.5) / cam["height"]) * cam["tan_y"]
    d = cam["forward"][None] + a[:, None] * cam["right"][None] + b[:, None] * cam["up"][None]
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("proj", ["polar_stereo", "gnomonic"])
@pytest.mark.parametrize("h0", [0.0, 850.0, -1200.0])
def test_flat_terrain_hit_is_the_sphere_intersection(proj, h0):
    n, g = 1024, 80.0
    h = np.full((n, n), h0, np.float32)
    cam = camera(64, 36)
    px = np.arange(64 * 36)
    u, v = oracle.view_hits(h, g, R, cam, px, proj=proj)
    d = _dirs(cam, px)
    C = cam["pos"]
    cd = d @ C
    disc = cd * cd - (C @ C - (R + h0) ** 2)
    hit = disc >= 0
    tau = -cd - np.sqrt(np.where(hit, disc, 0.0))
    x = C[None] + tau[:, None] * d
    got = ~np.isnan(u)
    # every oracle hit is a sphere hit; directions agree to ~1e-12 (1 um at R)
    assert got.sum() > 500
    assert np.all(hit[got])
    n_got = _inv_map(u[got], v[got], n, n, g, proj)
    n_exp = x[got] / np.linalg.norm(x[got], axis=1, keepdims=True)
    assert np.abs(n_got - n_exp).max() < 1e-11
    # sphere hits inside the tile (away from its edges) are oracle hits
    exp_dir = x / np.linalg.norm(x, axis=1, keepdims=True)
    if proj == "gnomonic":
        Xp = R * exp_dir[:, 0] / exp_dir[:, 2]
        Yp = R * exp_dir[:, 1] / exp_dir[:, 2]
    else:
        Xp = 2 * R * exp_dir[:, 0] / (1 + exp_dir[:, 2])
        Yp = 2 * R * exp_dir[:, 1] / (1 + exp_dir[:, 2])
    half = (n - 1) / 2.0 * g - 2 * g
    interior = hit & (np.abs(Xp) < half) & (np.abs(Yp) < half)
    assert np.all(got[interior])


def test_single_pixel_camera_looks_at_the_pole():
    n, g = 513, 40.0
    h = np.zeros((n, n), np.float32)
    cam = camera(1, 1)
    u, v = oracle.view_hits(h, g, R, cam, np.array([0]))
    assert abs(u[0] - 256.0) < 1e-6 and abs(v[0] - 256.0) < 1e-6


def _F(h, g, proj, x):
    """terrain clearance |x| - R - h(image of x) and in-tile flag (NumPy, vectorised)."""
    ny, nx = h.shape
    m = np.linalg.norm(x, axis=-1)
    if proj == "gnomonic":
        ok = x[..., 2] > 0
        X = R * x[..., 0] / np.where(ok, x[..., 2], 1.0)
        Y = R * x[..., 1] / np.where(ok, x[..., 2], 1.0)
    else:
        den = m + x[..., 2]
        ok = den > 0
        X = 2 * R * x[..., 0] / np.where(ok, den, 1.0)
        Y = 2 * R * x[..., 1] / np.where(ok, den, 1.0)
    u = X / g + (nx - 1) / 2.0
    v = Y / g + (ny - 1) / 2.0
    ok &= (u >= 0) & (u <= nx - 1) & (v >= 0) & (v <= ny - 1)
    i0 = np.clip(np.floor(np.where(ok, u, 0)).astype(np.int64), 0, nx - 2)
    j0 = np.clip(np.floor(np.where(ok, v, 0)).astype(np.int64), 0, ny - 2)
    fu = np.where(ok, u, 0) - i0
    fv = np.where(ok, v, 0) - j0
    hh = h.astype(np.float64)
    top = hh[j0, i0] + fu * (hh[j0, i0 + 1] - hh[j0, i0])
    bot = hh[j0 + 1, i0] + fu * (hh[j0 + 1, i0 + 1] - hh[j0 + 1, i0])
    return m - R - (top + fv * (bot - top)), ok


@pytest.mark.parametrize("proj", ["polar_stereo", "gnomonic"])
def test_brute_force_first_sample_on_rough_terrain(proj):
    n, g = 160, 150.0
    h = lunar_tile(n, g, seed=41, amplitude=3000.0, n_craters=6)
    cam = camera(48, 27)
    cam["step_m"] = 40.0
    cam["max_dist_m"] = 80e3
    rng = np.random.default_rng(5)
    px = np.sort(rng.choice(48 * 27, 300, replace=False))
    u, v = oracle.view_hits(h, g, R, cam, px, proj=proj)
    d = _dirs(cam, px)
    step = cam["step_m"]
    K = int(math.floor(cam["max_dist_m"] / step))
    taus = np.arange(1, K + 1) * step
    hits = 0
    for q in range(px.size):
        x = cam["pos"][None] + taus[:, None] * d[q][None]
        F, ok = _F(h, g, proj, x)
        below = ok & (F <= 0)
        if not below.any():
            assert np.isnan(u[q])
            continue
        hits += 1
        k = int(np.argmax(below))          # first sample below the terrain (0-based)
        assert not np.isnan(u[q])
        n_hit = _inv_map(np.array([u[q]]), np.array([v[q]]), n, n, g, proj)[0]
        # distance along the ray of the hit direction: solve C + tau d parallel to n_hit
        C = cam["pos"]
        A = np.stack([d[q], -n_hit], 1)
        sol = np.linalg.lstsq(A, -C, rcond=None)[0]
        tau_hit = sol[0]
        assert taus[k] - step - 1e-6 <= tau_hit <= taus[k] + 1e-6
        if k > 0 and ok[k - 1]:
            Fh, okh = _F(h, g, proj, (C + tau_hit * d[q])[None])
            assert okh[0] and abs(Fh[0]) < 1e-5
    assert hits > 100


def test_rays_above_the_horizon_hit_nothing():
    h = lunar_tile(256, 100.0, seed=3, amplitude=2000.0, n_craters=4)
    cam = camera(16, 9)
    cam["forward"] = cam["up"].copy()          # straight up from 10 km altitude
    cam["up"] = -camera(16, 9)["forward"]
    u, v = oracle.view_hits(h, 100.0, R, cam, np.arange(16 * 9))
    assert np.all(np.isnan(u)) and np.all(np.isnan(v))
