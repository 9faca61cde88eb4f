"""Seeded synthetic lunar terrain: fractional Brownian motion plus parabolic craters.

The paper's scenes use lunar south-pole terrain at up to 30 m/texel with crater
rims casting shadows tens of kilometres long and penumbrae about a seventh of
that (Sec. 3.1, Fig. 2; Sec. 1).  Those datasets are not available here, so
these seeded fields stand in for them with the same scales.

Everything is computed in float64 and returned as float32 row-major arrays
``h[row, col]`` (row = v / grid +y, col = u / grid +x).  Texel (col, row) sits at
plane coordinates ``x = (col - (nx-1)/2) * g``, ``y = (row - (ny-1)/2) * g``.

Nothing here evaluates shadows; it only makes heights, sun angles and ray origins.
"""
from __future__ import annotations

import math

import numpy as np


def _fade(s):
    # quintic smoothstep 6s^5 - 15s^4 + 10s^3 (Perlin's improved-noise fade curve)
    return s * s * s * (s * (s * 6.0 - 15.0) + 10.0)


def _corner_weights(coord, n_lat):
    """Separable factors of 2-D gradient noise along one axis.

    For lattice point l at distance s = coord - l the blend weight is
    fade(1 - |s|) when |s| < 1, else 0.  Returns (w, w*s), each [len(coord), n_lat].
    """
    s = coord[:, None] - np.arange(n_lat, dtype=np.float64)[None, :]
    a = np.abs(s)
    w = np.where(a < 1.0, _fade(np.clip(1.0 - a, 0.0, 1.0)), 0.0)
    return w, w * s


def gradient_noise(nx, ny, cells_x, cells_y, rng):
    """One octave of 2-D gradient noise sampled at texel centres.

    The tile spans ``cells_x`` x ``cells_y`` lattice cells; the lattice is shifted
    by a random sub-cell offset.  Evaluated in separable matrix form:
    noise = P @ GX @ Q^T + D @ GY @ W^T.
    """
    ox, oy = rng.random(2)
    xs = (np.arange(nx, dtype=np.float64) + 0.5) / nx * cells_x + ox
    ys = (np.arange(ny, dtype=np.float64) + 0.5) / ny * cells_y + oy
    lx = int(math.ceil(cells_x + 1.0)) + 1
    ly = int(math.ceil(cells_y + 1.0)) + 1
    theta = rng.random((ly, lx)) * (2.0 * math.pi)
    gx, gy = np.cos(theta), np.sin(theta)
    wxc, wxs = _corner_weights(xs, lx)   # [nx, lx]
    wyc, wys = _corner_weights(ys, ly)   # [ny, ly]
    return wyc @ gx @ wxs.T + wys @ gy @ wxc.T


def fbm(nx, ny, rng, octaves=8, hurst=0.8, lacunarity=2.0, amplitude=1500.0):
    """Octave sum of gradient noise; base wavelength = tile width; gain 2^-H.

    Mean removed, then scaled so that max |h| == amplitude.
    """
    h = np.zeros((ny, nx), dtype=np.float64)
    gain = 2.0 ** (-hurst)
    aspect = ny / nx
    for k in range(octaves):
        cells = lacunarity ** k
        h += (gain ** k) * gradient_noise(nx, ny, cells, cells * aspect, rng)
    h -= h.mean()
    m = np.abs(h).max()
    if m > 0:
        h *= amplitude / m
    return h


def crater_radii(n, rng, r_min=200.0, r_max=2000.0):
    """Radii with cumulative size-frequency N(>r) ~ r^-2, truncated to [r_min, r_max]."""
    u = rng.random(n)
    a, b = r_min ** -2.0, r_max ** -2.0
    return (a - u * (a - b)) ** -0.5


def add_craters(h, g, n, rng, r_min=200.0, r_max=2000.0):
    """Add ``n`` parabolic-bowl craters in place (float64 array, metres).

    Inside radius r: h += h_r + d((rho/r)^2 - 1), depth d = 0.2*(2r), rim h_r = 0.04*(2r).
    Outside: h += h_r (rho/r)^-3, truncated at 3r.
    """
    ny, nx = h.shape
    cx = (rng.random(n) - 0.5) * (nx - 1) * g
    cy = (rng.random(n) - 0.5) * (ny - 1) * g
    radii = crater_radii(n, rng, r_min, r_max)
    x0 = -(nx - 1) / 2.0 * g
    y0 = -(ny - 1) / 2.0 * g
    for xc, yc, r in zip(cx, cy, radii):
        d = 0.4 * r
        hr = 0.08 * r
        reach = 3.0 * r
        i0 = max(0, int(math.floor((xc - reach - x0) / g)))
        i1 = min(nx - 1, int(math.ceil((xc + reach - x0) / g)))
        j0 = max(0, int(math.floor((yc - reach - y0) / g)))
        j1 = min(ny - 1, int(math.ceil((yc + reach - y0) / g)))
        if i0 > i1 or j0 > j1:
            continue
        xs = x0 + np.arange(i0, i1 + 1) * g - xc
        ys = y0 + np.arange(j0, j1 + 1) * g - yc
        rho = np.sqrt(ys[:, None] ** 2 + xs[None, :] ** 2) / r
        inside = hr + d * (rho * rho - 1.0)
        outside = np.where(rho <= 3.0, hr * np.maximum(rho, 1.0) ** -3.0, 0.0)
        h[j0:j1 + 1, i0:i1 + 1] += np.where(rho < 1.0, inside, outside)
    return h


def lunar_tile(n, g, seed, amplitude=1500.0, n_craters=20, ny=None):
    """fBm (H=0.8, 8 octaves) + craters, as float32 [ny, n]."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    h = fbm(n, ny, rng, amplitude=amplitude)
    add_craters(h, g, n_craters, rng)
    return h.astype(np.float32)


def sun_list(n, seed, elev_deg=(0.2, 3.0), az_deg=(0.0, 360.0)):
    """``n`` (elevation, azimuth) pairs in radians, uniform over the given ranges."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(*elev_deg, size=n)
    a = rng.uniform(*az_deg, size=n)
    return [(math.radians(ei), math.radians(ai)) for ei, ai in zip(e, a)]


def random_origins(n, nx, ny, seed, margin=0.0):
    """``n`` ray origins (u, v) in continuous texel coordinates inside the tile."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(margin, nx - 1 - margin, size=n)
    v = rng.uniform(margin, ny - 1 - margin, size=n)
    return np.stack([u, v], axis=1).astype(np.float32)
