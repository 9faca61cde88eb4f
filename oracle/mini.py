"""Independent NumPy restatement of the oracle, for tiny inputs only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Written separately from
``shadow_oracle.c`` (vectorised over all samples of a ray, different indexing
code) so that a slip in either one shows up as a disagreement.

Definitions are the same as the C oracle's: Sec. 3.1 (shadow ray from p toward
the light centre; cost = clearance over distance, minimised along the ray),
Eq. discfrac (circular-segment light fraction), Sec. 3.2 (maximum mipmap).
"""
from __future__ import annotations

import math

import numpy as np


def _sun(elev, az):
    return np.array([math.cos(elev) * math.sin(az), math.cos(elev) * math.cos(az),
                     math.sin(elev)])


def _unit_dir(u, v, nx, ny, g, R, proj):
    X = (np.asarray(u, np.float64) - (nx - 1) / 2.0) * g
    Y = (np.asarray(v, np.float64) - (ny - 1) / 2.0) * g
    if proj == "gnomonic":
        vec = np.stack([X, Y, np.full_like(X, R)], axis=-1)
        return vec / np.linalg.norm(vec, axis=-1, keepdims=True)
    # inverse polar stereographic (projection from the antipode onto z = R)
    r2 = X * X + Y * Y
    den = 4 * R * R + r2
    return np.stack([4 * R * X / den, 4 * R * Y / den, (4 * R * R - r2) / den], axis=-1)


def _to_texel(q, nx, ny, g, R, proj):
    if proj == "gnomonic":
        ok = q[..., 2] > 0
        z = np.where(ok, q[..., 2], 1.0)
        X = R * q[..., 0] / z
        Y = R * q[..., 1] / z
    else:
        den = np.linalg.norm(q, axis=-1) + q[..., 2]
        ok = den > 0
        den = np.where(ok, den, 1.0)
        X = 2 * R * q[..., 0] / den
        Y = 2 * R * q[..., 1] / den
    return X / g + (nx - 1) / 2.0, Y / g + (ny - 1) / 2.0, ok


def _bilerp(h, u, v):
    ny, nx = h.shape
    i0 = np.clip(np.floor(u).astype(np.int64), 0, nx - 2)
    j0 = np.clip(np.floor(v).astype(np.int64), 0, ny - 2)
    fu = u - i0
    fv = v - j0
    top = h[j0, i0] + fu * (h[j0, i0 + 1] - h[j0, i0])
    bot = h[j0 + 1, i0] + fu * (h[j0 + 1, i0 + 1] - h[j0 + 1, i0])
    return top + fv * (bot - top)


def disc_light(d):
    d = np.clip(np.asarray(d, np.float64), -1.0, 1.0)
    return (np.pi - np.arccos(d) + d * np.sqrt(1.0 - d * d)) / np.pi


def shadow(h, g, radius, elev, az, alpha, lmax, step_texels=0.5, proj="gnomonic",
           uv=None, lift=None):
    """Returns (light, argmin (1-based, -1 none), cost) like ``oracle.cref.shadow``."""
    h = np.asarray(h, np.float64)
    ny, nx = h.shape
    if uv is None:
        vv, uu = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                             indexing="ij")
        uv = np.stack([uu.ravel(), vv.ravel()], axis=1)
        lift = np.zeros(uv.shape[0])
    else:
        uv = np.asarray(uv, np.float32).astype(np.float64).reshape(-1, 2)
        lift = np.zeros(uv.shape[0]) if lift is None else np.asarray(lift, np.float32).astype(np.float64)
    s = _sun(elev, az)
    delta = step_texels * g
    J = int(math.floor(lmax / delta))
    t = np.arange(1, J + 1, dtype=np.float64) * delta
    n = uv.shape[0]
    light = np.ones(n)
    argmin = np.full(n, -1, np.int64)
    cost = np.full(n, np.inf)
    for r in range(n):
        u0, v0 = uv[r]
        nr = _unit_dir(u0, v0, nx, ny, g, radius, proj)
        hp = _bilerp(h, np.array([u0]), np.array([v0]))[0] + lift[r]
        p = (radius + hp) * nr
        q = p[None, :] + t[:, None] * s[None, :]
        us, vs, ok = _to_texel(q, nx, ny, g, radius, proj)
        ok &= (us >= 0) & (us <= nx - 1) & (vs >= 0) & (vs <= ny - 1)
        if not ok.any():
            continue
        # only the first run of in-tile samples: the ray is not followed after it leaves
        first = int(np.argmax(ok))
        after = np.nonzero(~ok[first:])[0]
        if after.size:
            ok[first + after[0]:] = False
        H = np.linalg.norm(q, axis=1) - radius
        c = np.full(J, np.inf)
        c[ok] = (H[ok] - _bilerp(h, us[ok], vs[ok])) / t[ok]
        j = int(np.argmin(c))   # first occurrence of the minimum
        cost[r] = c[j]
        argmin[r] = j + 1
        se = float(nr @ s)
        ce = math.sqrt(max(0.0, 1.0 - se * se))
        light[r] = disc_light(cost[r] * ce / alpha)
    return light, argmin, cost


def sample_uv(h, g, radius, svec, j, step_texels=0.5, proj="gnomonic", uv=None, lift=None):
    """Texel coordinates [n, 2] of the image of sample j[r] of each ray (NaN where
    j[r] < 1), like ``oracle.cref.sample_uv``."""
    h = np.asarray(h, np.float64)
    ny, nx = h.shape
    if uv is None:
        vv, uu = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                             indexing="ij")
        uv = np.stack([uu.ravel(), vv.ravel()], axis=1)
        lift = np.zeros(uv.shape[0])
    else:
        uv = np.asarray(uv, np.float32).astype(np.float64).reshape(-1, 2)
        lift = np.zeros(uv.shape[0]) if lift is None else np.asarray(lift, np.float32).astype(np.float64)
    j = np.asarray(j, np.int64).reshape(-1)
    nr = _unit_dir(uv[:, 0], uv[:, 1], nx, ny, g, radius, proj)
    hp = _bilerp(h, uv[:, 0], uv[:, 1]) + lift
    p = (radius + hp)[:, None] * nr
    t = j.astype(np.float64) * step_texels * g
    q = p + t[:, None] * np.asarray(svec, np.float64)[None, :]
    us, vs, ok = _to_texel(q, nx, ny, g, radius, proj)
    ok &= j >= 1
    return np.stack([np.where(ok, us, np.nan), np.where(ok, vs, np.nan)], axis=1)


def maxmip(h):
    """Levels [h, ...] built by padding odd sizes with -inf and reshaping 2x2 blocks."""
    lv = [np.asarray(h, np.float32)]
    while lv[-1].shape != (1, 1):
        a = lv[-1]
        hh, w = a.shape
        pad = np.full((hh + (hh & 1), w + (w & 1)), -np.inf, np.float32)
        pad[:hh, :w] = a
        lv.append(pad.reshape(pad.shape[0] // 2, 2, pad.shape[1] // 2, 2).max(axis=(1, 3)))
    return lv
