"""Pins of the greedy-descent oracle (the paper's Algorithm 1, reproduced to
measure its error against the exact minimum).

  * flat terrain, sun along grid +y through the tile centre: every level's
    smallest sampled tip wins (the ray rises monotonically), so t* = T/2 with
    T the distance at which the ray's texel image has moved 2^(N'-1) texels --
    found here by root finding on the projection, not with Eq. maxstep -- and
    J = (|p + (T/2) s| - R - h0) / (T/2);
  * a NumPy restatement of the same steps (written separately, vectorised over
    nothing, indexing its own mipmap) agrees on random tiles, grid and list
    rays, several run layouts, both projections.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from workloads import lunar_tile, MOON_RADIUS_M

R = MOON_RADIUS_M


@pytest.mark.parametrize("levels", [(5,), (5, 5, 5), (7, 3)])
@pytest.mark.parametrize("elev_deg", [0.4, 1.5, 6.0])
def test_flat_terrain_closed_form(levels, elev_deg):
    n, g, h0 = 257, 20.0, 310.0
    h = np.full((n, n), h0, np.float32)
    elev, az = math.radians(elev_deg), 0.0            # sun toward grid +y
    alpha = math.radians(0.2665)
    c = (n - 1) // 2
    uv = np.array([[c, c]], np.float32)
    light, cost, tstar = oracle.greedy(h, g, R, elev, az, alpha, levels=levels, uv=uv)
    rho = R + h0
    p = np.array([0.0, 0.0, rho])
    s = np.array([0.0, math.cos(elev), math.sin(elev)])
    span = 2.0 ** (levels[0] - 1)

    def image_v(t):      # gnomonic texel row of p + t s, minus the target row
        q = p + t * s
        return R * q[1] / q[2] / g - span

    T = brentq(image_v, 1e-6, 1e6, xtol=1e-12)
    t_half = T / 2
    J = (np.linalg.norm(p + t_half * s) - R - h0) / t_half
    assert abs(tstar[0] - t_half) < 1e-6 * T
    assert abs(cost[0] - J) < 1e-12
    d = max(-1.0, min(1.0, J * 1.0 / alpha))          # cos(eps_p) = 1 at the centre
    F = (math.pi - math.acos(d) + d * math.sqrt(1 - d * d)) / math.pi
    assert abs(light[0] - F) < 1e-12


# ------------------------------------------------------------- NumPy restatement
def _maxmip(h):
    lv = [np.asarray(h, np.float32)]
    while lv[-1].shape != (1, 1):
        a = lv[-1]
        hh, w = a.shape
        pad = np.full((hh + (hh & 1), w + (w & 1)), -np.inf, np.float32)
        pad[:hh, :w] = a
        lv.append(pad.reshape(pad.shape[0] // 2, 2, pad.shape[1] // 2, 2).max(axis=(1, 3)))
    return lv


def _to_dir(u, v, nx, ny, g, proj):
    X, Y = (u - (nx - 1) / 2) * g, (v - (ny - 1) / 2) * g
    if proj == "gnomonic":
        d = np.array([X, Y, R])
        return d / np.linalg.norm(d)
    r2 = X * X + Y * Y
    return np.array([4 * R * X, 4 * R * Y, 4 * R * R - r2]) / (4 * R * R + r2)


def _to_tex(q, nx, ny, g, proj):
    if proj == "gnomonic":
        if q[2] <= 0:
            return None
        X, Y = R * q[0] / q[2], R * q[1] / q[2]
    else:
        den = np.linalg.norm(q) + q[2]
        if den <= 0:
            return None
        X, Y = 2 * R * q[0] / den, 2 * R * q[1] / den
    return X / g + (nx - 1) / 2, Y / g + (ny - 1) / 2


def _greedy_ray(h64, mips, g, proj, s, alpha, levels, u0, v0, lift):
    ny, nx = h64.shape
    i0 = min(max(int(math.floor(u0)), 0), nx - 2)
    j0 = min(max(int(math.floor(v0)), 0), ny - 2)
    fu, fv = u0 - i0, v0 - j0
    hp = ((1 - fu) * (1 - fv) * h64[j0, i0] + fu * (1 - fv) * h64[j0, i0 + 1]
          + (1 - fu) * fv * h64[j0 + 1, i0] + fu * fv * h64[j0 + 1, i0 + 1]) + lift
    nvec = _to_dir(u0, v0, nx, ny, g, proj)
    p = (R + hp) * nvec
    best, bestd, start = math.inf, -1.0, 0.0
    for Np in levels:
        Rs = p + start * s
        im = _to_tex(Rs, nx, ny, g, proj)
        lxy = math.hypot(s[0], s[1])
        if im is None or lxy == 0:
            break
        e = _to_dir(im[0] + 2 ** (Np - 1) * s[0] / lxy, im[1] + 2 ** (Np - 1) * s[1] / lxy,
                    nx, ny, g, proj)
        axe = np.cross(s, e)
        T = np.dot(np.cross(-Rs, e), axe) / np.dot(axe, axe)
        if not T > 0:
            break
        t = 1.0
        for k in range(Np):
            m = Np - 1 - k
            cands = [t, t - 2.0 ** -(k + 1), t - 2.0 ** -k]
            dbest, tbest = math.inf, -1.0
            for tc in cands:
                if tc <= 0:
                    continue
                q = p + (start + tc * T) * s
                im = _to_tex(q, nx, ny, g, proj)
                if im is None or not (0 <= im[0] <= nx - 1 and 0 <= im[1] <= ny - 1):
                    continue
                L = mips[m]
                I = min(max(int(math.floor((im[0] + 0.5) / 2 ** m)), 0), L.shape[1] - 1)
                Jv = min(max(int(math.floor((im[1] + 0.5) / 2 ** m)), 0), L.shape[0] - 1)
                dlt = np.linalg.norm(q) - R - float(L[Jv, I])
                if dlt < dbest:
                    dbest, tbest = dlt, tc
            t = tbest + 2.0 ** -(k + 1) if tbest > -1 else t - 2.0 ** -k
        if tbest > -1:
            dist = start + tbest * T
            if dbest / dist < best:
                best, bestd = dbest / dist, dist
        start += T
    if bestd <= 0:
        return 1.0, math.inf, -1.0
    se = float(nvec @ s)
    d = max(-1.0, min(1.0, best * math.sqrt(max(0.0, 1 - se * se)) / alpha))
    return (math.pi - math.acos(d) + d * math.sqrt(1 - d * d)) / math.pi, best, bestd


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
@pytest.mark.parametrize("levels", [(5, 5, 5), (4,), (6, 3, 2)])
def test_c_oracle_matches_numpy_restatement(proj, levels):
    n, g = 72, 25.0
    h = lunar_tile(n, g, seed=61, amplitude=300.0, n_craters=5, ny=57)
    elev, az, alpha = math.radians(1.1), math.radians(231.0), math.radians(1.0)
    s = np.array([math.cos(elev) * math.sin(az), math.cos(elev) * math.cos(az), math.sin(elev)])
    mips = _maxmip(h)
    h64 = h.astype(np.float64)
    rng = np.random.default_rng(9)
    uv = np.stack([rng.uniform(0, n - 1, 150), rng.uniform(0, 56, 150)], 1).astype(np.float32)
    lift = rng.uniform(0, 30, 150).astype(np.float32)
    for mode_uv, mode_lift in ((None, None), (uv, lift)):
        light, cost, tstar = oracle.greedy(h, g, R, elev, az, alpha, levels=levels, proj=proj,
                                           uv=mode_uv, lift=mode_lift)
        if mode_uv is None:
            ids = rng.choice(h.size, 200, replace=False)
            pts = [(float(i % n), float(i // n), 0.0) for i in ids]
        else:
            ids = np.arange(150)
            pts = [(float(uv[i, 0]), float(uv[i, 1]), float(lift[i])) for i in ids]
        for k, (u0, v0, lf) in zip(ids, pts):
            el, ec, et = _greedy_ray(h64, mips, g, proj, s, alpha, levels, u0, v0, lf)
            assert et == pytest.approx(tstar[k], abs=1e-9), (k, et, tstar[k])
            if math.isfinite(ec):
                assert ec == pytest.approx(cost[k], rel=1e-9, abs=1e-12)
            else:
                assert not math.isfinite(cost[k])
            assert el == pytest.approx(light[k], abs=1e-9)
