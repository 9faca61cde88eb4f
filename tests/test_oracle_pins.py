"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Tolerances: the oracle evaluates the ray height plainly as |q| - R in FP64 at
R = 1737.4 km, whose rounding is ~ulp(R) = 2.3e-10 m; divided by the first
sample distance (>= 5 m) that is <= ~1e-10 rad of cost, so costs are compared
to COST_TOL = 5e-10 rad and light fractions to LIGHT_TOL = 1e-7 (|dF/dc| <= 137/rad).

Each test checks the oracle against something other than itself:
  * Eq. discfrac: identities of the circular-segment area and a Monte-Carlo
    estimate of the lit area of a disc cut by a chord.
  * Sec. 3.1 on a sphere with flat terrain: the cost along the ray is
    increasing, so the argmin is the first sample, with a closed form.
  * An analytic ridge whose apex the shadow ray grazes: light is exactly 1/2,
    and for a raised/lowered apex light follows the disc formula.
  * Sec. 3.2 maximum mipmap: brute-force block maxima.
  * The C oracle against an independent NumPy statement (``oracle.mini``).
  * Finite differences of the oracle's own forward against its analytic gradient.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mini
from workloads import lunar_tile, random_origins, MOON_RADIUS_M

R = MOON_RADIUS_M
ALPHA = math.radians(0.2665)
COST_TOL = 5e-10
LIGHT_TOL = 1e-7


# ---------------------------------------------------------------- Eq. discfrac
def test_disc_light_identities():
    assert oracle.disc_light(-1.0) == 0.0
    assert oracle.disc_light(1.0) == 1.0
    assert abs(oracle.disc_light(0.0) - 0.5) < 1e-15
    assert oracle.disc_light(-3.0) == 0.0 and oracle.disc_light(7.0) == 1.0
    rng = np.random.default_rng(1)
    prev = -1.0
    for d in np.sort(rng.uniform(-1, 1, 200)):
        f = oracle.disc_light(d)
        assert abs(f + oracle.disc_light(-d) - 1.0) < 1e-14   # symmetry
        assert f >= prev                                        # monotone
        prev = f


def test_disc_light_monte_carlo_area():
    """Lit fraction of a unit disc whose horizon chord lies at distance d below
    its centre = area of {y > -d} within the disc, estimated by sampling."""
    rng = np.random.default_rng(2)
    n = 4_000_000
    r = np.sqrt(rng.random(n))
    th = rng.random(n) * 2 * np.pi
    y = r * np.sin(th)
    for d in (-0.9, -0.5, -0.1, 0.0, 0.3, 0.75, 0.95):
        est = np.mean(y > -d)
        f = oracle.disc_light(d)
        sigma = math.sqrt(max(f * (1 - f), 1e-12) / n)
        assert abs(est - f) < 4.5 * sigma, (d, est, f)


# ------------------------------------------------- Sec. 3.1, flat sphere closed form
def _flat_expected(nx, ny, g, h0, elev, az, proj="gnomonic", step=0.5):
    """Closed form for constant terrain height h0: c(t) = (sqrt(rho^2 + 2 t rho sin(eps)
    + t^2) - rho)/t is increasing (a convex function through 0 over t), so
    c* = c(delta) at the first sample; sin(eps) = n_p . s."""
    sinp = oracle.sin_elev(np.zeros((ny, nx)), g, R, elev, az, proj=proj)
    rho = R + h0
    dlt = step * g
    c = (np.sqrt(rho * rho + 2 * dlt * rho * sinp + dlt * dlt) - rho) / dlt
    # write as (2 rho sin + t) / (sqrt(...) + rho) to avoid cancellation
    c = (2 * rho * sinp + dlt) / (np.sqrt(rho * rho + 2 * dlt * rho * sinp + dlt * dlt) + rho)
    d = np.clip(c * np.sqrt(1 - sinp ** 2) / ALPHA, -1, 1)
    return c, mini.disc_light(d)


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
@pytest.mark.parametrize("elev_deg", [-0.5, -0.2, -0.1, 0.0, 0.05, 0.1, 0.15, 0.2, 0.3, 1.5])
def test_flat_sphere_closed_form(proj, elev_deg):
    nx, ny, g, h0 = 33, 29, 20.0, 123.25
    h = np.full((ny, nx), h0, np.float32)
    elev, az = math.radians(elev_deg), math.radians(37.0)
    light, argmin, cost = oracle.shadow(h, g, R, elev, az, ALPHA, 2000.0, proj=proj)
    c_exp, l_exp = _flat_expected(nx, ny, g, h0, elev, az, proj)
    inner = np.zeros((ny, nx), bool)
    inner[1:-1, 1:-1] = True
    inner = inner.ravel()
    assert np.all(argmin[inner] == 1)
    np.testing.assert_allclose(cost[inner], c_exp[inner], rtol=0, atol=COST_TOL)
    np.testing.assert_allclose(light[inner], l_exp[inner], rtol=0, atol=LIGHT_TOL)


def test_sun_below_horizon_is_dark_and_monotone_in_elevation():
    nx = ny = 21
    h = np.zeros((ny, nx), np.float32)
    lights = []
    for e in np.linspace(-2 * 0.2665, 2 * 0.2665, 41):
        light, _, _ = oracle.shadow(h, 20.0, R, math.radians(e), 0.3, ALPHA, 1000.0)
        lights.append(light.reshape(ny, nx)[1:-1, 1:-1].ravel())
    lights = np.array(lights)
    assert np.all(np.diff(lights, axis=0) >= -1e-15)
    light, _, _ = oracle.shadow(h, 20.0, R, math.radians(-1.0), 0.3, ALPHA, 1000.0)
    assert np.all(light.reshape(ny, nx)[1:-1, 1:-1] == 0.0)


def test_large_lift_is_fully_lit():
    h = lunar_tile(48, 20.0, seed=5)
    uv = random_origins(50, 48, 48, seed=6)
    light, _, _ = oracle.shadow(h, 20.0, R, math.radians(1.0), 0.4, ALPHA, 5000.0, uv=uv,
                                lift=np.full(50, 1e5, np.float32))
    assert np.all(light == 1.0)


# ---------------------------------------------------------- analytic ridge
def _ridge_case(proj, axis, sign, delta_m, j_apex=48):
    """Ridge of FP32 height A along a grid line; shadow ray from a flat-ground
    texel aimed so that it passes at height A + delta_m over the apex line.

    Returns (h, u_p, v_p, elev, az, step_texels, lmax, t_apex, sin_eps_p).
    """
    nx, ny, g, A, w = 64, 33, 20.0, np.float32(200.0), 2
    if axis == "v":          # ridge varies along v: swap the roles
        nx, ny = 33, 64
    h = np.zeros((ny, nx), np.float32)
    n_along = nx if axis == "u" else ny
    apex = 40 if sign > 0 else 23
    origin = 8 if sign > 0 else 55
    prof = np.maximum(0.0, 1.0 - np.abs(np.arange(n_along) - apex) / w).astype(np.float64)
    prof = (prof * float(A)).astype(np.float32)
    if axis == "u":
        h[:, :] = prof[None, :]
        up, vp, ua, va = float(origin), 16.0, float(apex), 16.0
    else:
        h[:, :] = prof[:, None]
        up, vp, ua, va = 16.0, float(origin), 16.0, float(apex)

    def unit(u, v):
        X = (u - (nx - 1) / 2.0) * g
        Y = (v - (ny - 1) / 2.0) * g
        if proj == "gnomonic":
            vec = np.array([X, Y, R])
            return vec / np.linalg.norm(vec)
        r2 = X * X + Y * Y
        return np.array([4 * R * X, 4 * R * Y, 4 * R * R - r2]) / (4 * R * R + r2)

    p = R * unit(up, vp)                                   # origin on flat ground (h=0)
    P = (R + float(A) + delta_m) * unit(ua, va)            # point the ray must pass
    t_apex = float(np.linalg.norm(P - p))
    s = (P - p) / t_apex
    elev = math.asin(s[2])
    az = math.atan2(s[0], s[1])
    step = t_apex / (j_apex * g)
    sin_p = float(unit(up, vp) @ s)
    return h, up, vp, elev, az, step, 1.5 * t_apex, t_apex, sin_p


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
@pytest.mark.parametrize("axis,sign", [("u", 1), ("u", -1), ("v", 1), ("v", -1)])
def test_ridge_grazing_ray_is_half_lit(proj, axis, sign):
    h, up, vp, elev, az, step, lmax, t_a, _ = _ridge_case(proj, axis, sign, 0.0)
    uv = np.array([[up, vp]], np.float32)
    light, argmin, cost = oracle.shadow(h, 20.0, R, elev, az, ALPHA, lmax, step_texels=step,
                                        proj=proj, uv=uv)
    assert argmin[0] == 48
    assert abs(cost[0]) < COST_TOL
    assert abs(light[0] - 0.5) < LIGHT_TOL


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
@pytest.mark.parametrize("d_target", [-1.3, -0.95, -0.6, -0.2, 0.1, 0.45, 0.8, 0.99, 1.2])
def test_ridge_penumbra_profile(proj, d_target):
    """Raise/lower the ray over the apex by delta: c* = delta / t_apex exactly, and
    light = F(c* cos(eps_p) / alpha) with F the circular-segment fraction."""
    # first pass to get t_apex and the elevation scale for the requested d
    _, _, _, _, _, _, _, t_a, sin_p = _ridge_case(proj, "u", 1, 0.0)
    delta = d_target * ALPHA * t_a / math.sqrt(1 - sin_p ** 2)
    h, up, vp, elev, az, step, lmax, t_a, sin_p = _ridge_case(proj, "u", 1, delta)
    uv = np.array([[up, vp]], np.float32)
    light, argmin, cost = oracle.shadow(h, 20.0, R, elev, az, ALPHA, lmax, step_texels=step,
                                        proj=proj, uv=uv)
    c_exp = delta / t_a
    d_exp = max(-1.0, min(1.0, c_exp * math.sqrt(1 - sin_p ** 2) / ALPHA))
    f_exp = (math.pi - math.acos(d_exp) + d_exp * math.sqrt(1 - d_exp ** 2)) / math.pi
    assert argmin[0] == 48
    assert abs(cost[0] - c_exp) < COST_TOL
    assert abs(light[0] - f_exp) < LIGHT_TOL


# ------------------------------------------------------------ Sec. 3.2 mipmap
@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (6, 1), (23, 37), (64, 64), (65, 31)])
def test_maxmip_block_maxima(shape):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    h = rng.normal(size=shape).astype(np.float32) * 1000
    levels = oracle.maxmip(h)
    ref = mini.maxmip(h)
    assert len(levels) == len(ref)
    ny, nx = shape
    for l, lv in enumerate(levels):
        assert np.array_equal(lv, ref[l])
        k = 1 << l
        for y in range(lv.shape[0]):
            for x in range(lv.shape[1]):
                assert lv[y, x] == h[y * k:(y + 1) * k, x * k:(x + 1) * k].max()
    assert levels[-1].shape == (1, 1) and levels[-1][0, 0] == h.max()


# -------------------------------------------- C oracle vs independent NumPy
@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
@pytest.mark.parametrize("elev_deg,az_deg", [(1.5, 30.0), (0.4, 200.0), (-0.3, 290.0),
                                             (3.0, 90.0), (0.8, 0.0)])
def test_c_oracle_matches_numpy_grid(proj, elev_deg, az_deg):
    h = lunar_tile(24, 20.0, seed=11, amplitude=300.0, n_craters=3, ny=20)
    args = (h, 20.0, R, math.radians(elev_deg), math.radians(az_deg), ALPHA, 1500.0)
    lc, ac, cc = oracle.shadow(*args, proj=proj)
    lm, am, cm = mini.shadow(*args, proj=proj)
    assert np.array_equal(ac, am)
    fin = np.isfinite(cc)
    assert np.array_equal(fin, np.isfinite(cm))
    np.testing.assert_allclose(cc[fin], cm[fin], rtol=0, atol=COST_TOL)
    np.testing.assert_allclose(lc, lm, rtol=0, atol=LIGHT_TOL)


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_c_oracle_matches_numpy_list_with_lift(proj):
    h = lunar_tile(32, 15.0, seed=12, amplitude=400.0, n_craters=4)
    uv = random_origins(300, 32, 32, seed=13)
    lift = np.random.default_rng(14).uniform(0, 30, 300).astype(np.float32)
    args = (h, 15.0, R, math.radians(1.1), math.radians(143.0), ALPHA, 1200.0)
    lc, ac, cc = oracle.shadow(*args, step_texels=0.37, proj=proj, uv=uv, lift=lift)
    lm, am, cm = mini.shadow(*args, step_texels=0.37, proj=proj, uv=uv, lift=lift)
    assert np.array_equal(ac, am)
    fin = np.isfinite(cc)
    np.testing.assert_allclose(cc[fin], cm[fin], rtol=0, atol=COST_TOL)
    np.testing.assert_allclose(lc, lm, rtol=0, atol=LIGHT_TOL)


def test_cost_is_min_over_all_samples():
    h = lunar_tile(40, 20.0, seed=21, amplitude=600.0, n_craters=5)
    elev, az = math.radians(1.2), math.radians(75.0)
    light, argmin, cost = oracle.shadow(h, 20.0, R, elev, az, ALPHA, 2000.0)
    rng = np.random.default_rng(0)
    for r in rng.choice(40 * 40, 60, replace=False):
        cs = oracle.ray_costs(h, 20.0, R, elev, az, 2000.0, r % 40, r // 40)
        if np.all(np.isnan(cs)):
            assert argmin[r] == -1 and light[r] == 1.0
            continue
        j = int(np.nanargmin(cs))
        assert argmin[r] == j + 1
        assert cost[r] == cs[j]


# ------------------------------------------------ gradient vs finite differences
def _fd_case(seed, proj):
    h = lunar_tile(40, 20.0, seed=seed, amplitude=500.0, n_craters=4).astype(np.float64)
    return h


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_grad_matches_central_differences(proj):
    """Per ray: analytic d light / d h (sample and origin texels) and d light /
    d (elevation, azimuth) against central differences, on rays with a unique
    argmin (gap to the runner-up cost >= 1e-4 rad) and |d| < 0.98.

    Steps: 1e-4 m on heights and 1e-5 rad on angles, so that the oracle's own
    rounding of |q| - R (~2e-10 m, i.e. up to ~2e-11 rad of cost at t = 10 m)
    stays far below the differences, while a step moves any sample cost by
    <= ~1e-5 rad, below the required gap."""
    g, lmax = 20.0, 1500.0
    elev, az = math.radians(2.0), math.radians(57.0)
    alpha = math.radians(3.0)      # a wide disc puts many rays in the penumbra
    h = _fd_case(31, proj)
    n = 1200
    uv = random_origins(n, 40, 40, seed=32, margin=1.0)
    lift = np.random.default_rng(33).uniform(0, 5, n).astype(np.float32)
    light, argmin, cost = oracle.shadow(h, g, R, elev, az, alpha, lmax, proj=proj, uv=uv,
                                        lift=lift)
    sinp = oracle.sin_elev(h, g, R, elev, az, proj=proj, uv=uv)
    d = cost * np.sqrt(1 - sinp ** 2) / alpha
    checked = 0
    for r in range(n):
        if argmin[r] < 0 or not (abs(d[r]) < 0.98):
            continue
        cs = oracle.ray_costs(h, g, R, elev, az, lmax, uv[r, 0], uv[r, 1], lift[r], proj=proj)
        srt = np.sort(cs[np.isfinite(cs)])
        if srt.size < 2 or srt[1] - srt[0] < 1e-4:
            continue
        one = uv[r:r + 1]
        lf = lift[r:r + 1]
        gh, gs = oracle.grad(h, g, R, elev, az, alpha, argmin[r:r + 1], np.ones(1), proj=proj,
                             uv=one, lift=lf)
        nz = np.argwhere(gh != 0)
        assert 1 <= len(nz) <= 8
        eps = 1e-4
        for (y, x) in nz:
            hp = h.copy(); hp[y, x] += eps
            hm = h.copy(); hm[y, x] -= eps
            lp = oracle.shadow(hp, g, R, elev, az, alpha, lmax, proj=proj, uv=one, lift=lf)[0][0]
            lm = oracle.shadow(hm, g, R, elev, az, alpha, lmax, proj=proj, uv=one, lift=lf)[0][0]
            fd = (lp - lm) / (2 * eps)
            # noise floor: |dF/dc| (<= (2/pi)/alpha ~ 12) * 2.3e-10 m / t (>= 10 m) / (2 eps)
            assert abs(fd - gh[y, x]) <= 1e-5 * abs(gh[y, x]) + 3e-6, (r, y, x, fd, gh[y, x])
        for k, (de, da) in enumerate(((1e-5, 0.0), (0.0, 1e-5))):
            lp = oracle.shadow(h, g, R, elev + de, az + da, alpha, lmax, proj=proj, uv=one, lift=lf)[0][0]
            lm = oracle.shadow(h, g, R, elev - de, az - da, alpha, lmax, proj=proj, uv=one, lift=lf)[0][0]
            fd = (lp - lm) / 2e-5
            assert abs(fd - gs[k]) <= 1e-5 * abs(gs[k]) + 1e-5, (r, k, fd, gs[k])
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_grad_sun_vector_matches_central_differences(proj):
    """The raw sun-direction gradient grad_sun[2:5] (s a free 3-vector: q = p + t s
    and sin(eps_p) = n_p . s, both linear in s) against central differences of
    the forward taken along each component of s and along s itself (the
    direction the elevation/azimuth pins above cannot see, since both of their
    tangents are orthogonal to s).  Rays with a unique argmin (runner-up cost at
    least 1e-4 rad above the minimum, from the oracle's own runner-up output) and
    |d| < 0.98; step 1e-5 moves any sample cost by ~1e-5 rad (|dc/ds| ~ 1 + terrain
    slope), below that gap, and the argmin is asserted unchanged.  Near |d| = 1
    the third derivative of F(d) = light grows like (1 - d^2)^-1.5, so the
    central difference's eps^2 error reaches ~2e-5 relative there; Richardson's
    extrapolation of the steps eps and eps/2, (4 D(eps/2) - D(eps)) / 3, removes
    that term."""
    g, lmax = 20.0, 1500.0
    elev, az = math.radians(2.0), math.radians(57.0)
    alpha = math.radians(3.0)
    h = _fd_case(31, proj)
    n = 1200
    uv = random_origins(n, 40, 40, seed=34, margin=1.0)
    lift = np.random.default_rng(35).uniform(0, 5, n).astype(np.float32)
    s = oracle.sun_vector(elev, az)
    light, argmin, cost, cost2 = oracle.shadow_svec(h, g, R, s, alpha, lmax, proj=proj, uv=uv,
                                                    lift=lift)
    # the vector form reproduces the elevation/azimuth form exactly
    l2, a2, c2 = oracle.shadow(h, g, R, elev, az, alpha, lmax, proj=proj, uv=uv, lift=lift)
    assert np.array_equal(a2, argmin) and np.array_equal(l2, light)
    sinp = oracle.sin_elev(h, g, R, elev, az, proj=proj, uv=uv)
    d = cost * np.sqrt(1 - sinp ** 2) / alpha
    ok = (argmin > 0) & (np.abs(d) < 0.98) & (cost2 - cost >= 1e-4)
    ids = np.nonzero(ok)[0]
    assert ids.size >= 20
    one_uv, one_lift = uv[ids], lift[ids]
    gL = np.zeros(ids.size)
    eps = 1e-5
    dirs = [np.eye(3)[i] for i in range(3)] + [s]
    for r_i, r in enumerate(ids):
        gL[:] = 0.0
        gL[r_i] = 1.0
        _, gs = oracle.grad(h, g, R, elev, az, alpha, argmin[ids], gL, proj=proj, uv=one_uv,
                            lift=one_lift)
        for e in dirs:
            dd = []
            for st in (eps, 0.5 * eps):
                lp, ap, _, _ = oracle.shadow_svec(h, g, R, s + st * e, alpha, lmax, proj=proj,
                                                  uv=one_uv[r_i:r_i + 1],
                                                  lift=one_lift[r_i:r_i + 1])
                lm, am, _, _ = oracle.shadow_svec(h, g, R, s - st * e, alpha, lmax, proj=proj,
                                                  uv=one_uv[r_i:r_i + 1],
                                                  lift=one_lift[r_i:r_i + 1])
                assert ap[0] == argmin[r] and am[0] == argmin[r]
                dd.append((lp[0] - lm[0]) / (2 * st))
            fd = (4.0 * dd[1] - dd[0]) / 3.0
            an = float(np.dot(gs[2:5], e))
            assert abs(fd - an) <= 1e-5 * abs(an) + 1e-5, (r, e, fd, an)


def test_runner_up_cost_is_second_smallest_sample_cost():
    """cost2 of the vector-form forward = the second smallest per-sample cost
    (brute force over the per-sample costs; equal costs count twice)."""
    h = lunar_tile(40, 20.0, seed=22, amplitude=600.0, n_craters=5)
    elev, az = math.radians(1.2), math.radians(75.0)
    s = oracle.sun_vector(elev, az)
    light, argmin, cost, cost2 = oracle.shadow_svec(h, 20.0, R, s, ALPHA, 2000.0)
    rng = np.random.default_rng(1)
    for r in rng.choice(40 * 40, 60, replace=False):
        cs = oracle.ray_costs(h, 20.0, R, elev, az, 2000.0, r % 40, r // 40)
        cs = np.sort(cs[np.isfinite(cs)])
        if cs.size < 2:
            assert np.isinf(cost2[r])
            continue
        assert cost[r] == cs[0] and cost2[r] == cs[1]
    # a tile whose every sample ties: the runner-up equals the minimum
    flat = np.zeros((20, 20))
    _, _, c, c2 = oracle.shadow_svec(flat, 20.0, R, s, ALPHA, 2000.0)
    assert np.all(c2 >= c)


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_sample_uv_matches_numpy_and_gradient_cells(proj):
    """sample_uv (C) against the NumPy restatement, and the texels the analytic
    gradient writes for a ray lie in the bilinear cell of its argmin sample's
    image or in the origin's cell."""
    g, lmax = 20.0, 1500.0
    h = _fd_case(31, proj)
    elev, az = math.radians(2.0), math.radians(57.0)
    s = oracle.sun_vector(elev, az)
    uv = random_origins(1500, 40, 40, seed=52, margin=1.0)
    lift = np.random.default_rng(53).uniform(0, 5, 1500).astype(np.float32)
    light, argmin, cost, _ = oracle.shadow_svec(h, g, R, s, math.radians(8.0), lmax, proj=proj,
                                                uv=uv, lift=lift)
    a = oracle.sample_uv(h, g, R, s, argmin, proj=proj, uv=uv, lift=lift)
    b = mini.sample_uv(h, g, R, s, argmin, proj=proj, uv=uv, lift=lift)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    fin = np.isfinite(a)
    assert fin.any()
    np.testing.assert_allclose(a[fin], b[fin], rtol=0, atol=1e-9)
    checked = 0
    for r in np.nonzero((light > 0) & (light < 1) & (argmin > 0))[0][:40]:
        one = np.zeros(1500)
        one[r] = 1.0
        gh, _ = oracle.grad(h, g, R, elev, az, math.radians(8.0), argmin, one, proj=proj, uv=uv,
                            lift=lift)
        i0 = min(int(np.floor(a[r, 0])), 38)
        j0 = min(int(np.floor(a[r, 1])), 38)
        oi = min(int(np.floor(uv[r, 0])), 38)
        oj = min(int(np.floor(uv[r, 1])), 38)
        for (y, x) in np.argwhere(gh != 0):
            assert (i0 <= x <= i0 + 1 and j0 <= y <= j0 + 1) or (oi <= x <= oi + 1 and
                                                                  oj <= y <= oj + 1)
        checked += 1
    assert checked >= 10


def test_grad_abs_and_count_outputs():
    """The per-texel |contribution| sum and count outputs of or_grad: with gL of
    one sign on a single ray, abs equals |grad| texel by texel on the sample
    texels; summed over rays, abs >= |grad| and the counts are whole numbers
    that add up to the non-zero contributions (at most 8 per ray)."""
    g, lmax = 20.0, 1500.0
    h = _fd_case(41, "gnomonic")
    elev, az = math.radians(1.7), math.radians(250.0)
    alpha = math.radians(3.0)
    light, argmin, _ = oracle.shadow(h, g, R, elev, az, alpha, lmax)
    gL = np.random.default_rng(43).normal(size=light.size)
    gh, gs, ah, ch = oracle.grad(h, g, R, elev, az, alpha, argmin, gL, with_abs=True)
    gh2, gs2 = oracle.grad(h, g, R, elev, az, alpha, argmin, gL)
    assert np.array_equal(gh, gh2) and np.array_equal(gs, gs2)
    assert np.all(ah >= np.abs(gh) * (1 - 1e-12))
    assert np.all(ch == np.round(ch)) and ch.sum() <= 8 * np.count_nonzero(gL)
    pen = np.nonzero((light > 0) & (light < 1))[0]
    assert pen.size > 10
    assert ch.sum() >= 4 * pen.size
    r = pen[0]
    one = np.zeros_like(gL)
    one[r] = 1.0
    g1, _, a1, c1 = oracle.grad(h, g, R, elev, az, alpha, argmin, one, with_abs=True)
    assert np.allclose(a1, np.abs(g1), rtol=1e-12, atol=0)
    assert 4 <= c1.sum() <= 8


def test_grad_is_sum_of_per_ray_gradients():
    g, lmax = 20.0, 1500.0
    h = _fd_case(41, "gnomonic")
    elev, az = math.radians(1.7), math.radians(250.0)
    light, argmin, _ = oracle.shadow(h, g, R, elev, az, ALPHA, lmax)
    gL = np.random.default_rng(42).normal(size=light.size)
    gh, gs = oracle.grad(h, g, R, elev, az, ALPHA, argmin, gL)
    acc_h = np.zeros_like(gh)
    acc_s = np.zeros(5)
    uv = np.stack([np.arange(light.size) % 40, np.arange(light.size) // 40], 1).astype(np.float32)
    for r in range(0, light.size, 37):
        gh1, gs1 = oracle.grad(h, g, R, elev, az, ALPHA, argmin[r:r + 1], gL[r:r + 1], uv=uv[r:r + 1])
        acc_h += gh1
        acc_s += gs1
    sub = np.zeros(light.size)
    sub[::37] = gL[::37]
    gh2, gs2 = oracle.grad(h, g, R, elev, az, ALPHA, argmin, sub)
    np.testing.assert_allclose(acc_h, gh2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(acc_s, gs2, rtol=1e-12, atol=1e-15)
