"""Full-size checks of the differentiable workload against the oracle (the
batched workload's full-size parity is in test_gpu_coverage.py).

* Differentiable: 1024^2, 4 suns, loss = mean over rays and suns of
  (light(H) - light(H'))^2 with H' = H + 64 seeded Gaussian bumps.
  - The GPU backward against the oracle's analytic gradient, texel by texel
    over the whole tile and on the sun angles.
  - The GPU gradient against FP64 central differences of the loss itself,
    computed with the oracle's forward, on the 64 x 64 window at the tile
    centre and on every sun's elevation and azimuth.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import bump_target, make_instance, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss
from _parity import grad_weights_mask, assert_grad_close, F32_UNIT, LIGHT_TOL

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M


# ----------------------------------------------------- differentiable config
# FD set-up (FP64, the oracle's forward).  The loss is restricted to the rays
# Omega with a unique argmin, runner-up cost >= GAP above the minimum, and
# |d| < D_MAX (away from the kinks of the clamp); every other ray gets no weight
# on either side.  A height step H_STEP moves any sample cost by at most
# H_STEP/delta (1 + ~1e-3) = 4e-6 rad < GAP/2 (delta = 5 m), and an angle step
# A_STEP by at most (1 + max slope) A_STEP (asserted below), so no ray of Omega
# changes its argmin within the steps (also asserted): the loss is smooth
# there, and a ray's light depends on a texel only through its argmin
# sample's bilinear cell and its origin, so each window texel's difference
# re-evaluates exactly those rays of Omega.  Central differences with
# Richardson's extrapolation (steps s and s/2) remove the s^2 error term,
# which near |d| = D_MAX is ~(1 - d^2)^-2 (dd)^2 / 6.
GAP = 1e-5
D_MAX = 0.99
H_STEP = 2e-5
A_STEP = 1e-6


@pytest.fixture(scope="module")
def diff_case():
    inst = make_instance("diff")
    h = inst["h"]
    g, alpha, lmax = inst["g"], inst["alpha"], inst["lmax"]
    target = bump_target(h, g, inst["seed"])
    per_sun = []
    for (e, a) in inst["suns"]:
        s = oracle.sun_vector(e, a)
        lo, ao, co, c2o = oracle.shadow_svec(h, g, R, s, alpha, lmax)
        lt, _, _ = oracle.shadow(target, g, R, e, a, alpha, lmax)
        sinp = oracle.sin_elev(h, g, R, e, a)
        d = co * np.sqrt(1.0 - sinp ** 2) / alpha
        with np.errstate(invalid="ignore"):
            omega = (ao > 0) & (np.abs(d) < D_MAX) & (c2o - co >= GAP)
        per_sun.append(dict(e=e, a=a, s=s, lo=lo, ao=ao, co=co, lt=lt, sinp=sinp, omega=omega))
    return dict(inst=inst, h=h, g=g, alpha=alpha, lmax=lmax, target=target, suns=per_sun)


def test_diff_config_full_size_gradient_vs_oracle_every_texel(diff_case):
    """dLoss/dH on every texel and dLoss/d(elevation, azimuth) per sun: the GPU
    backward against the oracle's analytic gradient (itself pinned by central
    differences), with dLoss/dlight from the oracle's lights.  Ties and rays at
    saturation get no weight on either side."""
    h, g, alpha, lmax = diff_case["h"], diff_case["g"], diff_case["alpha"], diff_case["lmax"]
    ny, nx = h.shape
    n_sun = len(diff_case["suns"])
    hf = ss.Heightfield(torch.from_numpy(h).cuda(), g, R)
    mip = ss.ss_build_maxmip(hf)
    gh_gpu_tot = np.zeros((ny, nx))
    gh_o_tot, ah_tot, ch_tot = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    for c in diff_case["suns"]:
        gl = 2.0 * (c["lo"] - c["lt"]) / (h.size * n_sun)          # dLoss/dlight
        sn = ss.Sun(c["e"], c["a"], alpha)
        res = ss.ss_shadow_forward(hf, mip, sn, lmax)
        am = res["argmin"].cpu().numpy().astype(np.int64)
        assert np.abs(res["light"].cpu().numpy() - c["lo"]).max() <= LIGHT_TOL
        gl[~grad_weights_mask(c["lo"], c["co"], c["sinp"], alpha, am, c["ao"])] = 0.0
        gl32 = gl.astype(np.float32)
        gh, gs = ss.ss_shadow_backward(hf, sn, lmax, res["argmin"], torch.from_numpy(gl32).cuda(),
                                       cost=res["cost"])
        torch.cuda.synchronize()
        gh_o, gs_o, ah, ch = oracle.grad(h, g, R, c["e"], c["a"], alpha, c["ao"],
                                         gl32.astype(np.float64), with_abs=True)
        # each sun's backward accumulates into its own zeroed buffer: add the
        # float32 results in FP64, and the bars texel by texel
        gh_gpu_tot += gh.cpu().numpy()
        gh_o_tot += gh_o
        ah_tot += ah
        ch_tot += ch
        np.testing.assert_allclose(gs.cpu().numpy()[:2], gs_o[:2], rtol=1e-4,
                                   atol=1e-6 * np.abs(gs_o[:2]).max() + 1e-12)
    st = assert_grad_close(gh_gpu_tot, gh_o_tot, ah_tot, ch_tot)
    assert st["texels"] > 10000
    c0 = (ny - 64) // 2, (nx - 64) // 2
    win = (slice(c0[0], c0[0] + 64), slice(c0[1], c0[1] + 64))
    assert np.count_nonzero(ch_tot[win]) >= 10


def test_diff_config_loss_central_differences_on_centre_window(diff_case):
    """Gradients against FP64 central differences of the loss itself (the
    oracle's forward; see GAP, D_MAX, H_STEP, A_STEP above), for two losses
    over the rays of Omega:
      (a) the config's loss, mean over rays and suns of (light(H) - light(H'))^2
          (only rays whose light the bumps change carry weight);
      (b) a linear loss, mean over rays and suns of c_r light(H) with seeded
          weights c_r ~ N(0, 1), so that every ray of Omega carries weight.
    The differences are taken of the forward, the light of each ray of Omega
    under each perturbation, and each loss's outer function is applied to them
    by the chain rule (loss (a): 2 (light - light(H')) dlight; loss (b):
    c_r dlight): a central difference of the square itself would carry, for
    rays whose light the bumps barely change, an error that is not
    proportional to the residual.
    Per texel of the 64 x 64 centre window and per sun angle:
      |g_gpu - fd| <= 1e-4 S + N + (cnt + 1) 2^-24 A
    with S the sum over rays of |per-ray difference| (the difference's own
    scale), N the rounding noise of the differences, A and cnt the oracle's
    |contribution| sum and count for the texel (float32 accumulation); texels
    no ray of Omega reads are exactly zero on the GPU.  N: a perturbation moves
    a ray's light through its cost c = (|q| - R - h)/t, which the oracle rounds
    to ~2^-53 (|q| - R and h terms: 2 max|h| for a sample texel, R once the
    origin or the sun moves q); the light moves |dl/dc| times that, and the
    Richardson central difference divides it by the step, so per ray
      N_r = 16 |dl/dc| 2^-53 L / (t step) |dLoss/dlight_r|,
    L = R or 2 max|h| (16 covers the extrapolation's (4 + 1)/3, the two
    evaluations and a margin); it matters only where the texel's weight in the
    ray's argmin cell is nearly zero.  The GPU gradient comes from ss_shadow_backward given dLoss/dlight from
    the oracle's lights; for loss (a) also from the autograd Function on the
    loss written with the GPU's own lights (their errors, <= LIGHT_TOL on each
    side, add 2 LIGHT_TOL |dlight/dh| / (n_rays n_sun) per ray to the bar)."""
    h, g, alpha, lmax = diff_case["h"], diff_case["g"], diff_case["alpha"], diff_case["lmax"]
    target = diff_case["target"]
    ny, nx = h.shape
    N = h.size
    n_sun = len(diff_case["suns"])
    wgt = 1.0 / (N * n_sun)
    c0 = (ny - 64) // 2, (nx - 64) // 2
    win = (slice(c0[0], c0[0] + 64), slice(c0[1], c0[1] + 64))
    h64 = h.astype(np.float64)                     # perturbed in place, restored after
    grid_uv = np.stack([np.arange(N) % nx, np.arange(N) // nx], 1).astype(np.float32)
    slope = max(np.abs(np.diff(h64, axis=0)).max(), np.abs(np.diff(h64, axis=1)).max()) / g
    assert (1.0 + slope) * A_STEP < GAP / 2
    cw = np.random.default_rng(20050672).normal(size=(n_sun, N))   # loss (b) weights

    hf = ss.Heightfield(torch.from_numpy(h).cuda(), g, R)
    mip = ss.ss_build_maxmip(hf)
    L = ("mse", "lin")
    gh_gpu = {l: np.zeros((ny, nx)) for l in L}
    fd_h = {l: np.zeros((64, 64)) for l in L}
    sc_h = {l: np.zeros((64, 64)) for l in L}
    nz_h = {l: np.zeros((64, 64)) for l in L}
    hmax2 = 2.0 * float(np.abs(h64).max())
    u64 = 2.0 ** -53
    ab_h = {l: np.zeros((ny, nx)) for l in L}
    cn_h = {l: np.zeros((ny, nx)) for l in L}
    ab1_h = np.zeros((ny, nx))              # sum over rays of |dlight/dh| (weight 1)
    gs_gpu = {l: [] for l in L}
    fd_s = {l: [] for l in L}
    sc_s = {l: [] for l in L}
    nz_s = {l: [] for l in L}
    n_fd_rays = 0
    for ks, c in enumerate(diff_case["suns"]):
        om = c["omega"]
        ids = np.nonzero(om)[0]
        assert ids.size > 1000
        lt = c["lt"]
        gls = {"mse": np.where(om, 2.0 * (c["lo"] - lt) * wgt, 0.0),
               "lin": np.where(om, cw[ks] * wgt, 0.0)}
        sn = ss.Sun(c["e"], c["a"], alpha)
        res = ss.ss_shadow_forward(hf, mip, sn, lmax)
        am = res["argmin"].cpu().numpy().astype(np.int64)
        # a unique argmin with a gap of GAP must be found exactly
        assert np.array_equal(am[ids], c["ao"][ids])
        # A sun-angle step moves every sample's texel image by up to
        # t step / g texels; bilinear heights have kinks at cell edges, so the
        # angle differences take the rays of Omega whose argmin sample is at
        # least 4 t* A_STEP / g from every edge of its cell (both sides drop the
        # others from the angle check)
        suv = oracle.sample_uv(h, g, R, c["s"], np.where(om, c["ao"], -1))
        fr = suv - np.floor(suv)
        dist = np.minimum(fr, 1.0 - fr)                    # NaN for rays outside Omega
        edge = np.where(np.isnan(dist).all(axis=1), -1.0,
                        np.min(np.where(np.isnan(dist), np.inf, dist), axis=1))
        t_star = np.maximum(c["ao"], 1) * 0.5 * g
        om_s = om & (edge > 4.0 * t_star * A_STEP / g)
        assert om_s.sum() > 0.9 * om.sum()
        ids_s = np.nonzero(om_s)[0]
        for l in L:
            gh, gs = ss.ss_shadow_backward(hf, sn, lmax, res["argmin"],
                                           torch.from_numpy(gls[l].astype(np.float32)).cuda(),
                                           cost=res["cost"])
            gls_s = np.where(om_s, gls[l], 0.0).astype(np.float32)
            _, gs_s = ss.ss_shadow_backward(hf, sn, lmax, res["argmin"],
                                            torch.from_numpy(gls_s).cuda(), cost=res["cost"])
            torch.cuda.synchronize()
            gh_gpu[l] += gh.cpu().numpy()
            gs_gpu[l].append(gs_s.cpu().numpy()[:2])
            _, _, ah, ch = oracle.grad(h, g, R, c["e"], c["a"], alpha, c["ao"], gls[l],
                                       with_abs=True)
            ab_h[l] += ah
            cn_h[l] += ch
        _, _, a1, _ = oracle.grad(h, g, R, c["e"], c["a"], alpha, c["ao"], om.astype(np.float64),
                                  with_abs=True)
        ab1_h += a1

        # rays of Omega per window texel: the argmin sample's cell and the origin
        i0 = np.clip(np.floor(suv[ids, 0]).astype(np.int64), 0, nx - 2)
        j0 = np.clip(np.floor(suv[ids, 1]).astype(np.int64), 0, ny - 2)
        touch = {}
        for di in (0, 1):
            for dj in (0, 1):
                for r, x, y in zip(ids, i0 + di, j0 + dj):
                    touch.setdefault((y, x), set()).add(r)
        for r in ids:
            touch.setdefault((r // nx, r % nx), set()).add(r)

        def terms(rays, s=None):
            out = oracle.shadow_svec(h64, g, R, c["s"] if s is None else s, alpha, lmax,
                                     uv=grid_uv[rays])
            assert np.array_equal(out[1], c["ao"][rays])       # no argmin switch
            return out[0]

        ce = np.sqrt(np.maximum(0.0, 1.0 - c["sinp"] ** 2))
        dd_ = np.clip(c["co"] * ce / alpha, -1.0, 1.0)
        dldc = (2.0 / np.pi) * np.sqrt(1.0 - dd_ ** 2) * ce / alpha     # |dlight/dc| per ray
        tstar = np.maximum(c["ao"], 1) * 0.5 * g
        wl = {"mse": 2.0 * (c["lo"] - lt) * wgt, "lin": cw[ks] * wgt}  # dLoss/dlight per ray

        def noise(rays, length, step):
            return {l: 16.0 * dldc[rays] * u64 * length / (tstar[rays] * step) *
                    np.abs(wl[l][rays]) for l in L}

        def central(rays, perturb, step):
            dd = []
            for stp in (step, 0.5 * step):
                dd.append((perturb(+stp, rays) - perturb(-stp, rays)) / (2 * stp))
            dl = (4.0 * dd[1] - dd[0]) / 3.0                     # dlight, per ray
            return {l: wl[l][rays] * dl for l in L}

        for (y, x), rs in touch.items():
            if not (win[0].start <= y < win[0].stop and win[1].start <= x < win[1].stop):
                continue
            rays = np.array(sorted(rs))
            n_fd_rays += rays.size

            def at_height(d, rr, y=y, x=x):
                old = h64[y, x]
                h64[y, x] = old + d
                t = terms(rr)
                h64[y, x] = old
                return t
            per_ray = central(rays, at_height, H_STEP)
            is_origin = (rays // nx == y) & (rays % nx == x)
            nzr = noise(rays, np.where(is_origin, R, hmax2), H_STEP)
            for l in L:
                fd_h[l][y - c0[0], x - c0[1]] += per_ray[l].sum()
                sc_h[l][y - c0[0], x - c0[1]] += np.abs(per_ray[l]).sum()
                nz_h[l][y - c0[0], x - c0[1]] += nzr[l].sum()

        # sun angles of this sun: every ray of Omega
        for l in L:
            fd_s[l].append([0.0, 0.0])
            sc_s[l].append([0.0, 0.0])
            nz_s[l].append([0.0, 0.0])
        for kk in range(2):
            def at_angle(d, rr, kk=kk):
                e = c["e"] + (d if kk == 0 else 0.0)
                az = c["a"] + (d if kk == 1 else 0.0)
                return terms(rr, s=oracle.sun_vector(e, az))
            per_ray = central(ids_s, at_angle, A_STEP)
            nzr = noise(ids_s, R, A_STEP)
            for l in L:
                fd_s[l][-1][kk] = per_ray[l].sum()
                sc_s[l][-1][kk] = np.abs(per_ray[l]).sum()
                nz_s[l][-1][kk] = nzr[l].sum()

    stats = {}
    bars = {}
    for l in L:
        gw = gh_gpu[l][win]
        bar = 1e-4 * sc_h[l] + nz_h[l] + (cn_h[l][win] + 1.0) * F32_UNIT * ab_h[l][win]
        touched = cn_h[l][win] > 0
        err = np.abs(gw - fd_h[l])
        assert np.all(err[touched] <= bar[touched]), (l, err[touched].max())
        assert np.all(gw[~touched] == 0.0), l
        for k in range(n_sun):
            for i in range(2):
                assert abs(gs_gpu[l][k][i] - fd_s[l][k][i]) <= 1e-4 * sc_s[l][k][i] + nz_s[l][k][i], (
                    l, k, i, gs_gpu[l][k][i], fd_s[l][k][i], sc_s[l][k][i], nz_s[l][k][i])
        stats[l] = dict(window_texels=int(touched.sum()),
                        max_err_over_bar=float((err / np.maximum(bar, 1e-300))[touched].max()))
        bars[l] = (bar, touched)
    assert stats["lin"]["window_texels"] >= 100 and stats["mse"]["window_texels"] >= 10
    assert n_fd_rays > 100

    # loss (a) through the autograd Function with the GPU's own lights
    ht = torch.from_numpy(h).cuda().requires_grad_(True)
    tgt = torch.from_numpy(target).cuda()
    loss = 0.0
    for c in diff_case["suns"]:
        ang = torch.tensor([c["e"], c["a"]], dtype=torch.float64)
        light = ss.shadow(ht, ang, g, R, alpha, lmax)
        with torch.no_grad():
            lt_gpu = ss.shadow(tgt, ang, g, R, alpha, lmax)
        mask = torch.from_numpy(c["omega"]).cuda()
        loss = loss + (torch.where(mask, light - lt_gpu, torch.zeros_like(light)) ** 2).sum() * wgt
    (ga,) = torch.autograd.grad(loss, [ht])
    ga = ga.cpu().numpy().astype(np.float64)[win]
    bar, touched = bars["mse"]
    bar_e2e = bar + 4.0 * LIGHT_TOL * wgt * ab1_h[win]
    err = np.abs(ga - fd_h["mse"])
    assert np.all(err[touched] <= bar_e2e[touched]), (err[touched].max(),)
    assert np.all(ga[~touched] == 0.0)
    print("config-5 FD:", stats, "fd rays", n_fd_rays)
