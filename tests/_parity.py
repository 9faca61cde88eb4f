"""Shared helpers for parity tests: compare the CUDA path with the FP64 oracle.

Bars (from the method's contract): light fraction within LIGHT_TOL = 1e-5
absolute; argmin equal except at ties, where the oracle's own costs at the two
indices must agree within TIE_TOL = 1e-6 rad; mipmap levels bit-exact.
"""
import math

import numpy as np

import oracle

LIGHT_TOL = 1e-5
TIE_TOL = 1e-6
# float32 cost output: rays whose light saturates keep the float32 sample
# value (|error| ~ 1e-7 * |terms|); penumbra rays are re-evaluated in FP64.
COST_ABS_TOL = 2e-6
COST_REL_TOL = 1e-5


def compare_to_oracle(h, g, R, sun, lmax, step, light, argmin, cost, ray_ids=None, uv=None,
                      lift=None, proj="gnomonic"):
    """Oracle on the given rays (grid ray ids, or list-mode uv/lift) vs GPU outputs
    (numpy arrays indexed the same way).  Returns a dict of statistics; asserts."""
    elev, az, alpha = sun
    if uv is None:
        ny, nx = h.shape
        ids = np.asarray(ray_ids)
        ouv = np.stack([ids % nx, ids // nx], 1).astype(np.float32)
        olift = None
    else:
        ouv, olift = uv, lift
    ol, oa, oc = oracle.shadow(h, g, R, elev, az, alpha, lmax, step_texels=step, proj=proj,
                               uv=ouv, lift=olift)
    light = np.asarray(light, np.float64)
    argmin = np.asarray(argmin, np.int64)
    cost = np.asarray(cost, np.float64)
    err = np.abs(light - ol)
    mism = np.nonzero(argmin != oa)[0]
    ties = 0
    for r in mism:
        assert argmin[r] >= 1 and oa[r] >= 1, (r, argmin[r], oa[r])
        cs = oracle.ray_costs(h, g, R, elev, az, lmax, ouv[r, 0], ouv[r, 1],
                              0.0 if olift is None else float(olift[r]), step_texels=step,
                              proj=proj)
        gap = abs(cs[argmin[r] - 1] - cs[oa[r] - 1])
        assert gap <= TIE_TOL, (r, argmin[r], oa[r], gap)
        ties += 1
    fin = np.isfinite(oc)
    assert np.array_equal(fin, np.isfinite(cost)), "finite-cost pattern differs"
    cerr = np.abs(cost[fin] - oc[fin]) if fin.any() else np.zeros(1)
    cbar = COST_ABS_TOL + COST_REL_TOL * (np.abs(oc[fin]) if fin.any() else np.zeros(1))
    stats = dict(n=len(ol), max_light_err=float(err.max()) if err.size else 0.0,
                 argmin_mismatch=len(mism), ties=ties, max_cost_err=float(cerr.max()),
                 penumbra=int(np.sum((ol > 0) & (ol < 1))))
    assert stats["max_light_err"] <= LIGHT_TOL, stats
    assert np.all(cerr <= cbar), stats
    return stats


# Gradient bars.  The GPU backward evaluates each ray's contributions in FP64
# (the same formulas as the oracle's analytic gradient) and accumulates them
# into float32 texels with atomic adds: a texel receiving cnt terms whose
# absolute values sum to A is off by at most (cnt + 1) 2^-24 A (each term
# rounded to float32 once, each partial sum once).  On top of that: 1e-6 A
# for the FP64 differences between the two sides (the GPU works in a local
# frame, the oracle computes |q| - R plainly: ~1e-10 m over t >= 5 m of cost,
# amplified near |d| = 1 by F''(d)/F'(d)), and GRAD_REL_TOL |g| per texel.
GRAD_REL_TOL = 1e-4
F32_UNIT = 2.0 ** -24
SAT_MARGIN = 1e-6


def grad_weights_mask(light_o, cost_o, sinp_o, alpha, argmin_gpu, argmin_o):
    """Rays that keep their dL/dlight in gradient comparisons: the GPU and the
    oracle agree on the argmin (at ties the two subgradients differ), and the
    oracle's |d| is not within SAT_MARGIN of 1 (there the two sides may
    disagree on whether the light is saturated, with a contribution of order
    sqrt(1 - |d|) either way)."""
    d = np.asarray(cost_o) * np.sqrt(np.maximum(0.0, 1.0 - np.asarray(sinp_o) ** 2)) / alpha
    near_sat = np.abs(np.abs(d) - 1.0) < SAT_MARGIN
    return (np.asarray(argmin_gpu) == np.asarray(argmin_o)) & ~near_sat


def assert_grad_close(gpu, ref, ref_abs, ref_cnt, rel=GRAD_REL_TOL, what="grad_h"):
    """Texel by texel: |gpu - ref| <= rel |ref| + ((cnt + 1) 2^-24 + 1e-6) A,
    with A (ref_abs) and cnt (ref_cnt) the oracle's per-texel sum of
    |contribution| and number of contributions; texels no ray contributes to
    must be exactly zero.  Returns statistics."""
    gpu = np.asarray(gpu, np.float64)
    err = np.abs(gpu - ref)
    bar = rel * np.abs(ref) + ((ref_cnt + 1.0) * F32_UNIT + 1e-6) * ref_abs
    bad = np.argwhere(err > bar)
    if bad.size:
        y, x = bad[0]
        raise AssertionError(
            f"{what}: {len(bad)} texels beyond the per-texel bar; first ({y},{x}): gpu "
            f"{gpu[y, x]!r} oracle {ref[y, x]!r} |err| {err[y, x]:.3e} bar {bar[y, x]:.3e} "
            f"(cnt {ref_cnt[y, x]:.0f}, abs {ref_abs[y, x]:.3e})")
    nz = ref_cnt > 0
    return dict(texels=int(nz.sum()), max_rel_err=float((err[nz] / np.maximum(
        np.abs(ref[nz]), 1e-300)).max()) if nz.any() else 0.0,
        max_err_over_bar=float((err[nz] / bar[nz]).max()) if nz.any() else 0.0)


def stratified_ids(light_gpu, n_uniform, n_penumbra, seed):
    """Ray ids for full-size parity: n_uniform seeded uniform ids plus up to
    n_penumbra seeded ids among the rays whose GPU light is in (0, 1) (the
    penumbra is a few percent of the rays and is where light errors can
    show).  Only the GPU's light is read, to pick the sample; every value
    compared comes from the oracle.  Sorted, distinct."""
    light_gpu = np.asarray(light_gpu)
    rng = np.random.default_rng(seed)
    n = light_gpu.size
    a = rng.choice(n, min(n_uniform, n), replace=False)
    pen = np.nonzero((light_gpu > 0) & (light_gpu < 1))[0]
    b = rng.choice(pen, min(n_penumbra, pen.size), replace=False) if pen.size else pen
    return np.union1d(a, b)


def random_ids(n_total, n, seed):
    """n distinct seeded ray ids (independent of any GPU output)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, min(n, n_total), replace=False))


def deg(x):
    return math.radians(x)
