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


def random_ids(n_total, n, seed):
    """n distinct seeded ray ids (independent of any GPU output)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, min(n, n_total), replace=False))


def deg(x):
    return math.radians(x)
