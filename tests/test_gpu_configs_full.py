"""Full-size checks of the batched and differentiable workloads against the oracle.

* Batched: the 64 uneven instances ({512..4096}^2, a sun each over a lunar day,
  50 km rays) in one persistent launch with the autotuner's starting shape; on
  every instance a seeded sample of rays is compared with the FP64 oracle
  (light within 1e-5, argmin equal except at ties).
* Differentiable: 1024^2, 4 suns, loss = mean over rays and suns of
  (light(H) - light(H'))^2 with H' = H + 64 seeded Gaussian bumps.  The oracle
  computes both lights itself, hence dLoss/dlight; the GPU backward and the
  oracle's analytic gradient (itself pinned against central differences) are
  compared on every texel, on the 64 x 64 window at the tile centre, and on the
  sun angles.
  Rays whose GPU and oracle argmin differ (ties) get no weight on either side.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import batched_instances, bump_target, make_instance, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss
from paper_2005_06671_gb300 import autotune
from _parity import compare_to_oracle, random_ids

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M


def test_batched_config_full_size_sampled_vs_oracle():
    insts = batched_instances()
    assert len(insts) == 64
    dev = torch.device("cuda:0")
    hfs = [ss.Heightfield(torch.from_numpy(d["h"]).to(dev), d["g"], d["radius"]) for d in insts]
    suns = [ss.Sun(d["suns"][0][0], d["suns"][0][1], d["alpha"]) for d in insts]
    b = ss.Batch(hfs, suns, insts[0]["lmax"], want_cost=True, **autotune.DEFAULT)
    outs = b.submit()
    torch.cuda.synchronize()
    penumbra = 0
    for k, (d, o) in enumerate(zip(insts, outs)):
        h = d["h"]
        ids = random_ids(h.size, 120, seed=4000 + k)
        got = {key: o[key].cpu().numpy()[ids] for key in ("light", "argmin", "cost")}
        st = compare_to_oracle(h, d["g"], R, (d["suns"][0][0], d["suns"][0][1], d["alpha"]),
                               d["lmax"], 0.5, got["light"], got["argmin"], got["cost"],
                               ray_ids=ids)
        penumbra += st["penumbra"]
    b.close()
    assert penumbra > 50


def test_diff_config_full_size_gradient_on_centre_window():
    inst = make_instance("diff")
    h, g = inst["h"], inst["g"]
    ny, nx = h.shape
    target = bump_target(h, g, inst["seed"])
    alpha, lmax = inst["alpha"], inst["lmax"]
    n_sun = len(inst["suns"])
    hf = ss.Heightfield(torch.from_numpy(h).cuda(), g, R)
    mip = ss.ss_build_maxmip(hf)
    c0 = (ny - 64) // 2, (nx - 64) // 2
    win = (slice(c0[0], c0[0] + 64), slice(c0[1], c0[1] + 64))
    gh_gpu_tot = np.zeros((ny, nx))
    gh_o_tot = np.zeros((ny, nx))
    for k, (e, a) in enumerate(inst["suns"]):
        lo, ao, _ = oracle.shadow(h, g, R, e, a, alpha, lmax)
        lt, _, _ = oracle.shadow(target, g, R, e, a, alpha, lmax)
        gl = 2.0 * (lo - lt) / (h.size * n_sun)                 # dLoss/dlight, oracle side
        s = ss.Sun(e, a, alpha)
        res = ss.ss_shadow_forward(hf, mip, s, lmax)
        am = res["argmin"].cpu().numpy().astype(np.int64)
        assert np.abs(res["light"].cpu().numpy() - lo).max() <= 1e-5
        gl[am != ao] = 0.0                                       # ties: subgradients differ
        gh, gs = ss.ss_shadow_backward(hf, s, lmax, res["argmin"],
                                       torch.from_numpy(gl.astype(np.float32)).cuda(),
                                       cost=res["cost"])
        torch.cuda.synchronize()
        gh_o, gs_o = oracle.grad(h, g, R, e, a, alpha, ao, gl.astype(np.float32).astype(np.float64))
        gh_gpu_tot += gh.cpu().numpy()
        gh_o_tot += gh_o
        np.testing.assert_allclose(gs.cpu().numpy()[:2], gs_o[:2], rtol=1e-4,
                                   atol=1e-6 * np.abs(gs_o[:2]).max() + 1e-12)
    # every texel of the tile, and the 64 x 64 centre window on its own scale
    scale = np.abs(gh_o_tot).max()
    assert scale > 0 and np.count_nonzero(gh_o_tot) > 1000
    assert np.abs(gh_gpu_tot - gh_o_tot).max() <= 1e-4 * scale
    w_gpu, w_o = gh_gpu_tot[win], gh_o_tot[win]
    assert np.abs(w_gpu - w_o).max() <= 1e-4 * max(np.abs(w_o).max(), 1e-3 * scale)
