"""View rays (ss_view_rays) against the FP64 view oracle, and the polar scene's
shadows on those rays against the shadow oracle.

The polar workload's shadow rays start at the terrain points an oblique camera
sees (3840 x 2160 pixels, camera 10 km up, 30 km from the pole, looking at it).
Bars: the same pixels hit; hit texel coordinates equal as float32 up to one
rounding step (both sides compute them in FP64 in a different order).  The
full-size polar scene (view rays and shadows over >= 10^6 sampled pixels) is
in test_gpu_coverage.py.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import camera, lunar_tile, make_instance, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss
from _parity import compare_to_oracle

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_view(h, g, proj, cam):
    hf = ss.Heightfield(_dev(h), g, R, projection=proj)
    mip = ss.ss_build_maxmip(hf)
    uv, pix = ss.ss_view_rays(hf, mip, cam)
    torch.cuda.synchronize()
    return hf, mip, uv, pix


def _check_hits(uv_gpu, pix_gpu, u_cpu, v_cpu, pixels):
    """GPU hit list (pixel order) vs CPU hits of `pixels`: same hit set, float32
    coordinates within one rounding step.  Returns (index into the GPU list,
    CPU float32 uv) of the common hits."""
    pix_gpu = np.asarray(pix_gpu)
    assert np.all(np.diff(pix_gpu) > 0), "GPU list not in pixel order"
    pos = np.searchsorted(pix_gpu, pixels)
    pos_c = np.minimum(pos, len(pix_gpu) - 1)
    gpu_hit = (pos < len(pix_gpu)) & (pix_gpu[pos_c] == pixels)
    cpu_hit = ~np.isnan(u_cpu)
    assert np.array_equal(gpu_hit, cpu_hit), (gpu_hit != cpu_hit).sum()
    idx = pos_c[cpu_hit]
    ref = np.stack([u_cpu[cpu_hit], v_cpu[cpu_hit]], 1).astype(np.float32)
    got = np.asarray(uv_gpu)[idx]
    ulp = np.spacing(np.abs(ref)).astype(np.float32)
    assert np.all(np.abs(got - ref) <= ulp), np.abs(got - ref).max()
    return idx, ref


@pytest.mark.parametrize("proj,n,g", [("polar_stereo", 2048, 5.0), ("polar_stereo", 1500, 40.0),
                                      ("gnomonic", 1200, 50.0)])
def test_view_rays_every_pixel_vs_oracle(proj, n, g):
    h = lunar_tile(n, g, seed=n + int(g), amplitude=2500.0, n_craters=30)
    cam = camera(192, 108)
    hf, mip, uv, pix = _gpu_view(h, g, proj, cam)
    px = np.arange(192 * 108)
    u, v = oracle.view_hits(h, g, R, cam, px, proj=proj)
    idx, ref = _check_hits(uv.cpu().numpy(), pix.cpu().numpy(), u, v, px)
    assert len(idx) > 2000


def test_view_rays_flat_terrain_hits_the_sphere():
    h = np.full((1024, 1024), 300.0, np.float32)
    cam = camera(64, 36)
    hf, mip, uv, pix = _gpu_view(h, 80.0, "polar_stereo", cam)
    u, v = oracle.view_hits(h, 80.0, R, cam, np.arange(64 * 36))
    _check_hits(uv.cpu().numpy(), pix.cpu().numpy(), u, v, np.arange(64 * 36))
