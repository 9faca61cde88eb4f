"""Non-finite inputs and the device status word (ss_outputs.status,
ss_shadow_backward_ws), and the deterministic backward.

* NaN heights: reported (SS_DEV_NONFINITE_HEIGHT, counted by the mipmap build);
  samples whose bilinear cell holds a NaN are skipped, as in the oracle's plain
  definition in IEEE arithmetic, so every ray still matches the oracle (light
  within 1e-5, argmin equal except at ties); maximum-mipmap levels ignore NaN.
* Infinite heights and NaN/infinite listed origins: reported, no fault, light
  in [0, 1]; a NaN origin has no usable sample.
* Non-finite dL/dlight: reported, the ray contributes nothing.
* Deterministic backward (SS_FLAG_DETERMINISTIC_BWD): the same bits over
  repeated runs and launch shapes, and the oracle's gradient within the
  per-texel bar.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import lunar_tile, make_instance, random_origins, MOON_RADIUS_M

import paper_2005_06671_gb300 as ss
from paper_2005_06671_gb300 import _abi
from _parity import compare_to_oracle, grad_weights_mask, assert_grad_close

pytestmark = pytest.mark.gpu
R = MOON_RADIUS_M
ALPHA = math.radians(0.2665)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _status():
    return torch.zeros(1, dtype=torch.int32, device="cuda")


def _tile_with(bad_value, n=128, count=40, seed=3):
    h = lunar_tile(n, 15.0, seed=seed, amplitude=500.0, n_craters=6)
    rng = np.random.default_rng(seed + 1)
    idx = rng.choice(h.size, count, replace=False)
    h.reshape(-1)[idx] = bad_value
    return h, idx


def test_clean_inputs_leave_the_status_word_zero():
    inst = make_instance("tiny", n=96)
    h = inst["h"]
    hf = ss.Heightfield(_dev(h), inst["g"], R)
    mip = ss.ss_build_maxmip(hf)
    st = _status()
    ss.ss_shadow_forward(hf, mip, ss.Sun(*inst["suns"][0], inst["alpha"]), inst["lmax"],
                         out=dict(status=st))
    ss.ss_shadow_uniform(hf, mip, ss.Sun(*inst["suns"][0], inst["alpha"]), inst["lmax"],
                         out=dict(status=st), light_only=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert ss.maxmip_nonfinite_count(mip, 96, 96) == 0


def test_nan_heights_reported_and_skipped_like_the_oracle():
    h, idx = _tile_with(np.nan, count=60)
    ny, nx = h.shape
    hf = ss.Heightfield(_dev(h), 15.0, R)
    mip = ss.ss_build_maxmip(hf)
    torch.cuda.synchronize()
    assert ss.maxmip_nonfinite_count(mip, nx, ny) == 60
    # levels ignore NaN texels: each is the fmax over its block of level 0
    lv = ss.maxmip_views(mip, nx, ny)
    for k, v in enumerate(lv, start=1):
        b = 2 ** k
        hp = np.full(((ny + b - 1) // b * b, (nx + b - 1) // b * b), np.nan, np.float32)
        hp[:ny, :nx] = h
        blocks = hp.reshape(hp.shape[0] // b, b, hp.shape[1] // b, b)
        with np.errstate(invalid="ignore"):
            want = np.fmax.reduce(np.fmax.reduce(blocks, axis=3), axis=1)
        got = v.cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(want)) and np.array_equal(
            got[~np.isnan(got)], want[~np.isnan(want)]), k
    nanm = np.isnan(h)
    cell = nanm[:-1, :-1] | nanm[1:, :-1] | nanm[:-1, 1:] | nanm[1:, 1:]   # cell of base (i, j)
    bi = np.minimum(np.arange(nx), nx - 2)
    bj = np.minimum(np.arange(ny), ny - 2)
    origin_cell_nan = cell[bj][:, bi].reshape(-1)
    assert origin_cell_nan.sum() < 0.05 * h.size
    for (e, a) in ((1.3, 40.0), (0.7, 200.0)):
        sun = (math.radians(e), math.radians(a), ALPHA)
        for method in ("dp", "uniform"):
            st = _status()
            fn = ss.ss_shadow_forward if method == "dp" else ss.ss_shadow_uniform
            res = fn(hf, mip, ss.Sun(*sun), 2500.0, out=dict(status=st))
            torch.cuda.synchronize()
            assert int(st.item()) & _abi.SS_DEV_NONFINITE_HEIGHT
            light = res["light"].cpu().numpy()
            assert np.all((light >= 0) & (light <= 1))
            # every ray except those whose origin cell holds a NaN: there the
            # oracle's weighted sum gives 0 * NaN = NaN for the origin height while
            # the GPU reads a grid ray's own texel (both are IEEE readings of an
            # interpolation at a texel centre; the header leaves it unspecified)
            ok = ~origin_cell_nan
            compare_to_oracle(h, 15.0, R, sun, 2500.0, 0.5, light[ok],
                              res["argmin"].cpu().numpy()[ok], res["cost"].cpu().numpy()[ok],
                              ray_ids=np.nonzero(ok)[0])
        # origins on a NaN texel have no usable sample
        res = ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), 2500.0)
        assert np.all(res["argmin"].cpu().numpy()[idx] == -1)
        assert np.all(res["light"].cpu().numpy()[idx] == 1.0)


@pytest.mark.parametrize("bad", [np.inf, -np.inf])
def test_infinite_heights_reported_without_fault(bad):
    h, _ = _tile_with(bad, count=25, seed=11)
    ny, nx = h.shape
    hf = ss.Heightfield(_dev(h), 15.0, R)
    mip = ss.ss_build_maxmip(hf)
    st = _status()
    sun = ss.Sun(math.radians(1.0), math.radians(75.0), ALPHA)
    res = ss.ss_shadow_forward(hf, mip, sun, 2500.0, out=dict(status=st))
    res2 = ss.ss_shadow_forward(hf, mip, sun, 2500.0, light_only=True)
    torch.cuda.synchronize()
    assert ss.maxmip_nonfinite_count(mip, nx, ny) == 25
    assert int(st.item()) & _abi.SS_DEV_NONFINITE_HEIGHT
    for r in (res, res2):
        light = r["light"].cpu().numpy()
        assert np.all((light >= 0) & (light <= 1))


def test_nonfinite_listed_origins_reported():
    inst = make_instance("tiny", n=128)
    h = inst["h"]
    hf = ss.Heightfield(_dev(h), inst["g"], R)
    mip = ss.ss_build_maxmip(hf)
    uv = random_origins(2000, 128, 128, seed=5)
    lift = np.zeros(2000, np.float32)
    uv[10] = (np.nan, 3.0)
    uv[20] = (7.0, np.nan)
    lift[30] = np.nan
    uv[40] = (np.inf, 5.0)
    lift[50] = np.inf
    sun = (inst["suns"][0][0], inst["suns"][0][1], inst["alpha"])
    for fn in (ss.ss_shadow_forward, ss.ss_shadow_uniform):
        st = _status()
        res = fn(hf, mip, ss.Sun(*sun), inst["lmax"], uv=_dev(uv), lift=_dev(lift),
                 out=dict(status=st))
        torch.cuda.synchronize()
        assert int(st.item()) == _abi.SS_DEV_NONFINITE_RAY
        light, arg = res["light"].cpu().numpy(), res["argmin"].cpu().numpy()
        assert np.all((light >= 0) & (light <= 1))
        for r in (10, 20, 30):                     # NaN origin or lift: no usable sample
            assert arg[r] == -1 and light[r] == 1.0
        ok = np.ones(2000, bool)
        ok[[10, 20, 30, 40, 50]] = False
        compare_to_oracle(h, inst["g"], R, sun, inst["lmax"], 0.5, light[ok], arg[ok],
                          res["cost"].cpu().numpy()[ok], uv=uv[ok], lift=lift[ok])


def test_batch_status_per_item():
    a = lunar_tile(96, 12.0, seed=31, amplitude=500.0, n_craters=4)
    b, _ = _tile_with(np.nan, n=80, count=10, seed=32)
    hfs = [ss.Heightfield(_dev(a), 12.0, R), ss.Heightfield(_dev(b), 12.0, R)]
    suns = [ss.Sun(math.radians(1.1), math.radians(30.0), ALPHA),
            ss.Sun(math.radians(0.9), math.radians(250.0), ALPHA)]
    bt = ss.Batch(hfs, suns, 2000.0)
    sts = [_status(), _status()]
    for i, s in enumerate(sts):
        bt.items[i].out.status = s.data_ptr()
    bt.submit()
    torch.cuda.synchronize()
    assert int(sts[0].item()) == 0
    assert int(sts[1].item()) == _abi.SS_DEV_NONFINITE_HEIGHT
    bt.close()


def _bwd_case():
    inst = make_instance("diff", n=160)
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][3]
    sun = (elev, az, math.radians(1.5))
    return h, g, sun, 3000.0


def test_nonfinite_grad_light_reported_and_skipped():
    h, g, sun, lmax = _bwd_case()
    hf = ss.Heightfield(_dev(h), g, R)
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    res = ss.ss_shadow_forward(hf, mip, s, lmax)
    light = res["light"].cpu().numpy()
    pen = np.nonzero((light > 0) & (light < 1))[0]
    assert pen.size > 50
    gl = np.random.default_rng(2).normal(size=h.size).astype(np.float32)
    bad = gl.copy()
    bad[pen[:5]] = np.nan
    bad[pen[5:8]] = np.inf
    ref = gl.copy()
    ref[pen[:8]] = 0.0
    for det in (False, True):
        st = _status()
        g1, s1 = ss.ss_shadow_backward(hf, s, lmax, res["argmin"], _dev(bad), cost=res["cost"],
                                       deterministic=det, status=st)
        g2, s2 = ss.ss_shadow_backward(hf, s, lmax, res["argmin"], _dev(ref), cost=res["cost"],
                                       deterministic=True)
        torch.cuda.synchronize()
        assert int(st.item()) == _abi.SS_DEV_NONFINITE_GRAD
        assert torch.isfinite(g1).all() and torch.isfinite(s1).all()
        if det:
            assert torch.equal(g1, g2) and torch.equal(s1, s2)
        else:
            assert torch.allclose(g1, g2, rtol=1e-5, atol=1e-6 * float(g2.abs().max()))


def test_deterministic_backward_repeatable_and_vs_oracle():
    h, g, sun, lmax = _bwd_case()
    hf = ss.Heightfield(_dev(h), g, R)
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    res = ss.ss_shadow_forward(hf, mip, s, lmax)
    am_gpu = res["argmin"].cpu().numpy().astype(np.int64)
    ol, oa, oc = oracle.shadow(h, g, R, sun[0], sun[1], sun[2], lmax)
    sinp = oracle.sin_elev(h, g, R, sun[0], sun[1])
    gl = np.random.default_rng(7).normal(size=h.size)
    gl[~grad_weights_mask(ol, oc, sinp, sun[2], am_gpu, oa)] = 0.0
    glt = _dev(gl.astype(np.float32))
    outs = []
    for block in (256, 256, 64, 160):
        outs.append(ss.ss_shadow_backward(hf, s, lmax, res["argmin"], glt, cost=res["cost"],
                                          deterministic=True, block_threads=block))
    torch.cuda.synchronize()
    for gh, gs in outs[1:]:
        assert torch.equal(gh.view(torch.int32), outs[0][0].view(torch.int32))
        assert torch.equal(gs.view(torch.int64), outs[0][1].view(torch.int64))
    gh_o, gs_o, ah, ch = oracle.grad(h, g, R, sun[0], sun[1], sun[2], oa,
                                     gl.astype(np.float32).astype(np.float64), with_abs=True)
    st = assert_grad_close(outs[0][0].cpu().numpy(), gh_o, ah, ch)
    assert st["texels"] > 50
    np.testing.assert_allclose(outs[0][1].cpu().numpy(), gs_o, rtol=1e-5,
                               atol=1e-6 * np.abs(gs_o).max())
    # accumulates into the given buffers, like the atomic path
    gh2 = outs[0][0].clone()
    gs2 = outs[0][1].clone()
    ss.ss_shadow_backward(hf, s, lmax, res["argmin"], glt, cost=res["cost"], deterministic=True,
                          grad_h=gh2, grad_sun=gs2)
    torch.cuda.synchronize()
    assert torch.allclose(gh2, 2 * outs[0][0], rtol=1e-6, atol=0)
    assert torch.allclose(gs2, 2 * outs[0][1], rtol=1e-12, atol=0)


def test_deterministic_backward_listed_rays_polar():
    n, g, lmax = 96, 400.0, 60e3
    h = lunar_tile(n, g, seed=5, amplitude=2000.0, n_craters=8)
    sun = (math.radians(1.1), math.radians(150.0), math.radians(1.5))
    hf = ss.Heightfield(_dev(h), g, R, projection="polar_stereo")
    mip = ss.ss_build_maxmip(hf)
    s = ss.Sun(*sun)
    uv = random_origins(4000, n, n, seed=9)
    lift = np.random.default_rng(10).uniform(0, 30, 4000).astype(np.float32)
    res = ss.ss_shadow_forward(hf, mip, s, lmax, uv=_dev(uv), lift=_dev(lift))
    am_gpu = res["argmin"].cpu().numpy().astype(np.int64)
    ol, oa, oc = oracle.shadow(h, g, R, sun[0], sun[1], sun[2], lmax, proj="polar_stereo", uv=uv,
                               lift=lift)
    sinp = oracle.sin_elev(h, g, R, sun[0], sun[1], proj="polar_stereo", uv=uv)
    gl = np.random.default_rng(11).normal(size=4000)
    gl[~grad_weights_mask(ol, oc, sinp, sun[2], am_gpu, oa)] = 0.0
    glt = _dev(gl.astype(np.float32))
    a = ss.ss_shadow_backward(hf, s, lmax, res["argmin"], glt, uv=_dev(uv), lift=_dev(lift),
                              deterministic=True)
    b = ss.ss_shadow_backward(hf, s, lmax, res["argmin"], glt, uv=_dev(uv), lift=_dev(lift),
                              deterministic=True, block_threads=96)
    torch.cuda.synchronize()
    assert torch.equal(a[0].view(torch.int32), b[0].view(torch.int32))
    assert torch.equal(a[1].view(torch.int64), b[1].view(torch.int64))
    gh_o, gs_o, ah, ch = oracle.grad(h, g, R, sun[0], sun[1], sun[2], oa,
                                     gl.astype(np.float32).astype(np.float64),
                                     proj="polar_stereo", uv=uv, lift=lift, with_abs=True)
    st = assert_grad_close(a[0].cpu().numpy(), gh_o, ah, ch)
    assert st["texels"] > 50
