"""The certified float32 usable-range search of stereographic rays against the
FP64 crossing search, on every ray (the first run of in-tile samples, reading
A14 of the paper's tile rule, Sec. 3.2/Appendix).

A check build of the library (SS_NVCC_FLAGS=-DSS_RANGE_CHECK, its own build
directory) runs both searches in every ray setup and prints each ray whose two
ranges differ (the first few).  This test builds it in a subprocess and runs
the polar test tiles through it: the reduced polar scene, wide tiles whose arcs
bend by several texels over a block, and listed origins inside and outside the
tile.  A printed difference fails the test.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import math, sys
    import numpy as np, torch
    sys.path.insert(0, {root!r})
    import paper_2005_06671_gb300 as ss
    from workloads import make_instance, lunar_tile, random_origins, MOON_RADIUS_M
    R = MOON_RADIUS_M
    def run(h, g, sun, lmax, uv=None, lift=None):
        hf = ss.Heightfield(torch.from_numpy(np.ascontiguousarray(h)).cuda(), g, R,
                            projection="polar_stereo")
        mip = ss.ss_build_maxmip(hf)
        kw = {{}}
        if uv is not None:
            kw = dict(uv=torch.from_numpy(uv).cuda(), lift=torch.from_numpy(lift).cuda())
        ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), lmax, **kw)
        ss.ss_shadow_forward(hf, mip, ss.Sun(*sun), lmax, light_only=True, **kw)
        torch.cuda.synchronize()
    inst = make_instance("polar", n=768)
    e, a = inst["suns"][0]
    run(inst["h"], inst["g"], (e, a, inst["alpha"]), inst["lmax"])
    for n, g, lmax, el, az in [(512, 300.0, 200e3, 1.0, 30.0), (384, 1000.0, 400e3, 2.5, 200.0),
                               (300, 600.0, 250e3, -0.3, 115.0)]:
        h = lunar_tile(n, g, seed=int(g) + n, amplitude=3000.0, n_craters=40)
        sun = (math.radians(el), math.radians(az), math.radians(0.2665))
        run(h, g, sun, lmax)
        rng = np.random.default_rng(n)
        uv = np.concatenate([random_origins(4000, n, n, seed=n + 1),
                             rng.uniform(-60, n + 60, (1000, 2))]).astype(np.float32)
        run(h, g, sun, lmax, uv, rng.uniform(0, 200, uv.shape[0]).astype(np.float32))
    print("range check ran with", ss._abi.lib()._name, flush=True)
""")


def test_float32_range_equals_fp64_range_on_every_ray(tmp_path):
    env = dict(os.environ)
    env["SS_NVCC_FLAGS"] = "-DSS_RANGE_CHECK"
    env["SS_BUILD_DIR"] = str(tmp_path / "build_rangecheck")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-3000:]
    assert "range check ran" in out, out[-3000:]
    # the check build itself was built and loaded (not the default library)
    lib = tmp_path / "build_rangecheck" / "libsoftshadow.so"
    assert lib.exists() and str(lib) in out, out[-3000:]
    assert "range mismatch" not in out, [l for l in out.splitlines() if "mismatch" in l][:8]
