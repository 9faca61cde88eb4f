"""ctypes binding of the C oracle (``shadow_oracle.c``, ``view_oracle.c``,
``greedy_oracle.c``, ``shade_oracle.c``).
Test infrastructure only.

``build_oracle()`` compiles the C files with gcc (FP64, IEEE semantics: no
fast-math, no FMA contraction, so x86 and Arm hosts give the same bits).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("shadow_oracle.c", "view_oracle.c", "greedy_oracle.c",
                                          "shade_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PROJ = {"gnomonic": 0, "polar_stereo": 1}


def library_path():
    return _LIB


def build_oracle(force=False):
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB)
            d, i32, i64, p = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            lib.or_disc_light.restype = d
            lib.or_disc_light.argtypes = [d]
            lib.or_shadow.restype = None
            lib.or_shadow.argtypes = [p, i32, i32, i64, d, d, i32, d, d, d, d, d, i32, i64,
                                      p, p, p, p, p]
            lib.or_ray_costs.restype = i64
            lib.or_ray_costs.argtypes = [p, i32, i32, i64, d, d, i32, d, d, d, d, d, d, d,
                                         p, i64]
            lib.or_sin_elev.restype = None
            lib.or_sin_elev.argtypes = [p, i32, i32, i64, d, d, i32, d, d, i32, i64, p, p]
            lib.or_shadow_svec.restype = None
            lib.or_shadow_svec.argtypes = [p, i32, i32, i64, d, d, i32, p, d, d, d, i32, i64,
                                           p, p, p, p, p, p]
            lib.or_sample_uv.restype = None
            lib.or_sample_uv.argtypes = [p, i32, i32, i64, d, d, i32, p, d, i32, i64, p, p, p,
                                         p]
            lib.or_sun_vector.restype = None
            lib.or_sun_vector.argtypes = [d, d, p]
            lib.or_grad.restype = None
            lib.or_grad.argtypes = [p, i32, i32, i64, d, d, i32, d, d, d, d, i32, i64, p, p,
                                    p, p, p, p, p, p]
            lib.or_maxmip.restype = i32
            lib.or_maxmip.argtypes = [p, i32, i32, i64, p]
            lib.ov_view_hits.restype = None
            lib.ov_view_hits.argtypes = [p, i32, i32, i64, d, d, i32, p, p, p, p, d, d, i32,
                                         i32, d, d, i64, p, p, p]
            lib.og_greedy.restype = None
            lib.og_greedy.argtypes = [p, p, i32, i32, d, d, i32, d, d, d, p, i32, i32, i64, p,
                                      p, p, p, p]
            lib.os_shade.restype = None
            lib.os_shade.argtypes = [p, i32, i32, d, d, i32, i32, i64, p, i32, p, p, p, p, p]
            lib.or_num_threads.restype = i32
            lib.or_num_threads.argtypes = []
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _heights(h):
    h64 = np.ascontiguousarray(h, dtype=np.float64)
    assert h64.ndim == 2
    return h64


def _rays(uv, lift):
    if uv is None:
        return 0, 0, None, None
    uv = np.ascontiguousarray(uv, dtype=np.float32).reshape(-1, 2)
    lift = None if lift is None else np.ascontiguousarray(lift, dtype=np.float32).reshape(-1)
    return 1, uv.shape[0], uv, lift


def num_threads():
    return int(_load().or_num_threads())


def disc_light(d):
    return float(_load().or_disc_light(float(d)))


def shadow(h, g, radius, elev, az, alpha, lmax, step_texels=0.5, proj="gnomonic",
           uv=None, lift=None):
    """Brute-force forward.  ``uv=None``: one ray per texel centre (row-major);
    else ``uv`` [n, 2] float32 texel coordinates with optional ``lift`` [n].

    Returns (light float64 [n], argmin int64 [n] (1-based, -1 none), cost float64 [n]).
    """
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    mode, n, uv, lift = _rays(uv, lift)
    nr = nx * ny if mode == 0 else n
    light = np.empty(nr, np.float64)
    argmin = np.empty(nr, np.int64)
    cost = np.empty(nr, np.float64)
    lib.or_shadow(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj], float(elev),
                  float(az), float(alpha), float(lmax), float(step_texels), mode, n,
                  _ptr(uv), _ptr(lift), _ptr(light), _ptr(argmin), _ptr(cost))
    return light, argmin, cost


def sun_vector(elev, az):
    """Unit sun direction (cos e sin a, cos e cos a, sin e) in the tile frame."""
    out = np.empty(3, np.float64)
    _load().or_sun_vector(float(elev), float(az), _ptr(out))
    return out


def shadow_svec(h, g, radius, svec, alpha, lmax, step_texels=0.5, proj="gnomonic",
                uv=None, lift=None):
    """Brute-force forward with the light direction given as a 3-vector ``svec``
    (used as is, not normalised), plus the runner-up cost of each ray.

    Returns (light, argmin, cost, cost2): cost2 is the smallest cost over the
    usable samples other than the argmin (+inf with fewer than two samples).
    """
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    mode, n, uv, lift = _rays(uv, lift)
    nr = nx * ny if mode == 0 else n
    sv = np.ascontiguousarray(svec, dtype=np.float64).reshape(3)
    light = np.empty(nr, np.float64)
    argmin = np.empty(nr, np.int64)
    cost = np.empty(nr, np.float64)
    cost2 = np.empty(nr, np.float64)
    lib.or_shadow_svec(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj], _ptr(sv),
                       float(alpha), float(lmax), float(step_texels), mode, n, _ptr(uv),
                       _ptr(lift), _ptr(light), _ptr(argmin), _ptr(cost), _ptr(cost2))
    return light, argmin, cost, cost2


def sample_uv(h, g, radius, svec, j, step_texels=0.5, proj="gnomonic", uv=None, lift=None):
    """Texel coordinates [n, 2] of the image of sample j[r] of every ray (NaN
    where j[r] < 1); the light direction as a 3-vector as in ``shadow_svec``."""
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    mode, n, uv, lift = _rays(uv, lift)
    nr = nx * ny if mode == 0 else n
    jj = np.ascontiguousarray(j, dtype=np.int64).reshape(-1)
    assert jj.size == nr
    sv = np.ascontiguousarray(svec, dtype=np.float64).reshape(3)
    out = np.empty((nr, 2), np.float64)
    lib.or_sample_uv(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj], _ptr(sv),
                     float(step_texels), mode, n, _ptr(uv), _ptr(lift), _ptr(jj), _ptr(out))
    return out


def ray_costs(h, g, radius, elev, az, lmax, u, v, lift=0.0, step_texels=0.5,
              proj="gnomonic"):
    """Cost of every sample j = 1..J along one ray (NaN where outside the tile)."""
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    J = int(np.floor(lmax / (step_texels * g)))
    out = np.empty(max(J, 1), np.float64)
    lib.or_ray_costs(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj],
                     float(elev), float(az), float(lmax), float(step_texels), float(u),
                     float(v), float(lift), _ptr(out), out.size)
    return out[:J]


def sin_elev(h, g, radius, elev, az, proj="gnomonic", uv=None):
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    mode, n, uv, _ = _rays(uv, None)
    nr = nx * ny if mode == 0 else n
    out = np.empty(nr, np.float64)
    lib.or_sin_elev(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj], float(elev),
                    float(az), mode, n, _ptr(uv), _ptr(out))
    return out


def grad(h, g, radius, elev, az, alpha, argmin, gL, step_texels=0.5, proj="gnomonic",
         uv=None, lift=None, with_abs=False):
    """Analytic gradient of sum(gL * light) at the given argmin.

    Returns (grad_h float64 [ny, nx], grad_sun float64 [5] =
    (d/d elev, d/d az, d/ds_x, d/ds_y, d/ds_z)); with ``with_abs`` also
    (abs_h, cnt_h) [ny, nx]: per texel the sum of |contribution| over the
    non-zero per-ray contributions, and their number.
    """
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    mode, n, uv, lift = _rays(uv, lift)
    argmin = np.ascontiguousarray(argmin, dtype=np.int64)
    gL = np.ascontiguousarray(gL, dtype=np.float64)
    gh = np.zeros((ny, nx), np.float64)
    gs = np.zeros(5, np.float64)
    ah = np.zeros((ny, nx), np.float64) if with_abs else None
    ch = np.zeros((ny, nx), np.float64) if with_abs else None
    lib.or_grad(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj], float(elev),
                float(az), float(alpha), float(step_texels), mode, n, _ptr(uv), _ptr(lift),
                _ptr(argmin), _ptr(gL), _ptr(gh), _ptr(gs), _ptr(ah), _ptr(ch))
    if with_abs:
        return gh, gs, ah, ch
    return gh, gs


def maxmip(h):
    """Maximum mipmap: list of float32 levels [level0 (copy), level1, ...]."""
    lib = _load()
    h32 = np.ascontiguousarray(h, dtype=np.float32)
    ny, nx = h32.shape
    total, w, hh = 0, nx, ny
    shapes = []
    while w > 1 or hh > 1:
        w, hh = (w + 1) // 2, (hh + 1) // 2
        shapes.append((hh, w))
        total += w * hh
    out = np.empty(max(total, 1), np.float32)
    L = lib.or_maxmip(_ptr(h32), nx, ny, nx, _ptr(out))
    assert L == len(shapes) + 1
    levels = [h32.copy()]
    off = 0
    for (hh, w) in shapes:
        levels.append(out[off:off + w * hh].reshape(hh, w).copy())
        off += w * hh
    return levels


def view_hits(h, g, radius, cam, pixels, proj="polar_stereo"):
    """First terrain hit of the view rays of the given pixels (indices into the
    cam["width"] x cam["height"] frame, row-major): float64 arrays (u, v) of the
    hit's texel coordinates, NaN where the pixel's ray hits nothing in the tile.
    ``cam`` holds pos, forward, right, up, tan_x, tan_y, width, height, step_m,
    max_dist_m (see ``workloads.camera``)."""
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    px = np.ascontiguousarray(pixels, dtype=np.int64)
    u = np.empty(px.size, np.float64)
    v = np.empty(px.size, np.float64)
    vec = {k: np.ascontiguousarray(cam[k], dtype=np.float64) for k in
           ("pos", "forward", "right", "up")}
    lib.ov_view_hits(_ptr(h64), nx, ny, nx, float(g), float(radius), PROJ[proj],
                     _ptr(vec["pos"]), _ptr(vec["forward"]), _ptr(vec["right"]), _ptr(vec["up"]),
                     float(cam["tan_x"]), float(cam["tan_y"]), int(cam["width"]),
                     int(cam["height"]), float(cam["step_m"]), float(cam["max_dist_m"]),
                     px.size, _ptr(px), _ptr(u), _ptr(v))
    return u, v


def greedy(h, g, radius, elev, az, alpha, levels=(5, 5, 5), proj="gnomonic", uv=None,
           lift=None):
    """The paper's greedy descent (Algorithm 1 with interval concatenation), FP64:
    returns (light, cost J [rad, +inf if nothing sampled], t* [m, -1]) per ray;
    ``levels`` = N' of each run."""
    lib = _load()
    h32 = np.ascontiguousarray(h, dtype=np.float32)
    h64 = h32.astype(np.float64)
    ny, nx = h32.shape
    mode, n, uvp, liftp = _rays(uv, lift)
    nr = nx * ny if mode == 0 else n
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    light = np.empty(nr)
    cost = np.empty(nr)
    tstar = np.empty(nr)
    lib.og_greedy(_ptr(h32), _ptr(h64), nx, ny, float(g), float(radius), PROJ[proj],
                  float(elev), float(az), float(alpha), _ptr(lv), lv.size, mode, n, _ptr(uvp),
                  _ptr(liftp), _ptr(light), _ptr(cost), _ptr(tstar))
    return light, cost, tstar


def shade(h, g, radius, lights, proj="gnomonic", uv=None):
    """Lambertian irradiance sum_l I_l s_l max(0, N . L_l) per ray (FP64).
    ``lights``: list of (elevation, azimuth, intensity, lit fraction array [n])."""
    lib = _load()
    h64 = _heights(h)
    ny, nx = h64.shape
    mode, n, uvp, _ = _rays(uv, None)
    nr = nx * ny if mode == 0 else n
    el = np.array([float(x[0]) for x in lights])
    az = np.array([float(x[1]) for x in lights])
    it = np.array([float(x[2]) for x in lights])
    fr = [np.ascontiguousarray(x[3], dtype=np.float64).reshape(-1) for x in lights]
    for f in fr:
        assert f.size == nr
    ptrs = (ctypes.c_void_p * len(fr))(*[f.ctypes.data for f in fr])
    E = np.empty(nr)
    lib.os_shade(_ptr(h64), nx, ny, float(g), float(radius), PROJ[proj], mode, n, _ptr(uvp),
                 len(lights), _ptr(el), _ptr(az), _ptr(it), ctypes.cast(ptrs, ctypes.c_void_p),
                 _ptr(E))
    return E
