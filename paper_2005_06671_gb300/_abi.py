"""ctypes mirror of include/softshadow.h and loader of libsoftshadow.so.

Argument marshalling only: every step of the shadow path runs in the CUDA
library.  Loading fails loudly (RuntimeError) when the library cannot be found
or built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

c_i32, c_i64, c_u32, c_f64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p

SS_OK = 0
STATUS = {0: "SS_OK", 1: "SS_ERR_INVALID_ARG", 2: "SS_ERR_BAD_SIZE", 3: "SS_ERR_OUT_OF_MEMORY",
          4: "SS_ERR_CUDA", 5: "SS_ERR_TIMEOUT", 6: "SS_ERR_INTERNAL", 7: "SS_ERR_UNSUPPORTED"}
SS_PROJ_GNOMONIC, SS_PROJ_POLAR_STEREO = 0, 1
SS_RAYS_GRID, SS_RAYS_LIST = 0, 1
SS_FLAG_COUNT_SAMPLES = 0x1
SS_FLAG_NO_EARLY_EXIT = 0x2
SS_FLAG_LIGHT_ONLY = 0x4
SS_FLAG_DETERMINISTIC_BWD = 0x8
SS_FLAG_LANE_LEAVES = 0x10
SS_DEV_NONFINITE_HEIGHT = 0x1
SS_DEV_NONFINITE_RAY = 0x2
SS_DEV_NONFINITE_GRAD = 0x4


class SSHeightfield(ctypes.Structure):
    _fields_ = [("h", c_vp), ("nx", c_i32), ("ny", c_i32), ("pitch", c_i64),
                ("texel_m", c_f64), ("radius_m", c_f64), ("projection", c_i32)]


class SSSun(ctypes.Structure):
    _fields_ = [("elevation_rad", c_f64), ("azimuth_rad", c_f64), ("angular_radius_rad", c_f64)]


class SSParams(ctypes.Structure):
    _fields_ = [("max_len_m", c_f64), ("step_texels", c_f64), ("flags", c_u32),
                ("block_threads", c_i32), ("leaf_level", c_i32), ("rays_per_thread", c_i32),
                ("refill_min", c_i32), ("ray_tile_w", c_i32), ("strip_len", c_i32),
                ("seed_width", c_i32)]


class SSBatchItem(ctypes.Structure):
    pass


class SSRays(ctypes.Structure):
    _fields_ = [("mode", c_i32), ("n", c_i64), ("uv", c_vp), ("lift_m", c_vp)]


class SSOutputs(ctypes.Structure):
    _fields_ = [("light", c_vp), ("argmin", c_vp), ("cost", c_vp), ("counters", c_vp),
                ("status", c_vp)]


SSBatchItem._fields_ = [("hf", SSHeightfield), ("mip", c_vp), ("sun", SSSun), ("out", SSOutputs)]


class SSLight(ctypes.Structure):
    _fields_ = [("elevation_rad", ctypes.c_double), ("azimuth_rad", ctypes.c_double),
                ("intensity", ctypes.c_double), ("lit", c_vp)]


class SSCamera(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("forward", ctypes.c_double * 3),
                ("right", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("tan_half_x", ctypes.c_double), ("tan_half_y", ctypes.c_double),
                ("width", c_i32), ("height", c_i32)]


P = ctypes.POINTER
_SIGNATURES = {
    "ss_status_string": (ctypes.c_char_p, [c_i32]),
    "ss_last_error_string": (ctypes.c_char_p, []),
    "ss_version": (ctypes.c_char_p, []),
    "ss_maxmip_levels": (c_i32, [c_i32, c_i32]),
    "ss_maxmip_bytes": (ctypes.c_size_t, [c_i32, c_i32]),
    "ss_maxmip_level_info": (c_i32, [c_i32, c_i32, c_i32, P(c_i32), P(c_i32), P(c_i64), P(c_i64)]),
    "ss_build_maxmip": (c_i32, [P(SSHeightfield), c_vp, c_vp]),
    "ss_shadow_forward": (c_i32, [P(SSHeightfield), c_vp, P(SSRays), P(SSSun), P(SSParams),
                                  P(SSOutputs), c_vp]),
    "ss_shadow_uniform": (c_i32, [P(SSHeightfield), c_vp, P(SSRays), P(SSSun), P(SSParams),
                                  P(SSOutputs), c_vp]),
    "ss_shadow_backward": (c_i32, [P(SSHeightfield), P(SSRays), P(SSSun), P(SSParams), c_vp,
                                   c_vp, c_vp, c_vp, c_vp, c_vp]),
    "ss_backward_workspace_bytes": (ctypes.c_size_t, [c_i32, c_i32, c_u32]),
    "ss_shadow_backward_ws": (c_i32, [P(SSHeightfield), P(SSRays), P(SSSun), P(SSParams), c_vp,
                                      c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp,
                                      c_vp]),
    "ss_batch_workspace_bytes": (ctypes.c_size_t, [c_i32]),
    "ss_batch_submit": (c_i32, [c_vp, c_i32, P(SSParams), c_vp, ctypes.c_size_t, c_vp]),
    "ss_batch_plan_create": (c_i32, [c_vp, c_i32, P(SSParams), c_vp, ctypes.c_size_t,
                                     P(c_vp)]),
    "ss_batch_plan_launch": (c_i32, [c_vp, c_vp]),
    "ss_batch_plan_destroy": (c_i32, [c_vp]),
    "ss_shadow_greedy": (c_i32, [P(SSHeightfield), c_vp, P(SSRays), P(SSSun), c_vp, c_i32,
                                 c_vp, c_vp, c_vp, c_vp]),
    "ss_shadow_greedy_f32": (c_i32, [P(SSHeightfield), c_vp, P(SSRays), P(SSSun), c_vp, c_i32,
                                     c_vp, c_vp, c_vp, c_vp]),
    "ss_shade": (c_i32, [P(SSHeightfield), P(SSRays), c_vp, c_i32, c_vp, c_vp]),
    "ss_view_workspace_bytes": (ctypes.c_size_t, [c_i32, c_i32]),
    "ss_view_rays": (c_i32, [P(SSHeightfield), c_vp, P(SSCamera), ctypes.c_double,
                             ctypes.c_double, c_vp, c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
}

_lock = threading.Lock()
_lib = None


def header_symbols():
    """Function names declared in include/*.h (the public ABI)."""
    inc = os.path.join(_build.ROOT, "include")
    names = []
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(ss_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def lib():
    """Load (building first if needed) libsoftshadow.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libsoftshadow.so missing at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class SoftShadowError(RuntimeError):
    def __init__(self, status, where):
        msg = STATUS.get(status, str(status))
        if status == 4:
            detail = lib().ss_last_error_string()
            msg += f" ({detail.decode() if detail else ''})"
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status, where):
    if status != SS_OK:
        raise SoftShadowError(status, where)
