"""PyTorch-facing binding of libsoftshadow (device memory and streams only).

Each ``ss_*`` function marshals tensors into the C ABI of the same name
(include/softshadow.h) and enqueues the work on the current CUDA stream.
``ShadowFn`` wraps forward + backward as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _abi
from ._abi import (SSHeightfield, SSOutputs, SSParams, SSRays, SSSun, check,
                   SS_FLAG_COUNT_SAMPLES, SS_FLAG_NO_EARLY_EXIT, SS_FLAG_LIGHT_ONLY)

PROJ = {"gnomonic": _abi.SS_PROJ_GNOMONIC, "polar_stereo": _abi.SS_PROJ_POLAR_STEREO}


@dataclass
class Heightfield:
    """A float32 CUDA tensor [ny, nx] of heights (m) with its mapping to the sphere."""
    h: torch.Tensor
    texel_m: float
    radius_m: float
    projection: str = "gnomonic"

    def c(self):
        h = self.h
        if not (h.is_cuda and h.dtype == torch.float32 and h.dim() == 2 and h.stride(1) == 1):
            raise ValueError("heights must be a 2-D float32 CUDA tensor with unit column stride")
        return SSHeightfield(h.data_ptr(), h.shape[1], h.shape[0], h.stride(0),
                             float(self.texel_m), float(self.radius_m), PROJ[self.projection])

    @property
    def shape(self):
        return tuple(self.h.shape)


@dataclass
class Sun:
    elevation: float
    azimuth: float
    angular_radius: float = math.radians(0.2665)

    def c(self):
        return SSSun(float(self.elevation), float(self.azimuth), float(self.angular_radius))


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def version():
    return _abi.lib().ss_version().decode()


# ------------------------------------------------------------------ mipmap
def maxmip_bytes(nx, ny):
    return int(_abi.lib().ss_maxmip_bytes(nx, ny))


def maxmip_layout(nx, ny):
    """[(width, height, pitch, offset_elems)] for levels 1..L-1, then the stats block."""
    L = _abi.lib()
    n = int(L.ss_maxmip_levels(nx, ny))
    out = []
    for lvl in range(1, n + 1):
        w, h, p, o = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        check(L.ss_maxmip_level_info(nx, ny, lvl, ctypes.byref(w), ctypes.byref(h),
                                     ctypes.byref(p), ctypes.byref(o)), "ss_maxmip_level_info")
        out.append((w.value, h.value, p.value, o.value))
    return out


def maxmip_views(mip, nx, ny):
    """Views of levels 1..L-1 of a mip buffer as 2-D tensors (padding excluded)."""
    views = []
    lay = maxmip_layout(nx, ny)
    for (w, h, p, o) in lay[:-1]:
        views.append(mip[o:o + p * h].view(h, p)[:, :w])
    return views


def maxmip_stats(mip, nx, ny):
    """(global max, global min) tensor view stored after the levels."""
    w, h, p, o = maxmip_layout(nx, ny)[-1]
    return mip[o:o + 2]


def maxmip_nonfinite_count(mip, nx, ny):
    """Number of non-finite heights counted by the build (stats word 2), on the host."""
    w, h, p, o = maxmip_layout(nx, ny)[-1]
    return int(mip[o + 2:o + 3].view(torch.int32).item())


def ss_build_maxmip(hf: Heightfield, mip=None, stream=None):
    ny, nx = hf.shape
    if mip is None:
        mip = torch.empty(maxmip_bytes(nx, ny) // 4, dtype=torch.float32, device=hf.h.device)
    check(_abi.lib().ss_build_maxmip(ctypes.byref(hf.c()), _ptr(mip), _stream_ptr(stream)),
          "ss_build_maxmip")
    return mip


# ----------------------------------------------------------------- forward
def _params(max_len_m, step_texels, flags, block_threads, leaf_level, rays_per_thread=0,
            refill_min=0, ray_tile_w=0, strip_len=0, seed_width=0):
    return SSParams(float(max_len_m), float(step_texels), int(flags), int(block_threads),
                    int(leaf_level), int(rays_per_thread), int(refill_min), int(ray_tile_w),
                    int(strip_len), int(seed_width))


def _rays(hf, uv, lift):
    if uv is None:
        ny, nx = hf.shape
        return SSRays(_abi.SS_RAYS_GRID, 0, None, None), nx * ny
    if not (uv.is_cuda and uv.dtype == torch.float32 and uv.is_contiguous() and uv.shape[-1] == 2):
        raise ValueError("uv must be a contiguous float32 CUDA tensor [n, 2]")
    if lift is not None and not (lift.is_cuda and lift.dtype == torch.float32 and lift.is_contiguous()):
        raise ValueError("lift must be a contiguous float32 CUDA tensor [n]")
    n = uv.numel() // 2
    return SSRays(_abi.SS_RAYS_LIST, n, uv.data_ptr(), None if lift is None else lift.data_ptr()), n


def _outputs(n, device, want_cost, count, out):
    if out is None:
        out = {}
    light = out.get("light")
    if light is None:
        light = torch.empty(n, dtype=torch.float32, device=device)
    argmin = out.get("argmin")
    if argmin is None:
        argmin = torch.empty(n, dtype=torch.int32, device=device)
    cost = out.get("cost")
    if cost is None and want_cost:
        cost = torch.empty(n, dtype=torch.float32, device=device)
    counters = out.get("counters")
    if counters is None and count:
        counters = torch.empty((n, 2), dtype=torch.int32, device=device)
    status = out.get("status")   # optional device int32/uint32 word (SS_DEV_* bits)
    if status is not None and not (status.is_cuda and status.dtype == torch.int32 and
                                   status.numel() >= 1):
        raise ValueError("status must be an int32 CUDA tensor of at least one element")
    c = SSOutputs(light.data_ptr(), argmin.data_ptr(), None if cost is None else cost.data_ptr(),
                  None if counters is None else counters.data_ptr(),
                  None if status is None else status.data_ptr())
    return c, dict(light=light, argmin=argmin, cost=cost, counters=counters, status=status)


def _forward(fn_name, hf, mip, sun, max_len_m, step_texels, uv, lift, flags, block_threads,
             leaf_level, want_cost, out, stream, rays_per_thread=0, refill_min=0, ray_tile_w=0,
             strip_len=0, seed_width=0):
    rays, n = _rays(hf, uv, lift)
    count = bool(flags & SS_FLAG_COUNT_SAMPLES)
    oc, res = _outputs(n, hf.h.device, want_cost, count, out)
    prm = _params(max_len_m, step_texels, flags, block_threads, leaf_level, rays_per_thread,
                  refill_min, ray_tile_w, strip_len, seed_width)
    fn = getattr(_abi.lib(), fn_name)
    check(fn(ctypes.byref(hf.c()), _ptr(mip), ctypes.byref(rays), ctypes.byref(sun.c()),
             ctypes.byref(prm), ctypes.byref(oc), _stream_ptr(stream)), fn_name)
    return res


def ss_shadow_forward(hf: Heightfield, mip, sun: Sun, max_len_m, step_texels=0.5, uv=None,
                      lift=None, count_samples=False, block_threads=0, leaf_level=-1,
                      want_cost=True, out=None, stream=None, rays_per_thread=0, refill_min=0,
                      ray_tile_w=0, light_only=False, strip_len=0, seed_width=0,
                      lane_leaves=False):
    """Exact max-mip descent.  Returns dict(light, argmin, cost, counters).
    light_only: saturation cutoffs (exact light; argmin/cost exact in the penumbra).
    strip_len: rays per seeded strip (0 = default, 1 = no seeding).
    seed_width: half-width of a seed window (0 = default).
    lane_leaves: leaf samples evaluated by each walking lane instead of as
    warp-wide tasks (grid rays on gnomonic tiles; same results)."""
    flags = ((SS_FLAG_COUNT_SAMPLES if count_samples else 0) |
             (SS_FLAG_LIGHT_ONLY if light_only else 0) |
             (_abi.SS_FLAG_LANE_LEAVES if lane_leaves else 0))
    return _forward("ss_shadow_forward", hf, mip, sun, max_len_m, step_texels, uv, lift, flags,
                    block_threads, leaf_level, want_cost, out, stream, rays_per_thread,
                    refill_min, ray_tile_w, strip_len, seed_width)


def ss_shadow_uniform(hf: Heightfield, mip, sun: Sun, max_len_m, step_texels=0.5, uv=None,
                      lift=None, count_samples=False, early_exit=True, block_threads=0,
                      want_cost=True, out=None, stream=None, rays_per_thread=0, refill_min=0,
                      ray_tile_w=0, light_only=False):
    """Uniform stepping over every sample (exact early exit unless disabled)."""
    flags = ((SS_FLAG_COUNT_SAMPLES if count_samples else 0) |
             (0 if early_exit else SS_FLAG_NO_EARLY_EXIT) | (SS_FLAG_LIGHT_ONLY if light_only else 0))
    return _forward("ss_shadow_uniform", hf, mip, sun, max_len_m, step_texels, uv, lift, flags,
                    block_threads, -1, want_cost, out, stream, rays_per_thread, refill_min,
                    ray_tile_w)


# ---------------------------------------------------------------- backward
def ss_shadow_backward(hf: Heightfield, sun: Sun, max_len_m, argmin, grad_light, step_texels=0.5,
                       uv=None, lift=None, grad_h=None, grad_sun=None, block_threads=0,
                       stream=None, cost=None, deterministic=False, status=None, workspace=None):
    """Accumulates dL/dh into grad_h [ny, nx] (float32) and dL/d(elev, az, s_x, s_y, s_z)
    into grad_sun (float64 [5]); allocates zeroed ones when not given.  ``cost``
    (the forward's cost output) lets saturated rays be skipped early.
    ``deterministic``: the same bits on every run (ss_shadow_backward_ws with
    SS_FLAG_DETERMINISTIC_BWD; ``workspace`` is allocated when not given).
    ``status``: optional int32 CUDA word OR-ed with SS_DEV_NONFINITE_GRAD."""
    rays, n = _rays(hf, uv, lift)
    if grad_h is None:
        grad_h = torch.zeros_like(hf.h)
    if grad_h.stride() != hf.h.stride() or grad_h.shape != hf.h.shape:
        raise ValueError("grad_h must have the heights' shape and strides")
    if grad_sun is None:
        grad_sun = torch.zeros(5, dtype=torch.float64, device=hf.h.device)
    argmin = argmin.contiguous()
    grad_light = grad_light.to(torch.float32).contiguous()
    flags = _abi.SS_FLAG_DETERMINISTIC_BWD if deterministic else 0
    prm = _params(max_len_m, step_texels, flags, block_threads, -1)
    cost = None if cost is None else cost.contiguous()
    if not deterministic and status is None:
        check(_abi.lib().ss_shadow_backward(ctypes.byref(hf.c()), ctypes.byref(rays),
                                            ctypes.byref(sun.c()), ctypes.byref(prm),
                                            _ptr(argmin), _ptr(cost), _ptr(grad_light),
                                            _ptr(grad_h), _ptr(grad_sun), _stream_ptr(stream)),
              "ss_shadow_backward")
        return grad_h, grad_sun
    ny, nx = hf.shape
    nb = int(_abi.lib().ss_backward_workspace_bytes(nx, ny, flags))
    if workspace is None and nb > 0:
        workspace = torch.empty(nb, dtype=torch.uint8, device=hf.h.device)
    if status is not None and not (status.is_cuda and status.dtype == torch.int32):
        raise ValueError("status must be an int32 CUDA tensor")
    check(_abi.lib().ss_shadow_backward_ws(ctypes.byref(hf.c()), ctypes.byref(rays),
                                           ctypes.byref(sun.c()), ctypes.byref(prm),
                                           _ptr(argmin), _ptr(cost), _ptr(grad_light),
                                           _ptr(grad_h), _ptr(grad_sun), _ptr(workspace),
                                           0 if workspace is None else workspace.numel(),
                                           _ptr(status), _stream_ptr(stream)),
          "ss_shadow_backward_ws")
    return grad_h, grad_sun


# ---------------------------------------------------------------- autograd
class ShadowFn(torch.autograd.Function):
    """light = shadow(h, sun_angles) with a hand-written adjoint.

    Inputs: h [ny, nx] float32 CUDA, sun_angles float64 tensor [2] =
    (elevation, azimuth) in rad.  Non-tensor arguments: texel_m, radius_m,
    alpha, max_len_m, step_texels.  Output: light [ny*nx] (grid mode).
    The gradient is a subgradient of the per-ray minimum (taken at the argmin).
    """

    @staticmethod
    def forward(ctx, h, sun_angles, texel_m, radius_m, alpha, max_len_m, step_texels=0.5):
        e, a = (float(x) for x in sun_angles.detach().cpu().tolist())
        hf = Heightfield(h.detach().contiguous(), texel_m, radius_m)
        sun = Sun(e, a, alpha)
        mip = ss_build_maxmip(hf)
        res = ss_shadow_forward(hf, mip, sun, max_len_m, step_texels, want_cost=True)
        ctx.save_for_backward(hf.h, res["argmin"], res["cost"])
        ctx.geom = (texel_m, radius_m, alpha, max_len_m, step_texels, e, a)
        ctx.sun_dtype = sun_angles.dtype
        ctx.sun_device = sun_angles.device
        return res["light"]

    @staticmethod
    def backward(ctx, grad_light):
        h, argmin, cost = ctx.saved_tensors
        texel_m, radius_m, alpha, max_len_m, step_texels, e, a = ctx.geom
        hf = Heightfield(h, texel_m, radius_m)
        gh, gs = ss_shadow_backward(hf, Sun(e, a, alpha), max_len_m, argmin,
                                    grad_light.contiguous(), step_texels, cost=cost)
        g_sun = gs[:2].to(device=ctx.sun_device, dtype=ctx.sun_dtype)
        return gh, g_sun, None, None, None, None, None


def shadow(h, sun_angles, texel_m, radius_m, alpha, max_len_m, step_texels=0.5):
    return ShadowFn.apply(h, sun_angles, texel_m, radius_m, alpha, max_len_m, step_texels)


# ----------------------------------------------------------------- batched
class Batch:
    """Inputs and outputs of one batch: grid-mode rays on gnomonic tiles.

    ``hfs``: list of Heightfield; ``suns``: list of Sun (one per tile).  Allocates
    the mipmap buffers, per-ray outputs and the device workspace once; they are
    reused by every submit/plan launch of this batch.
    """

    def __init__(self, hfs, suns, max_len_m, step_texels=0.5, count_samples=False,
                 want_cost=False, block_threads=0, leaf_level=-1, rays_per_thread=0,
                 refill_min=0, ray_tile_w=0, light_only=False, strip_len=0, seed_width=0,
                 lane_leaves=False):
        if len(hfs) != len(suns) or not hfs:
            raise ValueError("need one sun per heightfield, at least one item")
        self.hfs, self.suns = list(hfs), list(suns)
        dev = hfs[0].h.device
        flags = ((SS_FLAG_COUNT_SAMPLES if count_samples else 0) |
                 (SS_FLAG_LIGHT_ONLY if light_only else 0) |
                 (_abi.SS_FLAG_LANE_LEAVES if lane_leaves else 0))
        self.params = SSParams(float(max_len_m), float(step_texels), int(flags), int(block_threads),
                               int(leaf_level), int(rays_per_thread), int(refill_min),
                               int(ray_tile_w), int(strip_len), int(seed_width))
        n = len(hfs)
        self.items = (_abi.SSBatchItem * n)()
        self.mips, self.outs = [], []
        for i, (hf, sun) in enumerate(zip(hfs, suns)):
            ny, nx = hf.shape
            mip = torch.empty(maxmip_bytes(nx, ny) // 4, dtype=torch.float32, device=dev)
            oc, res = _outputs(nx * ny, dev, want_cost, count_samples, None)
            self.items[i].hf = hf.c()
            self.items[i].mip = mip.data_ptr()
            self.items[i].sun = sun.c()
            self.items[i].out = oc
            self.mips.append(mip)
            self.outs.append(res)
        nb = int(_abi.lib().ss_batch_workspace_bytes(n))
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=dev)
        self._plan = None

    def submit(self, stream=None):
        check(_abi.lib().ss_batch_submit(ctypes.cast(self.items, ctypes.c_void_p), len(self.hfs),
                                         ctypes.byref(self.params), _ptr(self.workspace),
                                         self.workspace.numel(), _stream_ptr(stream)),
              "ss_batch_submit")
        return self.outs

    def plan(self):
        """Capture the batch into a CUDA graph (uploads descriptors synchronously)."""
        if self._plan is None:
            h = ctypes.c_void_p()
            check(_abi.lib().ss_batch_plan_create(ctypes.cast(self.items, ctypes.c_void_p),
                                                  len(self.hfs), ctypes.byref(self.params),
                                                  _ptr(self.workspace), self.workspace.numel(),
                                                  ctypes.byref(h)), "ss_batch_plan_create")
            self._plan = h
        return self

    def launch(self, stream=None):
        """Replay the captured graph."""
        self.plan()
        check(_abi.lib().ss_batch_plan_launch(self._plan, _stream_ptr(stream)),
              "ss_batch_plan_launch")
        return self.outs

    def close(self):
        if self._plan is not None:
            _abi.lib().ss_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ss_batch_submit(hfs, suns, max_len_m, **kw):
    """One-shot batch: returns the per-item output dicts (light, argmin, cost, counters)."""
    b = Batch(hfs, suns, max_len_m, **kw)
    outs = b.submit()
    b.close()
    return outs


# ------------------------------------------------------------------ view rays
def _camera(cam):
    c = _abi.SSCamera()
    for k in ("pos", "forward", "right", "up"):
        v = [float(x) for x in cam[k]]
        getattr(c, k)[:] = v
    c.tan_half_x = float(cam["tan_x"])
    c.tan_half_y = float(cam["tan_y"])
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def ss_view_rays(hf: Heightfield, mip, cam, step_m=None, max_dist_m=None, stream=None):
    """Terrain points seen by a camera (first hit of each pixel's view ray), in
    pixel order: returns (uv float32 [n, 2], pixel int32 [n]) CUDA tensors.
    ``cam``: dict with pos, forward, right, up (3-vectors), tan_x, tan_y, width,
    height and optionally step_m, max_dist_m (as made by ``workloads.camera``)."""
    L = _abi.lib()
    step = float(cam["step_m"] if step_m is None else step_m)
    dist = float(cam["max_dist_m"] if max_dist_m is None else max_dist_m)
    W, H = int(cam["width"]), int(cam["height"])
    dev = hf.h.device
    uv = torch.empty((W * H, 2), dtype=torch.float32, device=dev)
    pixel = torch.empty(W * H, dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    wsb = L.ss_view_workspace_bytes(W, H)
    if wsb == 0:
        raise ValueError("bad camera size")
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    c = _camera(cam)
    st = L.ss_view_rays(ctypes.byref(hf.c()), _ptr(mip), ctypes.byref(c), step, dist, _ptr(uv),
                        _ptr(pixel), _ptr(count), _ptr(ws), wsb, _stream_ptr(stream))
    _abi.check(st, "ss_view_rays")
    n = int(count.item())
    return uv[:n], pixel[:n]


# ------------------------------------------------------------ greedy descent
def ss_shadow_greedy(hf: Heightfield, mip, sun: Sun, levels=(5, 5, 5), uv=None, lift=None,
                     stream=None, fp32=False):
    """The paper's greedy descent (an approximation of ss_shadow_forward's exact
    minimum): dict(light, cost [rad], t_star [m]) per ray; ``levels`` = N' per run.
    ``fp32``: the float32 build (ss_shadow_greedy_f32, gnomonic tiles)."""
    L = _abi.lib()
    rays, n = _rays(hf, uv, lift)
    dev = hf.h.device
    light = torch.empty(n, dtype=torch.float32, device=dev)
    cost = torch.empty(n, dtype=torch.float32, device=dev)
    t_star = torch.empty(n, dtype=torch.float32, device=dev)
    lv = (ctypes.c_int32 * len(levels))(*[int(x) for x in levels])
    fn = L.ss_shadow_greedy_f32 if fp32 else L.ss_shadow_greedy
    st = fn(ctypes.byref(hf.c()), _ptr(mip), ctypes.byref(rays), ctypes.byref(sun.c()),
            ctypes.cast(lv, ctypes.c_void_p), len(levels), _ptr(light), _ptr(cost), _ptr(t_star),
            _stream_ptr(stream))
    _abi.check(st, "ss_shadow_greedy_f32" if fp32 else "ss_shadow_greedy")
    return {"light": light, "cost": cost, "t_star": t_star}


# ---------------------------------------------------------- shading epilogue
def ss_shade(hf: Heightfield, lights, uv=None, out=None, stream=None):
    """Lambertian irradiance sum_l I_l s_l max(0, N . L_l) per ray.
    ``lights``: sequence of (elevation_rad, azimuth_rad, intensity, lit) with
    ``lit`` the float32 CUDA lit fractions of that light (ss_shadow_forward's light)."""
    L = _abi.lib()
    rays, n = _rays(hf, uv, None)
    arr = (_abi.SSLight * len(lights))()
    keep = []
    for k, (e, a, inten, lit) in enumerate(lights):
        if not (lit.is_cuda and lit.dtype == torch.float32 and lit.is_contiguous()
                and lit.numel() == n):
            raise ValueError("lit fractions must be contiguous float32 CUDA tensors [n rays]")
        keep.append(lit)
        arr[k] = _abi.SSLight(float(e), float(a), float(inten), lit.data_ptr())
    E = out if out is not None else torch.empty(n, dtype=torch.float32, device=hf.h.device)
    st = L.ss_shade(ctypes.byref(hf.c()), ctypes.byref(rays), ctypes.cast(arr, ctypes.c_void_p),
                    len(lights), _ptr(E), _stream_ptr(stream))
    _abi.check(st, "ss_shade")
    return E
