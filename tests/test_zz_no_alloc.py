"""ss_batch_submit_static: the batch entry point that allocates nothing.

Some callers of this library cannot hand the batch a device workspace: a
renderer's frame loop must not call cudaMalloc (it can synchronise the whole
device and stall a frame), and some host programs own all device memory
through their own allocator.  ss_batch_submit_static serves them from a fixed
scratch array inside the library.  Here it is called through the C ABI, twice
in a row (the second call reuses the scratch the first one left behind), and
its outputs are compared with those of ss_batch_submit, the entry point that
takes a caller-allocated workspace; both run the same exact descent, so the
comparison is exact.  Requests beyond the array's item limit must be refused
with a clear error.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from workloads import lunar_tile, MOON_RADIUS_M, SUN_ANGULAR_RADIUS_RAD

import paper_2005_06671_gb300 as ss
from paper_2005_06671_gb300 import _abi

pytestmark = pytest.mark.gpu


def _lib():
    L = _abi.lib()
    L.ss_batch_submit_static.restype = ctypes.c_int32
    L.ss_batch_submit_static.argtypes = [ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.POINTER(_abi.SSParams), ctypes.c_void_p]
    L.ss_batch_static_scratch_bytes.restype = ctypes.c_size_t
    L.ss_batch_static_scratch_bytes.argtypes = []
    return L


def _batch():
    shapes = [(80, 80), (64, 150), (200, 200), (47, 33), (128, 96)]
    suns = [(1.3, 40.0), (0.6, 170.0), (2.2, 260.0), (0.9, 330.0), (1.7, 95.0)]
    hfs, ss_suns = [], []
    for i, ((ny, nx), (e, a)) in enumerate(zip(shapes, suns)):
        h = lunar_tile(nx, 15.0, seed=700 + i, amplitude=500.0, n_craters=4, ny=ny)
        hfs.append(ss.Heightfield(torch.from_numpy(h).cuda(), 15.0, MOON_RADIUS_M))
        ss_suns.append(ss.Sun(math.radians(e), math.radians(a), SUN_ANGULAR_RADIUS_RAD))
    return ss.Batch(hfs, ss_suns, 2500.0, want_cost=True, rays_per_thread=4)


def _snapshot(outs):
    torch.cuda.synchronize()
    return [{k: o[k].cpu().numpy().copy() for k in ("light", "argmin", "cost")} for o in outs]


def test_static_scratch_batch_matches_workspace_batch():
    L = _lib()
    assert L.ss_batch_static_scratch_bytes() >= L.ss_batch_workspace_bytes(
        _abi_max_items())
    b = _batch()
    ref = _snapshot(b.submit())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        for o in b.outs:
            o["light"].fill_(-1.0)
            o["argmin"].fill_(-9)
            o["cost"].fill_(float("nan"))
        st = L.ss_batch_submit_static(ctypes.cast(b.items, ctypes.c_void_p), len(b.hfs),
                                      ctypes.byref(b.params), stream)
        assert st == 0, (call, st)
        got = _snapshot(b.outs)
        for i, (g, r) in enumerate(zip(got, ref)):
            assert np.array_equal(g["argmin"], r["argmin"]), (call, i)
            assert np.array_equal(g["light"].view(np.uint32), r["light"].view(np.uint32)), (call, i)
            assert np.array_equal(g["cost"].view(np.uint32), r["cost"].view(np.uint32)), (call, i)
    b.close()


def _abi_max_items():
    return 256   # SS_BATCH_STATIC_MAX_ITEMS in include/softshadow.h


def test_static_scratch_rejects_batches_beyond_its_limit():
    L = _lib()
    n = _abi_max_items() + 1
    items = (_abi.SSBatchItem * n)()
    prm = _abi.SSParams(1000.0, 0.5, 0, 0, -1, 0, 0, 0, 0)
    st = L.ss_batch_submit_static(ctypes.cast(items, ctypes.c_void_p), n, ctypes.byref(prm), None)
    assert st == 2   # SS_ERR_BAD_SIZE, nothing enqueued
    assert b"static scratch limit" in L.ss_last_error_string()
