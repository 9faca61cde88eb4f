"""Autotuner for the batched forward's launch shape.

Searches, by coordinate descent from the library defaults, over
  block_threads   threads per block
  rays_per_thread rays per warp = 32 x this (one queue chunk)
  ray_tile_w      chunk shape: 0 = runs of consecutive texels, w = w x (rays/w) rectangles
  refill_min      idle lanes that trigger a warp refill
  leaf_level      smallest bounded block = 2^(leaf_level+1) samples
  strip_len       0 = single rays with column seeds, S = seeded strips of S
                  rays, 1 = every ray walked from scratch
timing each candidate as CUDA-event-timed replays of a captured batch plan, and
keeps the best per (GPU name, tile-size class) in a JSON table.  Every candidate
gives the same outputs (the descent is exact); only the time changes.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from .shadow import Batch

SPACE = {
    "block_threads": (128, 256),
    "rays_per_thread": (8, 16, 32, 64, 128, 256),
    "ray_tile_w": (0, 16, 32, 64),
    "refill_min": (6, 10, 14, 18),
    "leaf_level": (1, 2, 3),
    "strip_len": (0, 1, 6, 10, 16),
}
# the starting point: 256 threads, 64 x 64 chunks (128 rays per lane), services at 14
# idle lanes, leaf blocks of 4 samples as warp tasks (64-instance batch on GB300:
# 332 ms against 350 ms for 32 x 64 chunks and 392 ms for the single-lane walk)
DEFAULT = {"block_threads": 256, "rays_per_thread": 128, "ray_tile_w": 64, "refill_min": 14,
           "leaf_level": 1, "strip_len": 0}


def default_table_path():
    return os.environ.get("SS_AUTOTUNE_TABLE") or os.path.join(
        os.path.expanduser("~"), ".cache", "softshadow_gb300", "autotune.json")


def size_class(nx, ny):
    """Power-of-two class of a tile's edge (geometric mean of nx, ny)."""
    return str(2 ** int(round(math.log2(max(1.0, math.sqrt(nx * ny))))))


def batch_class(hfs):
    """Size class of a batch: that of its median tile."""
    sizes = sorted(hf.shape[0] * hf.shape[1] for hf in hfs)
    m = sizes[len(sizes) // 2]
    return size_class(int(math.sqrt(m)), int(math.sqrt(m)))


def _valid(p):
    chunk = 32 * p["rays_per_thread"]
    return p["ray_tile_w"] == 0 or chunk % p["ray_tile_w"] == 0


def time_batch(hfs, suns, max_len_m, params, reps=3, step_texels=0.5):
    """Median ms of `reps` graph replays of the batch with these launch params."""
    b = Batch(hfs, suns, max_len_m, step_texels=step_texels, **params)
    try:
        b.launch()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            b.launch()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)
    finally:
        b.close()


def tune(hfs, suns, max_len_m, reps=3, rounds=2, step_texels=0.5, log=None):
    """Coordinate descent over SPACE; returns (best params, {key: ms})."""
    best = dict(DEFAULT)
    seen = {}

    def cost(p):
        key = json.dumps(p, sort_keys=True)
        if key not in seen:
            seen[key] = time_batch(hfs, suns, max_len_m, p, reps, step_texels)
            if log:
                log(f"autotune {key} {seen[key]:.3f} ms")
        return seen[key]

    best_ms = cost(best)
    for _ in range(rounds):
        improved = False
        for name, values in SPACE.items():
            for v in values:
                cand = dict(best, **{name: v})
                if cand == best or not _valid(cand):
                    continue
                ms = cost(cand)
                if ms < best_ms:
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    return best, seen


def load_table(path=None):
    path = path or default_table_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_table(table, path=None):
    path = path or default_table_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(hfs, table=None):
    """Tuned params for this batch's size class on this GPU, else the defaults."""
    table = load_table() if table is None else table
    key = f"{torch.cuda.get_device_name()}|{batch_class(hfs)}"
    return dict(table.get(key, {}).get("params", DEFAULT))


def tune_and_store(hfs, suns, max_len_m, path=None, **kw):
    best, seen = tune(hfs, suns, max_len_m, **kw)
    table = load_table(path)
    key = f"{torch.cuda.get_device_name()}|{batch_class(hfs)}"
    table[key] = {"params": best, "ms": min(seen.values()), "candidates": len(seen)}
    save_table(table, path)
    return best
