#!/usr/bin/env python3
"""Shadow rays/s of the exact max-mip descent on the 'mid' lunar workload.

Workload (one step): 4096 x 4096 float32 heightfield (10 m/texel, seeded fBm +
500 craters, +-1.5 km) on a sphere R = 1737.4 km, one shadow ray per texel
centre (16,777,216 rays), sun elevation 1.0 deg, azimuth 120 deg, angular
radius 0.2665 deg, max ray length 60 km (12,000 samples at 0.5 texel).
A step = maximum-mipmap build + exact descent forward (light + argmin per ray).
Inputs (64 MiB heights + 21 MiB pyramid) are smaller than L2, so L2 is flushed
(a 512 MiB write) before every timed step.

Printed JSON line: value = rays/s over all ranks (weak scaling: every rank runs
its own full tile).  Extra keys: the same-GPU uniform-stepping kernel (same
leaf values), forward+backward rays/s, the mipmap build alone, the roofline of
the descent kernel, the FP64 oracle timed on host cores, and clocks.

--impl reference times the FP64 CPU oracle (the reference arm of this
project: there is no runnable reference implementation) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shadow rays/s (DP+maxmip vs uniform stepping, same GB300, <=1e-5 err); fwd+bwd rays/s"
UNIT = "rays/s"
CONFIG = "mid"
# One launch of the descent kernel on the 4096x4096 workload, from one ncu capture
# (profiles/dp_task_grid4096.md; None until taken for the current kernel):
# dram__bytes_read.sum + dram__bytes_write.sum, and the issue counters
MID_DP_TRAFFIC_BYTES = 91520000 + 94630400
MID_DP_ISSUE = {"smsp__inst_executed.sum": 13104574673,
                "smsp__thread_inst_executed.sum": 312046763948,
                "sm__cycles_elapsed.avg": 29798239.3, "gpu__time_duration.sum_ns": 14402240}
SMS, SMSP_PER_SM = 152, 4
DESCENT_KERNEL = "dp_task_kernel"


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extras", action="store_true", help="skip uniform/backward/e2e/oracle legs")
    p.add_argument("--leaf-level", type=int, default=-1)
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-batched", action="store_true", help="skip the 64-instance batched leg")
    p.add_argument("--no-polar", action="store_true", help="skip the polar view leg")
    p.add_argument("--size", type=int, default=0,
                   help="profiling only: run the mid recipe at this tile size instead of 4096")
    p.add_argument("--polar-only", action="store_true",
                   help="profiling only: run the polar leg alone (at --size if given) and "
                        "print its numbers")
    return p.parse_args(argv)


# ----------------------------------------------------------------- ranks
def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def reduce_max(value, dist_mod, device=None):
    """Max of a float over all ranks (identity when not distributed)."""
    if dist_mod is None or not dist_mod.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(rays_per_rank, n_ranks, steps, seconds_max):
    """Whole-job throughput: every rank processes rays_per_rank per step."""
    return rays_per_rank * n_ranks * steps / seconds_max


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------- CPU oracle
def oracle_rate(inst, seconds, seed=2005):
    """The FP64 oracle as it stands, on a seeded sample of the workload's rays,
    sized to about `seconds` of work on all host cores.  Returns (rays/s, cores, sample)."""
    import numpy as np
    import oracle
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    ny, nx = h.shape
    rng = np.random.default_rng(seed)

    last = {}

    def run(n):
        ids = rng.choice(nx * ny, n, replace=False)
        uv = np.stack([ids % nx, ids // nx], 1).astype(np.float32)
        t0 = time.perf_counter()
        res = oracle.shadow(h, g, inst["radius"], elev, az, inst["alpha"], inst["lmax"], uv=uv)
        dt = time.perf_counter() - t0
        last.update(ids=ids, out=res)
        return dt

    # calibrate on growing samples until one takes >= 1/8 of the target
    n, t = 1024, run(1024)
    while t < seconds / 8 and n < 4_000_000:
        n = int(min(4_000_000, n * max(2.0, min(16.0, seconds / 8 / max(t, 1e-4)))))
        t = run(n)
    if t < 0.8 * seconds:
        n = int(min(4_000_000, n * seconds / t))
        t = run(n)
    cores = oracle.num_threads()
    sample = (f"{n} seeded random rays of the {nx}x{ny} tile (every one of the "
              f"{int(inst['lmax'] / (0.5 * g))} samples per ray evaluated in FP64)")
    return n / t, cores, sample, n, t, last


def parity_vs_oracle(inst, light, argmin, sampled, n_penumbra=500_000, seed=2006):
    """The timed step's outputs against the FP64 oracle: on the rays of the CPU
    baseline's last sample (seeded uniform) plus up to n_penumbra seeded rays
    among those whose GPU light is in (0, 1) (picked by reading only the GPU
    light).  Light within 1e-5; an argmin that differs from the oracle's counts
    as a tie when the oracle's costs at the two samples agree within 1e-6 rad."""
    import numpy as np
    import oracle
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    ny, nx = h.shape
    ids_u = sampled["ids"]
    lo_u, ao_u, _ = sampled["out"]
    pen = np.setdiff1d(np.nonzero((light > 0) & (light < 1))[0], ids_u)
    rng = np.random.default_rng(seed)
    ids_p = rng.choice(pen, min(n_penumbra, pen.size), replace=False) if pen.size else pen
    uv_p = np.stack([ids_p % nx, ids_p // nx], 1).astype(np.float32)
    lo_p, ao_p, _ = oracle.shadow(h, g, inst["radius"], elev, az, inst["alpha"], inst["lmax"],
                                  uv=uv_p)
    ids = np.concatenate([ids_u, ids_p])
    lo = np.concatenate([lo_u, lo_p])
    ao = np.concatenate([ao_u, ao_p])
    err = np.abs(light[ids].astype(np.float64) - lo)
    mism = np.nonzero(argmin[ids] != ao)[0]
    non_tie = 0
    for i in mism:
        r = ids[i]
        cs = oracle.ray_costs(h, g, inst["radius"], elev, az, inst["lmax"], r % nx, r // nx)
        jg, jo = int(argmin[r]), int(ao[i])
        if jg < 1 or jo < 1 or not abs(cs[jg - 1] - cs[jo - 1]) <= 1e-6:
            non_tie += 1
    return {"n": int(ids.size), "n_penumbra": int(((lo > 0) & (lo < 1)).sum()),
            "max_light_err": float(err.max()), "light_tol": 1e-5,
            "argmin_mismatch": int(mism.size), "argmin_mismatch_non_tie": non_tie,
            "outputs": "light and argmin of the last timed step",
            "rays": f"{ids_u.size} seeded uniform rays (the CPU baseline's sample) + "
                    f"{ids_p.size} seeded rays with GPU light in (0, 1)"}


# -------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import paper_2005_06671_gb300 as ss
    from workloads import make_instance

    rank, local_rank, world = rank_info()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

    inst = make_instance(CONFIG, n=args.size or None)
    h_np = inst["h"]
    ny, nx = h_np.shape
    n_rays = nx * ny
    elev, az = inst["suns"][0]
    lmax = inst["lmax"]
    hf = ss.Heightfield(torch.from_numpy(h_np).to(dev), inst["g"], inst["radius"])
    sun = ss.Sun(elev, az, inst["alpha"])
    mip = torch.empty(ss.maxmip_bytes(nx, ny) // 4, dtype=torch.float32, device=dev)
    light = torch.empty(n_rays, dtype=torch.float32, device=dev)
    argmin = torch.empty(n_rays, dtype=torch.int32, device=dev)
    bufs = dict(light=light, argmin=argmin)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    mip_launches = len(ss.maxmip_layout(nx, ny)) - 1
    mip_passes = math.ceil(mip_launches / 6)

    def step():
        ss.ss_build_maxmip(hf, mip)
        ss.ss_shadow_forward(hf, mip, sun, lmax, out=bufs, want_cost=False,
                             leaf_level=args.leaf_level, block_threads=args.block)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each, events on the launch stream
    sampler = ClockSampler(local_rank)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        ss.ss_build_maxmip(hf, mip)
        e1.record(stream)
        ss.ss_shadow_forward(hf, mip, sun, lmax, out=bufs, want_cost=False,
                             leaf_level=args.leaf_level, block_threads=args.block)
        e2.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    timed_light = light.cpu().numpy()          # the last timed step's outputs (parity)
    timed_argmin = argmin.cpu().numpy()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    mip_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    fwd_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    total_s = reduce_max(sum(step_ms) / 1e3, dist, dev)
    value = weak_scaling_value(n_rays, world, args.steps, total_s)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded fBm + crater lunar terrain)",
        "config": {"workload": f"mid: {nx}x{ny} f32 heightfield, 10 m/texel, one ray per texel "
                               f"({n_rays} rays), sun elev 1.0 deg az 120 deg, Lmax 60 km, "
                               f"0.5-texel samples; step = maxmip build + descent forward",
                   "rays_per_step": n_rays, "l2": "flushed before every timed step (512 MiB write)",
                   "parallelism": f"replicas x{world} (weak)"},
        "clocks": clocks,
        # per step: the mipmap passes, the descent and its FP64 refine pass
        "gpu_launches": (mip_passes + 2) * args.steps,
        "mip_build_ms": statistics.median(mip_ms),
        "forward_ms": statistics.median(fwd_ms),
    }
    if rank != 0 or args.no_extras:
        if rank == 0:
            print(json.dumps(out))
        if dist is not None:
            dist.destroy_process_group()
        return

    # events for the untimed extra legs (independent of --steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(3)]

    # ---- roofline of the descent kernel: gathered bytes from counted probes
    res = ss.ss_shadow_forward(hf, mip, sun, lmax, count_samples=True, want_cost=False,
                               leaf_level=args.leaf_level, block_threads=args.block)
    cnt = res["counters"].to(torch.int64).sum(0).cpu().numpy()
    bytes_fwd = 16.0 * (cnt[0] + cnt[1]) + 8.0 * n_rays
    fwd_s = statistics.mean(fwd_ms) / 1e3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_fwd / fwd_s / 1e9
    # DRAM bytes of one launch of this kernel, from an ncu capture of this exact
    # workload (profiles/dp_task_grid4096.md); reported only for the workload and
    # kernel settings it was taken on
    traffic = (MID_DP_TRAFFIC_BYTES if (nx, ny) == (4096, 4096) and args.leaf_level < 0
               and args.block == 0 else None)
    # the descent is bound by instruction issue: warp instructions over the issue
    # slots of its duration (one per SM sub-partition and cycle), from the same capture
    issue = None
    if traffic is not None and MID_DP_ISSUE is not None:
        wi = MID_DP_ISSUE["smsp__inst_executed.sum"]
        ti = MID_DP_ISSUE["smsp__thread_inst_executed.sum"]
        cyc = MID_DP_ISSUE["sm__cycles_elapsed.avg"]
        issue = {"warp_inst_per_ray": wi / n_rays, "thread_inst_per_ray": ti / n_rays,
                 "active_lanes_per_inst": ti / wi,
                 "issue_frac": wi / (SMS * SMSP_PER_SM * cyc),
                 "thread_inst_per_probe_or_leaf": ti / (float(cnt[0]) + float(cnt[1])),
                 "source": "ncu smsp__inst_executed.sum / (152 SMs x 4 sub-partitions x "
                           "sm__cycles_elapsed.avg), one launch (profiles/dp_task_grid4096.md)"}
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                       "frac": achieved / peak, "traffic": traffic, "issue": issue,
                       "kernel": DESCENT_KERNEL,
                       "algorithmic_bytes": bytes_fwd,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6800",
                       "mean_bound_probes_per_ray": float(cnt[0]) / n_rays,
                       "mean_leaf_samples_per_ray": float(cnt[1]) / n_rays}
    mip_bytes = 4.0 * n_rays + 4.0 * (ss.maxmip_bytes(nx, ny) / 4)
    out["mip_roofline"] = {"achieved": mip_bytes / (statistics.median(mip_ms) / 1e3) / 1e9,
                           "peak": peak, "unit": "GB/s"}

    # ---- same-GPU uniform stepping (same leaf values), timed the same way
    ures = ss.ss_shadow_uniform(hf, mip, sun, lmax, count_samples=True, want_cost=False)
    ucnt = ures["counters"].to(torch.int64).sum(0).cpu().numpy()
    u_ms = []
    for k in range(3):
        flush.zero_()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        ss.ss_build_maxmip(hf, mip)
        e1.record(stream)
        ss.ss_shadow_uniform(hf, mip, sun, lmax, out=bufs, want_cost=False)
        e2.record(stream)
        torch.cuda.synchronize()
        u_ms.append(e0.elapsed_time(e2))
    uni_value = n_rays / (statistics.mean(u_ms) / 1e3)
    out["uniform"] = {"value": uni_value, "unit": UNIT, "ms_per_step": statistics.mean(u_ms),
                      "mean_leaf_samples_per_ray": float(ucnt[1]) / n_rays,
                      "same_results_as_descent": bool(torch.equal(ures["argmin"], res["argmin"]))}
    out["speedup_vs_uniform"] = value / uni_value

    # ---- light-only mode (saturation cutoffs; exact light), both kernels
    lo = {}
    for name, fn in (("descent", ss.ss_shadow_forward), ("uniform", ss.ss_shadow_uniform)):
        ms_l = []
        for k in range(3):
            flush.zero_()
            e0, e1, e2 = ev[k]
            e0.record(stream)
            ss.ss_build_maxmip(hf, mip)
            e1.record(stream)
            fn(hf, mip, sun, lmax, out=bufs, want_cost=False, light_only=True)
            e2.record(stream)
            torch.cuda.synchronize()
            ms_l.append(e0.elapsed_time(e2))
        lo[name] = statistics.mean(ms_l)
    out["light_only"] = {"value": n_rays / (lo["descent"] / 1e3), "unit": UNIT,
                         "ms_per_step": lo["descent"],
                         "uniform_value": n_rays / (lo["uniform"] / 1e3),
                         "speedup_vs_uniform": lo["uniform"] / lo["descent"],
                         "note": "SS_FLAG_LIGHT_ONLY: same step, exact light; argmin exact "
                                 "in the penumbra only"}

    # ---- the paper's greedy descent (Algorithm 1, N' = {5,5,5}; an approximation):
    #      its speed here and its light error against the exact descent
    g_ms = []
    for k in range(3):
        flush.zero_()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        ss.ss_build_maxmip(hf, mip)
        e1.record(stream)
        gres = ss.ss_shadow_greedy(hf, mip, sun, levels=(5, 5, 5))
        e2.record(stream)
        torch.cuda.synchronize()
        g_ms.append(e0.elapsed_time(e2))
    gerr = (gres["light"] - res["light"]).abs()
    f_ms = []
    for k in range(3):
        flush.zero_()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        ss.ss_build_maxmip(hf, mip)
        e1.record(stream)
        fres = ss.ss_shadow_greedy(hf, mip, sun, levels=(5, 5, 5), fp32=True)
        e2.record(stream)
        torch.cuda.synchronize()
        f_ms.append(e0.elapsed_time(e2))
    ferr = (fres["light"] - res["light"]).abs()
    fdiff = (fres["light"] - gres["light"]).abs()
    out["greedy"] = {"value": n_rays / (statistics.mean(g_ms) / 1e3), "unit": UNIT,
                     "ms_per_step": statistics.mean(g_ms), "levels": [5, 5, 5],
                     "max_light_err_vs_exact": float(gerr.max()),
                     "mean_light_err_vs_exact": float(gerr.mean()),
                     "frac_rays_err_gt_1e-5": float((gerr > 1e-5).float().mean()),
                     "note": "the paper's Algorithm 1 with interval concatenation (FP64): "
                             "an approximation, not held to the 1e-5 bar",
                     "f32": {"value": n_rays / (statistics.mean(f_ms) / 1e3), "unit": UNIT,
                             "ms_per_step": statistics.mean(f_ms),
                             "max_light_err_vs_exact": float(ferr.max()),
                             "mean_light_err_vs_exact": float(ferr.mean()),
                             "frac_rays_err_gt_1e-5": float((ferr > 1e-5).float().mean()),
                             "frac_rays_differing_from_fp64_build_gt_1e-4":
                                 float((fdiff > 1e-4).float().mean()),
                             "note": "the same algorithm at the paper's float32 arithmetic "
                                     "(float-float for tips within the float32 margin of a "
                                     "texel edge, FP64 within 1e-6 texel)"}}

    # ---- shading epilogue: Sun and Earth lit fractions -> Lambertian irradiance
    from workloads import EARTH_LIGHT
    earth = ss.Sun(math.radians(EARTH_LIGHT["elevation_deg"]),
                   math.radians(EARTH_LIGHT["azimuth_deg"]),
                   math.radians(EARTH_LIGHT["angular_radius_deg"]))
    lit_s = torch.empty(n_rays, dtype=torch.float32, device=dev)
    lit_e = torch.empty(n_rays, dtype=torch.float32, device=dev)
    arg_e = torch.empty(n_rays, dtype=torch.int32, device=dev)
    irr = torch.empty(n_rays, dtype=torch.float32, device=dev)
    elev, az = inst["suns"][0]
    lights = [(elev, az, 1.0, lit_s),
              (earth.elevation, earth.azimuth, EARTH_LIGHT["intensity"], lit_e)]
    sh_ms, fr_ms = [], []
    for k in range(3):
        flush.zero_()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        ss.ss_build_maxmip(hf, mip)
        # the irradiance needs only the lit fractions: light-only descents (their
        # light is the exact descent's, bit for bit)
        ss.ss_shadow_forward(hf, mip, sun, lmax, out=dict(light=lit_s, argmin=argmin),
                             want_cost=False, light_only=True)
        ss.ss_shadow_forward(hf, mip, earth, lmax, out=dict(light=lit_e, argmin=arg_e),
                             want_cost=False, light_only=True)
        ss.ss_shade(hf, lights, out=irr)
        e2.record(stream)
        torch.cuda.synchronize()
        fr_ms.append(e0.elapsed_time(e2))
        flush.zero_()
        e0.record(stream)
        ss.ss_shade(hf, lights, out=irr)
        e1.record(stream)
        torch.cuda.synchronize()
        sh_ms.append(e0.elapsed_time(e1))
    shade_bytes = n_rays * (4.0 * len(lights) + 4.0 + 4.0)
    out["shade"] = {"value": n_rays / (statistics.mean(fr_ms) / 1e3), "unit": UNIT,
                    "ms_per_frame": statistics.mean(fr_ms),
                    "frame": "maxmip + light-only descents for the Sun and the Earth + shading",
                    "shade_kernel_ms": statistics.mean(sh_ms),
                    "shade_kernel_gbs": shade_bytes / (statistics.mean(sh_ms) / 1e3) / 1e9,
                    "shade_algorithmic_bytes": shade_bytes, "peak_gbs": peak}

    # ---- forward + backward (loss gradient of ones), rays/s
    gl = torch.ones(n_rays, dtype=torch.float32, device=dev)
    cost_buf = torch.empty(n_rays, dtype=torch.float32, device=dev)
    fb_bufs = dict(light=light, argmin=argmin, cost=cost_buf)
    gh = torch.zeros_like(hf.h)
    gs = torch.zeros(5, dtype=torch.float64, device=dev)
    fb_ms = []
    for k in range(3):
        flush.zero_()
        gh.zero_()
        gs.zero_()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        ss.ss_build_maxmip(hf, mip)
        ss.ss_shadow_forward(hf, mip, sun, lmax, out=fb_bufs)
        e1.record(stream)
        ss.ss_shadow_backward(hf, sun, lmax, argmin, gl, grad_h=gh, grad_sun=gs, cost=cost_buf)
        e2.record(stream)
        torch.cuda.synchronize()
        fb_ms.append(e0.elapsed_time(e2))
    out["fwd_bwd"] = {"value": n_rays / (statistics.mean(fb_ms) / 1e3), "unit": UNIT,
                      "ms_per_step": statistics.mean(fb_ms)}

    # ---- end to end through the public API with host buffers.  Every step copies
    # its heights in from pinned host memory and its light and argmin out.  Uploads
    # and downloads run on two streams of their own, so step k+1's upload and step
    # k-1's download overlap step k's kernels (two sets of device buffers; a set is
    # refilled once the step two back has finished reading it, and rewritten once
    # its results are out).  Timed from the first copy in to the last copy out.
    n_e2e = max(3, args.steps)
    h_host = torch.from_numpy(h_np).pin_memory()
    light_host = [torch.empty(n_rays, dtype=torch.float32).pin_memory() for _ in range(2)]
    arg_host = [torch.empty(n_rays, dtype=torch.int32).pin_memory() for _ in range(2)]
    sets = []
    for _ in range(2):
        hdev = torch.empty_like(hf.h)
        sets.append(dict(h=hdev, hf=ss.Heightfield(hdev, inst["g"], inst["radius"]),
                         mip=torch.empty_like(mip), light=torch.empty_like(light),
                         argmin=torch.empty_like(argmin)))
    h2d_stream = torch.cuda.Stream(device=dev)
    d2h_stream = torch.cuda.Stream(device=dev)

    def e2e_run():
        ev_in = [torch.cuda.Event() for _ in range(n_e2e)]
        ev_done = [torch.cuda.Event() for _ in range(n_e2e)]
        ev_out = [torch.cuda.Event() for _ in range(n_e2e)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        h2d_stream.wait_stream(stream)
        d2h_stream.wait_stream(stream)
        t0.record(h2d_stream)
        for k in range(n_e2e):
            b = sets[k % 2]
            with torch.cuda.stream(h2d_stream):
                if k >= 2:
                    h2d_stream.wait_event(ev_done[k - 2])   # set b's heights are read
                b["h"].copy_(h_host, non_blocking=True)
                ev_in[k].record(h2d_stream)
            stream.wait_event(ev_in[k])
            if k >= 2:
                stream.wait_event(ev_out[k - 2])            # set b's results are out
            ss.ss_build_maxmip(b["hf"], b["mip"], stream=stream)
            ss.ss_shadow_forward(b["hf"], b["mip"], sun, lmax,
                                 out=dict(light=b["light"], argmin=b["argmin"]),
                                 want_cost=False, stream=stream)
            ev_done[k].record(stream)
            with torch.cuda.stream(d2h_stream):
                d2h_stream.wait_event(ev_done[k])
                light_host[k % 2].copy_(b["light"], non_blocking=True)
                arg_host[k % 2].copy_(b["argmin"], non_blocking=True)
                ev_out[k].record(d2h_stream)
        t1.record(d2h_stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / n_e2e

    def e2e_serial():
        """The same steps one at a time on one stream (upload, kernels, download):
        what the copies cost when nothing overlaps them."""
        b = sets[0]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(n_e2e):
            b["h"].copy_(h_host, non_blocking=True)
            ss.ss_build_maxmip(b["hf"], b["mip"], stream=stream)
            ss.ss_shadow_forward(b["hf"], b["mip"], sun, lmax,
                                 out=dict(light=b["light"], argmin=b["argmin"]),
                                 want_cost=False, stream=stream)
            light_host[0].copy_(b["light"], non_blocking=True)
            arg_host[0].copy_(b["argmin"], non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / n_e2e

    e2e_run()                      # warm-up
    flush.zero_()
    torch.cuda.synchronize()
    e2e_ms = [e2e_run() for _ in range(2)]
    serial_ms = e2e_serial()
    ok = bool(torch.equal(torch.from_numpy(timed_light), light_host[(n_e2e - 1) % 2]))
    out["e2e"] = {"value": n_rays / (statistics.mean(e2e_ms) / 1e3), "unit": UNIT,
                  "h2d_bytes_per_step": int(h_host.numel() * 4),
                  "d2h_bytes_per_step": int(light_host[0].numel() * 4 + arg_host[0].numel() * 4),
                  "ms_per_step": statistics.mean(e2e_ms), "steps": n_e2e,
                  "pipelined": "uploads and downloads on their own streams overlap the "
                               "neighbouring steps' kernels; every step copies its own "
                               "inputs and results",
                  "same_light_as_timed_step": ok,
                  "serial": {"value": n_rays / (serial_ms / 1e3), "ms_per_step": serial_ms,
                             "note": "one step at a time: upload, kernels, download in order"}}

    # ---- batched: 64 uneven tiles in one persistent launch, CUDA-graph replay
    if not args.no_batched:
        out["batched"] = batched_leg(args, dev)

    # ---- polar scene: 16384^2 stereographic tile, rays from a 3840x2160 view
    if not args.no_polar:
        out["polar"] = polar_leg(args, dev, flush)

    # ---- CPU oracle on the machine's host cores (bounded sample)
    rate, cores, sample, n, t, last = oracle_rate(inst, args.cpu_seconds)
    out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": sample, "seconds": t}
    # ---- parity of the timed step's outputs with the oracle (>= 10^6 rays)
    out["parity"] = parity_vs_oracle(inst, timed_light, timed_argmin, last)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def batched_leg(args, dev):
    """The 'batched' workload: 64 tiles with sizes drawn from {512..4096}^2, a sun each
    (elevation 0.2-3 deg, azimuth 0-360 deg), 50 km rays, one launch; the launch shape
    is searched on every 8th instance, the search's pick and the default shape are
    timed on the whole batch, and the faster one is timed as graph replays (inputs
    and outputs, ~4 GB, exceed L2)."""
    import torch
    import paper_2005_06671_gb300 as ss
    from paper_2005_06671_gb300 import autotune
    from workloads import batched_instances
    t0 = time.perf_counter()
    insts = batched_instances()
    gen_s = time.perf_counter() - t0
    hfs = [ss.Heightfield(torch.from_numpy(d["h"]).to(dev), d["g"], d["radius"]) for d in insts]
    suns = [ss.Sun(d["suns"][0][0], d["suns"][0][1], d["alpha"]) for d in insts]
    lmax = insts[0]["lmax"]
    n_rays = sum(d["h"].size for d in insts)
    t0 = time.perf_counter()
    tuned = autotune.tune_and_store(hfs[::8], suns[::8], lmax, reps=2, rounds=1)
    # the search runs on every 8th instance; its pick and the default shape are
    # then timed on the whole batch, and the faster one is the leg's shape
    picks = {}
    for name, p in (("tuned", tuned), ("default", dict(autotune.DEFAULT))):
        bt = ss.Batch(hfs, suns, lmax, **p)
        bt.launch()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        bt.launch()
        e1.record()
        torch.cuda.synchronize()
        picks[name] = (e0.elapsed_time(e1), p)
        bt.close()
    choice = min(picks, key=lambda k: picks[k][0])
    params = picks[choice][1]
    tune_s = time.perf_counter() - t0
    b = ss.Batch(hfs, suns, lmax, **params)
    b.launch()
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.launch()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    b.close()
    sizes = sorted({d["h"].shape[0] for d in insts})
    return {"value": n_rays / (statistics.median(ms) / 1e3), "unit": UNIT,
            "ms_per_launch": statistics.median(ms), "instances": len(insts), "rays": n_rays,
            "tile_sizes": sizes, "params": params, "autotune_s": tune_s,
            "shape_choice": {k: {"ms": round(v[0], 2), "params": v[1]} for k, v in picks.items()},
            "generation_s": gen_s, "graph": True,
            "includes": "queue reset + 64 maxmip builds + one persistent descent launch"}


def polar_leg(args, dev, flush):
    """The 'polar' workload: a 16384x16384 polar stereographic tile (5 m, +-4 km,
    5000 craters), shadow rays from the terrain points a 3840x2160 oblique camera
    sees (ss_view_rays, timed separately), sun 0.5 deg, 100 km rays.  The descent
    over the whole ray list is timed like the headline step (L2 flushed; the
    1 GiB tile exceeds L2 anyway), next to uniform stepping on the same rays."""
    import torch
    import paper_2005_06671_gb300 as ss
    from workloads import make_instance, camera
    t0 = time.perf_counter()
    inst = make_instance("polar", n=(args.size or None) if args.polar_only else None)
    gen_s = time.perf_counter() - t0
    cam = camera()
    hf = ss.Heightfield(torch.from_numpy(inst["h"]).to(dev), inst["g"], inst["radius"],
                        projection=inst["proj"])
    mip = ss.ss_build_maxmip(hf)
    elev, az = inst["suns"][0]
    sun = ss.Sun(elev, az, inst["alpha"])
    lmax = inst["lmax"]
    ss.ss_view_rays(hf, mip, cam)               # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    view_ms = []
    for _ in range(2):
        e0.record()
        uv, pix = ss.ss_view_rays(hf, mip, cam)   # reads the hit count back (one sync)
        e1.record()
        torch.cuda.synchronize()
        view_ms.append(e0.elapsed_time(e1))
    n = uv.shape[0]
    light = torch.empty(n, dtype=torch.float32, device=dev)
    argmin = torch.empty(n, dtype=torch.int32, device=dev)
    bufs = dict(light=light, argmin=argmin)

    def timed(fn, reps):
        fn(hf, mip, sun, lmax, uv=uv, out=bufs, want_cost=False)
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0.record()
            fn(hf, mip, sun, lmax, uv=uv, out=bufs, want_cost=False)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    dp_ms = timed(ss.ss_shadow_forward, 3)
    uni_ms = timed(ss.ss_shadow_uniform, 2)
    lo_ms = timed(lambda *a, **k: ss.ss_shadow_forward(*a, light_only=True, **k), 3)
    shape = inst["h"].shape
    del hf, mip, uv, pix
    return {"value": n / (dp_ms / 1e3), "unit": UNIT, "ms_per_step": dp_ms, "rays": n,
            "pixels": cam["width"] * cam["height"], "view_ms": statistics.median(view_ms),
            "uniform_value": n / (uni_ms / 1e3), "speedup_vs_uniform": uni_ms / dp_ms,
            "light_only_value": n / (lo_ms / 1e3), "generation_s": gen_s,
            "workload": f"polar: {shape[1]}x{shape[0]} f32 polar "
                        "stereographic tile, 5 m/texel, rays "
                        "from a 3840x2160 view's visible terrain, sun elev 0.5 deg az 210 deg, "
                        "Lmax 100 km, 0.5-texel samples; list-mode rays"}


# ------------------------------------------------------- reference arm
def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return
    from workloads import make_instance
    import numpy as np
    import oracle
    inst = make_instance(CONFIG)
    ny, nx = inst["h"].shape
    # each step: a fixed seeded sample of the workload's rays, about 3 s of CPU work
    _, cores, _, n, t, _ = oracle_rate(inst, 3.0, seed=1)
    h, g = inst["h"], inst["g"]
    elev, az = inst["suns"][0]
    rng = np.random.default_rng(7)
    ids = rng.choice(nx * ny, n, replace=False)
    uv = np.stack([ids % nx, ids // nx], 1).astype(np.float32)

    def step():
        oracle.shadow(h, g, inst["radius"], elev, az, inst["alpha"], inst["lmax"], uv=uv)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = f"{n} seeded random rays of the {nx}x{ny} 'mid' tile per step (FP64, every sample)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded fBm + crater lunar terrain)",
        "config": {"workload": f"mid: {nx}x{ny} f32 heightfield, 10 m/texel, sun elev 1.0 deg "
                               f"az 120 deg, Lmax 60 km; bounded ray sample per step",
                   "rays_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main(argv=None):
    args = parse_args(argv)
    if args.polar_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"polar": polar_leg(args, dev, flush)}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
