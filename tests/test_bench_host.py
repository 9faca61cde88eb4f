"""Host-side logic of bench.py's multi-rank path, on CPU with world-size-2 gloo ranks:
max-over-ranks timing and whole-job (weak-scaling) throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.reduce_max(1.5 + rank, dist)      # rank 1 is the slower one
        r, lr, w = bench.rank_info()
        q.put((rank, t, r, w))
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [2.5, 2.5]
    assert [(g[2], g[3]) for g in got] == [(0, 2), (1, 2)]


def test_weak_scaling_value_and_single_rank_identity():
    assert bench.reduce_max(3.25, None) == 3.25
    # 2 ranks x 16.7M rays x 5 steps in 2.0 s (max over ranks)
    v = bench.weak_scaling_value(16_777_216, 2, 5, 2.0)
    assert v == pytest.approx(16_777_216 * 2 * 5 / 2.0)


def test_bench_cli_defaults():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
