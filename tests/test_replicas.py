"""Replica host logic of the bench under torch.distributed (gloo, world size 2, CPU):
distinct per-rank walker seeds, max-over-ranks timing and whole-job aggregation."""
import os

import pytest


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    plan = bench.replica_plan(rank, world, walkers=64)
    t_local = 10.0 + rank  # ms
    t_max = bench.max_over_ranks(t_local, dist, device="cpu")
    value = bench.aggregate_rate(plan["walkers"], steps=5, world=world, t_max_ms=t_max)
    out.put((rank, plan["config_seed"], t_max, value))
    dist.destroy_process_group()


def test_two_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0), (r1, s1, t1, v1) = res
    assert s0 != s1                      # each replica draws its own walkers
    assert t0 == t1 == 11.0              # max over ranks
    assert v0 == v1 == pytest.approx(2 * 64 * 5 / 0.011)
