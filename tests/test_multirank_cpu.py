"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).  The ranks
shard the views of one sweep (rank r renders views k = r mod N; weak scaling,
no collective on the data path); the only exchange is the max-over-ranks of
the timings, and the whole-job rate is the units all ranks processed over the
slowest rank's time.  The reference arm prints from rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [10.0, 12.5][rank]
        mx = bench.max_over_ranks(ms, world, torch.device("cpu"))
        mine = bench.shard_views(300, rank, world)
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        q.put((rank, mx, bench.job_rate(len(mine), world, mx), shards))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, mx, rate, shards in out:
        assert mx == 12.5  # the slower rank's time
        assert rate == pytest.approx(2 * 300 / 0.0125)
        # every view of the 600-view sweep is rendered by exactly one rank
        assert [len(s) for s in shards] == [300, 300]
        assert sorted(shards[0] + shards[1]) == list(range(600))


def test_sharded_sweep_views_are_distinct():
    import bench
    from paper_2412_20720_gb300 import synthetic as sy
    world = 4
    ts = set()
    for r in range(world):
        for k in bench.shard_views(5, r, world):
            v = sy.orbit_view(k, 5 * world, 64, 48)
            ts.add((float(v["t"]), tuple(float(x) for x in v["campos"])))
    assert len(ts) == 5 * world
    assert bench.shard_views(300, 0, 1) == list(range(300))  # N = 1: the plain sweep


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1, None) == 3.0
    assert bench.job_rate(300, 1, 150.0) == pytest.approx(2000.0)


def test_reference_arm_prints_from_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, n=1000)
    bench.run_reference(args, rank=1, world=2)  # other ranks exit without work
    assert capsys.readouterr().out == ""
