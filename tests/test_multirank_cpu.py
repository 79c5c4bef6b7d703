"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).  Every rank
renders its own sweep (weak scaling, no collective on the data path); the
only exchange is the max-over-ranks of the timings, and the whole-job rate is
the units all ranks processed over the slowest rank's time.  The reference
arm prints from rank 0 only."""
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
        q.put((rank, mx, bench.job_rate(300, world, mx)))
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
    for _, mx, rate in out:
        assert mx == 12.5  # the slower rank's time
        assert rate == pytest.approx(2 * 300 / 0.0125)


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
