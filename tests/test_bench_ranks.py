"""The multi-replica path of bench.py on CPU: two gloo ranks (one process each, spawned), the
max-over-ranks time, the whole-job throughput, and the rank gating of the reference arm."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        t_max = bench.reduce_max_over_ranks(times[rank], world, torch.device("cpu"))
        dist.barrier()
        q.put((rank, t_max, bench.job_throughput(world, 1000, 10, 3, t_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [5.0, 7.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [7.5, 7.5]  # every rank sees the slowest time
    # weak scaling: 2 replicas x 1000 nodes x 30 stage updates in 7.5 ms
    assert out[0][2] == pytest.approx(2 * 1000 * 10 * 3 / 7.5e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks(3.25, 1, None) == 3.25
    assert bench.job_throughput(1, 4194304, 100, 3, 771.9) == pytest.approx(1.63e9, rel=1e-3)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under torchrun every rank but 0 leaves the reference arm at once, printing nothing."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(workload="advected_wave", c2p=None, steps=1, warmup=3)
    bench.reference_arm(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
