"""The multi-rank host logic of bench.py on CPU: two gloo ranks (replicas) reduce their timings to the
slowest rank's, the job throughput counts the units of every rank, and the reference arm runs on rank
0 only (the other ranks return without work)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 20.0][rank]
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        e2e = bench.max_over_ranks([0.3, 0.1][rank], world, "cpu")

        class A:
            steps, warmup = 5, 3

        ref = bench.run_reference(A(), rank, world) if rank != 0 else "skipped"
        dist.barrier()
        q.put((rank, ms, e2e, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, e2e, ref in got:
        assert ms == 20.0 and e2e == pytest.approx(0.3)
        assert ref == ("skipped" if rank == 0 else None)


def test_job_throughput_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(1000, 10, 2.0, 1) == 5000.0
    assert bench.job_throughput(1000, 10, 2.0, 4) == 20000.0
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
