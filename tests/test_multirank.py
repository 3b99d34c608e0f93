"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas only, no data-path
collective).  The timed region is the slowest rank's, every rank receives it, and the
job throughput counts every replica's steps; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank  # rank 1 is the slow one
        worst = bench.max_over_ranks(mine, dist, "cpu")
        value = bench.job_throughput(world, 6, worst / 1e3)

        class Args:
            n, steps, warmup = 16, 1, 0
        ref_rc = bench.run_reference(Args, rank, world) if rank == 1 else 0
        q.put((rank, worst, value, ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    for rank, worst, value, ref_rc in out:
        assert worst == pytest.approx(15.0)            # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 6 / 0.015)   # both replicas' steps over that time
        assert ref_rc == 0                              # reference arm: rank 1 exits without work
