"""The N-replica path of bench.py on CPU ranks (gloo, world size 2): the
whole-job rate is the units all ranks processed over the slowest rank's time,
every rank sees the same maximum, and the reference arm does its work on rank
0 only (the other ranks return at once, without touching the oracle)."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank  # rank 1 is the slower one
        rate, ms_max = bench.whole_job_rate(world, 1000, ms_local, device="cpu")

        class Args:
            n, psize, steps, warmup = 64, 16, 1, 1
        ref = bench.run_reference(Args(), world, rank) if rank != 0 else "skipped"
        q.put((rank, rate, ms_max, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_whole_job_rate_and_rank0_only_reference():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, ms_max, ref in out:
        assert ms_max == 15.0
        assert rate == pytest.approx(2 * 1000 / 0.015)
    assert out[1][3] is None  # rank 1: no reference work, no output
