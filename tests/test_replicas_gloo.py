"""The multi-process ("replicas only") path of bench.py on CPU: two gloo ranks, each with its own
timings, agree on the slowest rank's times and report the whole-job rate from them.  The
library itself has no collective; this is the only cross-rank step."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r times (r + 1) ms for the step loop and (10 - r) ms end to end
        ms, e2e = bench.max_over_ranks([float(rank + 1), 10.0 - rank], world, torch.device("cpu"))
        q.put((rank, ms, e2e, bench.whole_job_rate(1024, 3, world, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, e2e, rate in got:
        assert ms == 2.0 and e2e == 10.0          # max over ranks, the same on every rank
        assert rate == pytest.approx(1024 * 3 * 2 / 0.002)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.whole_job_rate(1, 10, 1, 500.0) == pytest.approx(20.0)
