"""The multi-rank path of bench.py on the host: world_size 2 over gloo.

Each rank times its own instance; the job's time is the maximum over the ranks
and the whole-job throughput counts every rank's applies (weak scaling, no
data-path collective).  The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, ms, bench.job_value(world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_throughput():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 15.0                      # the slower rank sets the job's time
        assert abs(value - 2 * 1e3 / 15.0) < 1e-9


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert abs(bench.job_value(1, 12.5) - 80.0) < 1e-12
