"""The N-replica host logic of the benchmark on CPU: two gloo ranks report
different step times and the whole-job rate uses the slowest (the solve
itself has no collective: independent problems run as replicas)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        ms = [1200.0, 1500.0][rank]
        value, max_ms = bench.whole_job_rate(ms, 3, dist, world, "cpu")
        if rank == 0:
            with open(out, "w") as f:
                f.write("%r %r" % (value, max_ms))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "rate.txt")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    value, max_ms = (float(x) for x in open(out).read().split())
    assert max_ms == 1500.0
    assert abs(value - 2 * 3 / 1.5) < 1e-12


def test_single_rank_rate():
    import bench
    value, ms = bench.whole_job_rate(2000.0, 4, None, 1)
    assert ms == 2000.0 and abs(value - 2.0) < 1e-12
