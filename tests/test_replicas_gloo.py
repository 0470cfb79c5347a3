"""Multi-rank path of bench.py (replicas: one sort per rank, no collective on the data
path; the job's time is the slowest rank's and its rate sums all ranks' keys),
exercised on the CPU with two gloo ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # the ranks' own times
    dist.barrier()
    worst = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.job_rate(world, 1000 * (1 << 20), worst * 1e-3)
    out[rank] = (worst, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    worst, rate = res[0]
    assert worst == 15.0
    assert rate == pytest.approx(world * 1000 * (1 << 20) / 15e-3)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1, 100, 2.0) == 50.0
