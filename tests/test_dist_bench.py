"""Two-rank (gloo, CPU) check of the whole-job reduction used by bench.py:
each rank searches an independent beam, the job time is the slowest rank's and
the job's units are the sum over ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        assert (ws, r, local) == (world, rank, rank)
        # rank r: (1 + r) seconds for (10 + r) * 1e6 units
        t, units = bench.job_totals(1.0 + rank, (10 + rank) * 1e6)
        results[rank] = (t, units)
    finally:
        dist.destroy_process_group()


def test_job_totals_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, units = results[r]
        assert t == 2.0                    # max over ranks
        assert units == 21e6               # sum over ranks
    # whole-job throughput: all ranks' units over the slowest rank's time
    assert results[0][1] / results[0][0] == pytest.approx(10.5e6)


def test_job_totals_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(3.0, 5.0) == (3.0, 5.0)
