"""The multi-process path of bench.py on CPU ranks (gloo, world size 2): every rank
takes its own continuation point, the job's step time is the slowest rank's (the
only collective) and the job's value counts the units of all ranks."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2508_06302_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = I.workload_beam18()
    w = bench.rank_omega(wl, rank)
    ms_local = 10.0 + 5.0 * rank            # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, world, "cpu")
    val = bench.job_value(wl.N * wl.S1, world, ms)
    out[rank] = (w, ms, val)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_distinct_points_and_the_slowest_time():
    from paper_2508_06302_gb300 import inputs as I
    world, port = 2, 29731
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(100)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    wl = I.workload_beam18()
    (w0, ms0, v0), (w1, ms1, v1) = res[0], res[1]
    assert w0 == wl.omega1 and w1 == pytest.approx(1.01 * wl.omega1) and w0 != w1
    assert ms0 == ms1 == 15.0                 # max over ranks, seen by every rank
    assert v0 == v1 == pytest.approx(2 * wl.N * wl.S1 / 15e-3)
