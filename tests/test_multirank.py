"""The multi-rank host logic of bench.py on two gloo ranks (CPU): every rank
gets its own window (scene seed and Philox window id), times are combined as
the maximum over ranks, and the whole-job value counts the units of all
ranks over the slowest rank's time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = 1.0 + rank                      # rank 1 is the slowest
        m = bench.max_over_ranks(seconds, dist, "cpu")
        value = bench.whole_job_rate(world, 5e6, m)
        out[rank] = (m, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_on_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    m, value = res[0]
    assert m == 2.0
    assert value == pytest.approx(world * 5e6 / 2.0 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 2e6, 2.0) == 1.0


def test_ranks_get_distinct_windows():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    from paper_2104_06789_gb300 import synthetic
    # the replicas' scene seeds differ (rendered small to keep this quick)
    a = synthetic.driving(seed=3000, W=160, H=64, f=92.0, T=2)
    b = synthetic.driving(seed=3001, W=160, H=64, f=92.0, T=2)
    assert not np.array_equal(a.flows, b.flows)
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert "window_id=rank" in src and "seed=3000 + rank" in src
