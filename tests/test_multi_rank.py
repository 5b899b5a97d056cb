"""The benchmark's multi-GPU path on CPU ranks (gloo, world size 2): each rank runs
an independent replica of the workload (no data-path collective), the job time is
the slowest rank's, and the whole-job rate counts every rank's solves."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    k, f, b = bench.make_workload("grf", 31, bench.rank_seed(4, rank))
    out[rank] = (ms, bench.whole_job_rate(world, 3, ms), float(f[0]), b)
    dist.destroy_process_group()


def test_two_ranks_replicas_and_max_time():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (ms0, rate0, f0, b0), (ms1, rate1, f1, b1) = res[0], res[1]
    assert ms0 == ms1 == 15.0                      # the slowest rank's time on every rank
    assert rate0 == rate1 == pytest.approx(2 * 3 * 1e3 / 15.0)
    assert f0 != f1 and b0 != b1                   # independent problems per rank


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(1, 1, 50.0) == pytest.approx(20.0)
    assert bench.rank_seed(4, 0) == 4 and bench.rank_seed(4, 1) == 1004
