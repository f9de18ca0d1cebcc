"""The replicas-only multi-rank path of bench.py on CPU: two gloo ranks, each
with its own step time; the job time is the slowest rank's and the rate
counts every rank's elements (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank                     # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        out[rank] = (worst, bench.job_rate(world, 512, 5, worst / 1e3))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    world = 2
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for worst, rate in res.values():
        assert worst == 125.0
        assert rate == pytest.approx(2 * 512 * 5 / 0.125)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 8, 2, 0.5) == 32.0
