"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2):
per-rank workloads differ (seeds offset by rank), the job time is the
maximum over ranks, and the whole-job value counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, e2e = bench.max_over_ranks([10.0 + rank, 3.0 - rank], dist, "cpu")
        graphs = bench.workload(rank)
        out[rank] = (ms, e2e, graphs[0].num_edges, graphs[1].num_edges)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_by_maximum():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:2] == (11.0, 3.0) and res[1][:2] == (11.0, 3.0)
    assert res[0][2:] != res[1][2:]  # each rank solves its own graphs


def test_job_value_counts_every_rank():
    import bench
    assert bench.job_value(1e9, 5, 4, 1000.0) == pytest.approx(2e10)
    assert bench.max_over_ranks([1.0, 2.0], None, "cpu") == [1.0, 2.0]
