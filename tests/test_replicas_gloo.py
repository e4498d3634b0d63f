"""The N-GPU benchmark path (independent replicas) on two CPU ranks over gloo.

Replicas exchange nothing on the data path; the only collective is the
max-over-ranks of the timed region, which sets the whole-job rate.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        # per-rank timings of the mixed, FP64 and end-to-end legs; rank 1 is the slow one
        ms = bench.max_over_ranks([0.05 + 0.01 * r, 0.7 - 0.1 * r, 0.08], "cpu")
        dist.barrier()
        out[r] = (w, ms, bench.whole_job_rate(8192, w, ms[0]), bench.rank_seed(r))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_over_ranks_and_weak_scaling():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        w, ms, rate, seed = res[r]
        assert w == 2
        assert ms == pytest.approx([0.06, 0.7, 0.08])
        assert rate == pytest.approx(2 * 8192 / 0.06e-3)
    assert res[0][3] != res[1][3]  # each replica evaluates its own batch


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.whole_job_rate(100, 1, 2.0) == pytest.approx(5e4)
