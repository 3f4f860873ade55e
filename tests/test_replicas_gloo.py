"""The multi-GPU form is replicas only (every rank solves its own scene; no
data-path collective).  The host logic that turns per-rank times into the
whole-job rate (slowest rank's time, all ranks' iterations) runs here on two
CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 * (rank + 1)           # rank 1 is the slowest
        iters = 100 + 50 * rank
        out[rank] = bench.reduce_over_ranks(ms, iters, world, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_whole_job_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, value = res[rank]
        assert ms_max == 20.0
        assert value == pytest.approx((100 + 150) / 0.020)


def test_single_rank_is_its_own_rate():
    import bench
    ms, value = bench.reduce_over_ranks(40.0, 80, 1, "cpu")
    assert ms == 40.0 and value == pytest.approx(2000.0)
