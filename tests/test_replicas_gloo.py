"""The multi-replica path of bench.py on CPU: two gloo ranks time different
step lengths, every rank ends with the maximum, and the job's throughput
counts both replicas' targets (world_size 2, no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [10.0 + 5.0 * rank, 3.0 - rank, 7.0]      # rank 1 is slower on the first value
        got = bench.max_over_ranks(ms, torch.device("cpu"))
        dist.barrier()
        out[rank] = got + [bench.job_throughput(world, 1000, got[0])]
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r][:3] == [15.0, 3.0, 7.0]
        assert res[r][3] == pytest.approx(2 * 1000 / 0.015)


def test_one_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks([1.5, 2], None) == [1.5, 2.0]
    assert bench.job_throughput(1, 1 << 20, 8.0) == pytest.approx((1 << 20) / 0.008)
