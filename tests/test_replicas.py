"""Multi-GPU replicas, host side, on CPU: world_size-2 gloo ranks run the bench's reduction.

With one full problem per rank (no data-path collective), the job's step time is the slowest
rank's and its throughput counts the points of every rank; both reductions must give the same
answer on every rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms, bench.whole_job_value(ws, 1000, 2, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    ws, port = 2, _free_port()
    times = [12.5, 20.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, times, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 20.0
    assert value == pytest.approx(ws * 1000 * 2 / 0.020)


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.whole_job_value(1, 10, 1, 1000.0) == 10.0
