"""Replicas on several ranks, the multi-GPU layout of this library: every rank solves its own
copy of the workload and only the timing is exchanged.  The job's time is the slowest rank's
and the units add up over ranks.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        out[rank] = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1), ws, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time_and_sum_the_units():
    ws = 2
    # every helper process is spawned, never forked from this multi-threaded process
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        for r in range(ws):
            assert out[r] == (11.0, 300.0)


def test_one_rank_keeps_its_own_numbers():
    assert bench.reduce_over_ranks(5.0, 7, 1, "cpu") == (5.0, 7.0)
