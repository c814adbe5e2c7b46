"""Host-side logic of the N-rank benchmark path on CPU (gloo, world size 2).

The imaging units (channels of an integration) are independent, so ranks run
replicas with no data-path collective; only the timing is reduced (max over
ranks) and the job rate is every rank's units over the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_info()
        seconds = 2.0 + rank                      # rank 1 is the slowest
        tmax = bench.max_over_ranks(seconds, dist)
        out[rank] = (w, r, lr, tmax, bench.job_rate(1000, w, tmax))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, lr, tmax, rate = res[rank]
        assert (w, r, lr) == (world, rank, rank)
        assert tmax == 3.0                        # max over ranks, seen identically by all
        assert rate == pytest.approx(2000 / 3.0)  # all ranks' units / slowest time


def test_single_process_defaults():
    assert bench.rank_info() == (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                                 int(os.environ.get("LOCAL_RANK", "0")))
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
