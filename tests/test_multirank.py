"""The replica path of bench.py on two CPU ranks (gloo, world size 2, no GPU): each rank solves its
own shard of the workload's problem stream, and the only cross-rank steps are the timing barrier
and the max over ranks of the timings; the whole-job rate counts every rank's problems over the
slowest rank's time."""
import os
import socket

import numpy as np
import pytest

import spectra

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, per_rank, results):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first = bench.shard_first(rank, per_rank)
        d = spectra.batch(2, per_rank, 64, 4, 2, first=first)
        timings = [10.0 + rank, 5.0 * (world - rank)]  # rank 1 is slower on the first, faster on the second
        dist.barrier()
        results[rank] = (first, d["y"].tolist(), bench.max_over_ranks(timings, world))
    finally:
        dist.destroy_process_group()


def test_two_ranks_solve_disjoint_shards_and_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    world, per_rank = 2, 3
    with mp.Manager() as manager:
        results = manager.dict()
        mp.start_processes(_rank, args=(world, _free_port(), per_rank, results), nprocs=world,
                           start_method="spawn", join=True)
        results = dict(results)
    whole = spectra.batch(2, world * per_rank, 64, 4, 2, first=0)["y"]
    for rank in range(world):
        first, y, maxima = results[rank]
        assert first == rank * per_rank
        # the rank's shard is exactly its slice of the single-process stream: disjoint, complete
        np.testing.assert_array_equal(np.asarray(y, dtype=whole.dtype), whole[first:first + per_rank])
        # every rank sees the element-wise max over ranks
        assert maxima == [11.0, 10.0]


def test_whole_job_rate_counts_every_rank_over_the_slowest_time():
    import bench
    assert bench.whole_job_rate(4096, 2, 5, 2.0) == 4096 * 2 * 5 / 2.0
    assert bench.max_over_ranks([3.0, 1.0], 1) == [3.0, 1.0]
