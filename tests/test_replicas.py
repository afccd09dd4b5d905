"""The multi-GPU path is replicas only: each rank runs an independent filter
(its own seed) and the job's time is the slowest rank's.  The host logic of that
path is tested here with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import synthetic as S
from oracle import bpf


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        timings = [1.0 + rank, 10.0 - rank, 3.0]           # per-rank step time, e2e time, resident time
        mx = bench.max_over_ranks(timings, world, "cpu")
        out[rank] = (mx, bench.replica_seed(3000, rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_seeds_with_two_gloo_ranks():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == [2.0, 10.0, 3.0]
    assert out[0][1] != out[1][1]


def test_one_rank_is_the_identity():
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]


def test_job_throughput_counts_every_rank():
    assert bench.job_throughput(4, 1 << 20, 100, 2.0) == 4 * (1 << 20) * 100 / 2.0


def test_replicas_are_independent_filters():
    """Different replica seeds give different particle systems on the same data."""
    model = S.lg_scalar()
    y = S.simulate(model, 3, seed=1)[1]
    a = bpf.run(model, 256, (16, 16), bench.replica_seed(7, 0), y)
    b = bpf.run(model, 256, (16, 16), bench.replica_seed(7, 1), y)
    assert not np.array_equal(a["state"].x, b["state"].x)
