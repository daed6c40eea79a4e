"""Host logic of bench.py's multi-rank (torchrun) path, on CPU with gloo.

Templates are independent, so N ranks filter N disjoint shards of the same
shape (weak scaling) and the job's time is the slowest rank's: each rank's
shard is drawn from its own seed, and the reported time is the max over
ranks.  Two gloo ranks on 127.0.0.1 check both.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bank = bench.shard_bank("plain", rank)
        ms = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
        out[rank] = (bank.n_templates, bank.n_filters, float(np.abs(bank.a).sum()), ms)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_templates_and_take_the_slowest():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(worker, args=(world, free_port(), out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    (t0, l0, s0, ms0), (t1, l1, s1, ms1) = res[0], res[1]
    assert t0 == t1 and l0 == l1            # same shard shape (weak scaling)
    assert s0 != s1                         # different templates on each rank
    assert ms0 == ms1 == 11.0               # every rank reports the slowest rank's time


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
