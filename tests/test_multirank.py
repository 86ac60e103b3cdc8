"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
every rank evaluates its own system, the job time is the slowest rank's and
the value counts all ranks' particles; ranks draw different systems."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [2.0, 3.0][rank]
    n_local = [1000, 3000][rank]
    val, ms_max, n_tot = bench.aggregate(ms_local, n_local, dist)
    out[rank] = (val, ms_max, n_tot)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        val, ms_max, n_tot = out[r]
        assert ms_max == 3.0 and n_tot == 4000.0
        assert abs(val - 4000.0 / 3e-3 / 1e6) < 1e-12


def test_single_rank_aggregate():
    val, ms, n = bench.aggregate(2.0, 1000)
    assert ms == 2.0 and n == 1000.0 and abs(val - 0.5) < 1e-12


def test_ranks_get_different_systems():
    a = bench.workload("rpm", seed_offset=0)
    b = bench.workload("rpm", seed_offset=1)
    assert a["pos"].shape == b["pos"].shape
    assert not np.allclose(a["pos"], b["pos"])
