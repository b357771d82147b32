"""The multi-process (replicas) aggregation of bench.py on CPU ranks (gloo).

Each rank solves its own copy of the workload; the job's value is the summed
work over the slowest rank's time.  Two ranks with different times and work
must agree on (max time, total work)."""
from __future__ import annotations

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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, work = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1))
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert dict(out) == {0: (11.0, 300.0), 1: (11.0, 300.0)}


def test_reduce_over_ranks_single_process():
    import bench

    assert bench.reduce_over_ranks(5.0, 7.0) == (5.0, 7.0)
