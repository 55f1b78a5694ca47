"""Replica logic of bench.py under torch.distributed with gloo, two ranks on the CPU.

A single scene does not shard (one coupled Newton system), so N GPUs run N
independent replicas; the job throughput is the work of all ranks divided by
the slowest rank's time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    units = 3.0 + rank          # rank 0 did 3 solves, rank 1 did 4
    ms = 100.0 * (1 + rank)     # rank 1 is the slow one
    value, total_ms = bench.job_throughput(units, ms, world)
    out[rank] = (value, total_ms, bench.max_over_ranks(rank, world), bench.sum_over_ranks(1.0, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_throughput():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for rank in (0, 1):
        value, total_ms, mx, sm = out[rank]
        assert total_ms == 200.0
        assert abs(value - 7.0 / 0.2) < 1e-9
        assert mx == 1.0 and sm == 2.0


def test_single_rank_is_local():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    value, ms = bench.job_throughput(5.0, 250.0, 1)
    assert ms == 250.0 and abs(value - 20.0) < 1e-12
