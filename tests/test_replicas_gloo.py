"""Multi-process (world size 2, gloo, CPU) check of the bench's replica
aggregation: the path shards by instance with no collective in the data path,
so the only cross-rank operation is the timing/work reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 3.0, dist, torch.device("cpu"))
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == (15.0, 6.0) and out[1] == (15.0, 6.0)


def test_aggregation_without_process_group_is_identity():
    import bench
    assert bench.aggregate_over_ranks(7.0, 2.5) == (7.0, 2.5)
