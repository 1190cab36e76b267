"""CPU test of the multi-rank (replicas) path of bench.py with two gloo ranks:
every rank solves its own replica, the job time is the slowest rank's and the
work is the sum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 180.0][rank]
    evals = [60.0, 62.0][rank]
    out[rank] = bench.aggregate_ranks(ms, evals, "cpu")
    td.barrier()
    td.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        ms, ev = out[r]
        assert ms == 180.0 and ev == 122.0
