"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path
collective) agree on the barrier, the max-over-ranks time and the whole-job
units; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    r, w = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(w)
    units, sec = bench.aggregate(100.0, 1.0 + rank, w)       # rank r took 1 + r seconds
    args = type("A", (), {"n": 1000, "steps": 1, "warmup": 0})()
    ref = bench.run_reference(args, r, w) if r != 0 else "skipped"
    out[rank] = (units, sec, ref is None)
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_and_barrier():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][:2] == (200.0, 2.0) and out[1][:2] == (200.0, 2.0)
    assert out[1][2]                      # the reference arm does no work on rank 1
