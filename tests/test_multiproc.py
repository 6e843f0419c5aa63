"""Replica (multi-process) host logic of bench.py on CPU with gloo, world size 2.

The solve does not shard in this build; N processes each solve their own
copy and rank 0 reports max-over-ranks time.  These tests cover that host
logic: process-group setup from the torchrun environment, barrier, and
the max reduction, plus the reference arm's non-zero ranks exiting without
work."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    w, r, l = bench.dist_setup(world)
    assert (w, r, l) == (world, rank, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 + rank, w)
    # the reference arm: ranks other than 0 return immediately
    class A:
        workload = "c2"
        sample_iters = 1
        warmup = 0
        steps = 0
        gpus = world
    rc = bench.run_reference(A, w, r) if r != 0 else 0
    out[rank] = (m, rc)
    dist.destroy_process_group()


def test_replica_max_over_ranks_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == (11.0, 0) and out[1] == (11.0, 0)
