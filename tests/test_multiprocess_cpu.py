"""The multi-GPU form of the benchmark is replicas only: each rank solves its
own lattice and the ranks only agree on the elapsed time, the maximum over
ranks.  This checks that reduction with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v = bench.max_over_ranks(10.0 * (rank + 1), torch.device("cpu"))
    out.put((rank, v))
    dist.barrier()
    dist.destroy_process_group()


def test_elapsed_time_is_the_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 20.0, 1: 20.0}


def test_max_over_ranks_without_a_process_group():
    sys.path.insert(0, ROOT)
    import torch

    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
