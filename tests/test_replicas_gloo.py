"""The multi-GPU path of bench.py runs independent replicas (the D2Q37 step
has no data-path exchange on one lattice per GPU); what the ranks share is
the timing: a barrier and the maximum time over ranks.  Checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(torch, world)
    out[rank] = bench.dist_max(10.0 + rank, torch, world)
    dist.destroy_process_group()


def test_two_rank_max_over_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert dict(out) == {0: 11.0, 1: 11.0}
