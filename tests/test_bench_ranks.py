"""The benchmark's multi-process path on CPU (world size 2, gloo): the timed region's length is
the slowest rank's, per-rank rates add up to the whole-job value, and the reference arm runs
on rank 0 only (the other ranks exit 0 without work or output).  The GPU arm calls the same
helpers with NCCL tensors on each rank's device."""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cpu")
        t_max = bench.max_over_ranks(1.0 + 0.5 * rank, dist, dev)
        total = bench.sum_over_ranks(10.0 * (rank + 1), dist, dev)
        r, w, l = bench.dist_setup(None)
        buf = io.StringIO()
        if rank != 0:
            args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
            with redirect_stdout(buf):
                rc = bench.run_reference(args, rank, world)
        else:
            rc = 0
        out.put((rank, t_max, total, (r, w, l), rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, total, (r, w, l), rc, printed in res:
        assert t_max == 1.5            # the slower rank's time on every rank
        assert total == 30.0           # 10 + 20
        assert (r, w, l) == (rank, world, rank)
        assert rc == 0
        if rank != 0:
            assert printed == ""       # the reference arm prints on rank 0 only


def test_single_process_helpers_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.sum_over_ranks(7.0, None, None) == 7.0
