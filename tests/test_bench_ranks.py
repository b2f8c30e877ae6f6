"""The multi-rank path of bench.py on CPU (gloo, world size 2): replicas draw
their own point sources on the same graph, and the job's timing is the
slowest rank's time with the units of all ranks summed."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1))
    g, nodes = bench.make_workload(rank, n=20_000)
    out.put((rank, ms, units, int(g.nnz), sorted(int(x) for x in nodes)))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_draw_their_own_sources():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ms0, u0, nnz0, src0), (_, ms1, u1, nnz1, src1) = res
    assert ms0 == ms1 == 11.0           # max over ranks
    assert u0 == u1 == 300.0            # sum over ranks
    assert nnz0 == nnz1                 # the same graph on every rank
    assert src0 != src1 and len(src0) == len(src1) == 16


def test_single_process_is_unchanged():
    import bench
    assert bench.reduce_over_ranks(3.5, 7.0) == (3.5, 7.0)
