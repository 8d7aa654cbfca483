"""The benchmark's multi-process timing logic on CPU ranks (gloo, world size 2).

Every rank builds its own independent problem, so the only cross-rank work is
timing: a barrier, the maximum of the ranks' times and the sum of their pair
counts.
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d, r, local, ws = bench.dist_setup(None)
    assert (r, ws) == (rank, world) and d is not None
    bench.barrier(d)
    t_max = bench.max_over_ranks(d, 1.0 + rank)
    total = bench.sum_over_ranks(d, 10.0 * (rank + 1))
    q.put((rank, t_max, total))
    d.destroy_process_group()


def test_bench_timing_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.0, 30.0), (1, 2.0, 30.0)]
