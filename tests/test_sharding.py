"""Sharding by hash function (the distribution the paper leaves for future
work, Section VII), on the CPU oracle with gloo ranks.

G shards each cluster with t/G of the t functions (the run's functions
fn_offset .. fn_offset + t/G - 1) and compute their local rows; one exchange
of cluster counts gives each shard the run's number of its first cluster
(the greedy random starts draw with it), one exchange of the local rows and
the slot maps, concatenated in function order, gives every rank the inputs of
the merge: the graph equals the unsharded run's exactly.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2010_11497_gb300 import synth

K, T, B, N, SEED, THR, R = 8, 4, 8, 300, 13, 120, 3


def _data():
    return synth.random_profiles(900, 150, 12, 91, zipf_s=1.1)


def shard_rows(ptr, items, m, g, G, counts=None):
    """Shard g of G: its clustering, and its local rows once the cluster counts
    of the shards before it are known."""
    tg = T // G
    cl = oracle.frh_cluster_shard(ptr, items, m, tg, B, N, SEED, g * tg)
    if counts is None:
        return cl, None
    base = int(sum(counts[:g]))
    rows = oracle.cluster_knn_shard(ptr, items, cl["cptr"], cl["cusers"], K, SEED, THR, R, base)
    return cl, rows


def merged(ptr, parts):
    """Merge of the shards' rows in function order (the slot maps give the
    users; cluster boundaries only matter within a function)."""
    n = ptr.size - 1
    cusers = np.concatenate([cl["cusers"] for cl, _ in parts])
    li = np.concatenate([r[0] for _, r in parts])
    lc = np.concatenate([r[1] for _, r in parts])
    lu = np.concatenate([r[2] for _, r in parts])
    cptr = np.arange(0, cusers.size + 1, n, dtype=np.int32)   # one "cluster" per function
    return oracle.merge_topk(cptr, cusers, n, K, li, lc, lu)


@pytest.mark.parametrize("G", [1, 2, 4])
def test_logical_shards_equal_the_unsharded_build(G):
    ptr, items = _data()
    m = 150
    ref = oracle.build_graph(ptr, items, m, K, T, B, N, SEED, THR, R)
    counts = [shard_rows(ptr, items, m, g, G)[0]["n_clusters"] for g in range(G)]
    parts = [shard_rows(ptr, items, m, g, G, counts) for g in range(G)]
    got = merged(ptr, parts)
    for a, b in zip(got, ref[:3]):
        assert np.array_equal(a, b)
    assert sum(r[3] for _, r in parts) == ref[3]     # pair evaluations add up


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ptr, items = _data()
        m = 150
        cl, _ = shard_rows(ptr, items, m, rank, world)
        # exchange 1: the shards' cluster counts
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(counts, torch.tensor([cl["n_clusters"]], dtype=torch.int64))
        counts = [int(c.item()) for c in counts]
        _, rows = shard_rows(ptr, items, m, rank, world, counts)
        # exchange 2: slot maps and local rows, gathered in rank (= function) order
        mine = torch.from_numpy(np.concatenate([cl["cusers"][:, None], rows[0], rows[1], rows[2]],
                                               axis=1))
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        parts = [p.numpy() for p in parts]
        got = merged(ptr, [({"cusers": p[:, 0].copy()}, (p[:, 1:1 + K], p[:, 1 + K:1 + 2 * K],
                                                           p[:, 1 + 2 * K:1 + 3 * K]))
                           for p in parts])
        ref = oracle.build_graph(ptr, items, m, K, T, B, N, SEED, THR, R)
        out.put((rank, all(np.array_equal(a, b) for a, b in zip(got, ref[:3]))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_and_merge():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: True, 1: True}
