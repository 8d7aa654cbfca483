"""Cluster-and-Conquer sharded by hash function.

The paper names distribution as future work (Section VII): its t clusterings
are independent until the merge.  Shard g of G takes the run's functions
g*t/G .. (g+1)*t/G - 1 (c2_options.fn_offset) and clusters and builds its
local KNN graphs alone; two exchanges make the result the unsharded one:

1. the shards' cluster counts, so that shard g numbers its clusters from the
   run's number of its first cluster (c2_options.cluster_base; the greedy
   random starts draw with cluster numbers);
2. the shards' slot maps and local rows, which, concatenated in function
   order, are the merge's inputs of one call with all t functions.

`build_knn_graph_sharded` runs G logical shards one after another on the
current GPU, or, given a torch.distributed process group, one shard per rank
(every rank ends with the whole graph).  Every step runs in libc2.
"""
from __future__ import annotations

import torch

from . import _c2 as c2


def _shard_opts(base: dict, **kw):
    d = dict(base)
    d.update(kw)
    return c2.options(**d)


def _step1(ptr, items, n_items, tg, b, N, seed, g, opts_kw):
    return c2.c2_frh_cluster(ptr, items, n_items, tg, b, N, seed,
                             opts=_shard_opts(opts_kw, fn_offset=g * tg))


def _step2(ptr, items, n_items, tg, k, seed, cl, base, opts_kw):
    return c2.c2_cluster_knn(ptr, items, n_items, tg, cl["cptr_full"], cl["cusers"],
                             cl["n_clusters_dev"], k, seed,
                             opts=_shard_opts(opts_kw, cluster_base=base))


def build_knn_graph_sharded(ptr, items, n_items, k, t, b, N, seed, shards=None, group=None,
                            **opts_kw):
    """The whole method with its t functions split over G shards.

    shards: G logical shards on the current GPU (group is None); with a
    process group, G = its size and this rank computes shard `rank`.
    Returns (nbr_id, nbr_inter, nbr_union) of shape [n, k]."""
    n = ptr.numel() - 1
    if group is None:
        G = int(shards or 1)
        if G < 1 or t % G:
            raise ValueError("t must be a multiple of the number of shards")
        tg = t // G
        cls = [_step1(ptr, items, n_items, tg, b, N, seed, g, opts_kw) for g in range(G)]
        base = 0
        parts = []
        for g in range(G):
            parts.append((cls[g]["cusers"],
                          _step2(ptr, items, n_items, tg, k, seed, cls[g], base, opts_kw)))
            base += cls[g]["n_clusters"]
        cusers = torch.cat([p[0] for p in parts])
        rows = [torch.cat([p[1][i] for p in parts]) for i in range(3)]
        return c2.c2_merge_topk(cusers, n, t, k, *rows)

    import torch.distributed as dist
    G = dist.get_world_size(group)
    g = dist.get_rank(group)
    if t % G:
        raise ValueError("t must be a multiple of the number of ranks")
    tg = t // G
    dev = ptr.device
    cl = _step1(ptr, items, n_items, tg, b, N, seed, g, opts_kw)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(G)]
    dist.all_gather(counts, torch.tensor([cl["n_clusters"]], dtype=torch.int64, device=dev),
                    group=group)
    base = int(sum(int(c.item()) for c in counts[:g]))
    li, lc, lu = _step2(ptr, items, n_items, tg, k, seed, cl, base, opts_kw)
    mine = torch.cat([cl["cusers"].view(-1, 1), li, lc, lu], dim=1).contiguous()
    allp = [torch.empty_like(mine) for _ in range(G)]
    dist.all_gather(allp, mine, group=group)
    allp = torch.cat(allp)
    cusers = allp[:, 0].contiguous()
    rows = [allp[:, 1 + i * k:1 + (i + 1) * k].contiguous() for i in range(3)]
    return c2.c2_merge_topk(cusers, n, t, k, *rows)
