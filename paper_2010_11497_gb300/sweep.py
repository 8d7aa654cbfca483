"""Sensitivity of C^2 to its parameters (the paper's Section VI: number of
hash functions t, buckets b, and the split limit N) on a synthetic workload.

For each setting: device time per build (CUDA events, median of `reps` after a
warm-up build, inputs resident) and KNN quality (Eq. 2) against the exact
graph, which is computed once per workload.  One JSON line per setting.

Grids (--figure):
  one  one parameter at a time around the workload's own (t, b, N);
  4    Figure 4: t in {1, 2, 4, 8, 10} for each b in {512, 2048, 8192} (N fixed);
  5    Figure 5: N from 500 to 10,000 (t, b fixed);
  6    Figure 6: the sizes of the 100 largest clusters for N from 500 to
       10,000 and without splitting (clustering only, no KNN).

    python -m paper_2010_11497_gb300.sweep [--workload ml10m_like] [--figure one|4|5|6] [--reps 3]
"""
from __future__ import annotations

import argparse
import json
import statistics

import torch

import paper_2010_11497_gb300 as c2
from paper_2010_11497_gb300 import synth

FIG5_N = (500, 1000, 2000, 3000, 4000, 6000, 8000, 10000)


def settings(w, figure):
    """(t, b, N) triples of a grid."""
    if figure == "4":
        return [(t, b, w.N) for b in (512, 2048, 8192) for t in (1, 2, 4, 8, 10)]
    if figure == "5":
        return [(w.t, w.b, N) for N in FIG5_N]
    base = (w.t, w.b, w.N)
    out = [base]
    for t in (2, 4, 12):
        out.append((t, w.b, w.N))
    for b in (512, 1024, 16384):
        out.append((w.t, b, w.N))
    for N in (500, 1000, 4000):
        out.append((w.t, w.b, N))
    return out


def cluster_sizes(args, w, ptr, items, dev):
    """Figure 6: for each N (and N = n, no split), the 100 largest final
    clusters over all t functions, largest first."""
    n = w.n_users
    for N in FIG5_N + (n,):
        g = c2.c2_frh_cluster(ptr, items, w.n_items, w.t, w.b, N, w.seed)
        sizes = (g["cptr"][1:] - g["cptr"][:-1]).to(torch.int64)
        top = torch.sort(sizes, descending=True).values[:100].cpu().tolist()
        print(json.dumps({"workload": w.name, "t": w.t, "b": w.b, "N": N if N < n else None,
                          "n_clusters": g["n_clusters"], "top100": top}), flush=True)
    return 0


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ml10m_like")
    ap.add_argument("--figure", default="one", choices=["one", "4", "5", "6"])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    ptr_np, items_np, _ = synth.load(args.workload)
    dev = torch.device("cuda")
    ptr = torch.from_numpy(ptr_np).to(dev)
    items = torch.from_numpy(items_np).to(dev)
    if args.figure == "6":
        return cluster_sizes(args, w, ptr, items, dev)
    _, bin_, bun = c2.c2_bruteforce_knn(ptr, items, w.n_items, w.k)
    exact = c2.c2_avg_sim(bin_, bun)
    for t, b, N in settings(w, args.figure):
        opts = c2.options(greedy_threshold=w.greedy_threshold, greedy_rounds=w.greedy_rounds)
        ws = c2.workspace(c2.workspace_size(w.n_users, items_np.size, w.n_items, w.k, t, b, N,
                                            opts), dev)
        out = [torch.empty((w.n_users, w.k), dtype=torch.int32, device=dev) for _ in range(3)]
        c2.c2_build_knn_graph(ptr, items, w.n_items, w.k, t, b, N, w.seed, opts=opts, ws=ws,
                              out=out)
        ms = []
        for _ in range(args.reps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            c2.c2_build_knn_graph(ptr, items, w.n_items, w.k, t, b, N, w.seed, opts=opts, ws=ws,
                                  out=out, check=False)
            e.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        st = c2.c2_get_stats(ws)
        q = c2.c2_avg_sim(out[1], out[2]) / exact
        print(json.dumps({"workload": w.name, "t": t, "b": b, "N": N, "ms": statistics.median(ms),
                          "quality": q, "pairs": st["pairs"], "n_clusters": st["n_clusters"],
                          "max_cluster": st["max_cluster"],
                          "greedy_clusters": st["n_greedy_clusters"]}), flush=True)
        del ws, out
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
