"""Train the learned cluster proposer and compare it with FastRandomHash.

Positive pairs are the edges of KNN graphs built by plain Cluster-and-Conquer
(FastRandomHash clustering) on training datasets drawn with other seeds from
the same workload shape; the item universe is shared (same world seed), so a
model trained there applies to the target dataset.  The comparison builds the
target's graph both ways with the same t, b, N, k and reports build time and
quality (Eq. 2 against exact brute force).

    python -m paper_2010_11497_gb300.train_proposer --workload learned_ml20m \\
        --train-seeds 6 7 8 9 --steps 400

Every step runs in libc2 (graph builds, forward/backward kernels, Adam).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import _c2 as c2
from . import synth


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def positive_pairs(nbr_id: torch.Tensor) -> torch.Tensor:
    n, k = nbr_id.shape
    u = torch.arange(n, device=nbr_id.device, dtype=torch.int32).repeat_interleave(k)
    v = nbr_id.reshape(-1)
    keep = v >= 0
    return torch.stack([u[keep], v[keep]], 1).contiguous()


def timed(fn, reps=3):
    torch.cuda.synchronize()
    best = None
    out = None
    for _ in range(reps):
        a = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        t = time.perf_counter() - a
        best = t if best is None else min(best, t)
    return out, best


def quality(ptr, items, n_items, k, nbr_inter, nbr_union, judge=None):
    if judge is None:
        _, jin, jun = c2.c2_bruteforce_knn(ptr, items, n_items, k)
        judge = c2.c2_avg_sim(jin, jun)
    return c2.c2_avg_sim(nbr_inter, nbr_union) / judge, judge


def run(workload="learned_ml20m", train_seeds=(6, 7, 8, 9), steps=400, batch=8192, lr=2e-3,
        lam=3.0, dim=64, hidden=256, rows_log2=18, model_seed=2010, mu=0.0, log=print,
        lams=None):
    """Trains one model per balance weight in `lams` (default: [lam]) on the
    same training graphs; returns the results and the model of the best
    quality on the target."""
    lams = list(lams) if lams else [lam]
    w = synth.WORKLOADS[workload]
    k, t, b, N, thr = w.k, w.t, w.b, w.N, w.greedy_threshold
    opts = c2.options(greedy_threshold=thr, greedy_rounds=w.greedy_rounds)
    # training graphs (plain C^2 on other seeds)
    train = []
    t0 = time.perf_counter()
    for s in train_seeds:
        ptr, items, _ = synth.generate(w, s, mu=mu) if mu else synth.load(workload, s)
        dptr, ditems = dev(ptr), dev(items)
        nid, _, _ = c2.c2_build_knn_graph(dptr, ditems, w.n_items, k, t, b, N, s, opts=opts)
        train.append((dptr, ditems, positive_pairs(nid)))
    t_graphs = time.perf_counter() - t0
    # target dataset and the FastRandomHash reference
    ptr, items, _ = synth.generate(w, w.seed, mu=mu) if mu else synth.load(workload, w.seed)
    dptr, ditems = dev(ptr), dev(items)
    nnz = items.size
    ws = c2.workspace(c2.workspace_size(w.n_users, nnz, w.n_items, k, t, b, N, opts), "cuda")
    (fid, fin, fun), t_frh = timed(lambda: c2.c2_build_knn_graph(
        dptr, ditems, w.n_items, k, t, b, N, w.seed, opts=opts, ws=ws))
    frh_stats = c2.c2_get_stats(ws)
    q_frh, judge = quality(dptr, ditems, w.n_items, k, fin, fun)
    best = None
    results = []
    for lam in lams:
        r, model = _train_eval(w, train, steps, batch, lr, lam, dim, hidden, rows_log2, model_seed,
                               dptr, ditems, nnz, ws, opts, fid, judge, log)
        r.update(workload=workload, n_users=w.n_users, n_items=w.n_items, nnz=int(nnz), k=k, t=t,
                 b=b, N=N, mu=mu, train_seeds=list(train_seeds), train_graphs_s=t_graphs,
                 frh=dict(build_ms=t_frh * 1e3, quality=q_frh, pairs=frh_stats["pairs"],
                          n_clusters=frh_stats["n_clusters"],
                          max_cluster=frh_stats["max_cluster"]))
        r["gain_quality"] = r["learned"]["quality"] - q_frh
        r["speedup"] = t_frh * 1e3 / r["learned"]["total_ms"]
        log(json.dumps(r))
        results.append(r)
        if best is None or r["learned"]["quality"] > best[0]["learned"]["quality"]:
            best = (r, model)
    return results, best[1]


def _train_eval(w, train, steps, batch, lr, lam, dim, hidden, rows_log2, model_seed, dptr, ditems,
                nnz, ws, opts, fid, judge, log):
    k, t, b, N, thr = w.k, w.t, w.b, w.N, w.greedy_threshold
    model = c2.Model(t, b, dim, hidden, rows_log2, model_seed).init()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(model_seed)
    losses = []
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for step in range(steps):
        tptr, titems, pairs = train[step % len(train)]
        idx = torch.randint(0, pairs.shape[0], (batch,), device="cuda", generator=gen)
        losses.append(model.train_step(tptr, titems, pairs[idx].contiguous(), lr=lr, lam=lam))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    losses = torch.stack(losses).cpu().numpy()
    keys, t_prop = timed(lambda: model.propose(dptr, ditems))
    lopts = c2.options(greedy_threshold=thr, greedy_rounds=w.greedy_rounds, keys=keys)
    (lid, lin, lun), t_lbuild = timed(lambda: c2.c2_build_knn_graph(
        dptr, ditems, w.n_items, k, t, b, N, w.seed, opts=lopts, ws=ws))
    l_stats = c2.c2_get_stats(ws)
    q_learned, _ = quality(dptr, ditems, w.n_items, k, lin, lun, judge)
    kk = keys.cpu().numpy()
    cp = positive_pairs(fid).cpu().numpy()
    used = [int(np.unique(kk[j]).size) for j in range(t)]
    res = dict(
        steps=steps, batch=batch, lr=lr, lam=lam,
        loss_first=losses[:10].mean(0).tolist(), loss_last=losses[-10:].mean(0).tolist(),
        train_s=t_train,
        learned=dict(propose_ms=t_prop * 1e3, build_ms=t_lbuild * 1e3,
                     total_ms=(t_prop + t_lbuild) * 1e3, quality=q_learned,
                     pairs=l_stats["pairs"], n_clusters=l_stats["n_clusters"],
                     max_cluster=l_stats["max_cluster"], buckets_used_per_head=used,
                     frh_neighbour_pairs_sharing_a_key=float(
                         (kk[:, cp[:, 0]] == kk[:, cp[:, 1]]).any(0).mean())))
    return res, model


def time_propose(workload="learned_ml20m", chunk=65536, reps=10, dim=64, hidden=256,
                 rows_log2=18, model_seed=2010, log=print):
    """Times c2_model_propose of an untrained network (the workload's t and b)
    on the workload's target data with CUDA events: 3 warm-ups, then the mean
    of `reps` proposals of every user."""
    w = synth.WORKLOADS[workload]
    ptr, items, _ = synth.load(workload, w.seed)
    dptr, ditems = dev(ptr), dev(items)
    model = c2.Model(w.t, w.b, dim, hidden, rows_log2, model_seed).init()
    for _ in range(3):
        model.propose(dptr, ditems, chunk=chunk)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        model.propose(dptr, ditems, chunk=chunk)
    e1.record()
    torch.cuda.synchronize()
    r = dict(workload=workload, n_users=w.n_users, nnz=int(items.size), t=w.t, b=w.b, dim=dim,
             hidden=hidden, chunk=chunk, reps=reps, propose_ms=e0.elapsed_time(e1) / reps)
    log(json.dumps(r))
    return r


def time_train(workload="learned_ml20m", batch=8192, reps=20, dim=64, hidden=256, rows_log2=18,
               model_seed=2010, lam=3.0, log=print):
    """Times c2_model_train_step on the workload's target data with seeded
    random pairs (the GEMM shapes of training; the pairs' content does not
    change the work): 3 warm-up steps, then the mean of `reps` steps (CUDA
    events).  With batch a multiple of 32 the three large GEMMs of a step run
    on the tensor cores (tcgen05), otherwise on mma.sync."""
    w = synth.WORKLOADS[workload]
    ptr, items, _ = synth.load(workload, w.seed)
    dptr, ditems = dev(ptr), dev(items)
    model = c2.Model(w.t, w.b, dim, hidden, rows_log2, model_seed).init()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(model_seed)
    pairs = torch.randint(0, w.n_users, (batch, 2), device="cuda", generator=gen,
                          dtype=torch.int32)
    for _ in range(3):
        model.train_step(dptr, ditems, pairs, lam=lam)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        model.train_step(dptr, ditems, pairs, lam=lam)
    e1.record()
    torch.cuda.synchronize()
    r = dict(workload=workload, t=w.t, b=w.b, dim=dim, hidden=hidden, batch_pairs=batch,
             rows=2 * batch, reps=reps, train_step_ms=e0.elapsed_time(e1) / reps,
             gemm_flop_per_step=3 * 2 * (2 * batch) * hidden * w.t * w.b)
    log(json.dumps(r))
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--time-propose", action="store_true",
                    help="time proposals of an untrained network on the target data and exit")
    ap.add_argument("--time-train", action="store_true",
                    help="time training steps on random pairs of the target data and exit")
    ap.add_argument("--chunk", type=int, default=65536, help="users per proposal chunk")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--workload", default="learned_ml20m")
    ap.add_argument("--train-seeds", type=int, nargs="+", default=[6, 7, 8, 9])
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lam", type=float, default=3.0,
                    help="balance weight (3: best quality on the workload's own profiles; 10 on "
                         "profiles with community structure)")
    ap.add_argument("--lams", type=float, nargs="*", default=None)
    ap.add_argument("--mu", type=float, default=0.0)
    ap.add_argument("--save", default="")
    a = ap.parse_args()
    if a.time_propose:
        time_propose(a.workload, a.chunk, a.reps)
        return
    if a.time_train:
        time_train(a.workload, a.batch, a.reps, lam=a.lam)
        return
    _, model = run(a.workload, tuple(a.train_seeds), a.steps, a.batch, a.lr, a.lam, mu=a.mu,
                   lams=a.lams)
    if a.save:
        model.save(a.save)


if __name__ == "__main__":
    main()
