"""Benchmark: Cluster-and-Conquer KNN-graph build on one GB300 per rank.

One step = one whole build (FastRandomHash clustering with recursive split,
local KNN in every cluster, merge) of the ml20m-like synthetic workload, the
largest k=30 workload that fits one GPU: 138,493 users x 26,744 items, 20M
profile entries, k=30, t=8, b=4096, N=2000, brute force in every cluster
(the paper's rule rho*k^2 = 4500 > N).  --workload ml10m_like gives the
workload with greedy refinement (10 rounds in clusters of more than 500 users).

`value` is exact-Jaccard pair evaluations per second of the whole job,
device-timed with CUDA events around each step, inputs resident in HBM and
L2 flushed (a 512 MiB write) before every step; `intersections_per_step`
counts the pair intersections actually computed (brute-force pairs plus the
greedy clusters' count matrices; greedy rounds look counts up).  `e2e` repeats the build
through the host-buffer C entry point (pinned host CSR in, pinned host graph
out, copies inside the timed region).  With --impl reference the CPU oracle
is timed instead, on a bounded sample of the same workload.

Multi-GPU: every rank builds the graph of its own independent problem (the
same workload shape with seed + rank): weak scaling, no collective on the
data path; only the timing uses a barrier and a max over ranks.

Other workloads (--workload) and the MinHash-clustering variant of the
paper's Table 4 (--clustering minhash, optionally --split-N) use the same
line; past 200,000 users the quality is Eq. 2 on a seeded 4,096-user sample.
The line's `kernels` list gives each phase's share of the device time and,
where modelled, its kernel's rate against the roofline.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2010_11497_gb300 import synth  # noqa: E402

METRIC = "KNN-graph build s & exact-Jaccard pairs/s at k=30, quality≥0.95 vs brute force"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
HERE = os.path.dirname(os.path.abspath(__file__))
N_SM = 152
QUALITY_ALL_USERS = 200_000   # exact judge over every user up to this size
QUALITY_SAMPLE = 4096         # query users sampled beyond it
LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="c2", choices=["c2", "reference"])
    ap.add_argument("--workload", default="ml20m_like")
    ap.add_argument("--clustering", default="frh", choices=["frh", "minhash"],
                    help="first-level keys: FastRandomHash, or the MinHash variant (one cluster "
                         "per item, no split; Table 4)")
    ap.add_argument("--split-N", type=int, default=0,
                    help="MinHash variant: split clusters above this size with FastRandomHash "
                         "(0 = never, as in Table 4)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--similarity", default="exact", choices=["exact", "goldfinger"],
                    help="local KNN graphs on exact Jaccard, or on GoldFinger fingerprints "
                         "(Section II-F; quality is then Eq. 2 on the exact similarities of the "
                         "neighbours found)")
    ap.add_argument("--gf-bits", type=int, default=1024)
    ap.add_argument("--strategy", type=int, default=-1,
                    help="count-matrix strategy: -1 autotuned (default), 0 merge, 1-2 table, "
                         "3 tensor cores")
    ap.add_argument("--autotune-cache", default="",
                    help="autotuner table file: loaded before the warm-ups when present, saved "
                         "after them (a profiled run then repeats the decisions of a plain one)")
    ap.add_argument("--gram-budget-mb", type=int, default=0,
                    help="cap on count matrices held at once (0 = library default)")
    ap.add_argument("--cpu-full", action="store_true",
                    help="cpu_baseline: time the oracle's whole build once instead of a sample")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU seconds of the oracle sample")
    return ap.parse_args()


def peaks():
    p = dict(FALLBACK_PEAKS)
    src = "fallback"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            p.update(json.load(open(path)))
            src = "measured"
        except Exception:
            pass
    return p, src


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            busy = [x for x in sm if x > 0.5 * max(sm)] or sm
            out.update(sm_mhz=statistics.median(busy), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# ------------------------------------------------------------------ distributed
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        return dist, rank, local, ws
    return None, rank, local, ws


def barrier(dist, dev=None):
    if dist is not None:
        import torch
        if dev is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[dev.index])
        else:
            dist.barrier()


def max_over_ranks(dist, x: float, dev=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64,
                     device=dev if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float, dev=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64,
                     device=dev if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def host_cpu():
    """Host cores and CPU model (lscpu), for the CPU-baseline record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


SIZE_EDGES = (2, 9, 32, 128, 512, 2048, 1 << 62)


def oracle_sample(ptr, items, w, seed, budget_s, rng_seed=2010, clustering=None, t_cluster=None):
    """Times the oracle on a stratified systematic sample of the workload's
    clusters and extrapolates the time of the whole build.

    Step 1 (clustering) runs on the whole workload.  Every cluster of Step 2
    gets an estimate of its oracle work from its own profile lengths (a
    sorted-list merge per pair: (M-1) * sum of |P_u| for brute force;
    (k + R k^2) * 2 * sum of |P_u| for R greedy rounds).  Clusters are grouped
    into strata (brute force or greedy x size class); each stratum gets a
    share of the budget in proportion to its estimated work (at least 3%),
    and a systematic sample (every j-th cluster in increasing work, seeded
    offset, at least one cluster) that fits the share is timed alone.  Its
    time is scaled to the whole stratum by the estimated work; its pairs are
    exact for brute-force strata (M(M-1)/2 per cluster) and scaled by the
    members for greedy ones.  Returns (pairs/s of
    the extrapolated whole build, description, clustering)."""
    import oracle
    t0 = time.perf_counter()
    cl = clustering or oracle.frh_cluster(ptr, items, w.n_items, w.t, w.b, w.N, seed)
    if t_cluster is None:
        t_cluster = time.perf_counter() - t0
    cptr, cusers = cl["cptr"], cl["cusers"]
    sizes = np.diff(cptr).astype(np.int64)
    lens = np.diff(ptr).astype(np.int64)
    slot_len = lens[cusers]
    csum = np.concatenate([[0], np.cumsum(slot_len)])
    sum_len = (csum[cptr[1:]] - csum[cptr[:-1]]).astype(np.float64)
    greedy = sizes >= w.greedy_threshold
    work = np.where(greedy, (w.k + w.greedy_rounds * w.k * w.k) * 2.0 * sum_len,
                    np.maximum(sizes - 1, 0) * sum_len)
    est_s = work / 2.5e8
    size_cls = np.searchsorted(np.array(SIZE_EDGES), sizes, side="right") - 1
    stratum = np.where(sizes >= 2, size_cls * 2 + greedy.astype(np.int64), -1)
    ids = [s_ for s_ in np.unique(stratum) if s_ >= 0]
    est_total = float(est_s[stratum >= 0].sum())
    rng = np.random.default_rng(rng_seed)
    t_est, p_est, n_sampled, n_greedy_sampled, t_knn = 0.0, 0.0, 0, 0, 0.0
    for s_ in ids:
        members = np.flatnonzero(stratum == s_)
        members = members[np.argsort(work[members], kind="stable")]
        share = budget_s * max(0.03, float(est_s[members].sum()) / max(est_total, 1e-12))
        frac = min(1.0, share / max(float(est_s[members].sum()), 1e-12))
        step = max(1, int(round(1.0 / frac)))
        pick = members[int(rng.integers(0, step)) % members.size::step]
        only = np.zeros(sizes.size, np.uint8)
        only[pick] = 1
        t1 = time.perf_counter()
        _, _, _, pairs = oracle.cluster_knn(ptr, items, cptr, cusers, w.k, seed,
                                            w.greedy_threshold, w.greedy_rounds, 0, only=only)
        dt = time.perf_counter() - t1
        scale = float(work[members].sum()) / max(float(work[pick].sum()), 1.0)
        t_est += dt * scale
        if greedy[members[0]]:   # evaluations grow with the members
            p_est += pairs * float(sizes[members].sum()) / float(sizes[pick].sum())
        else:                    # brute force: exactly M(M-1)/2 per cluster
            p_est += float((sizes[members] * (sizes[members] - 1) // 2).sum())
        t_knn += dt
        n_sampled += int(pick.size)
        n_greedy_sampled += int(greedy[pick].sum())
    t_total = t_est + t_cluster
    desc = (f"oracle Step 1 on all {w.n_users} users ({t_cluster:.1f} s); Step 2 on a stratified "
            f"systematic sample of {n_sampled} of {int((sizes >= 2).sum())} clusters "
            f"({n_greedy_sampled} greedy; {len(ids)} strata by kind and size; {t_knn:.1f} s), "
            f"scaled to every cluster by estimated work: {p_est:.4g} pair evaluations in an "
            f"estimated {t_total:.1f} s for the whole build; single thread")
    return p_est / t_total, desc, cl


def oracle_full(ptr, items, w, seed):
    """Times the oracle's whole build once (Steps 1-3, single thread).
    Returns (pairs/s, description)."""
    import oracle
    t0 = time.perf_counter()
    _, _, _, pairs = oracle.build_graph(ptr, items, w.n_items, w.k, w.t, w.b, w.N, seed,
                                        w.greedy_threshold, w.greedy_rounds)
    dt = time.perf_counter() - t0
    return pairs / dt, (f"oracle whole build (Steps 1-3) of all {w.n_users} users: {pairs:.4g} "
                        f"pair evaluations in {dt:.1f} s; single thread")


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    dist, rank, local, world = dist_setup(args)
    if rank != 0:
        return 0
    w = synth.WORKLOADS[args.workload]
    ptr, items, _ = synth.load(args.workload, w.seed)
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    cl = oracle.frh_cluster(ptr, items, w.n_items, w.t, w.b, w.N, w.seed)
    t_cluster = time.perf_counter() - t0
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, _ = oracle_sample(ptr, items, w, w.seed, budget, rng_seed=2010 + i,
                                   clustering=cl, t_cluster=t_cluster)
        if i >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": w.name, **w.params()},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": desc, "host": host_cpu(),
                             "steps_values": vals},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ roofline
# DRAM traffic per launch of a kernel, from one ncu capture recorded in
# profiles/traffic.json together with a hash of the sources it was taken on;
# null once those sources change.
_CSRC = "paper_2010_11497_gb300/csrc/"
KERNEL_SOURCES = {
    "k_greedy_round": ["c2_knn.cu", "c2_internal.cuh"],
    "k_gram": ["c2_knn.cu", "c2_internal.cuh"],
    "k_gram_topk": ["c2_knn.cu", "c2_internal.cuh"],
    "k_gram_select": ["c2_knn.cu", "c2_internal.cuh"],
    "k_merge": ["c2_merge.cu", "c2_internal.cuh"],
    "k_minhash": ["c2_cluster.cu", "c2_internal.cuh"],
}


def sources_sha1(kernel):
    """Hash of the source files a kernel is built from."""
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(HERE, _CSRC + f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel, workload):
    path = os.path.join(HERE, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(kernel)
    if (not rec or kernel not in KERNEL_SOURCES or rec.get("workload") != workload
            or rec.get("sources_sha1") != sources_sha1(kernel)):
        return None
    return rec.get("bytes_per_launch")


def phase_model(dom, phase_ms, phase_calls, stats, w, nnz, pk, W, steps):
    """Roofline record of one phase's kernel: algorithmic work per launch over
    the launch's device time (CUDA events), against the measured peak.
    phase_ms and phase_calls are totals over `steps` builds; stats are those
    of one build."""
    n, t, k = w.n_users, w.t, w.k
    S = t * n
    calls = max(1, phase_calls.get(dom, 1))
    per_build = max(1.0, calls / max(1, steps))   # launches of the phase in one build
    ms = phase_ms[dom] / calls
    alu_peak = N_SM * LANES_PER_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12   # Tlane-op/s
    peak_note = f"peak = 152 SMs x 128 lanes x {pk.get('sm_max_mhz', 2070.0):.0f} MHz"

    def hbm(kernel, bytes_, model):
        achieved = bytes_ / (ms * 1e-3) / 1e9
        return {"kernel": kernel, "phase": dom, "bound": "hbm", "achieved": achieved,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                "traffic": recorded_traffic(kernel, w.name), "ms_per_launch": ms, "model": model}

    if dom == "greedy_rounds":
        # per examined neighbour-list entry: bitmap test-and-set (3), count and
        # length lookups (3), exact cross-multiplied comparison (6) = 12 lane-ops
        ms = phase_ms[dom] / (steps * max(1, w.greedy_rounds))   # one launch per round
        visits = stats.get("greedy_visits", 0) / max(1, w.greedy_rounds)
        ops = 12.0
        achieved = visits * ops / (ms * 1e-3) / 1e12
        return {"kernel": "k_greedy_round", "phase": dom, "bound": "alu", "achieved": achieved,
                "peak": alu_peak, "unit": "Tlane-op/s", "frac": achieved / alu_peak,
                "traffic": recorded_traffic("k_greedy_round", w.name), "ms_per_launch": ms,
                "model": f"{ops:.0f} integer lane-ops per neighbour-list entry examined "
                         f"({visits:.3e} entries/launch, {stats.get('greedy_computed', 0)} "
                         f"user-rounds computed of {stats.get('greedy_users', 0) * w.greedy_rounds}, "
                         f"{stats.get('greedy_evaluated', 0)} candidates looked up); {peak_note}"}
    if dom == "gram":
        visits = stats["item_visits_brute"] + stats["item_visits_greedy"]
        if W == 1:
            # bit-sliced counts: table load (1), item unpack (1), a carry-save
            # tree of 15 full adders of 2 logic ops per 16 items (1.875), the
            # weight-16 carry rippled through at most 12 planes (24 / 16 = 1.5)
            ops_per_visit = 1 + 1 + 30 / 16.0 + 24 / 16.0
        else:
            # 4-bit SWAR counters: table load (1), W words (W), spreading and
            # adding each word (12 W), flushing every 12 items (48 W / 12)
            ops_per_visit = 1 + W + 12 * W + 48 * W / 12.0
        achieved = visits / per_build * ops_per_visit / (ms * 1e-3) / 1e12
        return {"kernel": "k_gram<%d>" % W, "phase": dom, "bound": "alu", "achieved": achieved,
                "peak": alu_peak, "unit": "Tlane-op/s", "frac": achieved / alu_peak,
                "traffic": recorded_traffic("k_gram", w.name), "ms_per_launch": ms,
                "model": f"{ops_per_visit:.1f} integer lane-ops per candidate item visit "
                         f"({visits / per_build:.3e} visits/launch); {peak_note}"}
    if dom == "gram_tc" and stats.get("tc_macs"):
        # FP8 dense peak = the measured bf16 peak x the nominal fp8 / bf16
        # ratio (4.5 / 2.25 PFLOP/s)
        fp8_peak = 2.0 * pk["bf16_tflops"]
        flops = 2.0 * stats["tc_macs"] / per_build
        achieved = flops / (ms * 1e-3) / 1e12
        return {"kernel": "k_gram_mma", "phase": dom, "bound": "tensor", "achieved": achieved,
                "peak": fp8_peak, "unit": "TFLOP/s", "frac": achieved / fp8_peak,
                "traffic": None, "ms_per_launch": ms,
                "model": f"2 x {stats['tc_macs'] / per_build:.3e} FP8 multiply-adds issued per "
                         f"launch ({stats.get('tc_tiles', 0)} tiles of 128 x 256 over "
                         f"{stats.get('tc_clusters', 0)} clusters); peak = 2 x measured bf16 "
                         f"{pk['bf16_tflops']:.0f} TFLOP/s"}
    if dom == "brute_rows" and stats.get("brute_rows"):
        bytes_ = 2 * stats["brute_gram_elems"] + 12 * k * stats["brute_rows"]
        # exact selection serves keyed rows (every union below 2^16, clusters
        # below 2^14 members); the general top-k kernel the others
        keyed = 2 * stats.get("max_profile", 0) < 65536 and stats.get("max_cluster", 0) < 16384
        return hbm("k_gram_select" if keyed else "k_gram_topk", bytes_ / per_build,
                   f"count rows read once (2 B x {stats['brute_gram_elems']:.3e} elements) + "
                   f"12 k B of list per row ({stats['brute_rows']} rows)")
    if dom == "merge":
        return hbm("k_merge", 4 * S + 12 * S * k + 12 * n * k,
                   "t rows of k (id, inter, union) read per user, one row written, slot map read")
    if dom == "hash_minhash_level0":
        return hbm("k_minhash", 4 * (n + 1) + 4 * nnz + 12 * S,
                   "CSR read once plus three keys per (function, user) slot (the minimum and "
                   "the next two distinct values)")
    return None


def roofline(phase_ms, phase_calls, stats, w, nnz, pk, pk_src, W, steps):
    """Roofline of the dominant kernel phase (the largest share of device time)
    and the records of the other modelled phases."""
    candidates = {k_: v for k_, v in phase_ms.items() if v > 0 and not k_.startswith("round_")}
    if not candidates:
        return None, []
    dom = max(candidates, key=candidates.get)
    total = sum(candidates.values())
    rows = []
    for ph in sorted(candidates, key=candidates.get, reverse=True):
        rec = phase_model(ph, phase_ms, phase_calls, stats, w, nnz, pk, W, steps)
        row = {"phase": ph, "share": candidates[ph] / total}
        if rec:
            row.update({k_: rec[k_] for k_ in ("kernel", "bound", "achieved", "peak", "unit",
                                               "frac", "ms_per_launch", "traffic")})
        rows.append(row)
    rf = phase_model(dom, phase_ms, phase_calls, stats, w, nnz, pk, W, steps)
    if rf is None:   # an unmodelled phase dominates: CSR-read model as a floor
        rf = {"kernel": dom, "phase": dom, "bound": "hbm", "note": "no model for this phase"}
    return rf, rows


# ------------------------------------------------------------------ main arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2010_11497_gb300 as c2
    dist, rank, local, world = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS[args.workload]
    seed = w.seed + rank
    ptr_np, items_np, man = synth.load(args.workload, seed)
    nnz = int(items_np.size)
    ptr = torch.from_numpy(ptr_np).to(dev)
    items = torch.from_numpy(items_np).to(dev)
    minhash = args.clustering == "minhash"
    # the MinHash variant: keys are items (b = m + 1 buckets), clusters are never split
    wb, wN = (w.n_items + 1, args.split_N or w.n_users) if minhash else (w.b, w.N)
    keys = torch.empty((w.t, w.n_users), dtype=torch.int32, device=dev) if minhash else None
    kws = c2.workspace(256, dev)
    gf = args.similarity == "goldfinger"
    gf_out = None
    if gf:
        gbits = args.gf_bits
        gf_out = (torch.empty(w.n_users + 1, dtype=torch.int32, device=dev),
                  torch.empty(max(nnz, 1), dtype=torch.int32, device=dev),
                  torch.empty((w.n_users, gbits // 32), dtype=torch.int32, device=dev))
        gws = c2.workspace(int(c2.lib().c2_goldfinger_workspace_size(w.n_users)), dev)
    opts = c2.options(greedy_threshold=w.greedy_threshold, greedy_rounds=w.greedy_rounds,
                      gram_budget_bytes=args.gram_budget_mb << 20, keys=keys,
                      strategy=args.strategy,
                      sim=gf_out[:2] if gf else None, sim_n_items=args.gf_bits if gf else 0,
                      sim_bits=gf_out[2] if gf else None)
    ws = c2.workspace(c2.workspace_size(w.n_users, nnz, w.n_items, w.k, w.t, wb, wN, opts), dev)
    out = [torch.empty((w.n_users, w.k), dtype=torch.int32, device=dev) for _ in range(3)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        if minhash:
            c2.c2_minhash_keys(ptr, items, w.n_items, w.t, seed, out=keys, ws=kws, check=False)
        if gf:
            c2.c2_goldfinger(ptr, items, w.n_items, args.gf_bits, seed, ws=gws, check=False,
                             out=gf_out)
        c2.c2_build_knn_graph(ptr, items, w.n_items, w.k, w.t, wb, wN, seed, opts=opts, ws=ws,
                              out=out, check=False)

    if args.autotune_cache and os.path.exists(args.autotune_cache):
        c2.c2_autotune_load(args.autotune_cache)
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    assert c2.c2_get_status(ws) == 0, "build reported a device error"
    if args.autotune_cache:
        c2.c2_autotune_save(args.autotune_cache)
    stats = c2.c2_get_stats(ws)

    # timed region
    c2.c2_profile_enable(True)
    c2.c2_profile_report()                       # clear
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = c2.c2_kernel_launches()
    with ClockSampler(local) as clk:
        barrier(dist, dev)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        barrier(dist, dev)
    launches = c2.c2_kernel_launches() - launches0
    prof = c2.c2_profile_report()
    c2.c2_profile_enable(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    dev_s_max = max_over_ranks(dist, dev_s, dev)
    pairs = stats["pairs"]
    total_pairs = sum_over_ranks(dist, float(pairs) * args.steps, dev)
    value = total_pairs / dev_s_max
    clocks = clk.summary()

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e and not minhash and not gf:
        hptr = torch.from_numpy(ptr_np).pin_memory()
        hitems = torch.from_numpy(items_np).pin_memory()
        hws = c2.workspace(c2.workspace_size_host(w.n_users, nnz, w.n_items, w.k, w.t, w.b, w.N,
                                                  opts), dev)
        hout = [torch.empty((w.n_users, w.k), dtype=torch.int32).pin_memory() for _ in range(3)]
        for _ in range(max(3, args.warmup)):
            c2.c2_build_knn_graph_host(hptr, hitems, w.n_items, w.k, w.t, w.b, w.N, seed,
                                       opts=opts, ws=hws, out=hout)
        barrier(dist, dev)
        torch.cuda.synchronize()
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            c2.c2_build_knn_graph_host(hptr, hitems, w.n_items, w.k, w.t, w.b, w.N, seed,
                                       opts=opts, ws=hws, out=hout)
            e2e_s += time.perf_counter() - a
        e2e = e2e_s
        e2e_max = max_over_ranks(dist, e2e, dev)
        assert np.array_equal(hout[0].numpy(), out[0].cpu().numpy()), "host entry differs"
        e2e = {"value": total_pairs / e2e_max, "unit": "pairs/s",
               "h2d_bytes_per_step": int(ptr_np.nbytes + items_np.nbytes),
               "d2h_bytes_per_step": int(3 * w.n_users * w.k * 4),
               "ms_per_step": e2e_max / args.steps * 1e3}
        del hws

    # quality (Eq. 2) against the exact graph from the GPU judge
    quality = None
    if not args.no_quality and rank == 0:
        # with estimated similarities the graph's rows are rescored exactly
        ein, eun = c2.c2_exact_counts(ptr, items, out[0]) if gf else (out[1], out[2])
        if w.n_users <= QUALITY_ALL_USERS:
            bid, bin_, bun = c2.c2_bruteforce_knn(ptr, items, w.n_items, w.k)
            a_c2 = c2.c2_avg_sim(ein, eun)
            a_bf = c2.c2_avg_sim(bin_, bun)
            quality = {"avg_sim": a_c2, "avg_sim_bruteforce": a_bf, "quality": a_c2 / a_bf,
                       "users": "all"}
        else:
            # Eq. 2 on a seeded sample of query users (exact brute force of all
            # users is n^2 pairs): the same users' C^2 rows against their exact rows
            q = np.sort(np.random.default_rng(2010).choice(w.n_users, QUALITY_SAMPLE,
                                                           replace=False)).astype(np.int32)
            qd = torch.from_numpy(q).to(ptr.device).long()
            bid, bin_, bun = c2.c2_bruteforce_knn(ptr, items, w.n_items, w.k,
                                                  queries=qd.int().contiguous())
            a_c2 = c2.c2_avg_sim(ein[qd].contiguous(), eun[qd].contiguous())
            a_bf = c2.c2_avg_sim(bin_, bun)
            quality = {"avg_sim": a_c2, "avg_sim_bruteforce": a_bf, "quality": a_c2 / a_bf,
                       "users": f"{QUALITY_SAMPLE} seeded sample of {w.n_users}"}
        del bid, bin_, bun

    pk, pk_src = peaks()
    phase_ms = {k_: v["ms"] / args.steps for k_, v in prof.items()}
    phase_calls = {k_: v["calls"] / args.steps for k_, v in prof.items()}
    # table words per query of the shape the autotuner picked for this workload
    W = 2 if w.n_items * 8 + 40000 <= 227 * 1024 else 1
    for ent in c2.c2_autotune_report():
        if ent.get("n") == w.n_users and ent.get("m") == w.n_items and ent.get("buckets"):
            bk = ent["buckets"]
            W = bk[0]["words"] if ent.get("one_launch") else max(bk, key=lambda b: b["ms"])["words"]
    stats2 = dict(stats)
    rf, kernels = None, []
    try:
        rf, kernels = roofline({k_: v["ms"] for k_, v in prof.items()},
                               {k_: v["calls"] for k_, v in prof.items()}, stats2, w, nnz, pk,
                               pk_src, W, args.steps)
        if rf:
            rf["peak_source"] = pk_src
    except Exception as e:   # the measurement stands without the model
        rf = {"error": str(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        if args.cpu_full:
            v, desc = oracle_full(ptr_np, items_np, w, seed)
        else:
            v, desc, _ = oracle_sample(ptr_np, items_np, w, seed, args.cpu_seconds)
        cpu = {"value": v, "unit": "pairs/s", "cores": 1, "kind": "oracle", "sample": desc,
               "host": host_cpu()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": dev_s_max / args.steps * 1e3,
                "build_s": dev_s_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": w.name, "n_users": w.n_users, "n_items": w.n_items,
                           "nnz": nnz, **w.params(),
                           **({"clustering": "minhash", "b": wb, "N": wN} if minhash else {}),
                           **({"strategy": args.strategy} if args.strategy != -1 else {}),
                           **({"similarity": f"goldfinger{args.gf_bits}"} if gf else {}),
                           "l2": "flushed (512 MiB write) before each step",
                           "parallelism": f"replicas{world}" if world > 1 else "single"},
                "pairs_per_step": pairs, "gram_pairs_per_step": stats["gram_pairs"],
                "intersections_per_step": stats["brute_pairs"] + stats["greedy_pairs"],
                "pairs_split": {"brute_force": stats["brute_pairs"],
                                "greedy_evaluations": pairs - stats["brute_pairs"],
                                "greedy_count_matrix_pairs": stats["greedy_pairs"]},
                "quality": quality, "e2e": e2e, "gpu_launches": launches,
                "gpu_launches_per_step": launches / args.steps,
                "wall_s_timed": wall, "step_ms": step_ms,
                "phases_ms_per_step": phase_ms, "roofline": rf, "kernels": kernels,
                "cpu_baseline": cpu,
                "autotune": c2.c2_autotune_report(),
                "clocks": clocks, "stats": stats}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
