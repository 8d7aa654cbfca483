"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Everything here runs on the CPU.  Independent references are written with
Python sets and exact fractions, never by calling the oracle's own helpers.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2010_11497_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def csr_from_sets(rows):
    ptr = np.zeros(len(rows) + 1, np.int32)
    items = []
    for u, r in enumerate(rows):
        s = sorted(set(r))
        items.extend(s)
        ptr[u + 1] = ptr[u] + len(s)
    return ptr, np.array(items, np.int32)


def sets_from_csr(ptr, items):
    return [set(items[ptr[u]:ptr[u + 1]].tolist()) for u in range(ptr.size - 1)]


def py_topk(sets, u, cands, k):
    """Independent top-k: exact Fraction similarity, ties to the lower id, c > 0."""
    scored = []
    for v in cands:
        if v == u:
            continue
        c = len(sets[u] & sets[v])
        if c == 0:
            continue
        U = len(sets[u] | sets[v])
        scored.append((-Fraction(c, U), v, c, U))
    scored.sort()
    return [(v, c, U) for _, v, c, U in scored[:k]]


def rows_of(ids, inter, uni):
    out = []
    for r in range(ids.shape[0]):
        out.append([(int(a), int(b), int(c)) for a, b, c in zip(ids[r], inter[r], uni[r]) if a >= 0])
    return out


# ------------------------------------------------------------------ generators
def test_splitmix64_first_outputs():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014): the state advances by
    # the golden gamma before mixing; the published first outputs are these.
    g = 0x9E3779B97F4A7C15
    assert oracle.mix64(g) == 0xE220A8397B1DCDAF
    assert oracle.mix64((2 * g) % 2 ** 64) == 0x6E789E6AA1B965F4


def test_philox_known_answers():
    # Philox4x32-10 known-answer vectors published with Random123 (Salmon et al., SC'11).
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]).tolist() == \
        [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    f = 0xFFFFFFFF
    assert oracle.philox4x32_10([f, f, f, f], [f, f]).tolist() == \
        [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert oracle.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                [0xA4093822, 0x299F31D0]).tolist() == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_item_hash_range_and_uniformity():
    # h_i maps items onto [0, b) (Section II-D); a random function is uniform.
    b, m = 64, 64 * 400
    vals = np.array([oracle.item_hash(7, 3, x, b) for x in range(m)])
    assert vals.min() >= 0 and vals.max() < b
    counts = np.bincount(vals, minlength=b)
    chi2 = ((counts - 400.0) ** 2 / 400.0).sum()
    assert chi2 < 130  # 63 d.o.f.; p ~ 1e-6 cut
    # different functions are different
    other = np.array([oracle.item_hash(7, 4, x, b) for x in range(m)])
    assert (vals == other).mean() < 0.05


# ------------------------------------------------------------------ worked examples
def test_frh_worked_example():
    g = golden("frh_worked_example.json")
    b = g["b"]
    htab = np.array([np.array(g["h1"]) - 1, np.array(g["h2"]) - 1], np.int32)
    ptr, items = csr_from_sets([[i - 1 for i in g["P_u"]], [i - 1 for i in g["P_v"]]])
    keys = oracle.frh_keys(ptr, items, 5, 2, b, 0, htab=htab)
    assert keys[0].tolist() == [g["H1_u"] - 1, g["H1_v"] - 1]
    assert keys[1].tolist() == [g["H2_u"] - 1, g["H2_v"] - 1]
    cl = oracle.frh_cluster(ptr, items, 5, 2, b, 100, 0, htab=htab)
    co = cl["cluster_of"]
    assert co[0, 0] != co[0, 1]          # different clusters under h_1
    assert co[1, 0] == co[1, 1]          # same cluster under h_2
    assert cl["n_clusters"] == 3
    # within the shared cluster, each is the other's only neighbour with J = 1/5
    li, lc, lu, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], 2, 0, 10 ** 9)
    shared = co[1, 0]
    s0 = cl["cptr"][shared]
    assert li[s0].tolist() == [1, -1] and lc[s0, 0] == g["common_items_uv"] and lu[s0, 0] == g["union_items_uv"]
    nid, nin, nun = oracle.merge_topk(cl["cptr"], cl["cusers"], 2, 2, li, lc, lu)
    assert nid.tolist() == [[1, -1], [0, -1]]
    assert Fraction(int(nin[0, 0]), int(nun[0, 0])) == Fraction(1, 5)


def _figure3_profiles(res, mid, high, c2, c3):
    # items 0,1,2 hash to buckets 1,2,3 (0-based 0,1,2)
    rows = [[0]] * res + [[0, 1]] * mid + [[0, 2]] * high + [[1, 2]] * c2 + [[2]] * c3
    return csr_from_sets(rows)


def test_split_figure3():
    g = golden("split_figure3.json")
    s = g["split_of_bucket_1"]
    top = g["top_level_sizes_by_bucket"]
    ptr, items = _figure3_profiles(s["residual"], s["H_minus_1_eq_2"], s["H_minus_1_eq_3"],
                                   top["2"], top["3"])
    assert ptr.size - 1 == g["n_users"]
    htab = np.array([[0, 1, 2]], np.int32)
    # before split: N large
    cl0 = oracle.frh_cluster(ptr, items, 3, 1, g["b"], 10 ** 6, 0, htab=htab)
    sizes0 = np.diff(cl0["cptr"]).tolist()
    assert sizes0 == [top["1"], top["2"], top["3"]]
    assert cl0["n_clusters"] == g["n_clusters_before_split"]
    cl = oracle.frh_cluster(ptr, items, 3, 1, g["b"], g["N"], 0, htab=htab)
    sizes = np.diff(cl["cptr"]).tolist()
    assert cl["n_clusters"] == g["n_clusters_after_split"]
    # canonical order: residual of bucket 1 first, then its children, then buckets 2, 3
    assert sizes == [s["residual"], s["H_minus_1_eq_2"], s["H_minus_1_eq_3"], top["2"], top["3"]]
    meta = cl["cmeta"]
    assert meta[:, 2].tolist() == [1, 0, 0, 0, 0]          # residual flag
    assert meta[:, 1].tolist() == [0, 1, 1, 0, 0]          # depth
    assert meta[:, 3].tolist() == [0, 1, 2, 1, 2]          # last key
    # new sub-clusters are not merged with same-key top-level clusters
    assert cl["cluster_of"][0, 20] != cl["cluster_of"][0, 80]


def test_split_singletons_stay_in_residual():
    # A user alone in its new group stays in the split cluster (Section II-D).
    rows = [[0]] * 3 + [[0, 1]] * 4 + [[0, 2]]
    ptr, items = csr_from_sets(rows)
    htab = np.array([[0, 1, 2]], np.int32)
    cl = oracle.frh_cluster(ptr, items, 3, 1, 3, 5, 0, htab=htab)
    sizes = np.diff(cl["cptr"]).tolist()
    assert sizes == [4, 4]     # residual = 3 single-item users + the lone [0,2] user
    assert sorted(cl["cusers"][:4].tolist()) == [0, 1, 2, 7]


def test_recursive_split_goes_deeper():
    # groups still above N are split again using the new key as threshold
    rows = [[0, 1, 2]] * 6 + [[0, 1]] * 2 + [[0, 1, 3]] * 3
    ptr, items = csr_from_sets(rows)
    htab = np.array([[0, 1, 2, 3]], np.int32)
    cl = oracle.frh_cluster(ptr, items, 4, 1, 4, 4, 0, htab=htab)
    sizes = np.diff(cl["cptr"]).tolist()
    meta = cl["cmeta"]
    # bucket 0 (11 users) > 4 -> all go to eta'=1 group (11) > 4 -> split by eta''
    # eta''=2: 6 users (> 4, split again: all undefined -> residual 6, terminal)
    # eta''=3: 3 users; users [0,1]: undefined -> residual of the eta'=1 group
    assert sizes == [2, 6, 3]
    assert meta[:, 1].tolist() == [1, 2, 2]
    assert meta[:, 2].tolist() == [1, 1, 0]


# ------------------------------------------------------------------ invariants + brute force
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_c2_with_one_bucket_is_exact_brute_force(seed):
    # t=1, b=1: every user has key 0, one cluster; with N >= n nothing splits and
    # C^2 reduces to exact brute force.
    ptr, items = synth.random_profiles(120, 60, 8, seed)
    sets = sets_from_csr(ptr, items)
    k = 7
    nid, nin, nun, pairs = oracle.build_graph(ptr, items, 60, k, 1, 1, 1000, seed, 10 ** 9)
    got = rows_of(nid, nin, nun)
    for u in range(120):
        assert got[u] == py_topk(sets, u, range(120), k)
    assert pairs == 120 * 119 // 2


def test_bruteforce_matches_sets():
    ptr, items = synth.random_profiles(80, 40, 6, 11)
    sets = sets_from_csr(ptr, items)
    nid, nin, nun = oracle.bruteforce_knn(ptr, items, 5)
    got = rows_of(nid, nin, nun)
    for u in range(80):
        assert got[u] == py_topk(sets, u, range(80), 5)
    q = np.array([3, 17, 42], np.int32)
    qid, qin, qun = oracle.bruteforce_knn(ptr, items, 5, q)
    assert rows_of(qid, qin, qun) == [got[3], got[17], got[42]]


def _check_invariants(ptr, items, m, t, b, N, seed):
    n = ptr.size - 1
    cl = oracle.frh_cluster(ptr, items, m, t, b, N, seed)
    cptr, cusers, co, meta = cl["cptr"], cl["cusers"], cl["cluster_of"], cl["cmeta"]
    nc = cl["n_clusters"]
    assert cptr[0] == 0 and cptr[-1] == t * n
    sizes = np.diff(cptr)
    assert (sizes > 0).all()
    # every user in exactly one cluster per function, so in exactly t clusters
    for i in range(t):
        lo, hi = i * n, (i + 1) * n
        assert sorted(cusers[lo:hi].tolist()) == list(range(n))
        fn_clusters = np.nonzero(meta[:, 0] == i)[0]
        assert cptr[fn_clusters[0]] == lo and cptr[fn_clusters[-1] + 1] == hi
    for c in range(nc):
        mem = cusers[cptr[c]:cptr[c + 1]]
        assert (np.diff(mem) > 0).all()                      # ascending ids
        assert (co[meta[c, 0], mem] == c).all()
        if not meta[c, 2]:
            assert mem.size <= N                             # non-residual <= N
    # FRH keys agree with the top-level path element
    keys = oracle.frh_keys(ptr, items, m, t, b, seed)
    for c in range(nc):
        mem = cusers[cptr[c]:cptr[c + 1]]
        if meta[c, 1] == 0:
            assert (keys[meta[c, 0], mem] == meta[c, 3]).all()
    return cl


@pytest.mark.parametrize("N", [5, 12, 40])
def test_clustering_invariants(N):
    ptr, items = synth.random_profiles(300, 50, 6, 5, zipf_s=1.2)
    _check_invariants(ptr, items, 50, 4, 8, N, 99)


@pytest.mark.parametrize("t, b, N", [(64, 2, 2), (3, 65536, 2), (1, 2, 300)])
def test_clustering_invariants_at_parameter_limits(t, b, N):
    # the library's limits: 64 functions, 2 and 65,536 buckets, the smallest
    # split limit (N = 2 recurses until every non-residual cluster is a pair)
    ptr, items = synth.random_profiles(200, 80, 5, 6, zipf_s=1.0)
    _check_invariants(ptr, items, 80, t, b, N, 7)


def test_split_children_share_prefix_keys():
    # every member of a depth-d cluster has, as its d+1 smallest distinct hash
    # values, exactly the cluster's path (Section II-D: H\eta keeps values > eta)
    ptr, items = synth.random_profiles(400, 60, 7, 8, zipf_s=1.3)
    m, t, b, N, seed = 60, 3, 6, 10, 5
    cl = _check_invariants(ptr, items, m, t, b, N, seed)
    sets = sets_from_csr(ptr, items)
    htab = np.array([[oracle.item_hash(seed, i, x, b) for x in range(m)] for i in range(t)])
    for c in range(cl["n_clusters"]):
        fn, depth, resid, last = cl["cmeta"][c]
        mem = cl["cusers"][cl["cptr"][c]:cl["cptr"][c + 1]]
        for u in mem:
            hv = sorted({int(htab[fn, x]) for x in sets[u]})
            assert hv[depth] == last
            if not resid and depth > 0:
                assert len(hv) > depth


def test_local_knn_brute_force_per_cluster():
    ptr, items = synth.random_profiles(200, 40, 6, 21)
    sets = sets_from_csr(ptr, items)
    cl = oracle.frh_cluster(ptr, items, 40, 3, 4, 30, 3)
    k = 6
    li, lc, lu, pairs = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 3, 10 ** 9)
    got = rows_of(li, lc, lu)
    exp_pairs = 0
    for c in range(cl["n_clusters"]):
        mem = cl["cusers"][cl["cptr"][c]:cl["cptr"][c + 1]].tolist()
        exp_pairs += len(mem) * (len(mem) - 1) // 2
        for a, u in enumerate(mem):
            assert got[cl["cptr"][c] + a] == py_topk(sets, u, mem, k)
    assert pairs == exp_pairs


def test_merge_is_topk_of_union():
    ptr, items = synth.random_profiles(150, 40, 6, 4)
    sets = sets_from_csr(ptr, items)
    t, k = 4, 5
    cl = oracle.frh_cluster(ptr, items, 40, t, 4, 25, 8)
    li, lc, lu, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 8, 10 ** 9)
    nid, nin, nun = oracle.merge_topk(cl["cptr"], cl["cusers"], 150, k, li, lc, lu)
    got = rows_of(nid, nin, nun)
    # union of the t clusters' members is the candidate set
    co = cl["cluster_of"]
    for u in range(150):
        cand = set()
        for i in range(t):
            c = co[i, u]
            cand |= set(cl["cusers"][cl["cptr"][c]:cl["cptr"][c + 1]].tolist())
        assert got[u] == py_topk(sets, u, sorted(cand), k)


def test_merge_idempotent_on_copies():
    # merging t copies of one list gives that list back (Algorithm 3, dedupe)
    k, n = 4, 3
    base = np.array([[1, 2, -1, -1], [0, -1, -1, -1], [0, 1, -1, -1]], np.int32)
    inter = np.array([[3, 1, 0, 0], [3, 0, 0, 0], [1, 1, 0, 0]], np.int32)
    uni = np.array([[5, 6, 0, 0], [5, 0, 0, 0], [6, 6, 0, 0]], np.int32)
    t = 3
    cptr = np.arange(0, t * n + 1, n, dtype=np.int32)
    cusers = np.tile(np.arange(n, dtype=np.int32), t)
    li, lc, lu = np.tile(base, (t, 1)), np.tile(inter, (t, 1)), np.tile(uni, (t, 1))
    nid, nin, nun = oracle.merge_topk(cptr, cusers, n, k, li, lc, lu)
    assert (nid == base).all() and (nin == inter).all() and (nun == uni).all()


# ------------------------------------------------------------------ greedy
def test_greedy_equals_brute_force_when_cluster_fits_in_k():
    # with M <= k+1 the random start already holds every other member
    ptr, items = synth.random_profiles(40, 30, 6, 33)
    sets = sets_from_csr(ptr, items)
    cl = oracle.frh_cluster(ptr, items, 30, 2, 8, 100, 2)
    k = 31
    sizes = np.diff(cl["cptr"])
    assert sizes.max() <= k + 1
    li, lc, lu, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 2, 2, 3)
    got = rows_of(li, lc, lu)
    for c in range(cl["n_clusters"]):
        mem = cl["cusers"][cl["cptr"][c]:cl["cptr"][c + 1]].tolist()
        for a, u in enumerate(mem):
            assert got[cl["cptr"][c] + a] == py_topk(sets, u, mem, k)


def test_greedy_lists_improve_with_rounds():
    # the current list is always a candidate, so every user's list can only improve
    ptr, items = synth.random_profiles(300, 80, 10, 44)
    cl = oracle.frh_cluster(ptr, items, 80, 1, 1, 1000, 1)    # one cluster of 300
    k = 8
    prev = None
    for R in range(0, 5):
        li, lc, lu, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 1, 2, R)
        sims = [sorted((Fraction(int(c), int(U)) for c, U in zip(lc[s], lu[s]) if U > 0),
                       reverse=True) for s in range(300)]
        if prev is not None:
            for a, b in zip(prev, sims):
                b = b + [Fraction(0)] * (k - len(b))
                a = a + [Fraction(0)] * (k - len(a))
                assert all(y >= x for x, y in zip(a, b))
        prev = sims


def test_greedy_random_start_draws_distinct_others():
    # rounds=0 keeps the random start (minus zero-similarity entries)
    rows = [[0, 1]] * 50                   # everybody shares everything -> all c > 0
    ptr, items = csr_from_sets(rows)
    cl = oracle.frh_cluster(ptr, items, 2, 1, 1, 1000, 9)
    k = 10
    li, lc, lu, pairs = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 9, 2, 0)
    assert pairs == 50 * k
    for s in range(50):
        row = li[s].tolist()
        assert len(set(row)) == k and s not in row and all(0 <= v < 50 for v in row)
        # equal similarities -> ascending ids
        assert row == sorted(row)
    # the draws follow the Philox words: check user 0's first draw by hand
    w = oracle.philox4x32_10([0, 0, 0, 0], [9, 0])[0]
    x = int(w) % 49
    assert x + (1 if x >= 0 else 0) in li[0].tolist()


def test_greedy_improves_over_random_start():
    ptr, items = synth.random_profiles(400, 100, 12, 55, zipf_s=1.1)
    cl = oracle.frh_cluster(ptr, items, 100, 1, 1, 1000, 1)
    k = 10
    _, lc0, lu0, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 1, 2, 0)
    _, lc5, lu5, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 1, 2, 5)
    _, lcb, lub, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, 1, 10 ** 9, 0)
    a0, a5, ab = oracle.avg_sim(lc0, lu0), oracle.avg_sim(lc5, lu5), oracle.avg_sim(lcb, lub)
    assert a0 < a5 <= ab
    assert a5 > 0.9 * ab


# ------------------------------------------------------------------ quality (Eq. 1-2)
def test_avg_sim_definition_and_quality_bound():
    nin = np.array([[1, 2], [0, 0]], np.int32)
    nun = np.array([[5, 4], [0, 0]], np.int32)
    assert math.isclose(oracle.avg_sim(nin, nun), (0.2 + 0.5) / 4)
    ptr, items = synth.random_profiles(150, 50, 7, 66)
    k = 5
    nid, nin, nun, _ = oracle.build_graph(ptr, items, 50, k, 3, 8, 20, 3, 10 ** 9)
    bid, bin_, bun = oracle.bruteforce_knn(ptr, items, k)
    q = oracle.avg_sim(nin, nun) / oracle.avg_sim(bin_, bun)
    assert 0 < q <= 1.0


# ------------------------------------------------------------------ Theorems 1-2
def test_theorem2_numeric_example_reading():
    g = golden("theorem2_example.json")
    ell, b = g["ell"], g["b"]
    mean = ell * (ell - 1) / (2 * b)

    def bound(d):
        dens = (1 + d) * (ell - 1) / (2 * b)
        p = 1 - (math.exp(d) / (1 + d) ** (1 + d)) ** mean
        return dens, 3 * dens, p

    lo, hi, p = bound(g["d_reading"])
    # the paper prints 3 x the rounded lower gap (3 x 0.078 = 0.234)
    assert round(lo, 3) == g["lower_gap"] and abs(hi - g["upper_gap"]) < 1e-3
    assert round(p, 3) == g["probability"]
    lo5, hi5, p5 = bound(g["d_printed"])
    assert round(p5, 2) == 0.58 and round(lo5, 3) == 0.047


def test_theorem1_cohash_probability_band():
    # Empirical P[H(u1) = H(u2)] over many generative functions lies within
    # J - kappa/ell and J + 3 kappa/ell (+ sampling slack), Theorem 1.
    b, ell = 4096, 256
    rng = np.random.default_rng(3)
    universe = rng.permutation(10000)[:ell]
    shared = 64
    p1 = sorted(universe[:shared].tolist() + universe[shared:shared + 96].tolist())
    p2 = sorted(universe[:shared].tolist() + universe[shared + 96:].tolist())
    assert len(set(p1) | set(p2)) == ell
    J = shared / ell
    ptr, items = csr_from_sets([p1, p2])
    t = 4000
    keys = oracle.frh_keys(ptr, items, 10000, t, b, 77)
    freq = (keys[:, 0] == keys[:, 1]).mean()
    # expected collision density (ell-1)/(2b); Theorem 2 with d = 1.5 bounds it by 0.078
    kappa = 0.078
    slack = 4 * math.sqrt(J * (1 - J) / t)
    assert J - kappa - slack <= freq <= J + 3 * kappa + slack
    assert abs(freq - J) < 0.05


# ------------------------------------------------------------------ input validation
def test_validate_csr():
    ptr, items = csr_from_sets([[0, 2], [1]])
    assert oracle.validate_csr(ptr, items, 3) == 0
    assert oracle.validate_csr(ptr, np.array([2, 0, 1], np.int32), 3) == 2     # unsorted
    assert oracle.validate_csr(ptr, np.array([0, 0, 1], np.int32), 3) == 2     # duplicate
    assert oracle.validate_csr(ptr, np.array([0, 3, 1], np.int32), 3) == 2     # out of range
    assert oracle.validate_csr(np.array([1, 2, 3], np.int32), items, 3) == 2   # ptr[0] != 0
    assert oracle.validate_csr(np.array([0, 2, 1], np.int32), items, 3) == 2   # decreasing


def test_empty_profiles_use_sentinel_bucket():
    ptr, items = csr_from_sets([[0], [], [1], []])
    keys = oracle.frh_keys(ptr, items, 2, 1, 4, 0, htab=np.array([[2, 3]], np.int32))
    assert keys[0].tolist() == [2, 4, 3, 4]
    cl = oracle.frh_cluster(ptr, items, 2, 1, 4, 1, 0, htab=np.array([[2, 3]], np.int32))
    assert np.diff(cl["cptr"]).tolist() == [1, 1, 2]
    assert cl["cusers"].tolist() == [0, 2, 1, 3]


# ------------------------------------------------------------------ learned proposer (oracle)
def test_given_keys_one_cluster_split_equals_frh_groups():
    # One learned cluster holding everybody, split once (N < n): its sub-clusters
    # are the FastRandomHash clusters of >= 2 users, the rest is the residual.
    ptr, items = synth.random_profiles(400, 60, 6, 31, zipf_s=1.3)
    m, t, b, seed = 60, 2, 16, 7
    keys = np.zeros((t, 400), np.int32)
    cl = oracle.frh_cluster(ptr, items, m, t, b, 399, seed, keys=keys)
    frh = oracle.frh_cluster(ptr, items, m, t, b, 10 ** 6, seed)
    for i in range(t):
        sub = cl["cmeta"][:, 0] == i
        meta = cl["cmeta"][sub]
        sizes = np.diff(cl["cptr"])[sub]
        fsub = frh["cmeta"][:, 0] == i
        fsizes = np.diff(frh["cptr"])[fsub]
        assert meta[0, 2] == 1 and meta[0, 3] == -1        # residual of the learned cluster
        assert sizes[0] == (fsizes == 1).sum()
        assert sorted(sizes[1:].tolist()) == sorted(fsizes[fsizes >= 2].tolist())
        assert (meta[1:, 3] == frh["cmeta"][fsub][fsizes >= 2, 3]).all()


def _tiny_net(seed):
    rng = np.random.default_rng(seed)
    cfg = dict(dim=32, hidden=16, t=2, b=8, rows_log2=6, seed=5)
    T = cfg["t"] * cfg["b"]
    params = [rng.normal(0, 0.3, (64, 32)).astype(np.float32),
              rng.normal(0, 0.3, (32, 16)).astype(np.float32),
              rng.normal(0, 0.1, 16).astype(np.float32),
              rng.normal(0, 0.3, (16, T)).astype(np.float32),
              rng.normal(0, 0.1, T).astype(np.float32)]
    return cfg, params


def test_model_gradient_matches_finite_differences():
    # the oracle's backward pass against central differences of its own loss
    # (plain FP64, no BF16 rounding)
    cfg, params = _tiny_net(1)
    ptr, items = synth.random_profiles(30, 50, 5, 9)
    pairs = np.array([[0, 1], [2, 3], [4, 9], [7, 7], [11, 20]], np.int32)
    lam = 0.3
    oracle.model_exact(True)
    try:
        loss, grads = oracle.model_grads(cfg, params, ptr, items, pairs, lam)
        rng = np.random.default_rng(3)
        h = 1e-4
        for pi in range(5):
            flat = params[pi].ravel()
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                p_plus = [x.astype(np.float64).copy() for x in params]
                p_minus = [x.astype(np.float64).copy() for x in params]
                p_plus[pi].ravel()[idx] += h
                p_minus[pi].ravel()[idx] -= h
                # the oracle takes FP32 parameters: use a step FP32 represents well
                lp, _ = oracle.model_grads(cfg, [x.astype(np.float32) for x in p_plus], ptr, items, pairs, lam)
                lm, _ = oracle.model_grads(cfg, [x.astype(np.float32) for x in p_minus], ptr, items, pairs, lam)
                dp = (np.float32(p_plus[pi].ravel()[idx]) - np.float32(p_minus[pi].ravel()[idx]))
                fd = (lp.sum() - lm.sum()) / float(dp)
                an = grads[pi].ravel()[idx]
                assert abs(fd - an) <= 2e-3 * max(1.0, abs(an)) + 1e-5, (pi, idx, fd, an)
    finally:
        oracle.model_exact(False)


def test_model_keys_are_argmax_of_logits():
    cfg, params = _tiny_net(2)
    ptr, items = synth.random_profiles(40, 50, 6, 10)
    z, keys = oracle.model_forward(cfg, params, ptr, items)
    b = cfg["b"]
    for j in range(cfg["t"]):
        assert (keys[j] == np.argmax(z[:, j * b:(j + 1) * b], axis=1)).all()


# ------------------------------------------------------------------ MinHash variant
def test_minhash_keys_are_profile_items():
    # Section V-C / Table 4 variant: one cluster per item, the key is an item
    # of the user's own profile (m for an empty profile)
    ptr, items = synth.random_profiles(300, 500, 12, 51)
    ptr = np.concatenate([ptr, [ptr[-1]]])            # an empty last profile
    keys = oracle.minhash_keys(ptr, items, 500, 6, 3)
    n = ptr.size - 1
    for i in range(6):
        for u in range(n - 1):
            assert keys[i, u] in set(items[ptr[u]:ptr[u + 1]].tolist())
        assert keys[i, n - 1] == 500


def test_minhash_collision_rate_is_jaccard():
    # min-wise hashing (Broder, 1997): over random functions,
    # P[key(A) = key(B)] = |A n B| / |A u B|.  Three pairs, 4,000 functions:
    # J = 1/3, J = 9/11 and J = 0, each within 4.5 standard deviations.
    A = np.arange(0, 40)
    B = np.arange(20, 60)                 # |A n B| = 20, |A u B| = 60
    C_ = np.arange(0, 40)                 # a copy of A
    D = np.concatenate([np.arange(4, 40), np.arange(100, 104)])   # |C n D| = 36, |C u D| = 44
    E = np.arange(200, 240)               # disjoint from A
    rows = [A, B, C_, D, E]
    ptr = np.concatenate([[0], np.cumsum([r.size for r in rows])]).astype(np.int32)
    items = np.concatenate(rows).astype(np.int32)
    T = 4000
    keys = oracle.minhash_keys(ptr, items, 300, T, 12345)
    for (a, b), J in (((0, 1), 20 / 60), ((2, 3), 36 / 44), ((0, 4), 0.0)):
        freq = float((keys[:, a] == keys[:, b]).mean())
        sd = math.sqrt(max(J * (1 - J), 1e-12) / T)
        assert abs(freq - J) <= 4.5 * sd + 1e-12, (a, b, freq, J)
    # identical profiles always share the key
    assert (keys[:, 0] == keys[:, 2]).all()


# ------------------------------------------------------------------ greedy rounds, restated
def py_greedy(sets, members, cluster_no, k, seed, rounds, n_random):
    """Independent restatement of the synchronous greedy refinement (R11) with
    Python sets and exact Fractions.  Philox4x32-10 words are the only part
    taken from the oracle (the random source).  Returns the emitted rows
    [(id, inter, union)] per member and the method's evaluation count (R13):
    the random start's draws plus, per round, the candidates not already in
    the member's list."""
    M = len(members)
    key = [seed & 0xFFFFFFFF, seed >> 32]

    def draw(a, r, j):
        w = int(oracle.philox4x32_10([cluster_no, a, r, j], key)[0])
        x = w % (M - 1)
        return x + (1 if x >= a else 0)

    def rank(a, v):   # best first: larger Jaccard, then lower user id
        A, B = sets[members[a]], sets[members[v]]
        U = len(A | B)
        return (-(Fraction(len(A & B), U) if U else Fraction(0)), members[v])

    evals = 0
    cur = []
    for a in range(M):
        drawn, j = [], 0
        while len(drawn) < min(k, M - 1):
            v = draw(a, 0, j)
            if v not in drawn:
                drawn.append(v)
            j += 1
        evals += len(drawn)
        cur.append(sorted(drawn, key=lambda v: rank(a, v)))
    for r in range(1, rounds + 1):
        nxt = []
        for a in range(M):           # every member reads the previous round's lists
            cand = set(cur[a])
            for v in cur[a]:
                cand |= set(cur[v])
            cand |= {draw(a, r, j) for j in range(n_random)}
            cand.discard(a)
            evals += len(cand - set(cur[a]))
            nxt.append(sorted(cand, key=lambda v: rank(a, v))[:k])
        cur = nxt
    rows = []
    for a in range(M):
        A = sets[members[a]]
        row = []
        for v in cur[a]:
            B = sets[members[v]]
            c = len(A & B)
            if c > 0:
                row.append((members[v], c, len(A | B)))
        rows.append(row)
    return rows, evals


@pytest.mark.parametrize("rounds,n_random", [(1, 0), (2, 0), (3, 0), (2, 2), (3, 1)])
def test_greedy_rounds_match_set_restatement(rounds, n_random):
    # three greedy clusters of 23, 31 and 17 members over disjoint users,
    # numbered 0, 1, 2 (the cluster number enters the Philox counter)
    ptr, items = synth.random_profiles(71, 40, 7, 61, zipf_s=1.1)
    sets = sets_from_csr(ptr, items)
    rng = np.random.default_rng(7)
    perm = rng.permutation(71)
    groups = [np.sort(perm[:23]), np.sort(perm[23:54]), np.sort(perm[54:])]
    cptr = np.array([0, 23, 54, 71], np.int32)
    cusers = np.concatenate(groups).astype(np.int32)
    k, seed = 4, 0x1234_5678_9ABC
    li, lc, lu, pairs = oracle.cluster_knn(ptr, items, cptr, cusers, k, seed, 10, rounds, n_random)
    got = rows_of(li, lc, lu)
    total = 0
    for c, mem in enumerate(groups):
        rows, evals = py_greedy(sets, mem.tolist(), c, k, seed, rounds, n_random)
        total += evals
        for a in range(len(mem)):
            assert got[cptr[c] + a] == rows[a], (c, a)
    assert pairs == total


def test_greedy_pins_fail_on_planted_mistakes():
    # the restatement is sensitive to the mistakes it exists to catch: an
    # asynchronous update, a candidate set missing a neighbour's list, and an
    # evaluation count that includes listed ids each change rows or counts
    ptr, items = synth.random_profiles(40, 30, 6, 62, zipf_s=1.1)
    sets = sets_from_csr(ptr, items)
    mem = list(range(40))
    ref_rows, ref_evals = py_greedy(sets, mem, 0, 4, 99, 3, 0)

    def variant(async_update=False, skip_last=False, count_all=False):
        key = [99, 0]

        def draw(a, r, j):
            x = int(oracle.philox4x32_10([0, a, r, j], key)[0]) % 39
            return x + (1 if x >= a else 0)

        def rank(a, v):
            A, B = sets[a], sets[v]
            U = len(A | B)
            return (-(Fraction(len(A & B), U) if U else Fraction(0)), v)

        evals, cur = 0, []
        for a in range(40):
            drawn, j = [], 0
            while len(drawn) < 4:
                v = draw(a, 0, j)
                if v not in drawn:
                    drawn.append(v)
                j += 1
            evals += 4
            cur.append(sorted(drawn, key=lambda v: rank(a, v)))
        for r in range(1, 4):
            src = cur if async_update else [list(x) for x in cur]
            nxt = cur if async_update else [None] * 40
            for a in range(40):
                cand = set(src[a])
                for v in (src[a][:-1] if skip_last else src[a]):
                    cand |= set(src[v])
                cand.discard(a)
                evals += len(cand) if count_all else len(cand - set(src[a]))
                nxt[a] = sorted(cand, key=lambda v: rank(a, v))[:4]
            cur = nxt
        rows = [[(v, len(sets[a] & sets[v]), len(sets[a] | sets[v])) for v in cur[a]
                 if sets[a] & sets[v]] for a in range(40)]
        return rows, evals

    assert variant() == (ref_rows, ref_evals)
    for kw in (dict(async_update=True), dict(skip_last=True), dict(count_all=True)):
        assert variant(**kw) != (ref_rows, ref_evals), kw


# ------------------------------------------------------------------ learned forward, restated
def _splitmix64_mix(z):
    """SplitMix64's output function (Steele, Lea & Flood, OOPSLA 2014)."""
    m = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _bf16(x):
    """Round to the nearest BF16 value, ties to even (through torch's conversion)."""
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).double().numpy()


def np_forward(cfg, params, ptr, items, bf16):
    """The proposer's network in NumPy: bag of hashed embedding rows, ReLU
    hidden layer, logits; BF16 rounding where the library stores BF16."""
    E, W1, b1, W2, b2 = (np.asarray(x, np.float64) for x in params)
    rnd = _bf16 if bf16 else (lambda x: np.asarray(x, np.float64))
    E, W1, W2 = rnd(E), rnd(W1), rnd(W2)
    rows = 1 << cfg["rows_log2"]
    n = ptr.size - 1
    e = np.zeros((n, cfg["dim"]))
    for u in range(n):
        for x in items[ptr[u]:ptr[u + 1]]:
            e[u] += E[_splitmix64_mix(cfg["seed"] ^ int(x)) & (rows - 1)]
    e = rnd(e.astype(np.float32)) if bf16 else e
    h = np.maximum(e @ W1 + np.asarray(params[2], np.float64), 0.0)
    h = rnd(h.astype(np.float32)) if bf16 else h
    return h @ W2 + np.asarray(params[4], np.float64)


@pytest.mark.parametrize("exact", [True, False])
def test_model_forward_matches_numpy_restatement(exact):
    cfg, params = _tiny_net(3)
    ptr, items = synth.random_profiles(50, 70, 6, 11)
    assert all(_splitmix64_mix(z) == oracle.mix64(z) for z in (0, 1, 12345, (1 << 64) - 1))
    oracle.model_exact(exact)
    try:
        z, keys = oracle.model_forward(cfg, params, ptr, items)
    finally:
        oracle.model_exact(False)
    zn = np_forward(cfg, params, ptr, items, bf16=not exact)
    assert np.allclose(z, zn, rtol=1e-12, atol=1e-12)
    b = cfg["b"]
    for j in range(cfg["t"]):
        assert (keys[j] == np.argmax(zn[:, j * b:(j + 1) * b], axis=1)).all()


# ------------------------------------------------------------------ GoldFinger (R17)
def test_goldfinger_fingerprints_are_bit_sets_of_the_profile():
    # F_u is a set of bits in [0, B), no larger than the profile; the
    # fingerprint of a union is the union of the fingerprints (one bit per
    # item); an empty profile has an empty fingerprint
    rows = [[1, 5, 9, 40], [5, 9, 77], [1, 5, 9, 40, 77], [], list(range(300))]
    ptr, items = csr_from_sets(rows)
    for B in (16, 64, 1024):
        fp, fi = oracle.goldfinger(ptr, items, B, 11)
        F = sets_from_csr(fp, fi)
        for u, r in enumerate(rows):
            row = fi[fp[u]:fp[u + 1]]
            assert (np.diff(row) > 0).all() and (row >= 0).all() and (row < B).all()
            assert len(F[u]) <= min(len(r), B)
        assert F[2] == F[0] | F[1] and F[3] == set()
        if B == 16:
            assert F[4] == set(range(16))     # 300 items fill 16 bits


def test_goldfinger_bit_occupancy_matches_balls_in_bins():
    # over random seeds each item's bit is uniform on [0, B) and items are
    # independent: E|F| = B (1 - (1 - 1/B)^L) for a profile of L items, and two
    # items share a bit with probability 1/B
    L, B, S = 50, 64, 3000
    ptr, items = csr_from_sets([list(range(L))])
    sizes = [np.diff(oracle.goldfinger(ptr, items, B, s)[0])[0] for s in range(S)]
    expect = B * (1 - (1 - 1 / B) ** L)
    se = np.std(sizes) / np.sqrt(S)
    assert abs(np.mean(sizes) - expect) < 5 * se + 0.05, (np.mean(sizes), expect)
    ptr2, items2 = csr_from_sets([[3, 8]])
    same = sum(np.diff(oracle.goldfinger(ptr2, items2, B, s)[0])[0] == 1 for s in range(S))
    p = 1 / B
    assert abs(same / S - p) < 5 * np.sqrt(p * (1 - p) / S), same / S


def test_goldfinger_without_collisions_gives_the_exact_graph():
    # with B = 2^22 bits the 1,000 items of these profiles land on distinct
    # bits, so every estimate equals the exact Jaccard value: the build on
    # fingerprints equals the exact build, counts included
    ptr, items = synth.random_profiles(600, 1000, 15, 71, zipf_s=1.1)
    B, seed = 1 << 22, 5
    alli = np.arange(1000, dtype=np.int32)
    fpa, fia = oracle.goldfinger(np.array([0, 1000], np.int32), alli, B, seed)
    assert fpa[1] == 1000                  # no two items share a bit
    fp, fi = oracle.goldfinger(ptr, items, B, seed)
    k, t, b, N, thr = 8, 3, 16, 200, 120
    exact = oracle.build_graph(ptr, items, 1000, k, t, b, N, seed, thr, 3)
    est = oracle.build_graph_sim(ptr, items, 1000, fp, fi, k, t, b, N, seed, thr, 3)
    for a, e in zip(exact, est):
        assert np.array_equal(np.asarray(a), np.asarray(e))


def test_exact_counts_of_given_rows():
    ptr, items = synth.random_profiles(80, 60, 8, 72)
    sets = sets_from_csr(ptr, items)
    rng = np.random.default_rng(3)
    ids = rng.integers(-1, 80, (80, 5)).astype(np.int32)
    inter, uni = oracle.exact_counts(ptr, items, ids)
    for u in range(80):
        for j in range(5):
            v = ids[u, j]
            if v < 0:
                assert inter[u, j] == 0 and uni[u, j] == 0
            else:
                assert inter[u, j] == len(sets[u] & sets[v])
                assert uni[u, j] == len(sets[u] | sets[v])
