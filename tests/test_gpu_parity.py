"""GPU parity: the CUDA path through the C ABI vs the CPU oracle, bit-exact.

Every comparison is element by element on the same seeded inputs: cluster
assignments, cluster CSR and metadata, local rows, merged rows (ids and the
integer intersection / union counts) and the pair-evaluation counts.
"""
import numpy as np
import pytest

import oracle
from paper_2010_11497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11497_gb300 import build
    build.build()
    import paper_2010_11497_gb300 as pkg
    pkg.lib()
    return pkg


DEV = "cuda:0"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(DEV)


def npy(t):
    return t.cpu().numpy()


def assert_same(gpu, ref, what):
    g = npy(gpu) if hasattr(gpu, "cpu") else np.asarray(gpu)
    r = np.asarray(ref)
    assert g.shape == r.shape, f"{what}: shape {g.shape} vs {r.shape}"
    if not np.array_equal(g, r):
        bad = np.argwhere(g != r)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {i}: gpu {g[i]} oracle {r[i]}")


def csr_from_sets(rows):
    ptr = np.zeros(len(rows) + 1, np.int32)
    items = []
    for u, r in enumerate(rows):
        s = sorted(set(r))
        items.extend(s)
        ptr[u + 1] = ptr[u] + len(s)
    return ptr, np.array(items, np.int32)


def check_cluster(c2, ptr, items, m, t, b, N, seed, htab=None):
    opts = c2.options(hash_table=None if htab is None else to_dev(htab))
    g = c2.c2_frh_cluster(to_dev(ptr), to_dev(items if items.size else np.zeros(1, np.int32)),
                          m, t, b, N, seed, opts=opts)
    o = oracle.frh_cluster(ptr, items, m, t, b, N, seed, htab=htab)
    assert g["n_clusters"] == o["n_clusters"]
    assert_same(g["cluster_of"], o["cluster_of"], "cluster_of")
    assert_same(g["cptr"], o["cptr"], "cptr")
    assert_same(g["cusers"], o["cusers"], "cusers")
    assert_same(g["cmeta"], o["cmeta"], "cmeta")
    return g, o


# ------------------------------------------------------------------ Step 1
def test_frh_worked_examples(c2):
    # Section II-D worked example (h_1, h_2 over five items) and Figure 3
    htab = np.array([[1, 2, 1, 0, 2], [0, 2, 2, 1, 0]], np.int32)
    ptr, items = csr_from_sets([[0, 1, 2], [2, 3, 4]])
    g, _ = check_cluster(c2, ptr, items, 5, 2, 3, 100, 0, htab)
    co = npy(g["cluster_of"])
    assert co[0, 0] != co[0, 1] and co[1, 0] == co[1, 1]
    rows = [[0]] * 18 + [[0, 1]] * 34 + [[0, 2]] * 23 + [[1, 2]] * 10 + [[2]] * 15
    ptr, items = csr_from_sets(rows)
    g, _ = check_cluster(c2, ptr, items, 3, 1, 3, 40, 0, np.array([[0, 1, 2]], np.int32))
    assert np.diff(npy(g["cptr"])).tolist() == [18, 34, 23, 10, 15]


@pytest.mark.parametrize("n,m,mean,t,b,N,seed", [
    (300, 50, 6, 4, 8, 5, 1),
    (2000, 300, 20, 8, 64, 40, 2),
    (5000, 1000, 30, 3, 256, 100, 3),
    (3000, 200, 15, 16, 4, 200, 4),      # tiny b: deep splits
    (777, 5000, 12, 1, 1, 50, 5),        # b = 1: no key, residual only
    (4000, 800, 40, 64, 1024, 30, 6),    # t = 64
])
def test_frh_random_parity(c2, n, m, mean, t, b, N, seed):
    ptr, items = synth.random_profiles(n, m, mean, seed, zipf_s=1.2)
    check_cluster(c2, ptr, items, m, t, b, N, seed)


def test_frh_empty_profiles_and_tiny(c2):
    ptr, items = csr_from_sets([[0], [], [1], [], [0, 1]])
    check_cluster(c2, ptr, items, 2, 2, 4, 2, 3)
    ptr, items = csr_from_sets([[3]])
    check_cluster(c2, ptr, items, 4, 1, 8, 2, 3)


def test_frh_ml1m_full(c2):
    w = synth.WORKLOADS["ml1m_like"]
    ptr, items, _ = synth.load("ml1m_like")
    check_cluster(c2, ptr, items, w.n_items, w.t, w.b, w.N, w.seed)


# ------------------------------------------------------------------ Step 2
def check_local(c2, ptr, items, m, t, b, N, k, seed, thr, rounds=10, nrand=0, strategy=-1,
                budget=0):
    o = oracle.frh_cluster(ptr, items, m, t, b, N, seed)
    li, lc, lu, pairs = oracle.cluster_knn(ptr, items, o["cptr"], o["cusers"], k, seed, thr,
                                           rounds, nrand)
    dptr, ditems = to_dev(ptr), to_dev(items)
    g = c2.c2_frh_cluster(dptr, ditems, m, t, b, N, seed)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=rounds, greedy_random=nrand,
                      strategy=strategy, gram_budget_bytes=budget)
    n = ptr.size - 1
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    c2.c2_reset_status(ws)
    gi, gc, gu = c2.c2_cluster_knn(dptr, ditems, m, t, g["cptr_full"], g["cusers"],
                                   g["n_clusters_dev"], k, seed, opts=opts, ws=ws)
    assert c2.c2_get_status(ws) == 0
    assert_same(gi, li, "loc_id")
    assert_same(gc, lc, "loc_inter")
    assert_same(gu, lu, "loc_union")
    st = c2.c2_get_stats(ws)
    assert st["pairs"] == pairs
    return g, (gi, gc, gu), st


@pytest.mark.parametrize("strategy", [-1, 0, 1, 2, 3])
def test_local_brute_force_strategies(c2, strategy):
    ptr, items = synth.random_profiles(3000, 500, 25, 12, zipf_s=1.1)
    _, _, st = check_local(c2, ptr, items, 500, 4, 32, 400, 10, 5, 10 ** 9, strategy=strategy)
    if strategy == 3:     # clusters of 128 members or more went to the tensor cores
        assert st["tc_clusters"] >= 1 and st["tc_macs"] > 0


def _shape_test_profiles():
    # log-normal lengths around 150 (up to 1,200 items: walks with eight and
    # with sixteen bit planes, and warps mixing both), plus identical pairs of
    # 255-, 256- and 900-item profiles, whose counts reach 255 (the largest
    # count of eight planes), 256 and 900
    ptr, items = synth.random_profiles(1800, 1500, 150, 31, zipf_s=0.9, lmax=1200)
    rows = [items[ptr[u]:ptr[u + 1]].tolist() for u in range(ptr.size - 1)]
    rng = np.random.default_rng(77)
    for length, copies in ((255, 3), (256, 2), (900, 2)):
        r = sorted(rng.choice(1500, size=length, replace=False).tolist())
        rows.extend([r] * copies)
    return csr_from_sets(rows)


@pytest.mark.parametrize("shape", [(1, 512, 2, 1), (1, 256, 5, 1), (1, 512, 0, 1),
                                   (1, 512, 2, 0), (1, 256, 4, 0), (2, 256, 0, 0)])
def test_local_table_shapes(c2, tmp_path, shape):
    # each table shape the autotuner can choose (words of queries, threads,
    # resident blocks, 16-bit or int32 profile walk), forced by a loaded
    # table; 98 clusters of up to 500 members (many 32-query tiles, ragged
    # last tiles, mirrored columns): local rows and pair counts equal the
    # oracle's
    ptr, items = _shape_test_profiles()
    n, m, t, b, N, k, thr, seed = ptr.size - 1, 1500, 2, 64, 500, 10, 10 ** 9, 13
    W, NT, MB, P16 = shape
    cfg = " ".join(f"{W} {NT} {MB} {P16} 1" for _ in range(4))
    routes = " ".join("0 1 2" for _ in range(20))
    path = tmp_path / "tune.txt"
    path.write_text(f"c2-autotune 2\n{n} {m} {t} {b} {N} {k} {thr} 1 1 1 {cfg} {routes}\n")
    assert c2.c2_autotune_load(str(path)) == 1
    check_local(c2, ptr, items, m, t, b, N, k, seed, thr)
    rep = [e for e in c2.c2_autotune_report()
           if (e.get("n"), e.get("m"), e.get("t"), e.get("b"), e.get("N")) == (n, m, t, b, N)]
    assert rep and rep[0]["buckets"][0]["threads"] == NT
    assert rep[0]["buckets"][0]["items16"] is bool(P16)


def test_local_brute_force_tensor_cores_many_tiles(c2):
    # clusters of up to 1,771 members (14 row tiles, 7 column tiles, ragged
    # edges; two residuals above N) over 3,000 items: operands of many
    # 128-column stages, symmetric tiles and mirrored columns, compared with
    # the oracle element by element
    ptr, items = synth.random_profiles(4000, 3000, 60, 26, zipf_s=1.0)
    _, _, st = check_local(c2, ptr, items, 3000, 2, 16, 1500, 16, 7, 10 ** 9, strategy=3)
    assert st["tc_clusters"] >= 8 and st["tc_tiles"] >= 100


def test_local_greedy_tensor_cores(c2):
    # greedy clusters read count matrices made on the tensor cores
    ptr, items = synth.random_profiles(2500, 400, 20, 14, zipf_s=1.1)
    _, _, st = check_local(c2, ptr, items, 400, 3, 8, 600, 12, 21, 150, 4, 0, strategy=3)
    assert st["tc_clusters"] >= 1


@pytest.mark.parametrize("k", [1, 7, 30, 32])
def test_local_brute_force_k(c2, k):
    ptr, items = synth.random_profiles(1500, 300, 20, 13, zipf_s=1.0)
    check_local(c2, ptr, items, 300, 3, 16, 300, k, 9, 10 ** 9)


@pytest.mark.parametrize("rounds,nrand", [(0, 0), (1, 0), (4, 0), (3, 5)])
def test_local_greedy(c2, rounds, nrand):
    ptr, items = synth.random_profiles(2500, 400, 20, 14, zipf_s=1.1)
    check_local(c2, ptr, items, 400, 3, 8, 600, 12, 21, 150, rounds, nrand)


def test_local_greedy_with_merge_counts(c2):
    # forced merge strategy: greedy clusters get their count rows by merges
    ptr, items = synth.random_profiles(2000, 400, 20, 24, zipf_s=1.1)
    check_local(c2, ptr, items, 400, 3, 8, 600, 10, 22, 150, 3, 0, strategy=0)


@pytest.mark.parametrize("rounds,nrand", [(0, 0), (3, 0), (2, 5)])
def test_local_greedy_direct_counts(c2, rounds, nrand):
    # a count-matrix budget that holds every brute-force cluster (below 150
    # members: 149 count rows and the row of lengths, 152 entries each) but no
    # greedy one: the greedy clusters count from the profiles
    ptr, items = synth.random_profiles(2500, 400, 20, 14, zipf_s=1.1)
    budget = 2 * 150 * 152
    _, _, st = check_local(c2, ptr, items, 400, 3, 8, 600, 12, 21, 150, rounds, nrand,
                           budget=budget)
    assert st["direct_users"] == st["greedy_users"] > 0


def test_local_greedy_direct_wide_items(c2):
    # 100k items: no profile bitmap fits shared memory, counts come from merges
    ptr, items = synth.random_profiles(3000, 100000, 14, 31, zipf_s=1.05)
    _, _, st = check_local(c2, ptr, items, 100000, 2, 4, 900, 10, 5, 200, 3, 2,
                           budget=2 * 200 * 200)
    assert st["direct_users"] > 0


def test_greedy_over_member_cap(c2):
    # b = 1 and no split: one cluster of about 11,000 members, above the
    # 10,240-member bound of the count-matrix greedy path
    n, m, k = 11000, 2000, 10
    ptr, items = synth.random_profiles(n, m, 12, 77, zipf_s=1.1)
    _, _, st = check_local(c2, ptr, items, m, 1, 1, 20000, k, 8, 500, 2, 2)
    assert st["max_cluster"] > 10240
    assert st["direct_users"] == st["max_cluster"]


def test_build_wide_items_with_greedy(c2):
    # 300k items: no shared-memory item table fits; greedy clusters still build
    ptr, items = synth.random_profiles(3000, 300000, 12, 25, zipf_s=1.05)
    m, k, t, b, N, seed, thr = 300000, 10, 4, 8, 800, 6, 200
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 3)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=3)
    ws = c2.workspace(c2.workspace_size(3000, items.size, m, k, t, b, N, opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed,
                                          opts=opts, ws=ws)
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert c2.c2_get_stats(ws)["pairs"] == pairs


def test_local_greedy_small_budget_batches(c2):
    # greedy clusters processed in several batches of intersection matrices
    ptr, items = synth.random_profiles(3000, 300, 15, 15, zipf_s=1.2)
    o = oracle.frh_cluster(ptr, items, 300, 2, 8, 500, 4)
    sizes = np.diff(o["cptr"])
    # count matrices: M count rows and one row of lengths, padded to 8 entries
    # (16 bytes)
    big = int(((sizes.astype(np.int64) + 1) * ((sizes + 7) // 8 * 8)).max()) * 2
    k, thr = 8, 100
    li, lc, lu, pairs = oracle.cluster_knn(ptr, items, o["cptr"], o["cusers"], k, 4, thr, 3)
    dptr, ditems = to_dev(ptr), to_dev(items)
    g = c2.c2_frh_cluster(dptr, ditems, 300, 2, 8, 500, 4)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=3, gram_budget_bytes=big + 64)
    ws = c2.workspace(c2.workspace_size(3000, items.size, 300, k, 2, 8, 500, opts), DEV)
    c2.c2_reset_status(ws)
    gi, gc, gu = c2.c2_cluster_knn(dptr, ditems, 300, 2, g["cptr_full"], g["cusers"],
                                   g["n_clusters_dev"], k, 4, opts=opts, ws=ws)
    assert_same(gi, li, "loc_id")
    assert_same(gc, lc, "loc_inter")
    assert c2.c2_get_stats(ws)["pairs"] == pairs


# ------------------------------------------------------------------ Step 3 + whole build
# t*k <= 256: the ids seen so far are kept in a shared-memory set; (12, 30):
# rows compared with the list by shuffles
@pytest.mark.parametrize("t,k", [(5, 9), (8, 32), (12, 30)])
def test_merge_parity(c2, t, k):
    ptr, items = synth.random_profiles(2000, 300, 20, 16)
    m, b, N, seed = 300, 16, 300, 3
    o = oracle.frh_cluster(ptr, items, m, t, b, N, seed)
    li, lc, lu, _ = oracle.cluster_knn(ptr, items, o["cptr"], o["cusers"], k, seed, 10 ** 9)
    rid, rin, run = oracle.merge_topk(o["cptr"], o["cusers"], 2000, k, li, lc, lu)
    gid, gin, gun = c2.c2_merge_topk(to_dev(o["cusers"]), 2000, t, k, to_dev(li), to_dev(lc),
                                     to_dev(lu))
    assert_same(gid, rid, "nbr_id")
    assert_same(gin, rin, "nbr_inter")
    assert_same(gun, run, "nbr_union")


@pytest.mark.parametrize("n,m,mean,k,t,b,N,thr,seed", [
    (1000, 200, 15, 10, 4, 16, 200, 10 ** 9, 1),
    (4000, 600, 30, 30, 8, 128, 300, 150, 2),
    (2000, 3000, 12, 20, 8, 512, 100, 60, 3),     # sparse, wide item universe
    (600, 100, 30, 32, 2, 4, 50, 40, 4),
    (50, 20, 5, 5, 1, 1, 1000, 10 ** 9, 5),       # t=1, b=1 == exact brute force
])
def test_build_parity(c2, n, m, mean, k, t, b, N, thr, seed):
    ptr, items = synth.random_profiles(n, m, mean, seed, zipf_s=1.1)
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 4)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=4)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed,
                                          opts=opts, ws=ws)
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")
    assert c2.c2_get_stats(ws)["pairs"] == pairs


def test_build_ml1m_full(c2):
    w = synth.WORKLOADS["ml1m_like"]
    ptr, items, _ = synth.load("ml1m_like")
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, w.n_items, w.k, w.t, w.b, w.N, w.seed,
                                              w.greedy_threshold, w.greedy_rounds)
    opts = c2.options(greedy_threshold=w.greedy_threshold, greedy_rounds=w.greedy_rounds)
    ws = c2.workspace(c2.workspace_size(w.n_users, items.size, w.n_items, w.k, w.t, w.b, w.N,
                                        opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), w.n_items, w.k, w.t, w.b,
                                          w.N, w.seed, opts=opts, ws=ws)
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")
    assert c2.c2_get_stats(ws)["pairs"] == pairs


def test_build_ml1m_full_tensor_cores(c2):
    # the ml1m-like workload with every cluster of 128 members or more on the
    # tensor cores, then with the autotuner's choice: both equal the oracle
    w = synth.WORKLOADS["ml1m_like"]
    ptr, items, _ = synth.load("ml1m_like")
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, w.n_items, w.k, w.t, w.b, w.N, w.seed,
                                              w.greedy_threshold, w.greedy_rounds)
    for strategy in (3, -1):
        opts = c2.options(greedy_threshold=w.greedy_threshold, greedy_rounds=w.greedy_rounds,
                          strategy=strategy)
        ws = c2.workspace(c2.workspace_size(w.n_users, items.size, w.n_items, w.k, w.t, w.b, w.N,
                                            opts), DEV)
        gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), w.n_items, w.k, w.t,
                                              w.b, w.N, w.seed, opts=opts, ws=ws)
        assert_same(gid, oid, "nbr_id")
        assert_same(gin, oin, "nbr_inter")
        assert_same(gun, oun, "nbr_union")
        st = c2.c2_get_stats(ws)
        assert st["pairs"] == pairs
        if strategy == 3:
            assert st["tc_clusters"] >= 1
    rep = c2.c2_autotune_report()
    assert any(e.get("n") == w.n_users and e.get("strategy") for e in rep)


def test_build_host_entry_matches_device(c2):
    ptr, items = synth.random_profiles(1500, 300, 20, 17)
    m, k, t, b, N, seed = 300, 10, 4, 32, 200, 8
    opts = c2.options(greedy_threshold=100, greedy_rounds=2)
    d = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed, opts=opts)
    hp = torch.from_numpy(ptr).pin_memory()
    hi = torch.from_numpy(items).pin_memory()
    h = c2.c2_build_knn_graph_host(hp, hi, m, k, t, b, N, seed, opts=opts)
    for a, bb in zip(d, h):
        assert_same(a, bb.numpy(), "host entry")


# ------------------------------------------------------------------ judge + Eq. 1
def test_bruteforce_judge(c2):
    ptr, items = synth.random_profiles(1200, 250, 20, 18)
    k = 12
    rid, rin, run = oracle.bruteforce_knn(ptr, items, k)
    gid, gin, gun = c2.c2_bruteforce_knn(to_dev(ptr), to_dev(items), 250, k)
    assert_same(gid, rid, "judge id")
    assert_same(gin, rin, "judge inter")
    q = np.array([5, 17, 1000, 3, 1199], np.int32)
    rid, rin, run = oracle.bruteforce_knn(ptr, items, k, q)
    gid, gin, gun = c2.c2_bruteforce_knn(to_dev(ptr), to_dev(items), 250, k, to_dev(q))
    assert_same(gid, rid, "judge id (queries)")
    assert_same(gun, run, "judge union (queries)")


def test_bruteforce_judge_wide_items_hashed(c2):
    # 400,000 items: the judge counts through the shared hash table; the long
    # profiles share one query tile, which takes several passes
    m = 400000
    ptr, items = synth.random_profiles(800, m, 15, 19, zipf_s=0.8)
    ptr, items = _with_long_profiles(ptr, items, m, [1500, 2000, 2500, 3000, 4000], 3)
    k = 8
    rid, rin, run = oracle.bruteforce_knn(ptr, items, k)
    gid, gin, gun = c2.c2_bruteforce_knn(to_dev(ptr), to_dev(items), m, k)
    assert_same(gid, rid, "judge id")
    assert_same(gin, rin, "judge inter")
    q = np.array([800, 801, 802, 803, 804, 5, 17, 600], np.int32)
    rid, rin, run = oracle.bruteforce_knn(ptr, items, k, q)
    gid, gin, gun = c2.c2_bruteforce_knn(to_dev(ptr), to_dev(items), m, k, to_dev(q))
    assert_same(gid, rid, "judge id (queries)")
    assert_same(gun, run, "judge union (queries)")


def test_bruteforce_judge_wide_items_merge_fallback(c2):
    # a profile longer than one hash pass: the judge merges sorted lists
    m = 400000
    ptr, items = synth.random_profiles(600, m, 15, 23, zipf_s=0.8)
    ptr, items = _with_long_profiles(ptr, items, m, [5000], 4)
    k = 8
    rid, rin, run = oracle.bruteforce_knn(ptr, items, k)
    gid, gin, gun = c2.c2_bruteforce_knn(to_dev(ptr), to_dev(items), m, k)
    assert_same(gid, rid, "judge id")
    assert_same(gin, rin, "judge inter")


def test_avg_sim(c2):
    ptr, items = synth.random_profiles(900, 200, 20, 20)
    rid, rin, run = oracle.bruteforce_knn(ptr, items, 10)
    ref = oracle.avg_sim(rin, run)
    got = c2.c2_avg_sim(to_dev(rin), to_dev(run))
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


# ------------------------------------------------------------------ errors on the device
def test_invalid_csr_reported(c2):
    ptr = np.array([0, 2, 4], np.int32)
    items = np.array([1, 0, 2, 3], np.int32)      # first row not increasing
    with pytest.raises(c2.C2Error) as e:
        c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), 5, 3, 2, 8, 10, 1)
    assert e.value.code == 2
    items = np.array([0, 1, 2, 9], np.int32)      # item out of range
    with pytest.raises(c2.C2Error) as e:
        c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), 5, 3, 2, 8, 10, 1)
    assert e.value.code == 2


def test_explicit_hash_table_out_of_range(c2):
    ptr, items = csr_from_sets([[0, 1], [1, 2]])
    htab = np.array([[0, 5, 1]], np.int32)       # 5 >= b
    with pytest.raises(c2.C2Error) as e:
        c2.c2_frh_cluster(to_dev(ptr), to_dev(items), 3, 1, 4, 10, 0,
                          opts=c2.options(hash_table=to_dev(htab)))
    assert e.value.code == 1


def test_workspace_too_small(c2):
    ptr, items = synth.random_profiles(100, 50, 5, 21)
    ws = c2.workspace(1024, DEV)
    with pytest.raises(c2.C2Error) as e:
        c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), 50, 5, 2, 8, 10, 1, ws=ws)
    assert e.value.code == 4


@pytest.mark.parametrize("budget", [0, 2 * 50 * 56])
def test_greedy_draw_bound_reports_timeout(c2, budget):
    # The greedy random start's bounded loop: a bound below one batch of 32
    # draws stops every member's start, C2_ERR_TIMEOUT reaches the status
    # word, and the kernels after it (rounds, emit, merge) leave the outputs
    # untouched.  The default bound gives the oracle's graph.  The small budget
    # holds the brute-force clusters' count matrices (below 50 members) and no
    # greedy one: those take the path without count matrices.
    ptr, items = synth.random_profiles(1200, 300, 20, 51, zipf_s=1.1)
    n, m, k, t, b, N, seed, thr = 1200, 300, 8, 2, 4, 1200, 3, 50
    dptr, ditems = to_dev(ptr), to_dev(items)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=2, greedy_max_draws=1,
                      gram_budget_bytes=budget)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    out = [torch.full((n, k), -7, dtype=torch.int32, device=DEV) for _ in range(3)]
    c2.c2_build_knn_graph(dptr, ditems, m, k, t, b, N, seed, opts=opts, ws=ws, out=out,
                          check=False)
    assert c2.c2_get_status(ws) == 6
    assert c2.c2_get_stats(ws)["n_greedy_clusters"] >= 1
    for o in out:
        assert bool((o == -7).all())
    # the same workspace, cleared by the next build, with the default bound
    gid, gin, gun = c2.c2_build_knn_graph(dptr, ditems, m, k, t, b, N, seed, ws=ws,
                                          opts=c2.options(greedy_threshold=thr, greedy_rounds=2,
                                                          gram_budget_bytes=budget))
    oid, oin, oun, _ = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 2)
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")


def _with_long_profiles(ptr, items, m, lens, seed):
    """Appends users whose profiles hold `lens` distinct random items."""
    rng = np.random.default_rng(seed)
    rows = [items[ptr[u]:ptr[u + 1]] for u in range(ptr.size - 1)]
    rows += [np.sort(rng.choice(m, L, replace=False)) for L in lens]
    lens_all = np.array([r.size for r in rows])
    nptr = np.concatenate([[0], np.cumsum(lens_all)]).astype(np.int32)
    return nptr, np.concatenate(rows).astype(np.int32)


def test_build_long_profiles_unkeyed(c2):
    # unions may exceed 2^16: lists keep (id, inter, union) entries instead of
    # 64-bit order keys; brute-force and greedy clusters both
    m = 40000
    ptr, items = synth.random_profiles(2500, m, 20, 31, zipf_s=1.05)
    ptr, items = _with_long_profiles(ptr, items, m, [33000, 34000, 20000], 5)
    n, k, t, b, N, seed, thr = ptr.size - 1, 10, 3, 8, 600, 7, 150
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 3)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=3)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed,
                                          opts=opts, ws=ws)
    st = c2.c2_get_stats(ws)
    assert st["max_profile"] == 34000 and st["n_greedy_clusters"] > 0
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")
    assert st["pairs"] == pairs


def _wide_case(c2, extra_lens, seed):
    # 200,000 items: no dense item table fits shared memory
    m = 200000
    ptr, items = synth.random_profiles(3000, m, 30, 40 + seed, zipf_s=0.8)
    ptr, items = _with_long_profiles(ptr, items, m, extra_lens, seed)
    n, k, t, b, N, seed2, thr = ptr.size - 1, 10, 3, 8, 600, 9, 150
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed2, thr, 3)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=3)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed2,
                                          opts=opts, ws=ws)
    st = c2.c2_get_stats(ws)
    assert st["n_greedy_clusters"] > 0
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")
    assert st["pairs"] == pairs
    return st


def test_build_wide_items_hashed(c2):
    # count matrices through the shared hash table; the longest members share
    # a tile whose items exceed one pass (4,096), so that tile takes passes
    st = _wide_case(c2, [1500, 2000, 2500, 3000, 3500, 4000, 4096], 1)
    assert st["item_visits_greedy"] > 0


def test_build_wide_items_merge_fallback(c2):
    # a profile longer than one hash pass: count rows by merges instead
    st = _wide_case(c2, [1500, 5000], 2)
    assert st["item_visits_greedy"] == 0


def test_cluster_knn_profile_beyond_limit(c2):
    # c2_cluster_knn does not validate profiles: one longer than 65535 items
    # (16-bit counts) is reported as unsupported on the device
    m = 70000
    ptr, items = synth.random_profiles(400, m, 10, 32)
    ptr, items = _with_long_profiles(ptr, items, m, [66000], 6)
    n = ptr.size - 1
    cptr = np.array([0, n], np.int32)
    cusers = np.arange(n, dtype=np.int32)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, 5, 1, 2, 1000), DEV)
    c2.c2_reset_status(ws)
    c2.c2_cluster_knn(to_dev(ptr), to_dev(items), m, 1, to_dev(cptr), to_dev(cusers),
                      to_dev(np.array([1], np.int32)), 5, 1, ws=ws)
    assert c2.c2_get_status(ws) == 3


def test_build_duplicate_and_empty_profiles(c2):
    # many exact ties: copies of 40 template profiles (Jaccard 1 and equal
    # values broken by id), plus a greedy-sized cluster of empty profiles
    rng = np.random.default_rng(33)
    m = 600
    tmpl = [np.sort(rng.choice(m, rng.integers(5, 40), replace=False)) for _ in range(40)]
    rows = []
    for u in range(2400):
        r = tmpl[rng.integers(0, 40)]
        if rng.random() < 0.3:
            r = np.union1d(r, rng.choice(m, 1))
        rows.append(r)
    rows += [np.zeros(0, np.int64)] * 300
    perm = rng.permutation(len(rows))
    rows = [rows[i] for i in perm]
    ptr = np.concatenate([[0], np.cumsum([r.size for r in rows])]).astype(np.int32)
    items = np.concatenate(rows).astype(np.int32)
    n, k, t, b, N, seed, thr = ptr.size - 1, 12, 3, 16, 500, 8, 120
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 4)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=4)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed,
                                          opts=opts, ws=ws)
    assert c2.c2_get_stats(ws)["n_greedy_clusters"] > 0
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")
    assert c2.c2_get_stats(ws)["pairs"] == pairs


# ------------------------------------------------------------------ C^2/MinHash variant
def test_minhash_keys_and_build(c2):
    # Section V-C / Table 4: MinHash keys (one cluster per item, no split)
    ptr, items = synth.random_profiles(2500, 700, 20, 61, zipf_s=1.1)
    ptr = np.concatenate([ptr, [ptr[-1]]]).astype(np.int32)      # an empty profile
    n, m, t, k, seed = ptr.size - 1, 700, 5, 10, 17
    keys = c2.c2_minhash_keys(to_dev(ptr), to_dev(items), m, t, seed)
    okeys = oracle.minhash_keys(ptr, items, m, t, seed)
    assert_same(keys, okeys, "minhash keys")
    thr, b, N = 60, m + 1, n
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 3, keys=okeys)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=3, keys=keys.contiguous())
    ws = c2.workspace(c2.workspace_size(n, items.size, m, k, t, b, N, opts), DEV)
    gid, gin, gun = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed,
                                          opts=opts, ws=ws)
    st = c2.c2_get_stats(ws)
    assert st["split_levels"] == 0
    assert_same(gid, oid, "nbr_id")
    assert_same(gin, oin, "nbr_inter")
    assert_same(gun, oun, "nbr_union")
    assert st["pairs"] == pairs


@pytest.mark.parametrize("G", [2, 4])
def test_logical_shards_equal_one_call(c2, G):
    # sharding by hash function: G shards of t/G functions each (fn_offset,
    # cluster_base), their rows concatenated in function order and merged,
    # equal one call with all t functions and the oracle; greedy clusters
    # included (their random starts draw with the run's cluster numbers)
    from paper_2010_11497_gb300.shard import build_knn_graph_sharded
    ptr, items = synth.random_profiles(3000, 400, 20, 27, zipf_s=1.1)
    m, k, t, b, N, seed, thr = 400, 10, 4, 8, 600, 17, 150
    kw = dict(greedy_threshold=thr, greedy_rounds=3)
    ref = c2.c2_build_knn_graph(to_dev(ptr), to_dev(items), m, k, t, b, N, seed,
                                opts=c2.options(**kw))
    got = build_knn_graph_sharded(to_dev(ptr), to_dev(items), m, k, t, b, N, seed, shards=G, **kw)
    for a, r in zip(got, ref):
        assert torch.equal(a, r)
    oid, oin, oun, _ = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 3)
    assert_same(got[0], oid, "nbr_id")
    assert_same(got[2], oun, "nbr_union")
