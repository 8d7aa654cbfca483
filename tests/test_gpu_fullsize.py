"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (default options, the workload's k, t, b, N, threshold).

The oracle checks what it can finish: the whole clustering (bit-exact), the
local rows of a seeded sample of clusters (brute-force and greedy), and the
merge of the GPU's own local rows; the final graph is also checked for the
invariants of the method.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def same(g, r, what):
    g = g.cpu().numpy() if hasattr(g, "cpu") else np.asarray(g)
    r = np.asarray(r)
    assert g.shape == r.shape, what
    bad = np.argwhere(g != r)
    assert bad.size == 0, f"{what}: {len(bad)} mismatches, first {tuple(bad[0])}"


def check_workload(c2, name, n_brute_sample, greedy_sample, merge_users=None):
    w = synth.WORKLOADS[name]
    ptr, items, _ = synth.load(name)
    n, m = w.n_users, w.n_items
    dptr, ditems = dev(ptr), dev(items)
    opts = c2.options(greedy_threshold=w.greedy_threshold, greedy_rounds=w.greedy_rounds)
    ws = c2.workspace(c2.workspace_size(n, items.size, m, w.k, w.t, w.b, w.N, opts), "cuda")
    # Step 1: whole clustering, bit-exact
    g = c2.c2_frh_cluster(dptr, ditems, m, w.t, w.b, w.N, w.seed, opts=opts, ws=ws)
    o = oracle.frh_cluster(ptr, items, m, w.t, w.b, w.N, w.seed)
    assert g["n_clusters"] == o["n_clusters"]
    same(g["cptr"], o["cptr"], "cptr")
    same(g["cusers"], o["cusers"], "cusers")
    same(g["cluster_of"], o["cluster_of"], "cluster_of")
    same(g["cmeta"], o["cmeta"], "cmeta")
    # Step 2: local rows, sampled clusters
    c2.c2_reset_status(ws)
    li, lc, lu = c2.c2_cluster_knn(dptr, ditems, m, w.t, g["cptr_full"], g["cusers"],
                                   g["n_clusters_dev"], w.k, w.seed, opts=opts, ws=ws)
    assert c2.c2_get_status(ws) == 0
    sizes = np.diff(o["cptr"])
    rng = np.random.default_rng(7)
    brute = np.nonzero((sizes >= 2) & (sizes < w.greedy_threshold))[0]
    greedy = np.nonzero((sizes >= 2) & (sizes >= w.greedy_threshold))[0]
    # spread the brute sample over sizes: half uniform, half the largest ones
    pick = list(rng.choice(brute, size=min(n_brute_sample // 2, brute.size), replace=False))
    pick += list(brute[np.argsort(sizes[brute])[-(n_brute_sample // 2):]])
    if greedy.size and greedy_sample:
        pick += list(greedy[np.argsort(sizes[greedy])[:greedy_sample]])
    only = np.zeros(o["n_clusters"], np.uint8)
    only[np.array(pick, dtype=np.int64)] = 1
    ri, rc, ru, _ = oracle.cluster_knn(ptr, items, o["cptr"], o["cusers"], w.k, w.seed,
                                       w.greedy_threshold, w.greedy_rounds, 0, only=only)
    slots = np.concatenate([np.arange(o["cptr"][c], o["cptr"][c + 1]) for c in np.nonzero(only)[0]])
    same(li.cpu().numpy()[slots], ri[slots], "loc_id (sampled clusters)")
    same(lc.cpu().numpy()[slots], rc[slots], "loc_inter (sampled clusters)")
    same(lu.cpu().numpy()[slots], ru[slots], "loc_union (sampled clusters)")
    # Step 3: the GPU's local rows merged by the oracle (or checked on sampled users)
    nid, nin, nun = c2.c2_merge_topk(g["cusers"], n, w.t, w.k, li, lc, lu)
    li_h, lc_h, lu_h = li.cpu().numpy(), lc.cpu().numpy(), lu.cpu().numpy()
    if merge_users is None:
        rid, rin, run = oracle.merge_topk(o["cptr"], o["cusers"], n, w.k, li_h, lc_h, lu_h)
        same(nid, rid, "nbr_id")
        same(nin, rin, "nbr_inter")
        same(nun, run, "nbr_union")
    else:
        users = rng.choice(n, size=merge_users, replace=False)
        pos = np.empty(w.t * n, np.int64)
        for i in range(w.t):
            blk = o["cusers"][i * n:(i + 1) * n]
            pos[i * n + blk] = np.arange(i * n, (i + 1) * n)
        nid_h, nin_h = nid.cpu().numpy(), nin.cpu().numpy()
        from fractions import Fraction
        for u in users:
            cand = {}
            for i in range(w.t):
                s = pos[i * n + u]
                for j in range(w.k):
                    if li_h[s, j] >= 0:
                        cand[int(li_h[s, j])] = (int(lc_h[s, j]), int(lu_h[s, j]))
            best = sorted(cand.items(), key=lambda kv: (-Fraction(kv[1][0], kv[1][1]), kv[0]))[:w.k]
            assert [v for v, _ in best] == [int(x) for x in nid_h[u] if x >= 0]
            assert [cu[0] for _, cu in best] == [int(x) for x in nin_h[u][:len(best)]]
    # the whole build equals the three steps
    bid, bin_, bun = c2.c2_build_knn_graph(dptr, ditems, m, w.k, w.t, w.b, w.N, w.seed,
                                           opts=opts, ws=ws)
    same(bid, nid.cpu().numpy(), "build vs steps (id)")
    same(bun, nun.cpu().numpy(), "build vs steps (union)")
    # invariants of the final graph
    ids = bid.cpu().numpy()
    assert not np.any(ids == np.arange(n)[:, None]), "self edge"
    filled = ids >= 0
    srt = np.sort(np.where(filled, ids, -1 - np.arange(w.k)[None, :]), axis=1)
    assert not np.any((srt[:, 1:] == srt[:, :-1]) & (srt[:, 1:] >= 0)), "duplicate neighbour"
    assert np.all(filled[:, :-1] | ~filled[:, 1:]), "hole in a row"


def test_ml10m_like_full(c2):
    check_workload(c2, "ml10m_like", 40, 2)


def test_ml20m_like_full(c2):
    check_workload(c2, "ml20m_like", 40, 0)


@pytest.mark.slow
def test_sparse_wide_1m_full(c2):
    check_workload(c2, "sparse_wide_1m", 40, 1, merge_users=300)
