"""GoldFinger (Section II-F) on the GPU against the CPU oracle, bit-exact.

Fingerprints (CSR of set bits and packed rows), builds whose local KNN graphs
and merge use the fingerprints (shared-memory table, tensor cores on packed
rows), and the exact rescoring of a graph's rows.
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
    assert g.shape == r.shape, (what, g.shape, r.shape)
    bad = np.argwhere(g != r)
    assert bad.size == 0, f"{what}: {len(bad)} mismatches, first {tuple(bad[0])}"


@pytest.mark.parametrize("bits", [32, 1024, 8192])
def test_goldfinger_fingerprints_match_oracle(c2, bits):
    ptr, items = synth.random_profiles(2000, 5000, 40, 81, zipf_s=1.0)
    fptr, fitems, fbits = c2.c2_goldfinger(dev(ptr), dev(items), 5000, bits, 9, with_bits=True)
    optr, oitems = oracle.goldfinger(ptr, items, bits, 9)
    same(fptr, optr, "fp_ptr")
    same(fitems[:optr[-1]], oitems, "fp_items")
    # the packed rows hold the same bits
    words = fbits.cpu().numpy().view(np.uint32)
    for u in (0, 1, 777, 1999):
        got = [32 * w + b for w in range(bits // 32) for b in range(32) if (words[u, w] >> b) & 1]
        assert got == oitems[optr[u]:optr[u + 1]].tolist()


def _gf_build(c2, ptr, items, m, bits, k, t, b, N, seed, thr, rounds, strategy, with_bits):
    dptr, ditems = dev(ptr), dev(items)
    fptr, fitems, fbits = c2.c2_goldfinger(dptr, ditems, m, bits, seed, with_bits=with_bits)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=rounds, strategy=strategy,
                      sim=(fptr, fitems), sim_n_items=bits, sim_bits=fbits)
    ws = c2.workspace(c2.workspace_size(ptr.size - 1, items.size, m, k, t, b, N, opts), "cuda")
    out = c2.c2_build_knn_graph(dptr, ditems, m, k, t, b, N, seed, opts=opts, ws=ws)
    return out, c2.c2_get_stats(ws)


@pytest.mark.parametrize("strategy,with_bits", [(-1, False), (1, False), (3, True), (3, False)])
def test_goldfinger_build_matches_oracle(c2, strategy, with_bits):
    ptr, items = synth.random_profiles(4000, 3000, 60, 82, zipf_s=1.0)
    m, bits, k, t, b, N, seed, thr = 3000, 1024, 16, 3, 16, 1500, 4, 10 ** 9
    (gid, gin, gun), st = _gf_build(c2, ptr, items, m, bits, k, t, b, N, seed, thr, 3, strategy,
                                    with_bits)
    fp, fi = oracle.goldfinger(ptr, items, bits, seed)
    oid, oin, oun, pairs = oracle.build_graph_sim(ptr, items, m, fp, fi, k, t, b, N, seed, thr, 3)
    same(gid, oid, "nbr_id")
    same(gin, oin, "nbr_inter")
    same(gun, oun, "nbr_union")
    assert st["pairs"] == pairs
    if strategy == 3:
        assert st["tc_clusters"] >= 1


def test_goldfinger_greedy_on_tensor_cores_matches_oracle(c2):
    # greedy clusters whose count matrices come from packed fingerprint rows
    ptr, items = synth.random_profiles(3000, 600, 25, 83, zipf_s=1.1)
    m, bits, k, t, b, N, seed, thr = 600, 512, 12, 3, 8, 700, 21, 150
    (gid, gin, gun), st = _gf_build(c2, ptr, items, m, bits, k, t, b, N, seed, thr, 4, 3, True)
    fp, fi = oracle.goldfinger(ptr, items, bits, seed)
    oid, oin, oun, pairs = oracle.build_graph_sim(ptr, items, m, fp, fi, k, t, b, N, seed, thr, 4)
    same(gid, oid, "nbr_id")
    same(gun, oun, "nbr_union")
    assert st["pairs"] == pairs and st["tc_clusters"] >= 1 and st["n_greedy_clusters"] >= 1


def test_exact_counts_match_oracle(c2):
    ptr, items = synth.random_profiles(1500, 800, 30, 84)
    rng = np.random.default_rng(5)
    ids = rng.integers(-1, 1500, (1500, 20)).astype(np.int32)
    gin, gun = c2.c2_exact_counts(dev(ptr), dev(items), dev(ids))
    oin, oun = oracle.exact_counts(ptr, items, ids)
    same(gin, oin, "inter")
    same(gun, oun, "union")
