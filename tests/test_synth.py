"""CPU checks of the seeded synthetic workloads (the stand-ins for the paper's
datasets): shapes and statistics as declared, valid sets, reproducibility, the
Zipf rank sampler, and the community mixture's neighbourhood structure."""
import numpy as np
import pytest

from paper_2010_11497_gb300 import synth


@pytest.mark.parametrize("name, mean_len, lmax", [("ml1m_like", 95.0, 2300),
                                                  ("ml10m_like", 143.0, 10677)])
def test_workload_shapes_and_sets(name, mean_len, lmax):
    w = synth.WORKLOADS[name]
    ptr, items, man = synth.load(name)
    assert ptr.size == w.n_users + 1 and ptr[0] == 0
    L = np.diff(ptr.astype(np.int64))
    assert (L >= 20).all() and (L <= lmax).all()          # the paper keeps users with >= 20 items
    assert abs(L.mean() / mean_len - 1.0) < 0.03
    assert man["nnz"] == items.size == ptr[-1]
    assert items.min() >= 0 and items.max() < w.n_items
    # rows are sets: strictly increasing inside every row
    d = np.diff(items.astype(np.int64))
    row_start = np.zeros(items.size, bool)
    row_start[ptr[:-1][L > 0]] = True
    assert (d[~row_start[1:]] > 0).all()


def test_generation_is_seeded():
    a = synth.random_profiles(500, 300, 25, 7)
    b = synth.random_profiles(500, 300, 25, 7)
    c = synth.random_profiles(500, 300, 25, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


@pytest.mark.parametrize("s", [0.8, 1.0, 1.1])
def test_zipf_rank_sampler(s):
    # ranks drawn through the cumulative table follow P(r) = r^-s / H(m, s)
    m = 5000
    cdf = synth._zipf_cdf(m, s)
    rng = np.random.default_rng(3)
    r = np.searchsorted(cdf, rng.random(2_000_000), side="right")
    freq = np.bincount(r, minlength=m)[:20] / 2_000_000
    H = np.sum(np.arange(1, m + 1, dtype=np.float64) ** -s)
    want = np.arange(1, 21, dtype=np.float64) ** -s / H
    assert np.all(np.abs(freq / want - 1.0) < 0.05)


def test_head_items_are_the_most_frequent():
    w = synth.WORKLOADS["ml10m_like"]
    ptr, items, _ = synth.load("ml10m_like")
    by_rank = np.bincount(items, minlength=w.n_items)[synth.world_permutation(w.n_items)]
    assert by_rank[0] == by_rank.max()
    assert by_rank[0] > by_rank[9] > by_rank[99] > by_rank[999] > by_rank[9999]


def _contrast(ptr, items):
    """Mean Jaccard of each user's nearest neighbour over the mean of all pairs."""
    n = ptr.size - 1
    rows = [set(items[ptr[u]:ptr[u + 1]].tolist()) for u in range(n)]
    J = np.zeros((n, n))
    for u in range(n):
        for v in range(u + 1, n):
            c = len(rows[u] & rows[v])
            J[u, v] = J[v, u] = c / (len(rows[u]) + len(rows[v]) - c)
    return J.max(1).mean() / (J.sum() / (n * (n - 1)))


def test_community_mixture_adds_neighbourhood_structure():
    # with mu > 0 users draw part of their items from their community's own
    # ranking: nearest neighbours stand out from the average pair far more than
    # under pure Zipf popularity, where every pair shares the same popular head
    plain = synth.random_profiles(300, 2000, 30, 11)
    comm = synth.random_profiles(300, 2000, 30, 11, mu=0.8, n_comm=8)
    assert _contrast(*comm) > 2.0 * _contrast(*plain)
