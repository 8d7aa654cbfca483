"""Seeded synthetic user/item profiles: the input workloads of the KNN-graph build.

This module only draws inputs.  It holds none of the method's arithmetic (no
hashing, clustering, similarity or ranking), so both the CUDA path and the CPU
oracle may consume what it produces.

The paper evaluates Cluster-and-Conquer on binarised rating datasets (Section IV-A,
Table 1: MovieLens 1M/10M/20M, AmazonMovies, DBLP, Gowalla).  Those datasets are
not available here; the generators below stand in for them with the same
numbers of users and items and a profile-length / item-popularity shape of the
same kind:

* every user draws a profile length ``L`` (log-normal or a continuous power law,
  floored, never below 20 -- the paper keeps only users with at least 20 ratings,
  Section IV-A), then ``L`` *distinct* items;
* the item of rank ``r`` (1-based) is drawn with probability proportional to
  ``r ** -s`` (Zipf popularity) and mapped to an item id through a fixed random
  permutation of the item universe (the "world", seeded by ``WORLD_SEED``);
* distinct items are drawn by rejection (draw with replacement, keep first
  occurrences, stop at ``L`` distinct) when ``L <= m / 8``, otherwise by
  weighted sampling without replacement after Efraimidis & Spirakis (2006):
  key ``U ** (1 / w)`` per item, keep the ``L`` largest keys.

Profiles are returned as CSR (``ptr[n+1]``, ``items[nnz]``, int32), each row
sorted increasingly and free of duplicates.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

WORLD_SEED = 2010


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload plus the C^2 parameters it is run with."""

    name: str
    n_users: int
    n_items: int
    length: tuple          # ("lognormal", mean, sigma, lmin, lmax) | ("powerlaw", a_or_None, mean, lmin, lmax_or_None, nnz_target_or_None)
    zipf_s: float
    seed: int
    k: int
    t: int
    b: int
    N: int
    greedy_threshold: int  # brute force iff |C| < greedy_threshold (Algorithm 2)
    greedy_rounds: int = 10

    def params(self) -> dict:
        return dict(k=self.k, t=self.t, b=self.b, N=self.N,
                    greedy_threshold=self.greedy_threshold,
                    greedy_rounds=self.greedy_rounds, seed=self.seed)


# The five workloads.  Sizes follow Table 1 (ml1M, ml10M, ml20M) or the
# sparse/wide and learned-proposer stress cases; parameters follow Section IV-C
# (k=30, t=8, b=4096, N=2000, rho=5 so rho*k^2 = 4500) unless stated.
WORKLOADS = {
    "ml1m_like": Workload(
        "ml1m_like", 6040, 3706, ("lognormal", 95.0, 1.0, 20, 2300), 1.0, 1,
        k=30, t=8, b=1024, N=2000, greedy_threshold=5 * 30 * 30),
    "ml10m_like": Workload(
        "ml10m_like", 69878, 10677, ("powerlaw", None, 143.0, 20, None, None), 1.1, 2,
        k=30, t=8, b=4096, N=2000, greedy_threshold=501),
    "ml20m_like": Workload(
        "ml20m_like", 138493, 26744, ("powerlaw", 1.8, None, 20, None, 20_000_000), 1.0, 3,
        k=30, t=8, b=4096, N=2000, greedy_threshold=5 * 30 * 30),
    "sparse_wide_1m": Workload(
        "sparse_wide_1m", 1_000_000, 1_300_000, ("lognormal", 60.0, 1.0, 20, 10000), 0.8, 4,
        k=20, t=8, b=8192, N=4000, greedy_threshold=5 * 20 * 20),
    # sparse_wide_1m's shape at a fifth of its users: small enough for a full
    # profiler capture of the hashed count-matrix kernel (a few GB on the device)
    "sparse_wide_200k": Workload(
        "sparse_wide_200k", 200_000, 1_300_000, ("lognormal", 60.0, 1.0, 20, 10000), 0.8, 4,
        k=20, t=8, b=8192, N=4000, greedy_threshold=5 * 20 * 20),
    "learned_ml20m": Workload(
        "learned_ml20m", 138493, 26744, ("powerlaw", 1.8, None, 20, None, 20_000_000), 1.0, 5,
        k=30, t=8, b=1024, N=2000, greedy_threshold=5 * 30 * 30),
}


# ---------------------------------------------------------------- lengths
def _lognormal_mu(mean_total: float, sigma: float, lmin: int, lmax: int) -> float:
    """mu such that E[min(lmax, lmin + round(LogNormal(mu, sigma)))] ~= mean_total."""
    rng = np.random.default_rng(12345)
    z = rng.standard_normal(400_000)

    def mean_of(mu):
        return np.minimum(lmax, lmin + np.rint(np.exp(mu + sigma * z))).mean()

    lo, hi = -5.0, 15.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if mean_of(mid) < mean_total:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _powerlaw_mean(a: float, lo: float, hi: float) -> float:
    """Mean of the continuous density proportional to x**-a on [lo, hi]."""
    def integ(p):  # integral of x**p on [lo, hi]
        if abs(p + 1.0) < 1e-12:
            return math.log(hi / lo)
        return (hi ** (p + 1) - lo ** (p + 1)) / (p + 1)
    return integ(1.0 - a) / integ(-a)


def _bisect(f, lo, hi, target, iters=200):
    flo = f(lo) - target
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid) - target
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _powerlaw_sample(rng, n, a, lo, hi):
    u = rng.random(n)
    if abs(a - 1.0) < 1e-12:
        x = lo * (hi / lo) ** u
    else:
        p = 1.0 - a
        x = (lo ** p + u * (hi ** p - lo ** p)) ** (1.0 / p)
    return np.floor(x).astype(np.int64)


def draw_lengths(w: Workload, rng) -> tuple[np.ndarray, dict]:
    kind = w.length[0]
    if kind == "lognormal":
        _, mean, sigma, lmin, lmax = w.length
        lmax = min(lmax, w.n_items)
        mu = _lognormal_mu(mean, sigma, lmin, lmax)
        L = np.minimum(lmax, lmin + np.rint(np.exp(mu + sigma * rng.standard_normal(w.n_users))))
        return L.astype(np.int64), {"mu": mu, "sigma": sigma}
    _, a, mean, lmin, lmax, nnz_target = w.length
    if a is None:        # exponent fitted so the mean is `mean` on [lmin, m]
        hi = float(w.n_items)
        a = _bisect(lambda s: -_powerlaw_mean(s, lmin, hi), 1.01, 4.0, -(mean + 0.5))
    else:                # upper cut fitted so the total is nnz_target
        target = nnz_target / w.n_users + 0.5
        hi = _bisect(lambda h: _powerlaw_mean(a, lmin, h), lmin + 1.0, float(w.n_items), target)
    L = _powerlaw_sample(rng, w.n_users, a, float(lmin), hi)
    L = np.clip(L, lmin, w.n_items)
    return L, {"a": a, "upper": hi}


# ---------------------------------------------------------------- items
def world_permutation(n_items: int) -> np.ndarray:
    """Fixed rank -> item-id map of an item universe of size n_items."""
    return np.random.default_rng([WORLD_SEED, n_items]).permutation(n_items).astype(np.int64)


def _zipf_cdf(n_items: int, s: float) -> np.ndarray:
    w = np.arange(1, n_items + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _expected_draws(cdf: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Draws D with E[#distinct after D draws] >= L, per user (coupon collector)."""
    p = np.diff(np.concatenate(([0.0], cdf)))
    grid = np.unique(np.rint(np.geomspace(1, 64.0 * cdf.size, 400))).astype(np.int64)
    ed = np.array([np.sum(-np.expm1(d * np.log1p(-np.minimum(p, 1 - 1e-16)))) for d in grid])
    j = np.searchsorted(ed, L, side="left")
    j = np.minimum(j, grid.size - 1)
    return grid[j]


def _first_distinct(users, ranks, m, L):
    """Stream (user-major, draw order) -> first L distinct ranks per user, and counts."""
    key = users * m + ranks
    _, first = np.unique(key, return_index=True)
    first.sort()
    ku, kr = users[first], ranks[first]
    n_local = np.bincount(ku, minlength=L.size)
    start = np.concatenate(([0], np.cumsum(n_local)[:-1]))
    idx = np.arange(ku.size) - start[ku]
    sel = idx < L[ku]
    return ku[sel], kr[sel], np.minimum(n_local, L)


def _rejection_rows(rng, L, cdf, to_id=None):
    """Per user: draw items with replacement, keep first occurrences, stop at L distinct.

    A draw picks a Zipf rank; to_id(users, ranks) maps it to an item id (the
    identity when None).  All users' streams are drawn at once (with a
    coupon-collector estimate of the draws needed); users still short get
    their stream extended and re-scanned.
    """
    n, m = L.shape[0], cdf.size
    to_id = to_id or (lambda u, r: r)
    D = np.where(L > 0, (_expected_draws(cdf, L) * 1.15).astype(np.int64) + 16, 0)
    users = np.repeat(np.arange(n, dtype=np.int64), D)
    ranks = to_id(users, np.minimum(np.searchsorted(cdf, rng.random(users.size), side="right"), m - 1))
    ku, kr, got = _first_distinct(users, ranks, m, L)
    short = np.nonzero(got < L)[0]
    if short.size == 0:
        return ku, kr
    keep = got >= L
    out_u, out_r = [ku[keep[ku]]], [kr[keep[ku]]]
    mask = np.isin(users, short)
    su, sr = users[mask], ranks[mask]
    extra = np.maximum(D[short], 64)
    while True:
        nu = np.repeat(short, extra)
        nr = to_id(nu, np.minimum(np.searchsorted(cdf, rng.random(nu.size), side="right"), m - 1))
        su = np.concatenate([su, nu])
        sr = np.concatenate([sr, nr])
        order = np.argsort(su, kind="stable")      # user-major, draw order kept
        su, sr = su[order], sr[order]
        ku, kr, got = _first_distinct(su, sr, m, L)
        done = got[short] >= L[short]
        fin = short[done]
        sel = np.isin(ku, fin)
        out_u.append(ku[sel])
        out_r.append(kr[sel])
        short = short[~done]
        if short.size == 0:
            break
        mask = np.isin(su, short)
        su, sr = su[mask], sr[mask]
        extra = np.maximum(2 * extra[~done], 64)
    return np.concatenate(out_u), np.concatenate(out_r)


def _es_rows(rng, users, L, weights):
    """Efraimidis-Spirakis weighted sampling without replacement, per user."""
    out_u, out_r = [], []
    logw = np.log(weights)
    for u, l in zip(users, L):
        # key = U^(1/w)  <=>  log key = log(U) / w ; larger is better
        keys = np.log(rng.random(weights.size)) / weights
        top = np.argpartition(-keys, l - 1)[:l]
        out_u.append(np.full(l, u, np.int64))
        out_r.append(top.astype(np.int64))
    del logw
    if not out_u:
        return np.empty(0, np.int64), np.empty(0, np.int64)
    return np.concatenate(out_u), np.concatenate(out_r)


def generate(w: Workload, seed: int | None = None, mu: float = 0.0, n_comm: int = 64):
    """Return (ptr int32[n+1], items int32[nnz], manifest dict) for workload w.

    mu > 0 adds neighbourhood structure: every user belongs to one of n_comm
    communities (uniformly), and each draw takes, with probability mu, its
    item from the community's own rank order (a fixed permutation per
    community, part of the world) instead of the global one."""
    seed = w.seed if seed is None else seed
    rng = np.random.default_rng([seed, 0xC2])
    L, fit = draw_lengths(w, rng)
    m = w.n_items
    perm = world_permutation(m)
    cdf = _zipf_cdf(m, w.zipf_s)
    small = L <= m // 8
    to_id = None
    if mu > 0:
        comm = rng.integers(0, n_comm, w.n_users)
        cperm = np.stack([np.random.default_rng([WORLD_SEED, m, c + 1]).permutation(m)
                          for c in range(n_comm)])

        def to_id(users, ranks, _rng=np.random.default_rng([seed, 0xC3])):
            local = _rng.random(users.size) < mu
            return np.where(local, cperm[comm[users], ranks], perm[ranks])
    us, rs = _rejection_rows(rng, np.where(small, L, 0), cdf, to_id)
    if to_id is None:
        rs = perm[rs]
    big = np.nonzero(~small)[0]
    if big.size:
        weights = np.arange(1, m + 1, dtype=np.float64) ** (-w.zipf_s)
        bu, br = _es_rows(rng, big, L[big], weights)
        us = np.concatenate([us, bu])
        rs = np.concatenate([rs, perm[br]])
    items = rs
    order = np.lexsort((items, us))
    us, items = us[order], items[order]
    counts = np.bincount(us, minlength=w.n_users)
    assert np.array_equal(counts, L), "generator produced a wrong row length"
    ptr = np.zeros(w.n_users + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    assert ptr[-1] < 2 ** 31
    manifest = dict(workload=w.name, seed=seed, n_users=w.n_users, n_items=m,
                    nnz=int(ptr[-1]), mean_len=float(L.mean()), max_len=int(L.max()),
                    min_len=int(L.min()), zipf_s=w.zipf_s, length=list(w.length), fit=fit)
    return ptr.astype(np.int32), items.astype(np.int32), manifest


def cache_dir() -> str:
    d = os.environ.get("C2_CACHE_DIR") or os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), ".c2_cache")
    os.makedirs(d, exist_ok=True)
    return d


def load(name: str, seed: int | None = None):
    """generate() with an on-disk cache keyed by workload name and seed."""
    w = WORKLOADS[name]
    seed = w.seed if seed is None else seed
    path = os.path.join(cache_dir(), f"{name}_s{seed}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        import json
        return z["ptr"], z["items"], json.loads(str(z["manifest"]))
    ptr, items, man = generate(w, seed)
    import json
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, ptr=ptr, items=items, manifest=json.dumps(man))
    os.replace(tmp, path)
    return ptr, items, man


def random_profiles(n_users: int, n_items: int, mean_len: float, seed: int,
                    zipf_s: float = 1.0, lmin: int = 1, lmax: int | None = None,
                    mu: float = 0.0, n_comm: int = 64):
    """Small random CSR for unit tests (log-normal lengths, Zipf items,
    optional community structure mu)."""
    lmax = n_items if lmax is None else min(lmax, n_items)
    w = Workload("adhoc", n_users, n_items, ("lognormal", float(mean_len), 0.8, lmin, lmax),
                 zipf_s, seed, k=1, t=1, b=2, N=2, greedy_threshold=2)
    ptr, items, _ = generate(w, seed, mu=mu, n_comm=n_comm)
    return ptr, items
