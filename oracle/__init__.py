"""ctypes front end of the CPU oracle (oracle.cpp) -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the library's product path never imports it.  ``build()`` compiles
``liboracle.so`` next to this file with the host C++ compiler.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
U32P = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _opt(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.oracle_mix64.restype = C.c_uint64
        L.oracle_mix64.argtypes = [C.c_uint64]
        L.oracle_item_hash.restype = C.c_uint32
        L.oracle_item_hash.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int32]
        L.oracle_philox4x32_10.argtypes = [U32P, U32P, U32P]
        L.oracle_validate_csr.argtypes = [I32P, I32P, C.c_int32, C.c_int32]
        L.oracle_frh_keys.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_uint64, C.c_void_p, I32P]
        L.oracle_minhash_keys.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_int32,
                                          C.c_uint64, I32P]
        L.oracle_frh_cluster.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_int32, C.c_uint64, C.c_void_p, C.c_void_p, I32P, I32P,
                                         I32P, I32P, C.c_void_p]
        L.oracle_cluster_knn.argtypes = [I32P, I32P, C.c_int32, I32P, I32P, C.c_int32, C.c_int32,
                                         C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                         I32P, I32P, I32P, I64P]
        L.oracle_merge_topk.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_int32, I32P, I32P,
                                        I32P, I32P, I32P, I32P]
        L.oracle_build.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_int32, C.c_uint64, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_void_p, C.c_void_p, I32P, I32P, I32P, I64P]
        F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        L.oracle_model_exact.argtypes = [C.c_int32]
        L.oracle_model_forward.argtypes = [C.c_int32] * 5 + [C.c_uint64] + [F32P] * 5 + \
            [I32P, I32P, C.c_int32, C.c_void_p, I32P]
        L.oracle_model_grads.argtypes = [C.c_int32] * 5 + [C.c_uint64] + [F32P] * 5 + \
            [I32P, I32P, C.c_int32, I32P, C.c_int32, C.c_double] + [F64P] * 6
        L.oracle_bruteforce_knn.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_void_p,
                                            C.c_int32, I32P, I32P, I32P]
        L.oracle_frh_cluster_shard.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_int32,
                                               C.c_int32, C.c_int32, C.c_uint64, C.c_int32, I32P,
                                               I32P, I32P, I32P]
        L.oracle_cluster_knn_shard.argtypes = [I32P, I32P, C.c_int32, I32P, I32P, C.c_int32,
                                               C.c_int32, C.c_uint64, C.c_int32, C.c_int32,
                                               C.c_int32, I32P, I32P, I32P, I64P]
        L.oracle_goldfinger.argtypes = [I32P, I32P, C.c_int32, C.c_int32, C.c_uint64, I32P, I32P]
        L.oracle_build_sim.argtypes = [I32P, I32P, C.c_int32, C.c_int32, I32P, I32P, C.c_int32,
                                       C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32,
                                       C.c_int32, C.c_int32, I32P, I32P, I32P, I64P]
        L.oracle_exact_counts.argtypes = [I32P, I32P, C.c_int32, C.c_int32, I32P, I32P, I32P]
        L.oracle_avg_sim.restype = C.c_double
        L.oracle_avg_sim.argtypes = [I32P, I32P, C.c_int32, C.c_int32]
        _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------------ wrappers
def mix64(z: int) -> int:
    return int(lib().oracle_mix64(z))


def item_hash(seed: int, i: int, x: int, b: int) -> int:
    return int(lib().oracle_item_hash(seed, i, x, b))


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def validate_csr(ptr, items, m) -> int:
    ptr, items = _i32(ptr), _i32(items)
    if items.size == 0:
        items = np.zeros(1, np.int32)
    return lib().oracle_validate_csr(ptr, items, ptr.size - 1, m)


def frh_keys(ptr, items, m, t, b, seed, htab=None):
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    keys = np.zeros((t, n), np.int32)
    ht = None if htab is None else _i32(htab)
    lib().oracle_frh_keys(ptr, items if items.size else np.zeros(1, np.int32), n, m, t, b, seed,
                          _opt(ht), keys)
    return keys


def minhash_keys(ptr, items, m, t, seed):
    """Keys [t][n] of the C^2/MinHash variant: per function, the item of the
    profile with the least 64-bit value (m for an empty profile)."""
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    keys = np.zeros((t, n), np.int32)
    lib().oracle_minhash_keys(ptr, items if items.size else np.zeros(1, np.int32), n, m, t, seed,
                              keys)
    return keys


def frh_cluster(ptr, items, m, t, b, N, seed, htab=None, keys=None):
    """Returns dict(cluster_of[t,n], cptr[nc+1], cusers[t*n], n_clusters, cmeta[nc,4]).

    keys: optional first-level keys [t][n] (a learned proposer) instead of FRH."""
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    cluster_of = np.zeros((t, n), np.int32)
    cptr = np.zeros(t * n + 1, np.int32)
    cusers = np.zeros(max(t * n, 1), np.int32)
    nc = np.zeros(1, np.int32)
    cmeta = np.zeros((max(t * n, 1), 4), np.int32)
    ht = None if htab is None else _i32(htab)
    ky = None if keys is None else _i32(keys)
    rc = lib().oracle_frh_cluster(ptr, items if items.size else np.zeros(1, np.int32), n, m, t, b,
                                  N, seed, _opt(ht), _opt(ky), cluster_of, cptr, cusers, nc,
                                  cmeta.ctypes.data_as(C.c_void_p))
    if rc:
        raise ValueError(f"oracle_frh_cluster failed with status {rc}")
    c = int(nc[0])
    return dict(cluster_of=cluster_of, cptr=cptr[:c + 1].copy(), cusers=cusers[:t * n].copy(),
                n_clusters=c, cmeta=cmeta[:c].copy())


def cluster_knn(ptr, items, cptr, cusers, k, seed, greedy_threshold, greedy_rounds=10,
                greedy_random=0, only=None):
    """Local KNN rows [t*n, k] per slot; `only` = bool mask of clusters to compute."""
    ptr, items, cptr, cusers = _i32(ptr), _i32(items), _i32(cptr), _i32(cusers)
    n = ptr.size - 1
    nc = cptr.size - 1
    S = cusers.size
    li = np.full((S, k), -1, np.int32)
    lc = np.zeros((S, k), np.int32)
    lu = np.zeros((S, k), np.int32)
    pairs = np.zeros(1, np.int64)
    mask = None if only is None else np.ascontiguousarray(only, dtype=np.uint8)
    lib().oracle_cluster_knn(ptr, items, n, cptr, cusers, nc, k, seed, greedy_threshold,
                             greedy_rounds, greedy_random,
                             None if mask is None else mask.ctypes.data_as(C.c_void_p),
                             li, lc, lu, pairs)
    return li, lc, lu, int(pairs[0])


def frh_cluster_shard(ptr, items, m, t, b, N, seed, fn_offset):
    """Clustering of a shard: the run's functions fn_offset .. fn_offset + t - 1,
    numbered locally.  Returns dict(cptr, cusers, n_clusters)."""
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    cluster_of = np.zeros(t * n, np.int32)
    cptr = np.zeros(t * n + 1, np.int32)
    cusers = np.zeros(max(t * n, 1), np.int32)
    nc = np.zeros(1, np.int32)
    rc = lib().oracle_frh_cluster_shard(ptr, items if items.size else np.zeros(1, np.int32), n, m,
                                        t, b, N, seed, fn_offset, cluster_of, cptr, cusers, nc)
    if rc:
        raise ValueError(f"oracle_frh_cluster_shard failed with status {rc}")
    c = int(nc[0])
    return dict(cptr=cptr[:c + 1].copy(), cusers=cusers[:t * n].copy(), n_clusters=c)


def cluster_knn_shard(ptr, items, cptr, cusers, k, seed, greedy_threshold, greedy_rounds,
                      cluster_base):
    """Local rows of a shard whose first cluster is the run's cluster_base."""
    ptr, items, cptr, cusers = _i32(ptr), _i32(items), _i32(cptr), _i32(cusers)
    S = cusers.size
    li = np.full((S, k), -1, np.int32)
    lc = np.zeros((S, k), np.int32)
    lu = np.zeros((S, k), np.int32)
    pairs = np.zeros(1, np.int64)
    lib().oracle_cluster_knn_shard(ptr, items, ptr.size - 1, cptr, cusers, cptr.size - 1, k, seed,
                                   greedy_threshold, greedy_rounds, cluster_base, li, lc, lu,
                                   pairs)
    return li, lc, lu, int(pairs[0])


def merge_topk(cptr, cusers, n, k, li, lc, lu):
    cptr, cusers = _i32(cptr), _i32(cusers)
    out = [np.zeros((n, k), np.int32) for _ in range(3)]
    lib().oracle_merge_topk(cptr, cusers, cptr.size - 1, n, k, _i32(li), _i32(lc), _i32(lu), *out)
    return tuple(out)


def build_graph(ptr, items, m, k, t, b, N, seed, greedy_threshold, greedy_rounds=10,
                greedy_random=0, htab=None, keys=None):
    """The whole method.  Returns (nbr_id, nbr_inter, nbr_union, pairs)."""
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    out = [np.zeros((n, k), np.int32) for _ in range(3)]
    pairs = np.zeros(1, np.int64)
    ht = None if htab is None else _i32(htab)
    ky = None if keys is None else _i32(keys)
    rc = lib().oracle_build(ptr, items, n, m, k, t, b, N, seed, greedy_threshold, greedy_rounds,
                            greedy_random, _opt(ht), _opt(ky), *out, pairs)
    if rc:
        raise ValueError(f"oracle_build failed with status {rc}")
    return out[0], out[1], out[2], int(pairs[0])


def goldfinger(ptr, items, bits, seed):
    """GoldFinger fingerprints (R17): CSR (fptr, fitems) of each user's sorted bit positions."""
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    fptr = np.zeros(n + 1, np.int32)
    fitems = np.zeros(max(items.size, 1), np.int32)
    rc = lib().oracle_goldfinger(ptr, items, n, bits, seed, fptr, fitems)
    if rc:
        raise ValueError(f"oracle_goldfinger failed with status {rc}")
    return fptr, fitems[:fptr[n]].copy()


def build_graph_sim(ptr, items, m, sptr, sitems, k, t, b, N, seed, greedy_threshold,
                    greedy_rounds=10, greedy_random=0):
    """Step 1 on (ptr, items), Steps 2-3 on the similarity profiles (sptr, sitems).
    Returns (nbr_id, nbr_inter, nbr_union, pairs) with the similarity profiles' counts."""
    ptr, items, sptr, sitems = _i32(ptr), _i32(items), _i32(sptr), _i32(sitems)
    n = ptr.size - 1
    out = [np.zeros((n, k), np.int32) for _ in range(3)]
    pairs = np.zeros(1, np.int64)
    rc = lib().oracle_build_sim(ptr, items, n, m, sptr, sitems if sitems.size else np.zeros(1, np.int32),
                                k, t, b, N, seed, greedy_threshold, greedy_rounds, greedy_random,
                                *out, pairs)
    if rc:
        raise ValueError(f"oracle_build_sim failed with status {rc}")
    return out[0], out[1], out[2], int(pairs[0])


def exact_counts(ptr, items, nbr_id):
    """Exact (inter, union) of given neighbour rows [n, k] (id -1 = empty slot)."""
    ptr, items, nbr_id = _i32(ptr), _i32(items), _i32(nbr_id)
    n, k = nbr_id.shape
    out = [np.zeros((n, k), np.int32) for _ in range(2)]
    lib().oracle_exact_counts(ptr, items, n, k, nbr_id, *out)
    return tuple(out)


def bruteforce_knn(ptr, items, k, queries=None):
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    q = None if queries is None else _i32(queries)
    rows = n if q is None else q.size
    out = [np.zeros((rows, k), np.int32) for _ in range(3)]
    lib().oracle_bruteforce_knn(ptr, items, n, k, _opt(q), rows, *out)
    return tuple(out)


def avg_sim(nbr_inter, nbr_union) -> float:
    nbr_inter, nbr_union = _i32(nbr_inter), _i32(nbr_union)
    rows, k = nbr_inter.shape
    return float(lib().oracle_avg_sim(nbr_inter, nbr_union, rows, k))


# ------------------------------------------------------------------ learned proposer
def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def model_forward(cfg, params, ptr, items):
    """cfg = dict(dim, hidden, t, b, rows_log2, seed); params = (E, W1, b1, W2, b2) FP32.
    Returns (logits [n, t*b] float64, keys [t, n])."""
    ptr, items = _i32(ptr), _i32(items)
    n = ptr.size - 1
    T = cfg["t"] * cfg["b"]
    z = np.zeros((n, T), np.float64)
    keys = np.zeros((cfg["t"], n), np.int32)
    E, W1, b1, W2, b2 = (_f32(x) for x in params)
    lib().oracle_model_forward(cfg["dim"], cfg["hidden"], cfg["t"], cfg["b"], cfg["rows_log2"],
                               cfg["seed"], E, W1, b1, W2, b2, ptr, items, n,
                               z.ctypes.data_as(C.c_void_p), keys)
    return z, keys


def model_exact(on: bool):
    """Switch the network oracle to plain FP64 (no BF16 rounding) or back."""
    lib().oracle_model_exact(1 if on else 0)


def model_grads(cfg, params, ptr, items, pairs, lam):
    """FP64 loss [pair, balance] and gradients (gE, gW1, gb1, gW2, gb2)."""
    ptr, items = _i32(ptr), _i32(items)
    pairs = _i32(pairs).reshape(-1, 2)
    E, W1, b1, W2, b2 = (_f32(x) for x in params)
    loss = np.zeros(2)
    g = [np.zeros(x.size) for x in (E, W1, b1, W2, b2)]
    lib().oracle_model_grads(cfg["dim"], cfg["hidden"], cfg["t"], cfg["b"], cfg["rows_log2"],
                             cfg["seed"], E, W1, b1, W2, b2, ptr, items, ptr.size - 1,
                             pairs.ravel(), pairs.shape[0], float(lam), loss, *g)
    return loss, [gi.reshape(x.shape) for gi, x in zip(g, (E, W1, b1, W2, b2))]
