"""ctypes binding of libc2 (include/c2.h): argument marshalling only.

Every step of the method runs in libc2's CUDA kernels.  PyTorch provides the
device memory (tensors) and the stream; this module passes their raw pointers
through the C ABI with the same function names.  There is no fallback: if
libc2.so is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "libc2.so")
HEADER = os.path.join(ROOT, "include", "c2.h")

STRATEGY_AUTO, STRATEGY_MERGE, STRATEGY_TABLE32, STRATEGY_TABLE64, STRATEGY_MMA = -1, 0, 1, 2, 3
STATUS = {0: "C2_OK", 1: "C2_ERR_INVALID_ARG", 2: "C2_ERR_INVALID_CSR", 3: "C2_ERR_UNSUPPORTED",
          4: "C2_ERR_WORKSPACE", 5: "C2_ERR_CUDA", 6: "C2_ERR_TIMEOUT",
          7: "C2_ERR_QUALITY_FALLBACK"}


class C2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class Options(C.Structure):
    _fields_ = [("greedy_threshold", C.c_int32), ("greedy_rounds", C.c_int32),
                ("greedy_random", C.c_int32), ("strategy", C.c_int32),
                ("d_hash_table", C.c_void_p), ("gram_budget_bytes", C.c_int64),
                ("d_keys", C.c_void_p), ("greedy_max_draws", C.c_int32),
                ("sim_n_items", C.c_int32), ("d_sim_ptr", C.c_void_p), ("d_sim_items", C.c_void_p),
                ("d_sim_bits", C.c_void_p), ("fn_offset", C.c_int32),
                ("cluster_base", C.c_int32)]


class ModelConfig(C.Structure):
    _fields_ = [("t", C.c_int32), ("b", C.c_int32), ("dim", C.c_int32), ("hidden", C.c_int32),
                ("rows_log2", C.c_int32), ("reserved0", C.c_int32), ("seed", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("gram_pairs", C.c_int64), ("n_clusters", C.c_int32),
                ("split_levels", C.c_int32), ("n_greedy_clusters", C.c_int32),
                ("max_cluster", C.c_int32), ("max_profile", C.c_int32),
                ("greedy_users", C.c_int32), ("item_visits_brute", C.c_int64),
                ("item_visits_greedy", C.c_int64), ("greedy_visits", C.c_int64),
                ("greedy_computed", C.c_int64), ("greedy_evaluated", C.c_int64),
                ("brute_gram_elems", C.c_int64), ("brute_rows", C.c_int32),
                ("reserved", C.c_int32), ("brute_pairs", C.c_int64),
                ("greedy_pairs", C.c_int64), ("tc_macs", C.c_int64), ("tc_clusters", C.c_int32),
                ("tc_tiles", C.c_int32), ("select_general", C.c_int32), ("direct_users", C.c_int32)]


_lib = None
P = C.c_void_p
I32, I64, U64, SZ = C.c_int32, C.c_int64, C.c_uint64, C.c_size_t

_SIGS = {
    "c2_default_options": (None, [C.POINTER(Options)]),
    "c2_status_string": (C.c_char_p, [C.c_int]),
    "c2_workspace_size": (SZ, [I32, I64, I32, I32, I32, I32, I32, C.POINTER(Options)]),
    "c2_workspace_size_host": (SZ, [I32, I64, I32, I32, I32, I32, I32, C.POINTER(Options)]),
    "c2_minhash_keys": (C.c_int, [P, P, I32, I32, I32, U64, P, P, SZ, P]),
    "c2_frh_cluster": (C.c_int, [P, P, I32, I32, I32, I32, I32, U64, C.POINTER(Options), P, P, P,
                                 P, P, P, SZ, P]),
    "c2_cluster_knn": (C.c_int, [P, P, I32, I32, I32, P, P, P, I32, U64, C.POINTER(Options), P, P,
                                 P, P, SZ, P]),
    "c2_merge_topk": (C.c_int, [P, I32, I32, I32, P, P, P, P, P, P, P, SZ, P]),
    "c2_build_knn_graph": (C.c_int, [P, P, I32, I32, I32, I32, I32, I32, U64,
                                     C.POINTER(Options), P, P, P, P, SZ, P]),
    "c2_build_knn_graph_host": (C.c_int, [P, P, I32, I32, I32, I32, I32, I32, U64,
                                          C.POINTER(Options), P, P, P, P, SZ, P]),
    "c2_bruteforce_knn": (C.c_int, [P, P, I32, I32, I32, P, I32, P, P, P, P, SZ, P]),
    "c2_avg_sim": (C.c_int, [P, P, I32, I32, P, P, SZ, P]),
    "c2_get_status": (C.c_int, [P, P]),
    "c2_get_stats": (C.c_int, [P, P, C.POINTER(Stats)]),
    "c2_reset_status": (C.c_int, [P, P]),
    "c2_merge_topk_noalloc": (C.c_int, [P, I32, I32, I32, P, P, P, P, P, P, P]),
    "c2_goldfinger_workspace_size": (SZ, [I32]),
    "c2_goldfinger": (C.c_int, [P, P, I32, I32, I32, U64, P, P, P, P, SZ, P]),
    "c2_exact_counts": (C.c_int, [P, P, I32, I32, P, P, P, P]),
    "c2_model_state_bytes": (SZ, [C.POINTER(ModelConfig)]),
    "c2_workspace_size_learned": (SZ, [C.POINTER(ModelConfig), I32, I64, I32, I32, I32, I32,
                                       C.POINTER(Options)]),
    "c2_build_knn_graph_learned": (C.c_int, [C.POINTER(ModelConfig), P, P, P, I32, I64, I32, I32,
                                             I32, U64, C.POINTER(Options), C.c_float, I32, P, P,
                                             P, P, SZ, P, C.POINTER(C.c_double)]),
    "c2_model_workspace_size": (SZ, [C.POINTER(ModelConfig), I32, I32]),
    "c2_model_init": (C.c_int, [C.POINTER(ModelConfig), P, SZ, P]),
    "c2_model_propose": (C.c_int, [C.POINTER(ModelConfig), P, P, P, I32, P, P, SZ, P]),
    "c2_model_train_step": (C.c_int, [C.POINTER(ModelConfig), P, P, P, I32, P, I32, C.c_float,
                                      C.c_float, I32, P, P, SZ, P]),
    "c2_model_gradients": (C.c_int, [C.POINTER(ModelConfig), P, P, P, I32, P, I32, C.c_float, P,
                                     P, P, P, P, P, P, SZ, P]),
    "c2_model_params": (C.c_int, [C.POINTER(ModelConfig), P, C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "c2_merge_topk_noalloc_max_slots": (C.c_int64, []),
    "c2_kernel_launches": (C.c_int64, []),
    "c2_autotune_report": (C.c_size_t, [C.c_char_p, C.c_size_t]),
    "c2_autotune_save": (C.c_int32, [C.c_char_p]),
    "c2_autotune_load": (C.c_int32, [C.c_char_p]),
    "c2_profile_enable": (None, [C.c_int]),
    "c2_profile_report": (C.c_size_t, [C.c_char_p, C.c_size_t]),
}


def header_functions() -> list[str]:
    """Names of the functions include/c2.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(c2_[a-z0-9_]+)\s*\(", txt)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def options(greedy_threshold=0, greedy_rounds=-1, greedy_random=0, strategy=STRATEGY_AUTO,
            hash_table: torch.Tensor | None = None, gram_budget_bytes=0,
            keys: torch.Tensor | None = None, greedy_max_draws=0,
            sim: tuple | None = None, sim_n_items=0,
            sim_bits: torch.Tensor | None = None, fn_offset=0, cluster_base=0) -> Options:
    """Options of the build; sim = (ptr, items) similarity profiles over
    sim_n_items items (e.g. c2_goldfinger's fingerprints), sim_bits their
    packed rows."""
    o = Options()
    lib().c2_default_options(C.byref(o))
    o.greedy_threshold = greedy_threshold
    o.greedy_rounds = greedy_rounds
    o.greedy_random = greedy_random
    o.strategy = strategy
    o.d_hash_table = None if hash_table is None else hash_table.data_ptr()
    o.gram_budget_bytes = gram_budget_bytes
    o.d_keys = None if keys is None else keys.data_ptr()
    o.greedy_max_draws = greedy_max_draws
    o.sim_n_items = sim_n_items
    o.d_sim_ptr = None if sim is None else sim[0].data_ptr()
    o.d_sim_items = None if sim is None else sim[1].data_ptr()
    o.d_sim_bits = None if sim_bits is None else sim_bits.data_ptr()
    o.fn_offset = fn_offset
    o.cluster_base = cluster_base
    o._keep = (hash_table, keys, sim, sim_bits)   # keep the tensors alive with the options
    return o


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(rc, where):
    if rc != 0:
        raise C2Error(rc, where)


def _dev_i32(x, device):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32))
    return x.to(device=device, dtype=torch.int32).contiguous()


def workspace_size(n_users, nnz, n_items, k, t, b, N, opts=None) -> int:
    o = opts if opts is not None else options()
    sz = lib().c2_workspace_size(n_users, nnz, n_items, k, t, b, N, C.byref(o))
    if sz == 0:
        raise C2Error(1, "c2_workspace_size")
    return int(sz)


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """Workspace tensor with a cleared status header (its first 256 bytes)."""
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    ws[:256].zero_()
    return ws


# ------------------------------------------------------------------ entry points
def c2_minhash_keys(ptr, items, n_items, t, seed, out=None, ws=None, check=True, stream=None):
    """First-level keys [t, n] of the C^2/MinHash variant (one cluster per item).
    check=False skips the status read (no host synchronisation)."""
    dev = ptr.device
    n = ptr.numel() - 1
    keys = out if out is not None else torch.empty((t, max(n, 1)), dtype=torch.int32, device=dev)
    ws = ws if ws is not None else workspace(256, dev)
    _check(lib().c2_minhash_keys(_ptr(ptr), _ptr(items), n, n_items, t, seed, _ptr(keys),
                                 _ptr(ws), ws.numel(), _stream(stream)), "c2_minhash_keys")
    if check:
        _check(c2_get_status(ws, stream), "c2_minhash_keys (device)")
    return keys[:, :n]


def c2_frh_cluster(ptr, items, n_items, t, b, N, seed, opts=None, ws=None, stream=None):
    """Step 1.  Returns dict(cluster_of[t,n], cptr[nc+1], cusers[t*n], n_clusters, cmeta[nc,4])."""
    dev = ptr.device
    n = ptr.numel() - 1
    o = opts if opts is not None else options()
    if ws is None:
        ws = workspace(workspace_size(n, items.numel(), n_items, 1, t, b, N, o), dev)
    S = t * n
    cluster_of = torch.empty((t, n), dtype=torch.int32, device=dev)
    cptr = torch.empty(S + 1, dtype=torch.int32, device=dev)
    cusers = torch.empty(max(S, 1), dtype=torch.int32, device=dev)
    ncl = torch.zeros(1, dtype=torch.int32, device=dev)
    cmeta = torch.empty((max(S, 1), 4), dtype=torch.int32, device=dev)
    rc = lib().c2_frh_cluster(_ptr(ptr), _ptr(items), n, n_items, t, b, N, seed, C.byref(o),
                              _ptr(cluster_of), _ptr(cptr), _ptr(cusers), _ptr(ncl), _ptr(cmeta),
                              _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "c2_frh_cluster")
    _check(c2_get_status(ws, stream), "c2_frh_cluster (device)")
    nc = int(ncl.item())
    return dict(cluster_of=cluster_of, cptr=cptr[:nc + 1], cusers=cusers[:S], n_clusters=nc,
                cmeta=cmeta[:nc], n_clusters_dev=ncl, cptr_full=cptr)


def c2_cluster_knn(ptr, items, n_items, t, cptr, cusers, n_clusters_dev, k, seed, opts=None,
                   ws=None, stream=None):
    """Step 2.  Returns (loc_id, loc_inter, loc_union) of shape [t*n, k]."""
    dev = ptr.device
    n = ptr.numel() - 1
    o = opts if opts is not None else options()
    if ws is None:
        ws = workspace(workspace_size(n, items.numel(), n_items, k, t, 2, 2, o), dev)
    S = t * n
    out = [torch.empty((max(S, 1), k), dtype=torch.int32, device=dev) for _ in range(3)]
    rc = lib().c2_cluster_knn(_ptr(ptr), _ptr(items), n, n_items, t, _ptr(cptr), _ptr(cusers),
                              _ptr(n_clusters_dev), k, seed, C.byref(o), *[_ptr(x) for x in out],
                              _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "c2_cluster_knn")
    return tuple(x[:S] for x in out)


def c2_merge_topk(cusers, n_users, t, k, loc_id, loc_inter, loc_union, ws=None, stream=None):
    dev = cusers.device
    if ws is None:
        ws = workspace(workspace_size(n_users, 0, 0, k, t, 2, 2), dev)
    out = [torch.empty((n_users, k), dtype=torch.int32, device=dev) for _ in range(3)]
    rc = lib().c2_merge_topk(_ptr(cusers), n_users, t, k, _ptr(loc_id), _ptr(loc_inter),
                             _ptr(loc_union), *[_ptr(x) for x in out], _ptr(ws), ws.numel(),
                             _stream(stream))
    _check(rc, "c2_merge_topk")
    return tuple(out)


def c2_merge_topk_noalloc(cusers, n_users, t, k, loc_id, loc_inter, loc_union, stream=None):
    """Step 3 without a workspace (scratch in a fixed library array; see c2.h)."""
    dev = cusers.device
    out = [torch.empty((n_users, k), dtype=torch.int32, device=dev) for _ in range(3)]
    rc = lib().c2_merge_topk_noalloc(_ptr(cusers), n_users, t, k, _ptr(loc_id), _ptr(loc_inter),
                                     _ptr(loc_union), *[_ptr(x) for x in out], _stream(stream))
    _check(rc, "c2_merge_topk_noalloc")
    return tuple(out)


def c2_goldfinger(ptr, items, n_items, bits, seed, with_bits=False, ws=None, stream=None,
                  check=True, out=None):
    """GoldFinger fingerprints: (fp_ptr [n+1], fp_items [nnz capacity], fp_bits
    [n, bits/32] or None).  The CSR's rows are each user's set bits, increasing."""
    dev = ptr.device
    n = ptr.numel() - 1
    if out is not None:
        fptr, fitems, fbits = out
    else:
        fptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
        fitems = torch.empty(max(items.numel(), 1), dtype=torch.int32, device=dev)
        fbits = (torch.empty((max(n, 1), bits // 32), dtype=torch.int32, device=dev)
                 if with_bits else None)
    if ws is None:
        ws = workspace(int(lib().c2_goldfinger_workspace_size(n)), dev)
    _check(lib().c2_goldfinger(_ptr(ptr), _ptr(items), n, n_items, bits, seed, _ptr(fptr),
                               _ptr(fitems), _ptr(fbits), _ptr(ws), ws.numel(), _stream(stream)),
           "c2_goldfinger")
    if check:
        _check(c2_get_status(ws, stream), "c2_goldfinger (device)")
    return fptr, fitems, fbits


def c2_exact_counts(ptr, items, nbr_id, out=None, stream=None):
    """Exact (inter, union) of given neighbour rows [n, k]."""
    n, k = nbr_id.shape
    if out is None:
        out = [torch.empty((n, k), dtype=torch.int32, device=nbr_id.device) for _ in range(2)]
    _check(lib().c2_exact_counts(_ptr(ptr), _ptr(items), n, k, _ptr(nbr_id), _ptr(out[0]),
                                 _ptr(out[1]), _stream(stream)), "c2_exact_counts")
    return tuple(out)


def c2_merge_topk_noalloc_max_slots() -> int:
    return int(lib().c2_merge_topk_noalloc_max_slots())


def c2_build_knn_graph(ptr, items, n_items, k, t, b, N, seed, opts=None, ws=None, out=None,
                       stream=None, check=True):
    """The whole method.  Returns (nbr_id, nbr_inter, nbr_union) of shape [n, k]."""
    dev = ptr.device
    n = ptr.numel() - 1
    o = opts if opts is not None else options()
    if ws is None:
        ws = workspace(workspace_size(n, items.numel(), n_items, k, t, b, N, o), dev)
    if out is None:
        out = [torch.empty((n, k), dtype=torch.int32, device=dev) for _ in range(3)]
    rc = lib().c2_build_knn_graph(_ptr(ptr), _ptr(items), n, n_items, k, t, b, N, seed,
                                  C.byref(o), *[_ptr(x) for x in out], _ptr(ws), ws.numel(),
                                  _stream(stream))
    _check(rc, "c2_build_knn_graph")
    if check:
        _check(c2_get_status(ws, stream), "c2_build_knn_graph (device)")
    return tuple(out)


def workspace_size_host(n_users, nnz, n_items, k, t, b, N, opts=None) -> int:
    o = opts if opts is not None else options()
    sz = lib().c2_workspace_size_host(n_users, nnz, n_items, k, t, b, N, C.byref(o))
    if sz == 0:
        raise C2Error(1, "c2_workspace_size_host")
    return int(sz)


def c2_build_knn_graph_host(h_ptr, h_items, n_items, k, t, b, N, seed, opts=None, ws=None,
                            out=None, stream=None):
    """Whole method from host (ideally pinned) CPU tensors; results land in host tensors."""
    n = h_ptr.numel() - 1
    o = opts if opts is not None else options()
    if ws is None:
        ws = workspace(workspace_size_host(n, h_items.numel(), n_items, k, t, b, N, o))
    if out is None:
        out = [torch.empty((n, k), dtype=torch.int32).pin_memory() for _ in range(3)]
    rc = lib().c2_build_knn_graph_host(_ptr(h_ptr), _ptr(h_items), n, n_items, k, t, b, N, seed,
                                       C.byref(o), *[_ptr(x) for x in out], _ptr(ws), ws.numel(),
                                       _stream(stream))
    _check(rc, "c2_build_knn_graph_host")
    return tuple(out)


def c2_bruteforce_knn(ptr, items, n_items, k, queries=None, ws=None, stream=None):
    dev = ptr.device
    n = ptr.numel() - 1
    rows = n if queries is None else queries.numel()
    if ws is None:
        ws = workspace(workspace_size(n, items.numel(), n_items, k, 1, 1, 2), dev)
    out = [torch.empty((rows, k), dtype=torch.int32, device=dev) for _ in range(3)]
    rc = lib().c2_bruteforce_knn(_ptr(ptr), _ptr(items), n, n_items, k, _ptr(queries),
                                 rows if queries is not None else 0, *[_ptr(x) for x in out],
                                 _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "c2_bruteforce_knn")
    _check(c2_get_status(ws, stream), "c2_bruteforce_knn (device)")
    return tuple(out)


def c2_avg_sim(nbr_inter, nbr_union, ws=None, stream=None) -> float:
    dev = nbr_inter.device
    rows, k = nbr_inter.shape
    if ws is None:
        ws = workspace(workspace_size(1, 0, 0, k, 1, 1, 2), dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    rc = lib().c2_avg_sim(_ptr(nbr_inter), _ptr(nbr_union), rows, k, _ptr(out), _ptr(ws),
                          ws.numel(), _stream(stream))
    _check(rc, "c2_avg_sim")
    return float(out.item())


def c2_get_status(ws, stream=None) -> int:
    return int(lib().c2_get_status(_ptr(ws), _stream(stream)))


def c2_get_stats(ws, stream=None) -> dict:
    s = Stats()
    _check(lib().c2_get_stats(_ptr(ws), _stream(stream), C.byref(s)), "c2_get_stats")
    return dict(pairs=s.pairs, gram_pairs=s.gram_pairs, n_clusters=s.n_clusters,
                split_levels=s.split_levels, n_greedy_clusters=s.n_greedy_clusters,
                max_cluster=s.max_cluster, max_profile=s.max_profile,
                greedy_users=s.greedy_users, greedy_visits=s.greedy_visits,
                greedy_computed=s.greedy_computed, greedy_evaluated=s.greedy_evaluated,
                item_visits_brute=s.item_visits_brute, item_visits_greedy=s.item_visits_greedy,
                brute_gram_elems=s.brute_gram_elems, brute_rows=s.brute_rows,
                brute_pairs=s.brute_pairs, greedy_pairs=s.greedy_pairs, tc_macs=s.tc_macs,
                tc_clusters=s.tc_clusters, tc_tiles=s.tc_tiles, select_general=s.select_general,
                direct_users=s.direct_users)


def c2_reset_status(ws, stream=None):
    _check(lib().c2_reset_status(_ptr(ws), _stream(stream)), "c2_reset_status")


def c2_status_string(code: int) -> str:
    return lib().c2_status_string(code).decode()


def c2_autotune_save(path: str) -> int:
    return int(lib().c2_autotune_save(str(path).encode()))


def c2_autotune_load(path: str) -> int:
    return int(lib().c2_autotune_load(str(path).encode()))


def c2_autotune_report() -> list:
    import json
    need = lib().c2_autotune_report(None, 0)
    buf = C.create_string_buffer(int(need) + 1024)
    lib().c2_autotune_report(buf, len(buf))
    return json.loads(buf.value.decode() or "[]")


def c2_kernel_launches() -> int:
    return int(lib().c2_kernel_launches())


def c2_profile_enable(on: bool = True):
    lib().c2_profile_enable(1 if on else 0)


def c2_profile_report() -> dict:
    import json
    need = lib().c2_profile_report(None, 0)
    buf = C.create_string_buffer(int(need) + 4096)
    lib().c2_profile_report(buf, len(buf))
    return json.loads(buf.value.decode() or "{}")


# ------------------------------------------------------------------ learned proposer
class Model:
    """Device state of the learned cluster proposer (include/c2.h, c2_model_*)."""

    def __init__(self, t, b, dim=64, hidden=256, rows_log2=18, seed=2010, device="cuda"):
        self.cfg = ModelConfig(t, b, dim, hidden, rows_log2, 0, seed)
        nbytes = lib().c2_model_state_bytes(C.byref(self.cfg))
        if nbytes == 0:
            raise C2Error(3, "c2_model_state_bytes")
        self.state = torch.zeros(int(nbytes), dtype=torch.uint8, device=device)
        self._train_ws = None
        self._prop_ws = None
        self._prop_chunk = None
        self.step = 0

    def init(self, stream=None):
        _check(lib().c2_model_init(C.byref(self.cfg), _ptr(self.state), self.state.numel(),
                                   _stream(stream)), "c2_model_init")
        self.step = 0
        return self

    def config(self) -> dict:
        c = self.cfg
        return dict(t=c.t, b=c.b, dim=c.dim, hidden=c.hidden, rows_log2=c.rows_log2, seed=c.seed)

    def params(self):
        """FP32 master tensors (E, W1, b1, W2, b2) as views into the state buffer."""
        ptrs = [C.c_void_p() for _ in range(5)]
        _check(lib().c2_model_params(C.byref(self.cfg), _ptr(self.state), *[C.byref(p) for p in ptrs]),
               "c2_model_params")
        c = self.cfg
        T = c.t * c.b
        shapes = [(1 << c.rows_log2, c.dim), (c.dim, c.hidden), (c.hidden,), (c.hidden, T), (T,)]
        base = self.state.data_ptr()
        f = self.state.view(torch.uint8)
        out = []
        for p, shp in zip(ptrs, shapes):
            off = p.value - base
            n = int(np.prod(shp))
            out.append(f[off:off + 4 * n].view(torch.float32).view(*shp))
        return out

    def propose(self, ptr, items, stream=None, chunk=65536):
        n = ptr.numel() - 1
        keys = torch.empty((self.cfg.t, max(n, 1)), dtype=torch.int32, device=ptr.device)
        if self._prop_ws is None or self._prop_chunk != chunk:
            self._prop_ws = workspace(lib().c2_model_workspace_size(C.byref(self.cfg), chunk, 0),
                                      ptr.device)
            self._prop_chunk = chunk
        _check(lib().c2_model_propose(C.byref(self.cfg), _ptr(self.state), _ptr(ptr), _ptr(items),
                                      n, _ptr(keys), _ptr(self._prop_ws), self._prop_ws.numel(),
                                      _stream(stream)), "c2_model_propose")
        return keys[:, :n]

    def _ws(self, n_pairs, device):
        need = int(lib().c2_model_workspace_size(C.byref(self.cfg), n_pairs, 1))
        if self._train_ws is None or self._train_ws.numel() < need:
            self._train_ws = workspace(need, device)
        return self._train_ws

    def train_step(self, ptr, items, pairs, lr=1e-3, lam=0.1, stream=None):
        """One Adam step on pairs [P, 2] (int32, device).  Returns the device loss [2]."""
        P = pairs.shape[0]
        ws = self._ws(P, ptr.device)
        loss = torch.zeros(2, dtype=torch.float32, device=ptr.device)
        self.step += 1
        _check(lib().c2_model_train_step(C.byref(self.cfg), _ptr(self.state), _ptr(ptr), _ptr(items),
                                         ptr.numel() - 1, _ptr(pairs), P, lr, lam, self.step,
                                         _ptr(loss), _ptr(ws), ws.numel(), _stream(stream)),
               "c2_model_train_step")
        return loss

    def gradients(self, ptr, items, pairs, lam=0.1, stream=None):
        P = pairs.shape[0]
        ws = self._ws(P, ptr.device)
        E, W1, b1, W2, b2 = self.params()
        grads = [torch.empty_like(x) for x in (E, W1, b1, W2, b2)]
        loss = torch.zeros(2, dtype=torch.float32, device=ptr.device)
        _check(lib().c2_model_gradients(C.byref(self.cfg), _ptr(self.state), _ptr(ptr), _ptr(items),
                                        ptr.numel() - 1, _ptr(pairs), P, lam, _ptr(loss),
                                        *[_ptr(g) for g in grads], _ptr(ws), ws.numel(),
                                        _stream(stream)), "c2_model_gradients")
        return loss, grads

    def build_knn_graph(self, ptr, items, n_items, k, N, seed, opts=None, quality_threshold=0.95,
                        n_probe=2048, ws=None, stream=None):
        """Learned-proposer build with the FastRandomHash fallback.

        Returns ((nbr_id, nbr_inter, nbr_union), probed quality, fell_back)."""
        n = ptr.numel() - 1
        nnz = items.numel()
        o = opts if opts is not None else options()
        need = int(lib().c2_workspace_size_learned(C.byref(self.cfg), n, nnz, n_items, k, N,
                                                   n_probe, C.byref(o)))
        if need == 0:
            raise C2Error(1, "c2_workspace_size_learned")
        if ws is None or ws.numel() < need:
            ws = workspace(need, ptr.device)
        out = [torch.empty((n, k), dtype=torch.int32, device=ptr.device) for _ in range(3)]
        q = C.c_double(0.0)
        rc = lib().c2_build_knn_graph_learned(C.byref(self.cfg), _ptr(self.state), _ptr(ptr),
                                              _ptr(items), n, nnz, n_items, k, N, seed, C.byref(o),
                                              quality_threshold, n_probe, *[_ptr(x) for x in out],
                                              _ptr(ws), ws.numel(), _stream(stream), C.byref(q))
        if rc not in (0, 7):
            raise C2Error(rc, "c2_build_knn_graph_learned")
        return tuple(out), q.value, rc == 7

    def save(self, path):
        """Parameters and optimiser state, with a header (format, config, step)."""
        import json
        torch.cuda.synchronize()
        hdr = json.dumps(dict(format="c2-model-1", config=self.config(), step=self.step,
                              nbytes=self.state.numel())).encode()
        with open(path, "wb") as f:
            f.write(len(hdr).to_bytes(4, "little"))
            f.write(hdr)
            f.write(self.state.cpu().numpy().tobytes())

    @classmethod
    def load(cls, path, device="cuda"):
        import json
        with open(path, "rb") as f:
            n = int.from_bytes(f.read(4), "little")
            hdr = json.loads(f.read(n))
            data = np.frombuffer(f.read(), dtype=np.uint8)
        if hdr.get("format") != "c2-model-1":
            raise ValueError("not a c2 model file")
        c = hdr["config"]
        m = cls(c["t"], c["b"], c["dim"], c["hidden"], c["rows_log2"], c["seed"], device)
        if data.size != m.state.numel():
            raise ValueError("model file does not match its config")
        m.state.copy_(torch.from_numpy(data.copy()))
        m.step = hdr["step"]
        return m
