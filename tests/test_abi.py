"""CPU checks of the C ABI: the library builds, loads and exports every
function include/c2.h declares; host-side argument checks need no GPU."""
import ctypes as C

import pytest

import paper_2010_11497_gb300 as c2
from paper_2010_11497_gb300 import build as c2build


@pytest.fixture(scope="module")
def lib():
    c2build.build()
    return c2.lib()


def test_header_symbols_exported(lib):
    names = c2.header_functions()
    assert "c2_build_knn_graph" in names and "c2_frh_cluster" in names
    assert {"c2_cluster_knn", "c2_merge_topk", "c2_bruteforce_knn", "c2_avg_sim"} <= set(names)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/c2.h but not exported"


def test_status_strings(lib):
    for code in range(8):
        assert c2.c2_status_string(code)
    assert c2.c2_status_string(0) == "ok"


def test_default_options(lib):
    o = c2.options()
    assert o.greedy_threshold == 0 and o.greedy_rounds == -1 and o.strategy == -1
    assert o.fn_offset == 0 and o.cluster_base == 0 and o.d_keys is None and o.greedy_max_draws == 0
    assert o.d_sim_ptr is None and o.d_sim_bits is None and o.sim_n_items == 0


def test_workspace_size_validates(lib):
    ws = c2.workspace_size(1000, 20000, 500, 30, 8, 4096, 2000)
    assert ws > 0
    # larger problems need more
    assert c2.workspace_size(2000, 40000, 500, 30, 8, 4096, 2000) > ws
    bad = [(1000, 0, 500, 0, 8, 64, 10), (1000, 0, 500, 33, 8, 64, 10),
           (1000, 0, 500, 10, 65, 64, 10), (1000, 0, 500, 10, 8, 65537, 10),
           (1000, 0, 500, 10, 8, 64, 1), (-1, 0, 500, 10, 8, 64, 10)]
    for args in bad:
        o = c2.options()
        assert lib.c2_workspace_size(*args, C.byref(o)) == 0


def test_host_argument_errors_need_no_gpu(lib):
    o = c2.options()
    # NULL pointers are rejected before any CUDA call
    rc = lib.c2_build_knn_graph(None, None, 10, 10, 5, 2, 8, 4, 1, C.byref(o), None, None, None,
                                None, 0, None)
    assert rc == 1
    # k out of range
    rc = lib.c2_build_knn_graph(None, None, 10, 10, 40, 2, 8, 4, 1, C.byref(o), None, None, None,
                                None, 0, None)
    assert rc == 3
    # missing workspace
    fake = C.c_void_p(256)
    rc = lib.c2_build_knn_graph(fake, fake, 10, 10, 5, 2, 8, 4, 1, C.byref(o), fake, fake, fake,
                                None, 0, None)
    assert rc == 4
    # misaligned workspace
    rc = lib.c2_build_knn_graph(fake, fake, 10, 10, 5, 2, 8, 4, 1, C.byref(o), fake, fake, fake,
                                C.c_void_p(4096 + 8), 1 << 30, None)
    assert rc == 4
    # negative shard offsets
    o.fn_offset = -1
    rc = lib.c2_build_knn_graph(fake, fake, 10, 10, 5, 2, 8, 4, 1, C.byref(o), fake, fake, fake,
                                C.c_void_p(4096), 1 << 30, None)
    assert rc == 1


def test_minhash_keys_argument_errors_need_no_gpu(lib):
    fake = C.c_void_p(256)
    # NULL outputs
    assert lib.c2_minhash_keys(fake, fake, 10, 10, 4, 1, None, fake, 256, None) == 1
    # t beyond the 64 functions the library supports
    assert lib.c2_minhash_keys(fake, fake, 10, 10, 65, 1, fake, fake, 256, None) == 3
    # workspace missing, too small for the status header, or misaligned
    assert lib.c2_minhash_keys(fake, fake, 10, 10, 4, 1, fake, None, 256, None) == 4
    assert lib.c2_minhash_keys(fake, fake, 10, 10, 4, 1, fake, C.c_void_p(4096), 64, None) == 4
    assert lib.c2_minhash_keys(fake, fake, 10, 10, 4, 1, fake, C.c_void_p(4096 + 8), 256,
                               None) == 4


def test_goldfinger_and_exact_counts_argument_errors_need_no_gpu(lib):
    fake = C.c_void_p(256)
    ws = c2.lib().c2_goldfinger_workspace_size(100)
    assert ws >= 256
    # bits out of range or not a multiple of 32
    for bits in (16, 8224, 100):
        assert lib.c2_goldfinger(fake, fake, 100, 50, bits, 1, fake, fake, None, C.c_void_p(4096),
                                 ws, None) == 3
    # NULL outputs, missing or small workspace
    assert lib.c2_goldfinger(fake, fake, 100, 50, 1024, 1, None, fake, None, C.c_void_p(4096), ws,
                             None) == 1
    assert lib.c2_goldfinger(fake, fake, 100, 50, 1024, 1, fake, fake, None, None, ws, None) == 4
    assert lib.c2_goldfinger(fake, fake, 100, 50, 1024, 1, fake, fake, None, C.c_void_p(4096), 8,
                             None) == 4
    # k out of range, NULL rows
    assert lib.c2_exact_counts(fake, fake, 10, 33, fake, fake, fake, None) == 3
    assert lib.c2_exact_counts(fake, fake, 10, 5, None, fake, fake, None) == 1
    # similarity options: a CSR without its item universe, bit rows not in words of 32
    o = c2.options()
    o.d_sim_ptr = 256
    rc = lib.c2_build_knn_graph(fake, fake, 10, 10, 5, 2, 8, 4, 1, C.byref(o), fake, fake, fake,
                                C.c_void_p(4096), 1 << 30, None)
    assert rc == 1
    o = c2.options()
    o.d_sim_bits = 256
    o.sim_n_items = 100
    rc = lib.c2_build_knn_graph(fake, fake, 10, 10, 5, 2, 8, 4, 1, C.byref(o), fake, fake, fake,
                                C.c_void_p(4096), 1 << 30, None)
    assert rc == 1


def test_autotune_table_round_trip_needs_no_gpu(lib, tmp_path):
    # a saved table is read back into the process's table (host only)
    p = tmp_path / "tune.txt"
    routes = " ".join("%d 0.5 0.25" % (1 if i == 7 else -1) for i in range(20))
    shapes = " ".join("1 256 4 1 1.5" for _ in range(4))
    p.write_text("c2-autotune 2\n123 456 8 4096 2000 30 4500 1 1 1 " + shapes + " " + routes + "\n")
    assert c2.c2_autotune_load(str(p)) == 1
    rep = [e for e in c2.c2_autotune_report() if e.get("n") == 123]
    assert rep and rep[0]["m"] == 456 and rep[0]["buckets"][0]["threads"] == 256
    assert rep[0]["buckets"][0]["items16"] is True
    assert [s["use"] for s in rep[0]["strategy"]] == ["tensor"]
    q = tmp_path / "again.txt"
    assert c2.c2_autotune_save(str(q)) == 0
    assert "123 456 8 4096 2000 30 4500" in q.read_text()
    assert c2.c2_autotune_load(str(tmp_path / "missing.txt")) == -1
    (tmp_path / "bad.txt").write_text("not a table\n")
    assert c2.c2_autotune_load(str(tmp_path / "bad.txt")) == -1
