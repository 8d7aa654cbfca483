"""The workspace-free merge entry point (c2_merge_topk_noalloc).

It exists for callers that cannot allocate device memory when they merge
(plug-ins whose host application owns every allocation, loops that forbid
allocation after start-up); its scratch is a fixed array inside the library.  The local rows
it merges come from the CPU oracle, and its results are checked against the
oracle's merge (Algorithm 3) and against the workspace entry point
c2_merge_topk, on calls in a row.  This file is named so that pytest collects
it last.
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


def oracle_local_rows(n, m, t, k, seed):
    """Oracle clustering and local rows (greedy above 120 members, 3 rounds)."""
    ptr, items = synth.random_profiles(n, m, 20, seed, zipf_s=1.1)
    cl = oracle.frh_cluster(ptr, items, m, t, 32, 300, seed)
    li, lc, lu, _ = oracle.cluster_knn(ptr, items, cl["cptr"], cl["cusers"], k, seed, 120, 3)
    ref = oracle.merge_topk(cl["cptr"], cl["cusers"], n, k, li, lc, lu)
    return cl["cusers"], li, lc, lu, ref


def check(got, ref):
    for g, r in zip(got, ref):
        g = g.cpu().numpy()
        bad = np.argwhere(g != r)
        assert bad.size == 0, f"{len(bad)} mismatches, first {tuple(bad[0])}"


def test_noalloc_merge_matches_oracle_and_workspace_merge_twice(c2):
    n, m, t, k = 3000, 400, 6, 12
    cusers, li, lc, lu, ref = oracle_local_rows(n, m, t, k, 5)
    args = [dev(x) for x in (cusers, li, lc, lu)]
    ws_ref = c2.c2_merge_topk(args[0], n, t, k, *args[1:])
    torch.cuda.synchronize()
    check(ws_ref, ref)
    for _ in range(2):     # the shared scratch keeps the last call's contents
        got = c2.c2_merge_topk_noalloc(args[0], n, t, k, *args[1:])
        torch.cuda.synchronize()
        check(got, ref)                        # integer outputs: exact
        for a, b in zip(got, ws_ref):
            assert torch.equal(a, b)
    # a different, smaller problem afterwards still matches
    cusers2, li2, lc2, lu2, ref2 = oracle_local_rows(700, 200, 3, 7, 9)
    args2 = [dev(x) for x in (cusers2, li2, lc2, lu2)]
    got2 = c2.c2_merge_topk_noalloc(args2[0], 700, 3, 7, *args2[1:])
    torch.cuda.synchronize()
    check(got2, ref2)


def _raw_status(c2, fn, n, t, k, with_ws):
    d = torch.zeros(1, dtype=torch.int32, device="cuda").data_ptr()
    ws = c2.workspace(1 << 16, "cuda") if with_ws else None
    if with_ws:
        return fn(d, n, t, k, d, d, d, d, d, d, ws.data_ptr(), ws.numel(), None)
    return fn(d, n, t, k, d, d, d, d, d, d, None)


def test_noalloc_merge_argument_statuses_match_workspace_merge(c2):
    L = c2.lib()
    # k above 32, t above 64 (sizes beyond the limits), a negative size and k = 0
    for n, t, k in [(10, 2, 33), (10, 65, 5), (-1, 2, 5), (10, 2, 0)]:
        a = _raw_status(c2, L.c2_merge_topk, n, t, k, True)
        b = _raw_status(c2, L.c2_merge_topk_noalloc, n, t, k, False)
        assert a == b and a != 0, (n, t, k, a, b)
    assert _raw_status(c2, L.c2_merge_topk_noalloc, 10, 2, 33, False) == 3
    assert _raw_status(c2, L.c2_merge_topk_noalloc, -1, 2, 5, False) == 1


def test_noalloc_merge_rejects_oversize(c2):
    cap = c2.c2_merge_topk_noalloc_max_slots()
    assert cap == ((8 << 20) - 256) // 4
    t = 8
    n = cap // t + 1                     # one user too many; rejected on the host
    assert _raw_status(c2, c2.lib().c2_merge_topk_noalloc, n, t, 10, False) == 3
