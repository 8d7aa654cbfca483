"""The workspace-free merge entry point (c2_merge_topk_noalloc).

It exists for callers that cannot allocate device memory when they merge
(inside a stream capture without a memory pool, plug-ins whose host owns every
allocation); its scratch is a fixed array inside the library.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

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


def local_rows(c2, n, m, t, k, seed):
    ptr, items = synth.random_profiles(n, m, 20, seed, zipf_s=1.1)
    dptr = torch.from_numpy(ptr).cuda()
    ditems = torch.from_numpy(items).cuda()
    cl = c2.c2_frh_cluster(dptr, ditems, m, t, 32, 300, seed)
    opts = c2.options(greedy_threshold=120, greedy_rounds=3)
    li, lc, lu = c2.c2_cluster_knn(dptr, ditems, m, t, cl["cptr_full"], cl["cusers"],
                                   cl["n_clusters_dev"], k, seed, opts=opts)
    return cl["cusers"], li, lc, lu


def test_noalloc_merge_matches_workspace_merge_twice(c2):
    n, m, t, k = 3000, 400, 6, 12
    cusers, li, lc, lu = local_rows(c2, n, m, t, k, 5)
    ref = c2.c2_merge_topk(cusers, n, t, k, li, lc, lu)
    torch.cuda.synchronize()
    for _ in range(2):     # the shared scratch keeps the last call's contents
        got = c2.c2_merge_topk_noalloc(cusers, n, t, k, li, lc, lu)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)          # integer outputs: exact
    # a different, smaller problem afterwards still matches
    cusers2, li2, lc2, lu2 = local_rows(c2, 700, 200, 3, 7, 9)
    ref2 = c2.c2_merge_topk(cusers2, 700, 3, 7, li2, lc2, lu2)
    got2 = c2.c2_merge_topk_noalloc(cusers2, 700, 3, 7, li2, lc2, lu2)
    torch.cuda.synchronize()
    for a, b in zip(got2, ref2):
        assert torch.equal(a, b)


def test_noalloc_merge_rejects_oversize(c2):
    cap = c2.c2_merge_topk_noalloc_max_slots()
    assert cap == ((8 << 20) - 256) // 4
    t = 8
    n = cap // t + 1                     # one user too many; rejected on the host
    dummy = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(c2.C2Error) as e:
        c2.lib().c2_merge_topk_noalloc  # noqa: B018
        rc = c2.lib().c2_merge_topk_noalloc(dummy.data_ptr(), n, t, 10, dummy.data_ptr(),
                                            dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                            dummy.data_ptr(), dummy.data_ptr(), None)
        if rc:
            raise c2.C2Error(rc, "c2_merge_topk_noalloc")
    assert e.value.code == 3
