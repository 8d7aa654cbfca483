"""GPU checks of the learned cluster proposer against the CPU oracle.

- clustering and whole builds with caller-given first-level keys: bit-exact;
- model keys: equal to the oracle's argmax (FP64 logits on the same BF16
  operands) except where the oracle's two best logits are within 1e-3;
- gradients (BF16 operands, FP32 sums): element by element within 1e-2
  relative (above a floor of 1e-4 of the tensor's largest) of the FP64
  oracle on the same BF16 roundings, loss within 1e-3;
- training lowers the loss and raises the co-assignment of positive pairs;
- the learned build with its quality probe and FastRandomHash fallback.
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
    bad = np.argwhere(g != np.asarray(r))
    assert bad.size == 0, f"{what}: {len(bad)} mismatches, first {tuple(bad[0])}"


def test_cluster_and_build_with_given_keys(c2):
    ptr, items = synth.random_profiles(3000, 500, 20, 41, zipf_s=1.1)
    m, t, b, N, k, seed, thr = 500, 4, 16, 300, 10, 3, 200
    keys = np.random.default_rng(1).integers(0, b, (t, 3000)).astype(np.int32)
    keys[:, :900] = 5                  # one oversized learned cluster per function
    g = c2.c2_frh_cluster(dev(ptr), dev(items), m, t, b, N, seed,
                          opts=c2.options(keys=dev(keys)))
    o = oracle.frh_cluster(ptr, items, m, t, b, N, seed, keys=keys)
    assert g["n_clusters"] == o["n_clusters"]
    same(g["cptr"], o["cptr"], "cptr")
    same(g["cusers"], o["cusers"], "cusers")
    same(g["cmeta"], o["cmeta"], "cmeta")
    oid, oin, oun, pairs = oracle.build_graph(ptr, items, m, k, t, b, N, seed, thr, 3, keys=keys)
    opts = c2.options(greedy_threshold=thr, greedy_rounds=3, keys=dev(keys))
    ws = c2.workspace(c2.workspace_size(3000, items.size, m, k, t, b, N, opts), "cuda")
    gid, gin, gun = c2.c2_build_knn_graph(dev(ptr), dev(items), m, k, t, b, N, seed, opts=opts,
                                          ws=ws)
    same(gid, oid, "nbr_id")
    same(gun, oun, "nbr_union")
    assert c2.c2_get_stats(ws)["pairs"] == pairs


def _model(c2, t=4, b=32, dim=64, hidden=64, rows_log2=10, seed=11):
    return c2.Model(t, b, dim, hidden, rows_log2, seed).init()


def test_model_keys_match_oracle(c2):
    m = _model(c2)
    ptr, items = synth.random_profiles(1500, 800, 25, 42)
    keys = m.propose(dev(ptr), dev(items)).cpu().numpy()
    params = [x.cpu().numpy() for x in m.params()]
    z, okeys = oracle.model_forward(m.config(), params, ptr, items)
    b = m.cfg.b
    diff = np.argwhere(keys != okeys)
    for j, u in diff:
        zz = np.sort(z[u, j * b:(j + 1) * b])
        assert zz[-1] - zz[-2] < 1e-3 * max(1.0, abs(zz[-1])), (j, u)
    assert len(diff) <= 0.01 * keys.size


@pytest.mark.parametrize("t,b,hidden,n_pairs", [
    (4, 32, 64, 256),      # 512 rows: logits, dh and dW2 on the tensor cores (tcgen05)
    (4, 32, 64, 250),      # 500 rows (not a multiple of 64): the mma.sync GEMMs
    (2, 512, 256, 2048),   # 4,096 rows, 1,024 logits: several tiles, dW2 with K split
])
def test_model_gradients_match_oracle(c2, t, b, hidden, n_pairs):
    m = _model(c2, t=t, b=b, hidden=hidden)
    ptr, items = synth.random_profiles(600, 400, 20, 43)
    rng = np.random.default_rng(4)
    pairs = rng.integers(0, 600, (n_pairs, 2)).astype(np.int32)
    lam = 0.1
    loss, grads = m.gradients(dev(ptr), dev(items), dev(pairs), lam)
    params = [x.cpu().numpy() for x in m.params()]
    oloss, ograds = oracle.model_grads(m.config(), params, ptr, items, pairs, lam)
    loss = loss.cpu().numpy()
    assert abs(loss[0] - oloss[0]) <= 1e-3 * abs(oloss[0]) + 1e-6
    assert abs(loss[1] - oloss[1]) <= 1e-3 * abs(oloss[1]) + 1e-5
    # element by element: the oracle rounds to BF16 where the library stores
    # BF16 (operands, logit gradients, masked hidden gradients), so what is
    # left is FP32 accumulation order and the FP32 softmax: relative error
    # 1e-2 above a floor of 1e-4 of the tensor's largest gradient
    for name, g, og in zip(["E", "W1", "b1", "W2", "b2"], grads, ograds):
        g = g.cpu().numpy().astype(np.float64)
        floor = 1e-4 * np.abs(og).max()
        bad = np.abs(g - og) > 1e-2 * np.abs(og) + floor
        assert not bad.any(), (name, int(bad.sum()), np.argwhere(bad)[:3].tolist())


def _coassign(keys, pairs):
    return float((keys[:, pairs[:, 0]] == keys[:, pairs[:, 1]]).mean())


def test_training_lowers_loss_and_groups_pairs(c2):
    ptr, items = synth.random_profiles(4000, 2000, 30, 44, mu=0.8, n_comm=16)
    n, m_items, k, t, b, N, seed = 4000, 2000, 10, 4, 32, 400, 5
    dptr, ditems = dev(ptr), dev(items)
    gid, _, _ = c2.c2_build_knn_graph(dptr, ditems, m_items, k, t, b, N, seed)
    nid = gid.cpu().numpy()
    u = np.repeat(np.arange(n), k)
    v = nid.ravel()
    pairs = np.stack([u[v >= 0], v[v >= 0]], 1).astype(np.int32)
    model = _model(c2, t=t, b=b, seed=7)
    before = _coassign(model.propose(dptr, ditems).cpu().numpy(), pairs)
    rng = np.random.default_rng(0)
    losses = []
    for step in range(150):
        batch = dev(pairs[rng.integers(0, len(pairs), 2048)])
        losses.append(model.train_step(dptr, ditems, batch, lr=3e-3, lam=0.1))
    losses = torch.stack(losses).cpu().numpy()
    assert losses[-10:, 0].mean() < 0.8 * losses[:10, 0].mean()
    after = _coassign(model.propose(dptr, ditems).cpu().numpy(), pairs)
    assert after > before + 0.1, (before, after)


def test_learned_build_probe_and_fallback(c2):
    ptr, items = synth.random_profiles(3000, 1500, 30, 45, mu=0.8, n_comm=16)
    n, m_items, k, t, b, N, seed = 3000, 1500, 10, 4, 32, 300, 6
    model = _model(c2, t=t, b=b, seed=8)
    dptr, ditems = dev(ptr), dev(items)
    # threshold 0 never falls back: the graph is the keys' graph
    (gid, gin, gun), q, fell = model.build_knn_graph(dptr, ditems, m_items, k, N, seed,
                                                     quality_threshold=0.0, n_probe=500)
    assert not fell and 0.0 < q <= 1.0
    keys = model.propose(dptr, ditems).cpu().numpy()
    oid, oin, oun, _ = oracle.build_graph(ptr, items, m_items, k, t, b, N, seed, 5 * k * k, 10,
                                          keys=keys)
    same(gid, oid, "learned graph ids")
    # threshold above any quality falls back to the FastRandomHash graph
    (fid, fin, fun), q2, fell2 = model.build_knn_graph(dptr, ditems, m_items, k, N, seed,
                                                       quality_threshold=1.01, n_probe=500)
    assert fell2 and abs(q2 - q) < 1e-12
    rid, rin, run = c2.c2_build_knn_graph(dptr, ditems, m_items, k, t, b, N, seed)
    same(fid, rid.cpu().numpy(), "fallback graph ids")


def test_model_save_load_roundtrip(c2, tmp_path):
    m = _model(c2, seed=9)
    ptr, items = synth.random_profiles(300, 200, 10, 46)
    pairs = dev(np.random.default_rng(1).integers(0, 300, (64, 2)))
    m.train_step(dev(ptr), dev(items), pairs)
    path = tmp_path / "model.c2m"
    m.save(str(path))
    m2 = c2.Model.load(str(path))
    assert m2.step == m.step and torch.equal(m2.state, m.state)
    same(m2.propose(dev(ptr), dev(items)), m.propose(dev(ptr), dev(items)).cpu().numpy(), "keys")


def test_model_keys_fused_argmax_match_oracle(c2):
    # heads of 128 buckets: the argmax is fused into the logits GEMM
    m = _model(c2, t=2, b=256, dim=64, hidden=128, rows_log2=11, seed=12)
    ptr, items = synth.random_profiles(2500, 900, 25, 47)
    keys = m.propose(dev(ptr), dev(items)).cpu().numpy()
    params = [x.cpu().numpy() for x in m.params()]
    z, okeys = oracle.model_forward(m.config(), params, ptr, items)
    b = m.cfg.b
    diff = np.argwhere(keys != okeys)
    for j, u in diff:
        zz = np.sort(z[u, j * b:(j + 1) * b])
        assert zz[-1] - zz[-2] < 1e-3 * max(1.0, abs(zz[-1])), (j, u)
    assert len(diff) <= 0.01 * keys.size


def _sub_csr(ptr, items, users):
    lens = ptr[users + 1] - ptr[users]
    sp = np.zeros(len(users) + 1, np.int32)
    sp[1:] = np.cumsum(lens)
    si = np.concatenate([items[ptr[u]:ptr[u + 1]] for u in users]).astype(np.int32)
    return sp, si


def test_model_keys_tcgen05_full_shape(c2):
    # the learned workload's network (8 heads of 1024 buckets, hidden 256):
    # tcgen05 logits GEMM over 256-column slices, 157 row tiles x 32 slices
    # spread over the SMs (several tiles and a slice change per CTA, ring and
    # accumulator reuse), a ragged last tile (20011 = 156 * 128 + 43)
    m = c2.Model(8, 1024, 64, 256, 18, 13).init()
    n = 20011
    ptr, items = synth.random_profiles(n, 5000, 40, 48)
    keys = m.propose(dev(ptr), dev(items)).cpu().numpy()
    rng = np.random.default_rng(5)
    users = np.unique(np.concatenate([rng.choice(n, 500, replace=False), np.arange(128),
                                      np.arange(n - 171, n)]))
    sp, si = _sub_csr(ptr, items, users)
    params = [x.cpu().numpy() for x in m.params()]
    z, okeys = oracle.model_forward(m.config(), params, sp, si)
    b = m.cfg.b
    got = keys[:, users]
    diff = np.argwhere(got != okeys)
    for j, i in diff:
        zz = np.sort(z[i, j * b:(j + 1) * b])
        assert zz[-1] - zz[-2] < 1e-3 * max(1.0, abs(zz[-1])), (j, users[i])
    assert len(diff) <= 0.01 * got.size
    # chunked proposals (three chunks, the last ragged) give the same keys
    keys2 = m.propose(dev(ptr), dev(items), chunk=8192)
    same(keys2, keys, "keys with 8192-row chunks")


def test_model_keys_mma_fused_argmax_match_oracle(c2):
    # t*b = 384 (not a multiple of 256): the mma.sync logits GEMM with the
    # argmax of 128-column slices fused into its epilogue
    m = _model(c2, t=3, b=128, dim=64, hidden=128, rows_log2=11, seed=14)
    ptr, items = synth.random_profiles(2100, 900, 25, 49)
    keys = m.propose(dev(ptr), dev(items)).cpu().numpy()
    params = [x.cpu().numpy() for x in m.params()]
    z, okeys = oracle.model_forward(m.config(), params, ptr, items)
    b = m.cfg.b
    diff = np.argwhere(keys != okeys)
    for j, u in diff:
        zz = np.sort(z[u, j * b:(j + 1) * b])
        assert zz[-1] - zz[-2] < 1e-3 * max(1.0, abs(zz[-1])), (j, u)
    assert len(diff) <= 0.01 * keys.size


def test_learned_fallback_device_error_is_returned(c2):
    # A device error of the fallback build is returned, not the informational
    # fallback status.  An all-zero explicit hash table puts every user in one
    # FastRandomHash cluster per function (N = n: no split); the greedy
    # threshold sends it to the greedy phase, whose random start may make no
    # draw (greedy_max_draws = 1 is below one batch of 32): C2_ERR_TIMEOUT.
    # Every learned cluster is below the threshold (brute force), so the
    # learned build and its probe succeed, and a threshold above any quality
    # forces the fallback.
    n, m_items, k, t, b, seed = 2000, 900, 10, 4, 32, 6
    ptr, items = synth.random_profiles(n, m_items, 25, 50)
    model = _model(c2, t=t, b=b, seed=15)
    dptr, ditems = dev(ptr), dev(items)
    keys = model.propose(dptr, ditems).cpu().numpy()
    largest = max(int(np.bincount(keys[j], minlength=b).max()) for j in range(t))
    assert largest + 1 < n
    zeros = dev(np.zeros((t, m_items), np.int32))
    opts = c2.options(greedy_threshold=largest + 1, hash_table=zeros, greedy_max_draws=1)
    # the learned graph alone (threshold 0: no fallback) is fine
    _, q, fell = model.build_knn_graph(dptr, ditems, m_items, k, n, seed, opts=opts,
                                       quality_threshold=0.0, n_probe=200)
    assert not fell and 0.0 < q <= 1.0
    with pytest.raises(c2.C2Error) as e:
        model.build_knn_graph(dptr, ditems, m_items, k, n, seed, opts=opts,
                              quality_threshold=2.0, n_probe=200)
    assert e.value.code == 6


def test_trained_proposer_gains_over_frh_on_held_out_data(c2):
    # The gain of the network over the method without it: trained on the
    # plain-C^2 graphs of two seeds, evaluated on a third seed of the same
    # world (profiles with community structure), at equal t, b and N the
    # learned keys give a graph of higher quality (Eq. 2 against the exact
    # graph) than FastRandomHash keys.
    from paper_2010_11497_gb300.train_proposer import positive_pairs
    n, m_items, k, t, b, N = 5000, 2000, 10, 4, 32, 400

    def data(seed):
        ptr, items = synth.random_profiles(n, m_items, 30, seed, mu=0.8, n_comm=16)
        return dev(ptr), dev(items)

    train = []
    for s in (201, 202):
        dptr, ditems = data(s)
        nid, _, _ = c2.c2_build_knn_graph(dptr, ditems, m_items, k, t, b, N, s)
        train.append((dptr, ditems, positive_pairs(nid)))
    model = _model(c2, t=t, b=b, seed=16)
    rng = np.random.default_rng(0)
    for step in range(300):
        tptr, titems, pairs = train[step % 2]
        idx = torch.from_numpy(rng.integers(0, pairs.shape[0], 4096)).cuda()
        model.train_step(tptr, titems, pairs[idx].contiguous(), lr=3e-3, lam=3.0)
    dptr, ditems = data(203)
    _, jin, jun = c2.c2_bruteforce_knn(dptr, ditems, m_items, k)
    judge = c2.c2_avg_sim(jin, jun)
    _, fin, fun = c2.c2_build_knn_graph(dptr, ditems, m_items, k, t, b, N, 203)
    q_frh = c2.c2_avg_sim(fin, fun) / judge
    keys = model.propose(dptr, ditems)
    _, lin, lun = c2.c2_build_knn_graph(dptr, ditems, m_items, k, t, b, N, 203,
                                        opts=c2.options(keys=keys))
    q_learned = c2.c2_avg_sim(lin, lun) / judge
    assert q_learned > q_frh + 0.02, (q_frh, q_learned)
