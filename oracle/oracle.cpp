// Cluster-and-Conquer (C^2) CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of the method, written to be
// checked against the paper by eye.  Only the test-suite, the smoke check and
// the benchmark's CPU-baseline leg may load it; the library never does.  It
// shares no code, header, table or constant generator with the CUDA path.
//
// Paper: "Cluster-and-Conquer: When Randomness Meets Graph Locality"
// (Giakkoupis, Kermarrec, Ruas, Taiani), arXiv 2010.11497.
//
// Readings where the paper is silent (numbered as in the design notes):
//   R1  profiles are sets: CSR rows must be strictly increasing and in range.
//   R2  h_i(x) is a project-defined random function (the paper uses Jenkins'
//       hash, Section IV-E; Theorem 1 averages over any random h).  Parity of
//       the absolute hash values with the paper is unpinned.
//   R3  an empty profile gets FRH key b (a sentinel bucket).
//   R5  the residual of a split cluster is terminal (never split again).
//   R7  clusters are numbered by (hash function, path, residual first).
//   R8  v precedes w for user u iff c_v*U_w > c_w*U_v, ties to the lower id.
//   R9  candidates with no common item are never emitted.
//   R11 greedy refinement: Philox-seeded random start, synchronous rounds.
//   R12 merge reuses the carried (c, U) counts.
//   R17 GoldFinger (Section II-F) is named, not constructed: one random bit
//       of B per item; the estimate is the Jaccard of the bit sets.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

namespace {

// ------------------------------------------------------------------ hashing
// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Key of generative hash function number i (0-based) for a run seed: the
// (i+1)-th output of a SplitMix64 generator started at `seed`.
uint64_t function_key(uint64_t seed, int i) {
  return splitmix64_mix(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
}

// R2: generative hash h_i : items -> [0, b)  (Section II-D; 0-based buckets).
uint32_t item_hash(uint64_t seed, int i, int32_t x, int32_t b) {
  uint64_t z = splitmix64_mix(function_key(seed, i) ^ ((uint64_t)(uint32_t)x * 0xC2B2AE3D27D4EB4FULL));
  return (uint32_t)(((z >> 32) * (uint64_t)(uint32_t)b) >> 32);
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11).
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ------------------------------------------------------------------ profiles
struct Csr {
  const int32_t* ptr;
  const int32_t* items;
  int32_t n;
  int32_t len(int32_t u) const { return ptr[u + 1] - ptr[u]; }
  const int32_t* row(int32_t u) const { return items + ptr[u]; }
};

// |P_u intersect P_v| of two sorted sets (Section II-A).
int32_t common_items(const Csr& P, int32_t u, int32_t v) {
  const int32_t *a = P.row(u), *ae = a + P.len(u);
  const int32_t *b = P.row(v), *be = b + P.len(v);
  int32_t c = 0;
  while (a < ae && b < be) {
    if (*a < *b) ++a;
    else if (*b < *a) ++b;
    else { ++c; ++a; ++b; }
  }
  return c;
}

// One neighbour of some user: id, |P_u n P_v|, |P_u u P_v|.
struct Nbr {
  int32_t id, inter, uni;
};

// R8: strict "a is a better neighbour than b".  Jaccard a.inter/a.uni compared
// exactly by cross-multiplication; equal similarities go to the lower id.
bool better(const Nbr& a, const Nbr& b) {
  int64_t l = (int64_t)a.inter * b.uni, r = (int64_t)b.inter * a.uni;
  if (l != r) return l > r;
  return a.id < b.id;
}

Nbr make_nbr(const Csr& P, int32_t u, int32_t v) {
  int32_t c = common_items(P, u, v);
  return Nbr{v, c, P.len(u) + P.len(v) - c};
}

void write_row(const std::vector<Nbr>& lst, int32_t k, int32_t* id, int32_t* inter, int32_t* uni) {
  for (int32_t j = 0; j < k; ++j) {
    if (j < (int32_t)lst.size()) { id[j] = lst[j].id; inter[j] = lst[j].inter; uni[j] = lst[j].uni; }
    else { id[j] = -1; inter[j] = 0; uni[j] = 0; }
  }
}

// ------------------------------------------------------------------ clustering
struct Cluster {
  int fn;                      // hash function index i
  std::vector<int32_t> path;   // (key0, eta_1, eta_2, ...) -- R7
  std::vector<int32_t> members;
  bool residual;
  int32_t eta;                 // hash threshold of the next split: the path's last
                               // hash key, or -1 for a first-level key given by a proposer
};

// Recursive split of Section II-D ("Balancing large clusters through
// recursive splitting"): a cluster produced by hash value eta and larger than
// N re-hashes its users with H\eta(u) = min{h(x) : x in P_u, h(x) > eta}.
// Users for whom that is undefined, and users alone in their new group, stay
// in the cluster (its residual, R5); every other group is a new cluster that
// is split again while larger than N.  Emission is depth-first with the
// residual first, which is the canonical order R7.
void split_or_emit(const Csr& P, const std::vector<int32_t>& hfn, int32_t N, Cluster c,
                   std::vector<Cluster>& out) {
  if ((int32_t)c.members.size() <= N || c.residual) { out.push_back(std::move(c)); return; }
  const int32_t eta = c.eta;
  // H\eta(u) for every member; -1 where no item hashes above eta.
  std::vector<int32_t> next_key(c.members.size(), -1);
  std::map<int32_t, std::vector<int32_t>> groups;   // H\eta value -> users, ascending value
  for (size_t a = 0; a < c.members.size(); ++a) {
    int32_t u = c.members[a];
    for (int32_t j = 0; j < P.len(u); ++j) {
      int32_t hv = hfn[P.row(u)[j]];
      if (hv > eta && (next_key[a] < 0 || hv < next_key[a])) next_key[a] = hv;
    }
    if (next_key[a] >= 0) groups[next_key[a]].push_back(u);
  }
  Cluster res{c.fn, c.path, {}, true, c.eta};
  for (size_t a = 0; a < c.members.size(); ++a)
    if (next_key[a] < 0 || groups[next_key[a]].size() == 1) res.members.push_back(c.members[a]);
  if (!res.members.empty()) out.push_back(std::move(res));
  for (auto& g : groups) {
    if (g.second.size() < 2) continue;
    Cluster child{c.fn, c.path, g.second, false, g.first};
    child.path.push_back(g.first);
    split_or_emit(P, hfn, N, std::move(child), out);
  }
}

// Algorithm 1 (clustering with t FastRandomHash functions, Eq. 3) followed by
// the recursive split, for all t functions.
// With `keys` ([t][n], from a learned proposer) the first-level key of user u
// under function i is keys[i][u] instead of H_i(u); such clusters carry no
// hash threshold, so their first split uses the plain FRH key (eta = -1).
// fn_offset numbers the functions of a shard: local function i is the
// run's function fn_offset + i (its generative hash).
std::vector<Cluster> frh_clusters(const Csr& P, int32_t m, int32_t t, int32_t b, int32_t N,
                                  uint64_t seed, const int32_t* htab, const int32_t* keys,
                                  int32_t fn_offset = 0) {
  std::vector<Cluster> out;
  for (int i = 0; i < t; ++i) {
    std::vector<int32_t> hfn(m);
    for (int32_t x = 0; x < m; ++x)
      hfn[x] = htab ? htab[(size_t)i * m + x] : (int32_t)item_hash(seed, fn_offset + i, x, b);
    // B_i[key] <- users whose FRH key is `key` (Eq. 3: H_i(u) = min h_i(x)).
    std::vector<std::vector<int32_t>> B(b + 1);
    for (int32_t u = 0; u < P.n; ++u) {
      int32_t key = b;                                        // R3
      if (keys) key = keys[(size_t)i * P.n + u];
      else
        for (int32_t j = 0; j < P.len(u); ++j) key = std::min(key, hfn[P.row(u)[j]]);
      B[key].push_back(u);
    }
    for (int32_t key = 0; key <= b; ++key) {
      if (B[key].empty()) continue;
      // the empty-profile sentinel cannot split
      Cluster c{i, {key}, B[key], key == b, keys ? -1 : key};
      split_or_emit(P, hfn, N, std::move(c), out);
    }
  }
  return out;
}

// ------------------------------------------------------------------ local KNN
// Brute force inside one cluster (Algorithm 2, first branch; Section IV-B):
// every member is compared with every other member.
void brute_force_cluster(const Csr& P, const std::vector<int32_t>& mem, int32_t k,
                         std::vector<std::vector<Nbr>>& lists, int64_t& pairs) {
  const int32_t M = (int32_t)mem.size();
  lists.assign(M, {});
  for (int32_t a = 0; a < M; ++a) {
    std::vector<Nbr> cand;
    for (int32_t b2 = 0; b2 < M; ++b2) {
      if (b2 == a) continue;
      Nbr e = make_nbr(P, mem[a], mem[b2]);
      if (e.inter > 0) cand.push_back(e);                     // R9
    }
    std::sort(cand.begin(), cand.end(), better);
    if ((int32_t)cand.size() > k) cand.resize(k);
    lists[a] = cand;
  }
  pairs += (int64_t)M * (M - 1) / 2;
}

// Local index drawn for member l of a cluster of size M, from one Philox
// output word: uniform over the other M-1 members (R11).
int32_t draw_other(uint32_t r, int32_t l, int32_t M) {
  int32_t x = (int32_t)(r % (uint32_t)(M - 1));
  return x + (x >= l ? 1 : 0);
}

uint32_t philox_word0(uint64_t seed, uint32_t cluster_no, uint32_t l, uint32_t round, uint32_t j) {
  uint32_t ctr[4] = {cluster_no, l, round, j};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  philox4x32_10(ctr, key, out);
  return out[0];
}

// Greedy refinement inside one cluster (Algorithm 2, second branch; the
// Hyrec strategy of Section IV-B: each user is compared with the neighbours
// of its neighbours, starting from a random graph).  R11: fixed number of
// synchronous rounds; working lists keep zero-similarity entries.
// `pairs` counts similarity evaluations: the k random starting neighbours,
// then per round the candidates not already in the user's list.
struct LocalNbr {
  Nbr e;
  int32_t loc;   // local index inside the cluster
};

void greedy_cluster(const Csr& P, const std::vector<int32_t>& mem, uint32_t cluster_no,
                    int32_t k, uint64_t seed, int32_t rounds, int32_t n_random,
                    std::vector<std::vector<Nbr>>& lists, int64_t& pairs) {
  const int32_t M = (int32_t)mem.size();
  auto by_better = [](const LocalNbr& x, const LocalNbr& y) { return better(x.e, y.e); };
  auto evaluate = [&](int32_t a, int32_t v) { return LocalNbr{make_nbr(P, mem[a], mem[v]), v}; };
  std::vector<std::vector<LocalNbr>> cur(M);
  // Round 0: a random k-graph.
  const int32_t k0 = std::min(k, M - 1);
  for (int32_t a = 0; a < M; ++a) {
    std::vector<int32_t> drawn;
    for (uint32_t j = 0; (int32_t)drawn.size() < k0; ++j) {
      int32_t v = draw_other(philox_word0(seed, cluster_no, (uint32_t)a, 0, j), a, M);
      if (std::find(drawn.begin(), drawn.end(), v) == drawn.end()) drawn.push_back(v);
    }
    for (int32_t v : drawn) cur[a].push_back(evaluate(a, v));
    std::sort(cur[a].begin(), cur[a].end(), by_better);
    pairs += (int64_t)drawn.size();
  }
  // Rounds 1..R, synchronous: every user reads the previous round's lists.
  for (int32_t r = 1; r <= rounds; ++r) {
    std::vector<std::vector<LocalNbr>> next(M);
    for (int32_t a = 0; a < M; ++a) {
      std::set<int32_t> mine, cand;
      for (const LocalNbr& x : cur[a]) { mine.insert(x.loc); cand.insert(x.loc); }
      for (const LocalNbr& x : cur[a])
        for (const LocalNbr& y : cur[x.loc]) cand.insert(y.loc);
      for (int32_t j = 0; j < n_random; ++j)
        cand.insert(draw_other(philox_word0(seed, cluster_no, (uint32_t)a, (uint32_t)r, (uint32_t)j), a, M));
      cand.erase(a);
      std::vector<LocalNbr> scored;
      for (int32_t v : cand) {
        scored.push_back(evaluate(a, v));
        if (!mine.count(v)) ++pairs;
      }
      std::sort(scored.begin(), scored.end(), by_better);
      if ((int32_t)scored.size() > k) scored.resize(k);
      next[a] = scored;
    }
    cur.swap(next);
  }
  lists.assign(M, {});
  for (int32_t a = 0; a < M; ++a)
    for (const LocalNbr& x : cur[a])
      if (x.e.inter > 0) lists[a].push_back(x.e);              // R9
}

// ------------------------------------------------------------------ merge
// Algorithm 3: knn(u) is a bounded structure of size k; add(v, s) keeps the
// k best (R8) distinct neighbours seen so far, reusing the carried counts (R12).
struct BoundedKnn {
  std::vector<Nbr> e;
  void add(const Nbr& x, int32_t k) {
    for (const Nbr& y : e)
      if (y.id == x.id) return;
    e.push_back(x);
    std::sort(e.begin(), e.end(), better);
    if ((int32_t)e.size() > k) e.pop_back();
  }
};

}  // namespace

// ======================================================================
// C entry points (ctypes).  Every array is host memory owned by the caller.
// Return 0 on success, 2 on an invalid CSR, 1 on another invalid argument.
// ======================================================================
extern "C" {

// Shared bodies of the plain and sharded entry points (defined below).
int oracle_frh_cluster_impl(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m,
                            int32_t t, int32_t b, int32_t N, uint64_t seed, const int32_t* htab,
                            const int32_t* keys, int32_t fn_offset, int32_t* cluster_of,
                            int32_t* cptr, int32_t* cusers, int32_t* n_clusters, int32_t* cmeta);
int oracle_cluster_knn_impl(const int32_t* ptr, const int32_t* items, int32_t n,
                            const int32_t* cptr, const int32_t* cusers, int32_t n_clusters,
                            int32_t k, uint64_t seed, int32_t greedy_threshold,
                            int32_t greedy_rounds, int32_t greedy_random, const uint8_t* only,
                            int32_t cluster_base, int32_t* loc_id, int32_t* loc_inter,
                            int32_t* loc_union, int64_t* pairs_out);


uint64_t oracle_mix64(uint64_t z) { return splitmix64_mix(z); }

uint32_t oracle_item_hash(uint64_t seed, int32_t i, int32_t x, int32_t b) {
  return item_hash(seed, i, x, b);
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

// R1: profiles must be sets of valid items, listed in increasing order.
int oracle_validate_csr(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m) {
  if (n < 0 || m < 0) return 1;
  if (ptr[0] != 0) return 2;
  for (int32_t u = 0; u < n; ++u) {
    if (ptr[u + 1] < ptr[u]) return 2;
    for (int32_t j = ptr[u]; j < ptr[u + 1]; ++j) {
      if (items[j] < 0 || items[j] >= m) return 2;
      if (j > ptr[u] && items[j] <= items[j - 1]) return 2;
    }
  }
  return 0;
}

// FRH keys H_i(u) = min_{x in P_u} h_i(x) (Eq. 3), output [t][n].
int oracle_frh_keys(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m, int32_t t,
                    int32_t b, uint64_t seed, const int32_t* htab, int32_t* keys) {
  Csr P{ptr, items, n};
  for (int i = 0; i < t; ++i)
    for (int32_t u = 0; u < n; ++u) {
      int32_t key = b;
      for (int32_t j = 0; j < P.len(u); ++j) {
        int32_t x = P.row(u)[j];
        int32_t hv = htab ? htab[(size_t)i * m + x] : (int32_t)item_hash(seed, i, x, b);
        key = std::min(key, hv);
      }
      keys[(size_t)i * n + u] = key;
    }
  return 0;
}

// MinHash keys of the C^2/MinHash variant (Section V-C, Table 4; Section
// II-E): function i gives every item x a 64-bit value
//   v_i(x) = SplitMix64(K_i xor (x * 0xD6E8FEB86659FD93)),  K_i = function_key(seed, i),
// and user u's key is the item of P_u with the least value (ties to the lower
// item); an empty profile gets m.  One cluster per item, no splitting.
int oracle_minhash_keys(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m, int32_t t,
                        uint64_t seed, int32_t* keys) {
  Csr P{ptr, items, n};
  for (int i = 0; i < t; ++i) {
    const uint64_t K = function_key(seed, i);
    for (int32_t u = 0; u < n; ++u) {
      int32_t key = m;
      uint64_t best = 0;
      for (int32_t j = 0; j < P.len(u); ++j) {
        const int32_t x = P.row(u)[j];
        const uint64_t v = splitmix64_mix(K ^ ((uint64_t)(uint32_t)x * 0xD6E8FEB86659FD93ULL));
        if (key == m || v < best || (v == best && x < key)) {
          best = v;
          key = x;
        }
      }
      keys[(size_t)i * n + u] = key;
    }
  }
  return 0;
}

// Step 1 (Algorithm 1 + recursive split).  Outputs, for t functions:
//   cluster_of[t][n]  final cluster number of user u under function i
//   cptr[n_clusters+1], cusers[t*n]  cluster CSR, members ascending
//   cmeta[n_clusters][4] (optional): function, depth, residual flag, last key
// A shard's clustering (functions fn_offset .. fn_offset + t - 1 of the run,
// numbered locally from 0).
int oracle_frh_cluster_shard(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m,
                             int32_t t, int32_t b, int32_t N, uint64_t seed, int32_t fn_offset,
                             int32_t* cluster_of, int32_t* cptr, int32_t* cusers,
                             int32_t* n_clusters) {
  return oracle_frh_cluster_impl(ptr, items, n, m, t, b, N, seed, nullptr, nullptr, fn_offset,
                                 cluster_of, cptr, cusers, n_clusters, nullptr);
}

int oracle_frh_cluster(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m, int32_t t,
                       int32_t b, int32_t N, uint64_t seed, const int32_t* htab,
                       const int32_t* keys, int32_t* cluster_of, int32_t* cptr, int32_t* cusers,
                       int32_t* n_clusters, int32_t* cmeta) {
  return oracle_frh_cluster_impl(ptr, items, n, m, t, b, N, seed, htab, keys, 0, cluster_of, cptr,
                                 cusers, n_clusters, cmeta);
}

int oracle_frh_cluster_impl(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m,
                            int32_t t, int32_t b, int32_t N, uint64_t seed, const int32_t* htab,
                            const int32_t* keys, int32_t fn_offset, int32_t* cluster_of,
                            int32_t* cptr, int32_t* cusers, int32_t* n_clusters, int32_t* cmeta) {
  if (oracle_validate_csr(ptr, items, n, m)) return 2;
  if (keys)
    for (size_t s2 = 0; s2 < (size_t)t * n; ++s2)
      if (keys[s2] < 0 || keys[s2] >= b) return 1;
  Csr P{ptr, items, n};
  std::vector<Cluster> cl = frh_clusters(P, m, t, b, N, seed, htab, keys, fn_offset);
  int32_t pos = 0;
  cptr[0] = 0;
  for (size_t c = 0; c < cl.size(); ++c) {
    for (int32_t u : cl[c].members) {
      cusers[pos++] = u;
      cluster_of[(size_t)cl[c].fn * n + u] = (int32_t)c;
    }
    cptr[c + 1] = pos;
    if (cmeta) {
      cmeta[4 * c + 0] = cl[c].fn;
      cmeta[4 * c + 1] = (int32_t)cl[c].path.size() - 1;
      cmeta[4 * c + 2] = cl[c].residual ? 1 : 0;
      cmeta[4 * c + 3] = cl[c].eta;
    }
  }
  *n_clusters = (int32_t)cl.size();
  return 0;
}

// Step 2: local KNN of every cluster (Algorithm 2).  Brute force iff
// |C| < greedy_threshold.  Output rows are per cluster slot (position in
// cusers), [t*n][k], sorted by R8 and padded with id -1.  `only` (optional,
// one byte per cluster) restricts the work to the marked clusters; rows of
// the others are left untouched.
// cluster_base: the run's number of this shard's first cluster (the clusters
// of the functions before it), which the greedy random start draws with.
int oracle_cluster_knn_shard(const int32_t* ptr, const int32_t* items, int32_t n,
                             const int32_t* cptr, const int32_t* cusers, int32_t n_clusters,
                             int32_t k, uint64_t seed, int32_t greedy_threshold,
                             int32_t greedy_rounds, int32_t cluster_base, int32_t* loc_id,
                             int32_t* loc_inter, int32_t* loc_union, int64_t* pairs_out) {
  return oracle_cluster_knn_impl(ptr, items, n, cptr, cusers, n_clusters, k, seed,
                                 greedy_threshold, greedy_rounds, 0, nullptr, cluster_base, loc_id,
                                 loc_inter, loc_union, pairs_out);
}

int oracle_cluster_knn(const int32_t* ptr, const int32_t* items, int32_t n, const int32_t* cptr,
                       const int32_t* cusers, int32_t n_clusters, int32_t k, uint64_t seed,
                       int32_t greedy_threshold, int32_t greedy_rounds, int32_t greedy_random,
                       const uint8_t* only, int32_t* loc_id, int32_t* loc_inter,
                       int32_t* loc_union, int64_t* pairs_out) {
  return oracle_cluster_knn_impl(ptr, items, n, cptr, cusers, n_clusters, k, seed,
                                 greedy_threshold, greedy_rounds, greedy_random, only, 0, loc_id,
                                 loc_inter, loc_union, pairs_out);
}

int oracle_cluster_knn_impl(const int32_t* ptr, const int32_t* items, int32_t n,
                            const int32_t* cptr, const int32_t* cusers, int32_t n_clusters,
                            int32_t k, uint64_t seed, int32_t greedy_threshold,
                            int32_t greedy_rounds, int32_t greedy_random, const uint8_t* only,
                            int32_t cluster_base, int32_t* loc_id, int32_t* loc_inter,
                            int32_t* loc_union, int64_t* pairs_out) {
  Csr P{ptr, items, n};
  int64_t pairs = 0;
  for (int32_t c = 0; c < n_clusters; ++c) {
    if (only && !only[c]) continue;
    std::vector<int32_t> mem(cusers + cptr[c], cusers + cptr[c + 1]);
    std::vector<std::vector<Nbr>> lists;
    if ((int32_t)mem.size() < greedy_threshold || mem.size() < 2)
      brute_force_cluster(P, mem, k, lists, pairs);
    else
      greedy_cluster(P, mem, (uint32_t)(c + cluster_base), k, seed, greedy_rounds, greedy_random,
                     lists, pairs);
    for (size_t a = 0; a < mem.size(); ++a) {
      size_t s = (size_t)cptr[c] + a;
      write_row(lists[a], k, loc_id + s * k, loc_inter + s * k, loc_union + s * k);
    }
  }
  if (pairs_out) *pairs_out = pairs;
  return 0;
}

// Step 3 (Algorithm 3): fold, for every user, the local lists of the t
// clusters it belongs to, function by function and cluster by cluster.
int oracle_merge_topk(const int32_t* cptr, const int32_t* cusers, int32_t n_clusters, int32_t n,
                      int32_t k, const int32_t* loc_id, const int32_t* loc_inter,
                      const int32_t* loc_union, int32_t* nbr_id, int32_t* nbr_inter,
                      int32_t* nbr_union) {
  std::vector<BoundedKnn> knn(n);
  for (int32_t c = 0; c < n_clusters; ++c)
    for (int32_t s = cptr[c]; s < cptr[c + 1]; ++s) {
      int32_t u = cusers[s];
      for (int32_t j = 0; j < k; ++j) {
        size_t e = (size_t)s * k + j;
        if (loc_id[e] < 0) continue;
        knn[u].add(Nbr{loc_id[e], loc_inter[e], loc_union[e]}, k);
      }
    }
  for (int32_t u = 0; u < n; ++u)
    write_row(knn[u].e, k, nbr_id + (size_t)u * k, nbr_inter + (size_t)u * k,
              nbr_union + (size_t)u * k);
  return 0;
}

// The whole method: Step 1, Step 2, Step 3.
int oracle_build(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m, int32_t k,
                 int32_t t, int32_t b, int32_t N, uint64_t seed, int32_t greedy_threshold,
                 int32_t greedy_rounds, int32_t greedy_random, const int32_t* htab,
                 const int32_t* keys, int32_t* nbr_id, int32_t* nbr_inter, int32_t* nbr_union,
                 int64_t* pairs_out) {
  std::vector<int32_t> cluster_of((size_t)t * n), cptr((size_t)t * n + 1), cusers((size_t)t * n);
  int32_t nc = 0;
  int rc = oracle_frh_cluster(ptr, items, n, m, t, b, N, seed, htab, keys, cluster_of.data(),
                              cptr.data(), cusers.data(), &nc, nullptr);
  if (rc) return rc;
  std::vector<int32_t> li((size_t)t * n * k), lc((size_t)t * n * k), lu((size_t)t * n * k);
  oracle_cluster_knn(ptr, items, n, cptr.data(), cusers.data(), nc, k, seed, greedy_threshold,
                     greedy_rounds, greedy_random, nullptr, li.data(), lc.data(), lu.data(),
                     pairs_out);
  return oracle_merge_topk(cptr.data(), cusers.data(), nc, n, k, li.data(), lc.data(), lu.data(),
                           nbr_id, nbr_inter, nbr_union);
}

// ------------------------------------------------------------------ GoldFinger
// Section II-F computes the local KNN graphs with GoldFinger, a 64- to
// 8096-bit summary of each profile from which Jaccard values are estimated
// (1024 bits in Section IV-E), without giving its construction.  R17: item x
// sets one bit of B,
//   fp(x) = floor((SplitMix64(K_g ^ x * 0xC2B2AE3D27D4EB4F) >> 32) * B / 2^32),
//   K_g = SplitMix64(seed ^ 0x474F4C4446494E47),
// the fingerprint of u is the set F_u = {fp(x) : x in P_u}, and J(u, v) is
// estimated by |F_u n F_v| / |F_u u F_v|: the Jaccard similarity of the
// fingerprints, so Steps 2-3 run unchanged on the fingerprints as profiles.
uint32_t fingerprint_bit(uint64_t seed, int32_t x, int32_t bits) {
  const uint64_t key = splitmix64_mix(seed ^ 0x474F4C4446494E47ULL);
  const uint64_t z = splitmix64_mix(key ^ ((uint64_t)(uint32_t)x * 0xC2B2AE3D27D4EB4FULL));
  return (uint32_t)(((z >> 32) * (uint64_t)(uint32_t)bits) >> 32);
}

// Fingerprints of every user as a CSR of sorted bit positions (rows never
// longer than the profiles, so out_items needs at most nnz entries).
int oracle_goldfinger(const int32_t* ptr, const int32_t* items, int32_t n, int32_t bits,
                      uint64_t seed, int32_t* out_ptr, int32_t* out_items) {
  if (bits < 1) return 1;
  out_ptr[0] = 0;
  for (int32_t u = 0; u < n; ++u) {
    std::set<int32_t> f;
    for (int32_t e = ptr[u]; e < ptr[u + 1]; ++e) f.insert((int32_t)fingerprint_bit(seed, items[e], bits));
    int32_t o = out_ptr[u];
    for (int32_t x : f) out_items[o++] = x;
    out_ptr[u + 1] = o;
  }
  return 0;
}

// The method with estimated similarities: Step 1 on the profiles (ptr,
// items, m items), Steps 2 and 3 on the similarity profiles (sptr, sitems),
// e.g. GoldFinger fingerprints.
int oracle_build_sim(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m,
                     const int32_t* sptr, const int32_t* sitems, int32_t k, int32_t t, int32_t b,
                     int32_t N, uint64_t seed, int32_t greedy_threshold, int32_t greedy_rounds,
                     int32_t greedy_random, int32_t* nbr_id, int32_t* nbr_inter,
                     int32_t* nbr_union, int64_t* pairs_out) {
  std::vector<int32_t> cluster_of((size_t)t * n), cptr((size_t)t * n + 1), cusers((size_t)t * n);
  int32_t nc = 0;
  int rc = oracle_frh_cluster(ptr, items, n, m, t, b, N, seed, nullptr, nullptr, cluster_of.data(),
                              cptr.data(), cusers.data(), &nc, nullptr);
  if (rc) return rc;
  std::vector<int32_t> li((size_t)t * n * k), lc((size_t)t * n * k), lu((size_t)t * n * k);
  oracle_cluster_knn(sptr, sitems, n, cptr.data(), cusers.data(), nc, k, seed, greedy_threshold,
                     greedy_rounds, greedy_random, nullptr, li.data(), lc.data(), lu.data(),
                     pairs_out);
  return oracle_merge_topk(cptr.data(), cusers.data(), nc, n, k, li.data(), lc.data(), lu.data(),
                           nbr_id, nbr_inter, nbr_union);
}

// Exact |P_u n P_v| and |P_u u P_v| of given neighbour rows (id -1: empty
// slot, counts 0), for Eq. 1 on exact similarities.
int oracle_exact_counts(const int32_t* ptr, const int32_t* items, int32_t n, int32_t k,
                        const int32_t* nbr_id, int32_t* out_inter, int32_t* out_union) {
  Csr P{ptr, items, n};
  for (int32_t u = 0; u < n; ++u)
    for (int32_t j = 0; j < k; ++j) {
      const size_t e = (size_t)u * k + j;
      if (nbr_id[e] < 0) {
        out_inter[e] = out_union[e] = 0;
        continue;
      }
      Nbr x = make_nbr(P, u, nbr_id[e]);
      out_inter[e] = x.inter;
      out_union[e] = x.uni;
    }
  return 0;
}

// Exact KNN by global brute force (Section IV-B, "Brute force"): for each
// query user, all other users are candidates.  queries == NULL means all.
int oracle_bruteforce_knn(const int32_t* ptr, const int32_t* items, int32_t n, int32_t k,
                          const int32_t* queries, int32_t nq, int32_t* nbr_id, int32_t* nbr_inter,
                          int32_t* nbr_union) {
  Csr P{ptr, items, n};
  int32_t rows = queries ? nq : n;
  for (int32_t q = 0; q < rows; ++q) {
    int32_t u = queries ? queries[q] : q;
    std::vector<Nbr> cand;
    for (int32_t v = 0; v < n; ++v) {
      if (v == u) continue;
      Nbr e = make_nbr(P, u, v);
      if (e.inter > 0) cand.push_back(e);
    }
    std::sort(cand.begin(), cand.end(), better);
    if ((int32_t)cand.size() > k) cand.resize(k);
    write_row(cand, k, nbr_id + (size_t)q * k, nbr_inter + (size_t)q * k, nbr_union + (size_t)q * k);
  }
  return 0;
}

// Eq. 1: average edge similarity, sum_u sum_{v in knn(u)} J(u,v) / (k * rows),
// summed in row order then slot order.  Empty slots count as similarity 0.
double oracle_avg_sim(const int32_t* nbr_inter, const int32_t* nbr_union, int32_t rows, int32_t k) {
  double s = 0.0;
  for (int32_t r = 0; r < rows; ++r)
    for (int32_t j = 0; j < k; ++j) {
      size_t e = (size_t)r * k + j;
      if (nbr_union[e] > 0) s += (double)nbr_inter[e] / (double)nbr_union[e];
    }
  return s / ((double)k * (double)rows);
}

// ======================================================================
// Learned proposer (no counterpart in the paper): the network of the
// library's proposer written out in FP64, with the operands rounded to BF16
// where the library stores them in BF16 (table, weights, bag sums, hidden
// activations; in the backward pass the logit gradients and the ReLU-masked
// hidden gradients).  Parameters are given as FP32 masters.
// ======================================================================
}  // extern "C"

namespace {

// Round-to-nearest-even of an FP32 value to BF16 (the upper 16 bits).
double to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return (double)r;
}

struct Net {
  int D, H, t, b, T, rows;
  uint64_t seed;
  std::vector<double> E, W1, b1, W2, b2;   // E, W1, W2 rounded to BF16
};

bool g_exact = false;   // true: no BF16 rounding anywhere (finite-difference checks)

double rnd(float f) { return g_exact ? (double)f : to_bf16(f); }

Net make_net(int D, int H, int t, int b, int rows_log2, uint64_t seed, const float* E,
             const float* W1, const float* b1, const float* W2, const float* b2) {
  Net n{D, H, t, b, t * b, 1 << rows_log2, seed, {}, {}, {}, {}, {}};
  n.E.resize((size_t)n.rows * D);
  for (size_t i = 0; i < n.E.size(); ++i) n.E[i] = rnd(E[i]);
  n.W1.resize((size_t)D * H);
  for (size_t i = 0; i < n.W1.size(); ++i) n.W1[i] = rnd(W1[i]);
  n.b1.assign(b1, b1 + H);
  n.W2.resize((size_t)H * n.T);
  for (size_t i = 0; i < n.W2.size(); ++i) n.W2[i] = rnd(W2[i]);
  n.b2.assign(b2, b2 + n.T);
  return n;
}

size_t emb_row(const Net& n, int32_t x) {
  return (size_t)(splitmix64_mix(n.seed ^ (uint64_t)(uint32_t)x) & (uint64_t)(n.rows - 1));
}

struct Fwd {
  std::vector<double> e, e16, hpre, h16, z;
};

// e = bag of rows; hpre = W1^T e16 + b1; h16 = bf16(ReLU(hpre)); z = W2^T h16 + b2
Fwd forward(const Net& n, const Csr& P, int32_t u) {
  Fwd f;
  f.e.assign(n.D, 0.0);
  for (int32_t j = 0; j < P.len(u); ++j) {
    const size_t r = emb_row(n, P.row(u)[j]);
    for (int d = 0; d < n.D; ++d) f.e[d] += n.E[r * n.D + d];
  }
  f.e16.resize(n.D);
  for (int d = 0; d < n.D; ++d) f.e16[d] = g_exact ? f.e[d] : to_bf16((float)f.e[d]);
  f.hpre.assign(n.H, 0.0);
  f.h16.assign(n.H, 0.0);
  for (int h = 0; h < n.H; ++h) {
    double s = n.b1[h];
    for (int d = 0; d < n.D; ++d) s += f.e16[d] * n.W1[(size_t)d * n.H + h];
    f.hpre[h] = s;
    f.h16[h] = g_exact ? std::max(s, 0.0) : to_bf16((float)std::max(s, 0.0));
  }
  f.z.assign(n.T, 0.0);
  for (int c = 0; c < n.T; ++c) {
    double s = n.b2[c];
    for (int h = 0; h < n.H; ++h) s += f.h16[h] * n.W2[(size_t)h * n.T + c];
    f.z[c] = s;
  }
  return f;
}

}  // namespace

extern "C" {

// 1: compute the network in plain FP64 without BF16 rounding (for finite
// differences); 0 (default): round where the library stores BF16.
void oracle_model_exact(int32_t on) { g_exact = on != 0; }

// Logits z[n_users][t*b] of every user and keys[t][n_users] = argmax per head
// (ties to the lower bucket).
int oracle_model_forward(int32_t D, int32_t H, int32_t t, int32_t b, int32_t rows_log2,
                         uint64_t seed, const float* E, const float* W1, const float* b1,
                         const float* W2, const float* b2, const int32_t* ptr,
                         const int32_t* items, int32_t n, double* z, int32_t* keys) {
  Net net = make_net(D, H, t, b, rows_log2, seed, E, W1, b1, W2, b2);
  Csr P{ptr, items, n};
  for (int32_t u = 0; u < n; ++u) {
    Fwd f = forward(net, P, u);
    if (z) std::copy(f.z.begin(), f.z.end(), z + (size_t)u * net.T);
    for (int j = 0; j < t; ++j) {
      int best = 0;
      for (int c = 1; c < b; ++c)
        if (f.z[(size_t)j * b + c] > f.z[(size_t)j * b + best]) best = c;
      keys[(size_t)j * n + u] = best;
    }
  }
  return 0;
}

// Loss of a batch of pairs and its gradients, in FP64 (the library's training
// objective): rows 0..P-1 are the pairs' first users, P..2P-1 the second;
//   L = sum_{i,j} -log(S_ij + 1e-9) / (P t) + lambda sum_j sum_c m_jc log(b m_jc) / t,
//   S_ij = sum_c p_{u_i,jc} p_{v_i,jc},  m_jc = mean over the 2P rows of p_jc.
int oracle_model_grads(int32_t D, int32_t H, int32_t t, int32_t b, int32_t rows_log2,
                       uint64_t seed, const float* E, const float* W1, const float* b1,
                       const float* W2, const float* b2, const int32_t* ptr,
                       const int32_t* items, int32_t n, const int32_t* pairs, int32_t Pn,
                       double lambda, double* loss, double* gE, double* gW1, double* gb1,
                       double* gW2, double* gb2) {
  Net net = make_net(D, H, t, b, rows_log2, seed, E, W1, b1, W2, b2);
  Csr P{ptr, items, n};
  const int R = 2 * Pn, T = net.T;
  std::vector<Fwd> f(R);
  std::vector<double> p((size_t)R * T);
  for (int r = 0; r < R; ++r) {
    const int32_t u = r < Pn ? pairs[2 * r] : pairs[2 * (r - Pn) + 1];
    f[r] = forward(net, P, u);
    for (int j = 0; j < t; ++j) {
      double mx = -1e300, sum = 0.0;
      for (int c = 0; c < b; ++c) mx = std::max(mx, f[r].z[(size_t)j * b + c]);
      for (int c = 0; c < b; ++c) sum += std::exp(f[r].z[(size_t)j * b + c] - mx);
      for (int c = 0; c < b; ++c)
        p[(size_t)r * T + (size_t)j * b + c] = std::exp(f[r].z[(size_t)j * b + c] - mx) / sum;
    }
  }
  std::vector<double> m(T, 0.0);
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < T; ++c) m[c] += p[(size_t)r * T + c] / R;
  // dL/dp
  std::vector<double> g((size_t)R * T, 0.0);
  double lp = 0.0, lb = 0.0;
  const double scale = 1.0 / ((double)Pn * t), eps = 1e-9;
  for (int i = 0; i < Pn; ++i)
    for (int j = 0; j < t; ++j) {
      const double* pu = &p[(size_t)i * T + (size_t)j * b];
      const double* pv = &p[(size_t)(i + Pn) * T + (size_t)j * b];
      double S = 0.0;
      for (int c = 0; c < b; ++c) S += pu[c] * pv[c];
      lp += -std::log(S + eps) * scale;
      for (int c = 0; c < b; ++c) {
        g[(size_t)i * T + (size_t)j * b + c] += -pv[c] / (S + eps) * scale;
        g[(size_t)(i + Pn) * T + (size_t)j * b + c] += -pu[c] / (S + eps) * scale;
      }
    }
  for (int c = 0; c < T; ++c) {
    if (m[c] > 0) lb += lambda * m[c] * std::log((double)b * m[c]) / t;
    const double gb = lambda * (std::log(std::max((double)b * m[c], 1e-300)) + 1.0) / ((double)R * t);
    for (int r = 0; r < R; ++r) g[(size_t)r * T + c] += gb;
  }
  loss[0] = lp;
  loss[1] = lb;
  // softmax backward, then the layers
  std::fill(gE, gE + (size_t)net.rows * D, 0.0);
  std::fill(gW1, gW1 + (size_t)D * H, 0.0);
  std::fill(gb1, gb1 + H, 0.0);
  std::fill(gW2, gW2 + (size_t)H * T, 0.0);
  std::fill(gb2, gb2 + T, 0.0);
  for (int r = 0; r < R; ++r) {
    std::vector<double> dz(T);
    for (int j = 0; j < t; ++j) {
      double s = 0.0;
      for (int c = 0; c < b; ++c) s += p[(size_t)r * T + (size_t)j * b + c] * g[(size_t)r * T + (size_t)j * b + c];
      for (int c = 0; c < b; ++c) {
        const size_t q = (size_t)j * b + c;
        dz[q] = p[(size_t)r * T + q] * (g[(size_t)r * T + q] - s);
        if (!g_exact) dz[q] = to_bf16((float)dz[q]);   // stored in BF16 for the backward GEMMs
      }
    }
    std::vector<double> dh(H, 0.0);
    for (int c = 0; c < T; ++c) {
      gb2[c] += dz[c];
      for (int h = 0; h < H; ++h) {
        gW2[(size_t)h * T + c] += f[r].h16[h] * dz[c];
        dh[h] += dz[c] * net.W2[(size_t)h * T + c];
      }
    }
    std::vector<double> de(D, 0.0);
    for (int h = 0; h < H; ++h) {
      if (f[r].hpre[h] <= 0.0) continue;
      if (!g_exact) dh[h] = to_bf16((float)dh[h]);     // the masked dh, stored in BF16
      gb1[h] += dh[h];
      for (int d = 0; d < D; ++d) {
        gW1[(size_t)d * H + h] += f[r].e16[d] * dh[h];
        de[d] += dh[h] * net.W1[(size_t)d * H + h];
      }
    }
    const int32_t u = r < Pn ? pairs[2 * r] : pairs[2 * (r - Pn) + 1];
    for (int32_t j = 0; j < P.len(u); ++j) {
      const size_t row = emb_row(net, P.row(u)[j]);
      for (int d = 0; d < D; ++d) gE[row * D + d] += de[d];
    }
  }
  return 0;
}

}  // extern "C"
