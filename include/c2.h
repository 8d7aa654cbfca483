/*
 * c2.h -- C ABI of the GB300 (sm_103a) Cluster-and-Conquer KNN-graph library.
 *
 * Cluster-and-Conquer (C^2), Giakkoupis, Kermarrec, Ruas & Taiani,
 * arXiv 2010.11497.  The library builds an approximate k-nearest-neighbour
 * graph of users described by binary item profiles, under the Jaccard
 * similarity J(u,v) = |P_u n P_v| / |P_u u P_v| (Section II-A), in three steps:
 *
 *   1. clustering with t FastRandomHash functions, H_i(u) = min h_i(x) over
 *      the user's items (Eq. 3, Algorithm 1), with recursive splitting of
 *      clusters larger than N (Section II-D);
 *   2. a KNN graph inside every cluster, by brute force for clusters with
 *      fewer than `greedy_threshold` users and by greedy neighbours-of-
 *      neighbours refinement otherwise (Algorithm 2, Section II-F);
 *   3. a merge of each user's t cluster-local lists into one top-k list
 *      (Algorithm 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are DEVICE pointers (CUDA global memory of the current
 *   device); pointers named h_* are HOST pointers.  All are owned by the
 *   caller and only borrowed until the work queued on `stream` completes.
 * - Profiles are CSR: d_csr_ptr[n_users+1] (int32, d_csr_ptr[0] == 0,
 *   non-decreasing) and d_csr_items[nnz] (int32 item ids in [0, n_items),
 *   strictly increasing within a row: profiles are sets).
 * - Every function is asynchronous on `stream` unless stated otherwise.  The
 *   library allocates no device memory: scratch space comes from the caller's
 *   workspace `d_ws` of at least c2_workspace_size() bytes (256-byte aligned).
 * - A workspace must start with a cleared status header (its first 256
 *   bytes zero, or c2_reset_status()); c2_frh_cluster, c2_build_knn_graph,
 *   c2_bruteforce_knn and c2_build_knn_graph_host clear it themselves.
 * - Host-detected argument errors are returned at once.  Errors detected on
 *   the device (an invalid CSR, a bounded wait that ran out) are recorded in
 *   a status word inside the workspace; read it with c2_get_status().  Once a
 *   device error is recorded, later kernels of the same workspace return
 *   without touching memory.
 * - Neighbour lists are rows of k slots: id, |P_u n P_v| (inter) and
 *   |P_u u P_v| (union), sorted best first.  "Better" compares Jaccard values
 *   exactly by integer cross-multiplication, equal values going to the lower
 *   user id.  Users with no common item are never listed; unused slots hold
 *   id -1 and counts 0.  Users, items and buckets are 0-based.
 * - Limits: 1 <= k <= 32, 1 <= t <= 64, 1 <= b <= 65536, N >= 2,
 *   nnz < 2^31, t * n_users < 2^31, every profile shorter than 65536 items.
 *   Anything else returns C2_ERR_UNSUPPORTED (profile lengths: on the device).
 */
#ifndef C2_H
#define C2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* c2_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  C2_OK = 0,
  C2_ERR_INVALID_ARG = 1,  /* a NULL pointer, a negative size, k/t/b/N out of range      */
  C2_ERR_INVALID_CSR = 2,  /* profiles are not sorted sets of valid item ids            */
  C2_ERR_UNSUPPORTED = 3,  /* a size beyond the documented limits                        */
  C2_ERR_WORKSPACE = 4,    /* d_ws NULL, misaligned or smaller than c2_workspace_size()  */
  C2_ERR_CUDA = 5,         /* a CUDA runtime call failed                                 */
  C2_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                         */
  C2_ERR_QUALITY_FALLBACK = 7 /* informational: the learned proposer fell back to FRH    */
} c2_status;

/* Strategy used to count common items inside clusters (Step 2).  When the
 * item universe is too large for a shared-memory item table (more than about
 * 57,000 items), every strategy but MERGE counts through a shared-memory hash
 * table of the 32 query users' items instead, provided no profile exceeds
 * 4,096 items; otherwise rows are counted by merges. */
enum {
  C2_STRATEGY_AUTO = -1,   /* per (cluster size, density) bucket: table or tensor cores,
                              whichever the autotuner measured faster; tuned table shape  */
  C2_STRATEGY_MERGE = 0,   /* sorted-list merge, one warp per query user                  */
  C2_STRATEGY_TABLE32 = 1, /* shared-memory item table, 32 query users per block          */
  C2_STRATEGY_TABLE64 = 2, /* shared-memory item table, 64 query users per block          */
  C2_STRATEGY_MMA = 3      /* 0/1 FP8 products on the tensor cores (tcgen05, exact FP32
                              sums) for every cluster of 128 members or more whose items
                              held by two members or more number 1 to 65,536, in item
                              universes of at most 524,288 items; the table otherwise      */
};

typedef struct {
  int32_t greedy_threshold; /* brute force iff |C| < greedy_threshold (Algorithm 2);
                               <= 0 selects the paper's rho*k^2 with rho = 5 (Section II-F) */
  int32_t greedy_rounds;    /* synchronous refinement rounds; < 0 selects 10               */
  int32_t greedy_random;    /* extra random candidates per user and round; default 0       */
  int32_t strategy;         /* C2_STRATEGY_*                                               */
  const int32_t* d_hash_table; /* optional explicit generative hashes h_i(x), device int32
                               [t][n_items] with values in [0, b); NULL = the library's
                               seeded hash (a test hook for hand-worked examples)          */
  int64_t gram_budget_bytes;/* cap on the intersection-count matrices of greedy clusters
                               held at once; <= 0 selects 2 GiB                            */
  const int32_t* d_keys;    /* optional first-level cluster keys, device int32 [t][n_users]
                               in [0, b), e.g. from c2_model_propose; NULL = FastRandomHash.
                               Oversized clusters are then split by FastRandomHash with no
                               threshold (the first split key is H_i(u) itself)            */
  int32_t greedy_max_draws; /* bound on the Philox draws per member for the random start of
                               a greedy cluster (round 0), made 32 at a time; <= 0 selects
                               2^24, which uniform draws never reach.  When the bound stops
                               the draws before min(k, M-1) distinct members are found (any
                               bound below 32, for instance), C2_ERR_TIMEOUT is recorded in
                               the status word                                             */
  int32_t sim_n_items;      /* item universe of d_sim_ptr/d_sim_items (below)              */
  const int32_t* d_sim_ptr; /* optional similarity profiles for Steps 2-3 of
                               c2_build_knn_graph (device CSR [n_users+1] / items in
                               [0, sim_n_items), sets, no more entries than the
                               profiles), e.g. GoldFinger fingerprints from
                               c2_goldfinger: clusters come from the profiles, the local
                               KNN graphs and the merge from these (Section II-F); NULL =
                               the profiles themselves                                     */
  const int32_t* d_sim_items;
  const uint32_t* d_sim_bits; /* optional packed bit rows of the profiles the local KNN
                               graphs are computed on (d_sim_* in c2_build_knn_graph, the
                               CSR itself in c2_cluster_knn): [n_users][sim_n_items / 32]
                               words, as c2_goldfinger's d_fp_bits; with sim_n_items a
                               multiple of 128 the tensor-core count matrices then read
                               whole rows (no per-cluster remap)                          */
  int32_t fn_offset;        /* sharding by hash function: this call's functions 0 .. t-1 are
                               the run's functions fn_offset .. fn_offset + t - 1 (their
                               generative hashes); default 0                              */
  int32_t cluster_base;     /* sharding by hash function: the run's number of this call's
                               first cluster (the clusters of the functions before
                               fn_offset), which the greedy random starts draw with;
                               default 0.  G shards' local rows and slot maps,
                               concatenated in function order, merge to the graph of one
                               call with all t functions                                   */
} c2_options;

/* Run statistics, filled by c2_get_stats(). */
typedef struct {
  int64_t pairs;            /* similarity evaluations of the method: M(M-1)/2 per
                               brute-force cluster plus the greedy candidate evaluations   */
  int64_t gram_pairs;       /* count-matrix elements (rows padded to 8) of every cluster
                               with a count matrix (brute force of 9 members or more, and
                               greedy)                                                     */
  int32_t n_clusters;       /* clusters after splitting, all t functions                   */
  int32_t split_levels;     /* recursive-split levels that found an oversized cluster      */
  int32_t n_greedy_clusters;
  int32_t max_cluster;      /* largest cluster                                             */
  int32_t max_profile;      /* longest profile                                             */
  int32_t greedy_users;     /* users (slots) in greedy clusters                            */
  int64_t item_visits_brute;/* profile items walked by the shared-memory table kernel:     */
  int64_t item_visits_greedy; /* brute-force clusters / greedy intersection matrices       */
  int64_t greedy_visits;    /* neighbour-list entries examined by greedy rounds            */
  int64_t greedy_computed;  /* (user, round) pairs a greedy round computed, not repeated  */
  int64_t greedy_evaluated; /* fresh candidates whose counts a greedy round looked up (the
                               method's other evaluations come from neighbour lists known
                               to repeat the previous round's candidates)                 */
  int64_t brute_gram_elems; /* count-matrix elements (rows padded to 8) of brute-force
                               clusters with a count matrix                                */
  int32_t brute_rows;       /* users of those clusters (rows ranked by the row kernel)     */
  int32_t reserved;
  int64_t brute_pairs;      /* M(M-1)/2 over brute-force clusters                          */
  int64_t greedy_pairs;     /* M(M-1)/2 over greedy clusters: with brute_pairs, the pairs
                               whose intersections were counted (greedy rounds look counts
                               up in their clusters' count matrices)                       */
  int64_t tc_macs;          /* tensor-core multiply-adds issued for count matrices          */
  int32_t tc_clusters;      /* count matrices computed on the tensor cores                 */
  int32_t tc_tiles;         /* their 128 x 256 tiles                                       */
  int32_t select_general;   /* brute-force rows with more than 64 candidates tied at their
                               k-th value, ranked by the general path                      */
  int32_t direct_users;     /* members of greedy clusters refined without a count matrix
                               (over 10,240 members, or a matrix beyond gram_budget_bytes):
                               their counts come from the profiles, one warp per member    */
} c2_stats;

/* Fills *opt with the defaults described above.  Never fails. */
void c2_default_options(c2_options* opt);

/* Human-readable name of a status code (static storage). */
const char* c2_status_string(c2_status s);

/* Bytes of workspace the entry points below need for these sizes (the
 * maximum over all of them).  Returns 0 on invalid sizes.  Host only. */
size_t c2_workspace_size(int32_t n_users, int64_t nnz, int32_t n_items, int32_t k, int32_t t,
                         int32_t b, int32_t N, const c2_options* opt);

/* Step 1 (Algorithm 1 + recursive split of Section II-D).  For each hash
 * function i < t and user u, cluster_of[i*n_users+u] is the number of u's
 * final cluster.  Clusters are numbered by function, then by their path of
 * hash keys (key, then each split key) with a split cluster's residual --
 * the users left in it -- before its sub-clusters; members are listed in
 * increasing user id.  The residual of a split is never split again.
 * Outputs (device, caller-allocated):
 *   d_cluster_of[t*n_users], d_cptr[t*n_users+1] (cluster offsets into
 *   d_cusers; entries past *d_n_clusters are left undefined),
 *   d_cusers[t*n_users], d_n_clusters (one int32),
 *   d_cmeta (optional, [t*n_users][4]: function, split depth, residual flag,
 *   last key of the cluster's path -- the hash threshold its split used, -1
 *   for a first-level key given through c2_options.d_keys).
 * This call synchronises `stream` once per split level to read the number of
 * oversized clusters. */
c2_status c2_frh_cluster(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                         int32_t n_items, int32_t t, int32_t b, int32_t N, uint64_t seed,
                         const c2_options* opt, int32_t* d_cluster_of, int32_t* d_cptr,
                         int32_t* d_cusers, int32_t* d_n_clusters, int32_t* d_cmeta, void* d_ws,
                         size_t ws_bytes, c2_stream_t stream);

/* First-level keys of the C^2/MinHash variant (Section V-C, Table 4, which
 * replaces FastRandomHash by MinHash; Section II-E compares the two).  Function
 * i < t gives item x the 64-bit value
 *   v_i(x) = SplitMix64(K_i ^ (x * 0xD6E8FEB86659FD93)),
 *   K_i = SplitMix64(seed + (i + 1) * 0x9E3779B97F4A7C15)
 * (SplitMix64 = the output function of Steele, Lea & Flood, OOPSLA 2014), and
 * d_keys[i*n_users+u] = the item of u's profile with the least value (ties to
 * the lower item), n_items for an empty profile.  The variant clusters users
 * by these keys, one cluster per item and no splitting: pass d_keys through
 * c2_options.d_keys to c2_build_knn_graph with b = n_items + 1 (at most 65,536)
 * and N = n_users.  The CSR is validated first (C2_ERR_INVALID_CSR through the
 * status word).  Workspace: one 256-byte status header (d_ws 256-byte aligned,
 * ws_bytes >= 256).  Asynchronous on `stream`. */
c2_status c2_minhash_keys(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                          int32_t n_items, int32_t t, uint64_t seed, int32_t* d_keys, void* d_ws,
                          size_t ws_bytes, c2_stream_t stream);

/* Step 2 (Algorithm 2): the KNN graph inside every cluster given by
 * (d_cptr, d_cusers, d_n_clusters) as produced by c2_frh_cluster.  Outputs
 * one row of k per cluster slot s (a position in d_cusers):
 * d_loc_id/d_loc_inter/d_loc_union[t*n_users][k].
 * Greedy clusters start from a random k-graph drawn with Philox4x32-10
 * (key = seed, counter = (cluster number, member index, round, draw)) and
 * refine every member's list with its neighbours' neighbours for
 * greedy_rounds synchronous rounds.  A greedy cluster of more than 10,240
 * members, or whose M x round_up(M, 8) 16-bit count matrix exceeds
 * gram_budget_bytes, counts its similarities from the profiles instead (one
 * warp per member; needs k + k^2 + greedy_random <= 1536, else
 * C2_ERR_UNSUPPORTED); the rows are the same.  The CSR is not validated
 * again: it must be the one c2_frh_cluster validated.  Synchronises `stream`
 * once to size the greedy phase. */
c2_status c2_cluster_knn(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                         int32_t n_items, int32_t t, const int32_t* d_cptr,
                         const int32_t* d_cusers, const int32_t* d_n_clusters, int32_t k,
                         uint64_t seed, const c2_options* opt, int32_t* d_loc_id,
                         int32_t* d_loc_inter, int32_t* d_loc_union, void* d_ws,
                         size_t ws_bytes, c2_stream_t stream);

/* Step 3 (Algorithm 3): per user, the k best distinct neighbours found in its
 * t cluster-local rows.  d_cusers[t*n_users] maps slots to users (each
 * function's slots are one permutation of the users).  Outputs
 * d_nbr_id/d_nbr_inter/d_nbr_union[n_users][k]. */
c2_status c2_merge_topk(const int32_t* d_cusers, int32_t n_users, int32_t t, int32_t k,
                        const int32_t* d_loc_id, const int32_t* d_loc_inter,
                        const int32_t* d_loc_union, int32_t* d_nbr_id, int32_t* d_nbr_inter,
                        int32_t* d_nbr_union, void* d_ws, size_t ws_bytes, c2_stream_t stream);

/* The whole method: Steps 1-3.  Outputs d_nbr_*[n_users][k]. */
c2_status c2_build_knn_graph(const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                             int32_t n_users, int32_t n_items, int32_t k, int32_t t, int32_t b,
                             int32_t N, uint64_t seed, const c2_options* opt, int32_t* d_nbr_id,
                             int32_t* d_nbr_inter, int32_t* d_nbr_union, void* d_ws,
                             size_t ws_bytes, c2_stream_t stream);

/* The whole method from HOST buffers: copies the profiles to the device
 * workspace, builds the graph and copies the three [n_users][k] result arrays
 * back.  h_* buffers should be pinned for full copy speed.  Synchronous: it
 * returns after the results are in host memory.  The workspace must hold
 * c2_workspace_size_host() bytes. */
size_t c2_workspace_size_host(int32_t n_users, int64_t nnz, int32_t n_items, int32_t k,
                              int32_t t, int32_t b, int32_t N, const c2_options* opt);
c2_status c2_build_knn_graph_host(const int32_t* h_csr_ptr, const int32_t* h_csr_items,
                                  int32_t n_users, int32_t n_items, int32_t k, int32_t t,
                                  int32_t b, int32_t N, uint64_t seed, const c2_options* opt,
                                  int32_t* h_nbr_id, int32_t* h_nbr_inter, int32_t* h_nbr_union,
                                  void* d_ws, size_t ws_bytes, c2_stream_t stream);

/* Exact KNN by brute force (the judge of Section IV-B): for each query user
 * (d_queries[n_queries], or every user when d_queries is NULL) the k best of
 * all other users.  Outputs d_nbr_*[rows][k]. */
c2_status c2_bruteforce_knn(const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                            int32_t n_users, int32_t n_items, int32_t k,
                            const int32_t* d_queries, int32_t n_queries, int32_t* d_nbr_id,
                            int32_t* d_nbr_inter, int32_t* d_nbr_union, void* d_ws,
                            size_t ws_bytes, c2_stream_t stream);

/* Eq. 1: average similarity of the rows d_nbr_inter/d_nbr_union[rows][k],
 * sum of J over filled slots divided by k*rows, accumulated in FP64 in row
 * order.  Writes one double to d_out. */
c2_status c2_avg_sim(const int32_t* d_nbr_inter, const int32_t* d_nbr_union, int32_t rows,
                     int32_t k, double* d_out, void* d_ws, size_t ws_bytes, c2_stream_t stream);

/* Synchronises `stream` and returns the device status word of d_ws. */
c2_status c2_get_status(const void* d_ws, c2_stream_t stream);

/* Synchronises `stream` and copies the run statistics of d_ws to *out. */
c2_status c2_get_stats(const void* d_ws, c2_stream_t stream, c2_stats* out);

/* Clears the device status word and statistics of d_ws (asynchronous). */
c2_status c2_reset_status(void* d_ws, c2_stream_t stream);

/* GoldFinger fingerprints (Section II-F: the prototype estimates Jaccard
 * similarities from a 64- to 8096-bit summary of each profile, 1024 bits in
 * Section IV-E; the construction is not given, so this reading is the
 * library's own).  Item x sets bit
 *   fp(x) = floor((SplitMix64(K_g ^ x * 0xC2B2AE3D27D4EB4F) >> 32) * bits / 2^32),
 *   K_g = SplitMix64(seed ^ 0x474F4C4446494E47)
 * of the user's fingerprint, and the estimate of J(u, v) is the Jaccard
 * similarity of the two fingerprints' bit sets.  Outputs (device):
 * d_fp_ptr[n_users+1] and d_fp_items[<= nnz] (each user's set bits,
 * increasing: a CSR over an item universe of `bits`), and optionally
 * d_fp_bits[n_users][bits/32] (the packed words, bit b of word w = position
 * 32w + b).  32 <= bits <= 8192, a multiple of 32 (C2_ERR_UNSUPPORTED
 * otherwise).  The profiles are validated (C2_ERR_INVALID_CSR through the
 * status word).  Workspace: c2_goldfinger_workspace_size() bytes.
 * Asynchronous on `stream`.  Pass the fingerprints as c2_options.d_sim_* to
 * c2_build_knn_graph for the method with estimated similarities. */
size_t c2_goldfinger_workspace_size(int32_t n_users);
c2_status c2_goldfinger(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                        int32_t n_items, int32_t bits, uint64_t seed, int32_t* d_fp_ptr,
                        int32_t* d_fp_items, uint32_t* d_fp_bits, void* d_ws, size_t ws_bytes,
                        c2_stream_t stream);

/* Exact |P_u n P_v| and |P_u u P_v| of given neighbour rows d_nbr_id[n_users][k]
 * (id -1: empty slot, counts 0), e.g. to evaluate Eq. 1 on exact similarities
 * for a graph built on estimated ones.  Asynchronous on `stream`; no
 * workspace. */
c2_status c2_exact_counts(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                          int32_t k, const int32_t* d_nbr_id, int32_t* d_nbr_inter,
                          int32_t* d_nbr_union, c2_stream_t stream);

/* Step 3 without a workspace, for callers that cannot allocate device memory
 * when they merge (plug-ins whose host application owns every allocation,
 * real-time loops that forbid allocation after start-up).  The paper has no counterpart: this is a deployment variant of
 * c2_merge_topk with the same arguments and results, minus the workspace.
 * Its scratch (a status word and one index per (function, user) pair) lives
 * in an 8 MiB array inside the library that every GPU loading the library
 * holds until the process exits, so t * n_users may not exceed
 * c2_merge_topk_noalloc_max_slots() (2,097,088); larger inputs return
 * C2_ERR_UNSUPPORTED.  Arguments are checked as c2_merge_topk checks them,
 * with the same statuses.  It calls no allocation routine.  The first call on a
 * device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.  All
 * calls share the one array: calls that overlap on the GPU (different
 * streams, or another thread) race and must be serialised by the caller.
 * Device-side errors are not reported through a workspace status word. */
int64_t c2_merge_topk_noalloc_max_slots(void);
c2_status c2_merge_topk_noalloc(const int32_t* d_cusers, int32_t n_users, int32_t t, int32_t k,
                                const int32_t* d_loc_id, const int32_t* d_loc_inter,
                                const int32_t* d_loc_union, int32_t* d_nbr_id,
                                int32_t* d_nbr_inter, int32_t* d_nbr_union, c2_stream_t stream);

/* ---------------------------------------------------------------------------
 * Learned cluster proposer (no counterpart in the paper: a stand-in for
 * FastRandomHash as the source of first-level cluster keys).  For user u:
 *   e_u = sum over items x of E[SplitMix64(seed xor x) mod 2^rows_log2]
 *   (BF16 table, FP32 sums);  h_u = ReLU(W1^T e_u + b1) (dim -> hidden);
 *   z_u = W2^T h_u + b2 (hidden -> t*b);  key_j(u) = argmax of head j's b
 *   logits, ties to the lower bucket.  GEMMs run BF16 x BF16 -> FP32 on the
 *   tensor cores.  The model lives in a caller-owned device state buffer of
 *   c2_model_state_bytes() (FP32 masters, Adam moments, BF16 copies).
 * Training minimises, over positive pairs (u, v) -- e.g. neighbours in
 *   graphs built by plain C^2 -- and heads j, -log(sum_c p_u,jc p_v,jc + 1e-9)
 *   / (P t), p = softmax of a head, plus lambda * sum_j KL(batch mean of
 *   p_j || uniform) / t; one Adam step (beta 0.9 / 0.999, eps 1e-8) per call.
 * --------------------------------------------------------------------------- */
typedef struct {
  int32_t t, b;          /* heads and buckets per head: keys for t functions in [0, b)   */
  int32_t dim, hidden;   /* embedding width (32..128, multiple of 32) and hidden width   */
  int32_t rows_log2;     /* embedding table rows 2^rows_log2 (4..26)                     */
  int32_t reserved0;     /* must be zero                                                 */
  uint64_t seed;         /* item-row hash and initialisation seed                        */
} c2_model_config;

size_t c2_model_state_bytes(const c2_model_config* cfg);
/* Workspace of c2_model_propose (rows = users per chunk, train = 0) or of a
 * training step on max_rows pairs (train = 1). */
size_t c2_model_workspace_size(const c2_model_config* cfg, int32_t max_rows, int32_t train);
/* Deterministic initialisation (uniform, Philox-seeded), zero Adam moments. */
c2_status c2_model_init(const c2_model_config* cfg, void* d_state, size_t state_bytes,
                        c2_stream_t stream);
/* First-level keys d_keys[t][n_users] for every user. */
c2_status c2_model_propose(const c2_model_config* cfg, const void* d_state,
                           const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                           int32_t* d_keys, void* d_ws, size_t ws_bytes, c2_stream_t stream);
/* One Adam step on n_pairs pairs d_pairs[n_pairs][2] (user ids); step counts
 * from 1 for bias correction; d_loss[2] (optional) receives the pair loss and
 * the balance loss of the batch before the step. */
c2_status c2_model_train_step(const c2_model_config* cfg, void* d_state,
                              const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                              int32_t n_users, const int32_t* d_pairs, int32_t n_pairs, float lr,
                              float lambda, int32_t step, float* d_loss, void* d_ws,
                              size_t ws_bytes, c2_stream_t stream);
/* Loss and gradients of one batch without a step (for checking): shapes
 * E [2^rows_log2][dim], W1 [dim][hidden], b1 [hidden], W2 [hidden][t*b], b2 [t*b]. */
c2_status c2_model_gradients(const c2_model_config* cfg, const void* d_state,
                             const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                             const int32_t* d_pairs, int32_t n_pairs, float lambda, float* d_loss,
                             float* d_gE, float* d_gW1, float* d_gb1, float* d_gW2, float* d_gb2,
                             void* d_ws, size_t ws_bytes, c2_stream_t stream);
/* The learned path end to end: keys from the model, clustering (oversized
 * learned clusters split by FastRandomHash), local KNN and merge; then a
 * quality probe (Eq. 2 on every (n_users / n_probe)-th user against exact
 * brute force).  If the probed quality is below quality_threshold the graph
 * is rebuilt with FastRandomHash keys and C2_ERR_QUALITY_FALLBACK (an
 * informational status) is returned; *h_quality (optional) receives the
 * probed quality of the learned graph.  The device status is read after the
 * learned build, after the probe and after the fallback build: a device
 * error of any of them is returned instead (before any fallback status).  nnz = d_csr_ptr[n_users].
 * Synchronises the stream.  Workspace: c2_workspace_size_learned(). */
size_t c2_workspace_size_learned(const c2_model_config* cfg, int32_t n_users, int64_t nnz,
                                 int32_t n_items, int32_t k, int32_t N, int32_t n_probe,
                                 const c2_options* opt);
c2_status c2_build_knn_graph_learned(const c2_model_config* cfg, const void* d_state,
                                     const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                                     int32_t n_users, int64_t nnz, int32_t n_items, int32_t k,
                                     int32_t N, uint64_t seed, const c2_options* opt,
                                     float quality_threshold, int32_t n_probe,
                                     int32_t* d_nbr_id, int32_t* d_nbr_inter,
                                     int32_t* d_nbr_union, void* d_ws, size_t ws_bytes,
                                     c2_stream_t stream, double* h_quality);

/* Device addresses of the FP32 master parameters inside a state buffer. */
c2_status c2_model_params(const c2_model_config* cfg, const void* d_state, float** E, float** W1,
                          float** b1, float** W2, float** b2);

/* Instrumentation (no counterpart in the paper; the paper reports wall-clock
 * time only, Section IV-E).  c2_kernel_launches() returns how many CUDA
 * kernels this library has launched in the process.  With profiling enabled
 * the library records a CUDA event pair on the caller's stream around every
 * phase of the build; c2_profile_report() synchronises on those events,
 * writes a JSON object {"phase": {"ms": total, "calls": n, "launches": n}}
 * into buf (NUL-terminated, truncated to len) and clears the records; with
 * buf == NULL it only returns the size.  It returns the number of bytes the
 * full report needs.  Host only; the
 * profiler state is process-wide and guarded by a mutex. */
int64_t c2_kernel_launches(void);
/* Autotuner (batching of uneven clusters; no counterpart in the paper).  With
 * strategy C2_STRATEGY_AUTO, the first c2_cluster_knn / c2_build_knn_graph
 * call for given sizes (n_users, n_items, t, b, N, k, threshold) times every
 * shared-memory table shape (item words 1-2 x 128-512 threads per block, and
 * for item universes below 2^16 whether the profiles are walked as a 16-bit
 * copy) on each cluster-size bucket (32-127, 128-511, 512-2047, 2048+ users)
 * and keeps the fastest for later calls; results never depend on the choice.  This
 * writes the process-wide table as a JSON array into buf (like
 * c2_profile_report) and returns the bytes the full report needs. */
size_t c2_autotune_report(char* buf, size_t len);
/* The autotuner's table on disk (a text file, one line per problem size):
 * c2_autotune_save writes the process's table to `path` (0, or -1 when the
 * file cannot be written); c2_autotune_load merges a saved table into the
 * process's (entries of the same sizes are replaced; table shapes this
 * library does not have are measured again) and returns the number of
 * entries read, or -1 when `path` is missing or not such a table.  Loaded
 * decisions are used as if measured in this process, so later builds repeat
 * them (e.g. under a profiler, which changes the timings).  Host only. */
int32_t c2_autotune_save(const char* path);
int32_t c2_autotune_load(const char* path);
void c2_profile_enable(int on);
size_t c2_profile_report(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* C2_H */
