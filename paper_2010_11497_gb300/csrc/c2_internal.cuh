// Internal declarations of the sm_103a Cluster-and-Conquer library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/c2.h"

namespace c2 {

constexpr int kMaxK = 32;
constexpr int kMaxT = 64;
constexpr int kMaxB = 65536;
constexpr int kMaxProfile = 65535;

// ---------------------------------------------------------------- device header
// First 256 bytes of every workspace: the device status word and run counters.
struct DevHeader {
  int32_t status;              // first device-detected c2_status (0 = OK)
  int32_t n_labels;            // labels (clusters) of the current split level
  int32_t n_oversized;         // oversized labels found at the current level
  int32_t split_levels;
  int32_t max_profile;
  int32_t max_cluster;
  int32_t n_greedy;            // greedy clusters
  int32_t n_work;              // table work items
  unsigned long long pairs;    // method pair evaluations
  unsigned long long gram_pairs;
  unsigned long long greedy_gram_elems;  // sum of M*M over greedy clusters
  unsigned int work_counter[8];  // persistent-kernel work counters
  unsigned long long item_visits[2];  // table kernel: candidate items walked (brute, greedy)
  int32_t greedy_users;
  int32_t n_gwork;             // greedy round work items of the current batch
  unsigned long long greedy_visits;    // candidate entries examined by computed users
  unsigned long long greedy_computed;  // (user, round) pairs computed (not skipped)
  int32_t knn_max_len;         // longest profile among the clustered users
  int32_t pad0;
  unsigned long long greedy_evaluated;  // candidates looked up by greedy rounds
  unsigned long long brute_gram_elems;  // count-matrix elements of brute-force clusters
  int32_t brute_rows;          // users of brute-force clusters with a count matrix
  int32_t pad1;
  unsigned long long brute_pairs;  // M(M-1)/2 over brute-force clusters (intersections computed)
  unsigned long long greedy_pairs; // M(M-1)/2 over greedy clusters (their count matrices)
  unsigned long long tc_macs;      // tensor-core multiply-adds issued for count matrices
  int32_t tc_clusters;             // count matrices computed on the tensor cores
  int32_t tc_tiles;                // their 128 x 256 tiles
  int32_t select_general;          // brute-force rows the select kernel handed to the keyed path
  int32_t direct_users;            // members of greedy clusters without a count matrix
  unsigned long long gram_len_elems;  // elements of the count matrices' length rows
};
static_assert(sizeof(DevHeader) <= 256, "header must fit 256 bytes");

__device__ __forceinline__ bool dev_failed(const DevHeader* h) {
  return *(volatile const int32_t*)&h->status != 0;
}
__device__ __forceinline__ void dev_fail(DevHeader* h, int code) { atomicCAS(&h->status, 0, code); }

// ---------------------------------------------------------------- label flags
// Per-cluster metadata during splitting: terminal | residual | fn | depth.
__host__ __device__ __forceinline__ int32_t lf_pack(int terminal, int residual, int fn, int depth) {
  return (terminal & 1) | ((residual & 1) << 1) | ((fn & 63) << 2) | (depth << 8);
}
__host__ __device__ __forceinline__ int lf_terminal(int32_t f) { return f & 1; }
__host__ __device__ __forceinline__ int lf_residual(int32_t f) { return (f >> 1) & 1; }
__host__ __device__ __forceinline__ int lf_fn(int32_t f) { return (f >> 2) & 63; }
__host__ __device__ __forceinline__ int lf_depth(int32_t f) { return f >> 8; }

// ---------------------------------------------------------------- workspace
// Offsets (bytes) of every scratch array inside the caller's workspace.  The
// same function sizes the workspace (base 0) and binds it (real base).
struct Ws {
  char* base = nullptr;
  size_t top = 0;
  template <class T>
  T* take(size_t count) {
    size_t off = (top + 255) & ~size_t(255);
    top = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

struct Sizes {
  int32_t n, m, k, t, b, N;
  int64_t nnz;
  int64_t S;           // t * n slots
  int32_t tp;          // t rounded up to a multiple of 8 (hash-table row)
  int64_t omax;        // max oversized clusters in one split level
  int64_t gram_budget; // bytes
  int64_t rl_pn;       // per-function stride of the remapped lists (0: nnz unknown or no tensor cores)
  bool tc;             // the tensor-core count matrices are allowed (strategy, item universe)
};

// The workspace tail holds, from its start: the padded profiles (int32, rows
// padded to 4 items: (nnz + 3n + 64) entries), then, 256-byte aligned, a
// 16-bit copy of the profiles for item universes below 2^16 (rows padded to
// 8 items: (nnz + 7n + 64) entries), then the remapped lists of the
// tensor-core count matrices: one area of rl_stride() uint16 entries per
// function.
inline size_t p16_offset(int64_t nnz, int32_t n) {
  return ((size_t)(nnz + 3 * (int64_t)n + 64) * 4 + 255) & ~size_t(255);
}
inline size_t p16_bytes(int64_t nnz, int32_t n) {
  return ((size_t)(nnz + 7 * (int64_t)n + 64) * 2 + 255) & ~size_t(255);
}
inline int64_t rl_stride(int64_t nnz, int32_t n) { return (nnz + 3 * (int64_t)n + 4) & ~int64_t(3); }
inline size_t rl_offset(int64_t nnz, int32_t n) { return p16_offset(nnz, n) + p16_bytes(nnz, n); }
inline size_t rl_tail_bytes(int64_t nnz, int32_t n, int32_t t) {
  return (size_t)t * rl_stride(nnz, n) * 2 + 256;
}

// Item universes up to this size can use the tensor-core count matrices (the
// remap kernels hold three 32-bit words per 32 items in shared memory).
constexpr int kGramTcMaxItems = 1 << 19;

struct ClusterWs {
  DevHeader* hdr;
  uint16_t* htab;          // [m][tp]
  int32_t* key;            // [S] level-0 keys, then next keys
  int32_t* key2;           // [S] second smallest distinct hash value (b: none)
  int32_t* key3;           // [S] third smallest distinct hash value (b: none)
  int32_t *lab, *lab2;     // [S] per-slot labels
  int32_t* hist;           // [t*(b+1)+1]
  int32_t* binlab;         // [t*(b+1)+1]
  int32_t* ovlist;         // [S]
  int32_t *lsize, *lsize2; // [S+1] per-label sizes
  int32_t *leta, *leta2;   // [S]
  int32_t *lflag, *lflag2; // [S]
  int32_t* ovidx;          // [S+1]
  int32_t* nchild;         // [S+1]
  int32_t* subcnt;         // [omax][b+1]
  int32_t* subrank;        // [omax][b+1]
  int32_t* sub_resid;      // [omax]
  uint32_t *skey, *skey2;  // [S] radix sort keys
  int32_t *sval, *sval2;   // [S] radix sort values
  uint32_t* shist;         // radix histograms
  int32_t* scan_tmp;       // scan scratch
};

struct KnnWs {
  DevHeader* hdr;
  int32_t* pptr16;         // [n+1] row offsets of the 16-bit profile copy (rows padded to 8)
  uint16_t* pitems16;      // the 16-bit profile copy in the tail (null: not built)
  int32_t* slot2c;         // [S] slot -> cluster
  int32_t* slen;           // [S] profile length of the slot's user
  int32_t* small_cnt;      // [S+1] members of clusters for the merge kernel, per cluster
  int32_t* small_off;      // [S+1] their prefix sums
  int32_t* small_slot;     // [S+1] slots of those clusters
  int32_t* gflag;          // [S+1] greedy cluster flag
  int32_t* gidx;           // [S+1]
  int32_t* work_c;         // [S+1] work item -> cluster
  int32_t* work_t;         // [S+1] work item -> query tile
  int32_t* gcl;            // [S] greedy cluster list
  int32_t* gsz;            // [S] greedy cluster sizes
  int64_t* gsq;            // [S+1] squared sizes
  int64_t* goff;           // [S+1] their prefix sums
  int64_t* gofs;           // [S] per-cluster offset into gram, -1 = none
  int32_t *bt_cnt, *bt_off, *bu_cnt, *bu_off;  // [S+1] greedy batch tiles / users
  int32_t *gu_slot, *gu_g; // [S] greedy users of a batch
  int32_t *gw_g, *gw_t;    // [S+1] greedy round work items: greedy index, user chunk
  int32_t *bw_cnt, *bw_off;// [S+1] chunks per greedy cluster of a batch
  int32_t* gseq;           // [S+1] 0, 1, 2, ...
  int32_t* gkind_c;        // [S+1] per cluster: greedy (1) or brute force (0)
  int32_t* gkind;          // [S+1] per count-matrix cluster
  int32_t *bb_cnt, *bb_off;// [S+1] brute-force users per cluster of a batch
  int32_t *ub_slot, *ub_g; // [S+1] brute-force users of a batch
  int32_t* ipos;           // [S+1] slot -> internal position in its cluster
  int2* iinfo;             // [S+1] internal slot -> (local index, profile length)
  int4* islot;             // [S+1] internal slot -> (int32 padded offset, 16-bit padded
                           //        offset, profile length, user)
  int32_t *chg0, *chg1;    // [S+1] greedy: list changed in the last round
  int32_t* gfresh;         // [S+1] greedy: evaluations of the last computed round
  int32_t* pptr;           // [n+1] padded CSR offsets
  int32_t* pitems;         // padded CSR items: the workspace tail
  int64_t pitems_cap;      // capacity of pitems (elements)
  int64_t tail_bytes;      // bytes of the workspace tail from pitems on
  int32_t *wl0, *wl1;      // [S*k] greedy working lists (local indices)
  uint16_t* gram;          // gram_budget bytes
  int32_t* pos_of;         // [S] (function, user) -> slot
  // tensor-core count matrices (c2_gram_tc.cu)
  int32_t* gk2;            // [S+1] per count-matrix cluster: items held by two members or more
  int64_t* gsum;           // [S+1] per count-matrix cluster: total profile length
  int32_t* groute;         // [S+1] per count-matrix cluster: 0 table, 1 tensor cores, -1 none
  int32_t* gorder;         // [S+1] per batch position: cluster (batch-relative), cost order
  int32_t* gt_list;        // [S+1] tensor-core clusters (count-matrix indices)
  int32_t* rl_len;         // [S+1] per slot: entries of its remapped list
  int32_t *bg_flag, *bg_off, *bg_slot;  // [S+1] greedy members without a count matrix
  int4* gt_work;           // [gt_work_cap] (cluster, row tile, column tile, stages)
  int64_t gt_work_cap;
  uint16_t* rl;            // [t][rl_pn] remapped lists (absent when unused)
  int64_t rl_pn;
  double* partial;         // [1024] reduction partials
  int32_t* scan_tmp;
  int32_t* scan_tmp2;      // scan scratch of work on the side stream
  int64_t* scan_tmp64;
};

// Host checks shared by the entry points (c2_api.cu): argument errors
// (C2_ERR_INVALID_ARG), then sizes beyond the documented limits
// (C2_ERR_UNSUPPORTED), then the options' reserved fields.
c2_status check_common(int32_t n, int32_t m, int32_t k, int32_t t, int32_t b, int32_t N,
                       const c2_options* opt);
Sizes make_sizes(int32_t n, int64_t nnz, int32_t m, int32_t k, int32_t t, int32_t b, int32_t N,
                 const c2_options* opt);
void bind_cluster_ws(Ws& w, const Sizes& s, ClusterWs& c);
void bind_knn_ws(Ws& w, const Sizes& s, KnnWs& c);
size_t scan_tmp_elems(int64_t n);
size_t sort_hist_elems(int64_t n);

// ---------------------------------------------------------------- primitives
// Exclusive prefix sum of d_in[n] into d_out[n+1] (d_out[n] = total).
// In-place allowed.  tmp needs scan_tmp_elems(n) ints.
cudaError_t scan_exclusive(const int32_t* d_in, int32_t* d_out, int64_t n, int32_t* tmp,
                           cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
// Result ends in (k0, v0); k1/v1 are scratch of the same size.
cudaError_t radix_sort_pairs(uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int64_t n,
                             int bits, uint32_t* hist, int32_t* scan_tmp, cudaStream_t st);

// ---------------------------------------------------------------- device math
// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014), GPU side.
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), GPU side.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Exact neighbour order: (c1/u1, id1) before (c2/u2, id2) iff the Jaccard
// value is larger, or equal with the smaller id.  Cross-multiplied in 64 bits.
__device__ __forceinline__ bool nbr_better(uint32_t c1, uint32_t u1, int32_t id1, uint32_t c2,
                                           uint32_t u2, int32_t id2) {
  uint64_t l = (uint64_t)c1 * u2, r = (uint64_t)c2 * u1;
  return l > r || (l == r && (uint32_t)id1 < (uint32_t)id2);
}

// Warp-held sorted list: lane j < k holds entry j (id -1 = empty, worst).
struct WarpList {
  int32_t id;
  uint32_t c, u;
};

// True iff the candidate beats entry `e` (an empty entry is beaten by all).
__device__ __forceinline__ bool beats(const WarpList& e, int32_t id, uint32_t c, uint32_t u) {
  return e.id < 0 || nbr_better(c, u, id, e.c, e.u, e.id);
}

// Inserts a candidate known to all lanes into the warp list of length k when
// it ranks among the first k.  Returns true if inserted.
__device__ __forceinline__ bool warp_list_insert(WarpList& e, int k, int32_t id, uint32_t c,
                                                 uint32_t u) {
  const int lane = threadIdx.x & 31;
  bool mine_better = lane < k && !beats(e, id, c, u);
  int pos = __popc(__ballot_sync(0xffffffffu, mine_better));
  if (pos >= k) return false;
  int32_t pid = __shfl_up_sync(0xffffffffu, e.id, 1);
  uint32_t pc = __shfl_up_sync(0xffffffffu, e.c, 1);
  uint32_t pu = __shfl_up_sync(0xffffffffu, e.u, 1);
  if (lane > pos) { e.id = pid; e.c = pc; e.u = pu; }
  if (lane == pos) { e.id = id; e.c = c; e.u = u; }
  return true;
}

// Strict order on warp-list entries: better neighbour first, empty last.
__device__ __forceinline__ bool entry_better(const WarpList& a, const WarpList& b) {
  return a.id >= 0 && (b.id < 0 || nbr_better(a.c, a.u, a.id, b.c, b.u, b.id));
}

__device__ __forceinline__ WarpList shfl_entry_xor(const WarpList& e, int m) {
  WarpList o;
  o.id = __shfl_xor_sync(0xffffffffu, e.id, m);
  o.c = __shfl_xor_sync(0xffffffffu, e.c, m);
  o.u = __shfl_xor_sync(0xffffffffu, e.u, m);
  return o;
}

// Bitonic sort of one entry per lane, best first (32 lanes).
__device__ __forceinline__ void warp_sort32(WarpList& e) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      const WarpList o = shfl_entry_xor(e, j);
      const bool best_first = size == 32 || (lane & size) == 0;
      const bool lower = (lane & j) == 0;
      const bool take = (lower == best_first) ? entry_better(o, e) : entry_better(e, o);
      if (take) e = o;
    }
  }
}

// Merges a warp batch `b` (one candidate per lane, id -1 = none) into the
// sorted list `e` of length k and returns the new list: the batch is sorted,
// the two sorted runs form a bitonic sequence holding the best 32, which is
// cleaned.  Not inlined (large; called on a uniform branch).
static __device__ __noinline__ WarpList warp_list_merge(WarpList e, int k, WarpList b) {
  const int lane = threadIdx.x & 31;
  warp_sort32(b);
  if (lane >= k) e.id = -1;
  WarpList r;
  r.id = __shfl_sync(0xffffffffu, b.id, 31 - lane);
  r.c = __shfl_sync(0xffffffffu, b.c, 31 - lane);
  r.u = __shfl_sync(0xffffffffu, b.u, 31 - lane);
  if (entry_better(r, e)) e = r;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const WarpList o = shfl_entry_xor(e, j);
    const bool lower = (lane & j) == 0;
    const bool take = lower ? entry_better(o, e) : entry_better(e, o);
    if (take) e = o;
  }
  if (lane >= k) e.id = -1;
  return e;
}

// Merges a batch `b` already sorted best first (id -1 = none, at the end)
// into the sorted list `e` of length k: max of the list and the reversed
// batch is a bitonic sequence holding the best 32, which is cleaned.
static __device__ __noinline__ WarpList warp_list_merge_sorted(WarpList e, int k, WarpList b) {
  const int lane = threadIdx.x & 31;
  if (lane >= k) e.id = -1;
  WarpList r;
  r.id = __shfl_sync(0xffffffffu, b.id, 31 - lane);
  r.c = __shfl_sync(0xffffffffu, b.c, 31 - lane);
  r.u = __shfl_sync(0xffffffffu, b.u, 31 - lane);
  if (entry_better(r, e)) e = r;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const WarpList o = shfl_entry_xor(e, j);
    const bool lower = (lane & j) == 0;
    const bool take = lower ? entry_better(o, e) : entry_better(e, o);
    if (take) e = o;
  }
  if (lane >= k) e.id = -1;
  return e;
}

// Adds the lanes' candidates flagged `pass` to the list: one by one when few
// pass, by a sort-and-merge when many do.
__device__ __forceinline__ void warp_list_add(WarpList& e, int k, bool pass, int32_t id,
                                              uint32_t c, uint32_t u) {
  unsigned mask = __ballot_sync(0xffffffffu, pass);
  if (__popc(mask) > 16) {
    WarpList b;
    b.id = pass ? id : -1;
    b.c = c;
    b.u = u;
    e = warp_list_merge(e, k, b);
    return;
  }
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    warp_list_insert(e, k, __shfl_sync(0xffffffffu, id, src), __shfl_sync(0xffffffffu, c, src),
                     __shfl_sync(0xffffffffu, u, src));
  }
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Streaming top-k of one warp.  Candidates that beat the current k-th entry
// (the filter `T`, the same in all lanes) are staged in a per-warp shared
// buffer of 64 entries; every 32 staged candidates are merged at once and the
// filter is refreshed.  The final list is the k best of all offered
// candidates under the neighbour order whatever the offering order, so long
// as the offered candidates are distinct and not already in the list.
struct WarpTopk {
  WarpList L;      // lane i < k: i-th best (id -1 = empty)
  WarpList T;      // k-th entry
  int n, k;        // staged entries (uniform), list length
  int32_t* sid;    // shared [64]
  uint2* scu;      // shared [64]: (intersection, union)

  __device__ __forceinline__ void refresh() {
    T.id = __shfl_sync(0xffffffffu, L.id, k - 1);
    T.c = __shfl_sync(0xffffffffu, L.c, k - 1);
    T.u = __shfl_sync(0xffffffffu, L.u, k - 1);
  }
  __device__ __forceinline__ void start(const WarpList& l0, int k_, int32_t* sid_, uint2* scu_) {
    L = l0;
    k = k_;
    n = 0;
    sid = sid_;
    scu = scu_;
    refresh();
  }
  // True iff the candidate may enter the list (it beats the k-th entry).
  __device__ __forceinline__ bool filter(int32_t id, uint32_t c, uint32_t u) const {
    return beats(T, id, c, u);
  }
  __device__ __forceinline__ void drain32() {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    WarpList b;
    b.id = sid[lane];
    const uint2 cu = scu[lane];
    b.c = cu.x;
    b.u = cu.y;
    const int rest = n - 32;
    int32_t rid = 0;
    uint2 rcu = make_uint2(0u, 0u);
    if (lane < rest) { rid = sid[32 + lane]; rcu = scu[32 + lane]; }
    __syncwarp();
    if (lane < rest) { sid[lane] = rid; scu[lane] = rcu; }
    __syncwarp();
    n = rest;
    L = warp_list_merge(L, k, b);
    refresh();
  }
  // Stages the lanes' candidates flagged `pass` (already filtered).
  __device__ __forceinline__ void stage(bool pass, int32_t id, uint32_t c, uint32_t u) {
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if (m == 0u) return;
    if (pass) {
      const int p = n + __popc(m & lanemask_lt());
      sid[p] = id;
      scu[p] = make_uint2(c, u);
    }
    n += __popc(m);
    if (n >= 32) drain32();
  }
  // Merges what is still staged; the buffer is free again afterwards.
  __device__ __forceinline__ void finish() {
    if (n == 0) return;
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const bool pass = lane < n;
    int32_t id = -1;
    uint2 cu = make_uint2(0u, 0u);
    if (pass) { id = sid[lane]; cu = scu[lane]; }
    __syncwarp();
    n = 0;
    warp_list_add(L, k, pass, id, cu.x, cu.y);
    refresh();
  }
};

// floor(a / u) for a <= 0xFFFF0000 and 0 < u < 2^16 with a quotient below
// 2^17, without an integer division (estimate and correct): the float
// quotient is within one of a / u (relative error below 2^-21), corrected by
// one integer step either way (every product stays below 2^32).
__device__ __forceinline__ uint32_t udiv16(uint32_t a, uint32_t u) {
  uint32_t q = __float2uint_rz(__fdividef((float)a, (float)u));
  if (q * u > a) --q;
  else if ((q + 1u) * u <= a) ++q;
  return q;
}

// ------------------------------------------------------------ keyed lists
// Exact order key of a neighbour (c common items, u union, local index `lid`
// in the cluster's user-id order, position `pos` in the cluster's internal
// order) when u < 2^16 (hence c <= u < 2^16) and the cluster has fewer than
// 2^14 members:  K << 31 | (16383 - lid) << 17 | pos << 1 | mark.
// K = floor(c * 2^32 / u) keeps equal Jaccard values equal and separates
// different ones (they differ by at least 1/(u u') > 2^-32); 16383 - lid
// ranks the lower id first among equal values; pos and the one-bit mark only
// ride along (lid already differs between candidates).  Larger key = better
// neighbour; 0 = empty.  K comes from two exact 16-bit quotient steps:
// c*2^16 = q1*u + r1, then r1*2^16 / u (c, r1 < 2^16), by udiv16.
__device__ __forceinline__ uint64_t nbr_key(uint32_t c, uint32_t u, int32_t lid, int32_t pos,
                                            uint32_t mark = 0u) {
  const uint32_t ud = u ? u : 1u;            // c = u = 0 only for two empty profiles
  const uint32_t a = c << 16;
  const uint32_t q1 = udiv16(a, ud), r1 = a - q1 * ud;
  const uint32_t q2 = udiv16(r1 << 16, ud);
  const uint64_t K = c ? (((uint64_t)q1 << 16) | q2) : 0ull;
  return (K << 31) | ((uint64_t)(16383u - (uint32_t)lid) << 17) |
         ((uint64_t)(uint32_t)pos << 1) | (uint64_t)(mark & 1u);
}
__device__ __forceinline__ int32_t key_id(uint64_t key) {
  return key ? (int32_t)(16383u - (uint32_t)((key >> 17) & 0x3fffu)) : -1;
}
__device__ __forceinline__ int32_t key_pos(uint64_t key) {
  return key ? (int32_t)((key >> 1) & 0x3fffu) : -1;
}
__device__ __forceinline__ uint32_t key_mark(uint64_t key) { return (uint32_t)key & 1u; }

// Bitonic sort of one key per lane, largest first (32 lanes).
__device__ __forceinline__ uint64_t warp_sort32_keys(uint64_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, x, j);
      const bool best_first = size == 32 || (lane & size) == 0;
      const bool lower = (lane & j) == 0;
      const bool take = (lower == best_first) ? (o > x) : (x > o);
      x = take ? o : x;
    }
  }
  return x;
}

// Merges a batch of keys (one per lane, 0 = none) into the sorted key list
// `e` of length k: max of the list and the reversed sorted batch is a bitonic
// sequence holding the best 32, which is cleaned.  Not inlined (called on a
// uniform branch).
static __device__ __noinline__ uint64_t key_list_merge(uint64_t e, int k, uint64_t b) {
  const int lane = threadIdx.x & 31;
  b = warp_sort32_keys(b);
  if (lane >= k) e = 0ull;
  const uint64_t r = __shfl_sync(0xffffffffu, b, 31 - lane);
  e = r > e ? r : e;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const uint64_t o = __shfl_xor_sync(0xffffffffu, e, j);
    const bool lower = (lane & j) == 0;
    e = lower ? (o > e ? o : e) : (o < e ? o : e);
  }
  return lane < k ? e : 0ull;
}

// Inserts a key known to all lanes into the key list (keys are distinct).
__device__ __forceinline__ void key_list_insert(uint64_t& e, int k, uint64_t key) {
  const int lane = threadIdx.x & 31;
  const int pos = __popc(__ballot_sync(0xffffffffu, lane < k && e > key));
  if (pos >= k) return;
  const uint64_t p = __shfl_up_sync(0xffffffffu, e, 1);
  if (lane > pos) e = p;
  if (lane == pos) e = key;
  if (lane >= k) e = 0ull;
}

// Key of a staged candidate (pos | lid << 16, c | u << 16).
__device__ __forceinline__ uint64_t staged_key(uint2 x) {
  return nbr_key(x.y & 0xffffu, x.y >> 16, (int32_t)(x.x >> 16), (int32_t)(x.x & 0xffffu));
}

// Merges the 32 oldest of n >= 32 staged candidates into the key list and
// moves the rest down; returns the new list.  Not inlined, so that the call
// sites in unrolled candidate loops stay small.
static __device__ __noinline__ uint64_t key_drain32(uint64_t L, int k, uint2* stg, int n) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const uint2 x = stg[lane];
  const int rest = n - 32;
  uint2 y = make_uint2(0u, 0u);
  if (lane < rest) y = stg[32 + lane];
  __syncwarp();
  if (lane < rest) stg[lane] = y;
  __syncwarp();
  return key_list_merge(L, k, staged_key(x));
}

// WarpTopk on order keys, for rows whose unions are below 2^16 in clusters
// of fewer than 2^14 members: the filter compares 32-bit cross products
// against the k-th entry, staged candidates get their keys in one batch, and
// lists are merged and shifted as single 64-bit keys.  Candidates carry their
// local index (order) and internal position (storage); CU maps an internal
// position to its (common, union) counts, used to refresh the filter after
// the list changed.
template <class CU>
struct KeyTopk {
  uint64_t L;      // lane i < k: key of the i-th best (0 = empty)
  uint32_t Tc, Tu;
  uint32_t Tid;    // k-th entry; the floor while the list is not full
  uint32_t Fc, Fu, Fid;   // floor: (0, 1, 0x7fffffff) passes every candidate
  int n, k;        // staged entries (uniform), list length
  uint2* stg;      // shared [64]: (pos | lid << 16, c | u << 16)
  CU cu;

  __device__ __forceinline__ void refresh() {
    const uint64_t kth = __shfl_sync(0xffffffffu, L, k - 1);
    if (kth == 0ull) {
      Tc = Fc; Tu = Fu; Tid = Fid;
    } else {
      Tid = (uint32_t)key_id(kth);
      const uint2 x = cu(key_pos(kth));
      Tc = x.x; Tu = x.y;
    }
  }
  __device__ __forceinline__ void start(uint64_t key0, int k_, uint2* stg_, CU cu_) {
    L = key0;
    k = k_;
    n = 0;
    stg = stg_;
    cu = cu_;
    Fc = 0u; Fu = 1u; Fid = 0x7fffffffu;
    refresh();
  }
  // Floor for the filter while the list is not full: the key of a candidate
  // known to rank no lower than the final k-th entry (0 = none).  That
  // candidate itself still passes (its id is the floor's id minus one).
  __device__ __forceinline__ void set_floor(uint64_t key) {
    if (key == 0ull) return;
    const uint2 x = cu(key_pos(key));
    Fc = x.x; Fu = x.y; Fid = (uint32_t)key_id(key) + 1u;
    refresh();
  }
  __device__ __forceinline__ bool filter(int32_t lid, uint32_t c, uint32_t u) const {
    const uint32_t l = c * Tu, r = Tc * u;
    return l > r || (l == r && (uint32_t)lid < Tid);
  }
  __device__ __forceinline__ void drain32() {
    L = key_drain32(L, k, stg, n);
    n -= 32;
    refresh();
  }
  __device__ __forceinline__ void stage(bool pass, int32_t pos, int32_t lid, uint32_t c, uint32_t u) {
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if (m == 0u) return;
    if (pass)
      stg[n + __popc(m & lanemask_lt())] =
          make_uint2((uint32_t)pos | ((uint32_t)lid << 16), c | (u << 16));
    n += __popc(m);
    if (n >= 32) drain32();
  }
  __device__ __forceinline__ void finish() {
    if (n == 0) return;
    const int lane = threadIdx.x & 31;
    __syncwarp();
    uint64_t key = 0ull;
    if (lane < n) key = staged_key(stg[lane]);
    __syncwarp();
    if (n > 8) {
      L = key_list_merge(L, k, key);
    } else {
      for (int j = 0; j < n; ++j) key_list_insert(L, k, __shfl_sync(0xffffffffu, key, j));
    }
    n = 0;
    refresh();
  }
  __device__ __forceinline__ int32_t id() const { return key_id(L); }
  __device__ __forceinline__ int32_t pos() const { return key_pos(L); }
};

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- launches
// Every kernel launch of the library goes through C2_LAUNCH, which counts it.
extern std::atomic<long long> g_launches;
#define COMMA ,
#define C2_LAUNCH(kern, grid, block, smem, st, ...)            \
  do {                                                         \
    kern<<<(grid), (block), (smem), (st)>>>(__VA_ARGS__);      \
    ::c2::g_launches.fetch_add(1, std::memory_order_relaxed);  \
  } while (0)

// Optional per-phase CUDA-event timing (off unless c2_profile_enable(1)):
// a Prof object records an event pair around its scope on `st`.
class Prof {
 public:
  Prof(cudaStream_t st, const char* name);
  ~Prof() { end(); }
  void end();   // records the closing event (once)
 private:
  cudaStream_t st_;
  const char* name_;
  int idx_;
  long long launches0_;
};

#define C2_CUDA_TRY(expr)                         \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return C2_ERR_CUDA;    \
  } while (0)

// ---------------------------------------------------------------- phases
c2_status run_frh_cluster(const int32_t* ptr, const int32_t* items, const Sizes& s, uint64_t seed,
                          const c2_options& opt, int32_t* cluster_of, int32_t* cptr,
                          int32_t* cusers, int32_t* n_clusters, int32_t* cmeta, ClusterWs& w,
                          cudaStream_t st);
c2_status run_cluster_knn(const int32_t* ptr, const int32_t* items, const Sizes& s,
                          const int32_t* cptr, const int32_t* cusers, const int32_t* n_clusters,
                          uint64_t seed, const c2_options& opt, int32_t* lid, int32_t* lin,
                          int32_t* lun, KnnWs& w, cudaStream_t st);
c2_status run_merge(const int32_t* cusers, const Sizes& s, const int32_t* lid, const int32_t* lin,
                    const int32_t* lun, int32_t* nid, int32_t* nin, int32_t* nun, KnnWs& w,
                    cudaStream_t st);
c2_status run_bruteforce(const int32_t* ptr, const int32_t* items, const Sizes& s,
                         const int32_t* queries, int32_t nq, int32_t* nid, int32_t* nin,
                         int32_t* nun, KnnWs& w, cudaStream_t st);
c2_status run_avg_sim(const int32_t* nin, const int32_t* nun, int32_t rows, int32_t k, double* out,
                      DevHeader* hdr, double* partial, cudaStream_t st);
c2_status run_validate(const int32_t* ptr, const int32_t* items, const Sizes& s, DevHeader* hdr,
                       cudaStream_t st);

// tcgen05 logits GEMM with a fused per-slice argmax (c2_tc.cu):
// part[r][s] = (max, argmax) of A[r] . Bt[j] + bias[j] over the tc_slice_width() columns j
// of slice s; A [M][K] and Bt [N][K] row-major BF16.  Timeouts of its bounded
// waits are recorded in *status.
bool tc_logits_ok(int K, int N, int b);
// C[M][N] (FP32, row stride ldc) = A[M][K] . B[N][K]^T (+ bias[N]) on the tensor
// cores (tcgen05), BF16 row-major operands, K a multiple of 64; 16-byte aligned
// pointers.  Device-side timeouts go to *status.
bool tc_gemm_ok(int M, int N, int K);
c2_status tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K,
                  const float* bias, float* C, int ldc, int32_t* status, cudaStream_t st);
int tc_slice_width();
c2_status tc_transpose_bf16(const __nv_bfloat16* B, int K, int N, __nv_bfloat16* Bt,
                            cudaStream_t st);
c2_status tc_logits_argmax(const __nv_bfloat16* A, int M, int K, const __nv_bfloat16* Bt, int N,
                           const float* bias, float2* part, int32_t* status, cudaStream_t st);

// Tensor-core count matrices (c2_gram_tc.cu).  gram_tc_count: per
// count-matrix cluster g of `list` (every g < nlist when list is NULL, those of
// fewer than min_m members skipped) the items held by two members or more and
// the total profile length; gram_tc_remap: the remapped lists of the clusters
// of `list`; gram_tc_run: the count matrices of the work items
// (cluster, row tile, column tile, stages).
c2_status gram_tc_count(const int32_t* list, int nlist, int min_m, const int32_t* gsz,
                        const int32_t* gcl, const int32_t* cptr, const int32_t* cusers,
                        const int32_t* ptr, const int32_t* items, int m, bool whole, int32_t* k2,
                        int64_t* sumlen, DevHeader* hdr, cudaStream_t st);
c2_status gram_tc_remap(const int32_t* list, int nlist, const int32_t* gcl, const int32_t* cptr,
                        const int32_t* cusers, const int32_t* ptr, const int32_t* items, int m,
                        const int32_t* pptr, int64_t PN, int n, uint16_t* rl, int32_t* rl_len,
                        DevHeader* hdr, cudaStream_t st);
c2_status gram_tc_run(const int4* work, int n_work, const int32_t* cptr, const int32_t* cusers,
                      const int2* iinfo, const int32_t* pptr, const uint16_t* rl, int64_t PN,
                      int n, const int32_t* rl_len, const int64_t* gofs, uint16_t* gram,
                      const uint32_t* bits, int row_words, DevHeader* hdr, cudaStream_t st);
int gram_tc_tile_rows();
int gram_tc_tile_cols();
int gram_tc_stage_cols();

// Greedy clusters without a count matrix (c2_greedy_big.cu).
bool big_greedy_supported(int32_t k, int32_t n_random);
c2_status run_big_greedy(const int32_t* ptr, const int32_t* items, int32_t m, const int32_t* cptr,
                         const int32_t* cusers, const int32_t* slot2c, const int32_t* gkind_c,
                         int64_t S, int64_t n_users, int32_t k, int32_t rounds, int32_t n_random,
                         int32_t max_draws, uint32_t cluster_base, uint2 key, int32_t* flag,
                         int32_t* off, int32_t* bslot, int32_t* scan_tmp, int32_t* wl0,
                         int32_t* wl1, int32_t* out_id, int32_t* out_in, int32_t* out_un,
                         DevHeader* hdr, cudaStream_t st);

// GoldFinger fingerprints and exact rescoring (c2_goldfinger.cu).
size_t goldfinger_ws_bytes(int32_t n);
c2_status run_goldfinger(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m,
                         int32_t bits, uint64_t seed, int32_t* fptr, int32_t* fitems,
                         uint32_t* fbits, DevHeader* hdr, int32_t* scan_tmp, cudaStream_t st);
c2_status run_exact_counts(const int32_t* ptr, const int32_t* items, int32_t n, int32_t k,
                           const int32_t* nbr, int32_t* out_in, int32_t* out_un, cudaStream_t st);

int num_sms();
size_t autotune_report(char* buf, size_t len);
int autotune_save(const char* path);
int autotune_load(const char* path);

}  // namespace c2
