// Step 2 of Cluster-and-Conquer on sm_103a: the KNN graph inside every
// cluster (Algorithm 2), by brute force below the greedy threshold and by
// synchronous greedy neighbours-of-neighbours rounds above it.
//
// Counting |P_u n P_v| exactly:
// * "table" kernels take a tile of Q = 32*W query users, mark their items in
//   a shared-memory table T[item] (bit j of word w = query 32w+j holds the
//   item) and stream the candidates: one thread per candidate walks its
//   profile once and adds T[x] into 4-bit SWAR lanes (15 items per flush) and
//   then 16-bit counters, giving the counts of all Q queries at once.
// * a "merge" kernel (one warp per query, one lane per candidate,
//   sorted-list merge) serves item universes too large for the table.
// Top-k lists live in warp registers (lane j = entry j) and are updated with
// an exact cross-multiplied comparison.
#include <algorithm>
#include <vector>

#include "c2_internal.cuh"

namespace c2 {

cudaError_t scan_exclusive64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* tmp,
                             cudaStream_t st);

namespace {

constexpr int kNT = 256;
constexpr int kMaxGreedyM = 32768;            // greedy cluster size limit (shared bitmap)
constexpr int kBitmapWords = kMaxGreedyM / 32;

// ------------------------------------------------------------------ table kernel
struct TableArgs {
  const int32_t* ptr;
  const int32_t* items;
  int32_t n_items, k;
  const int32_t* work_c;   // cluster of each work item (cluster mode)
  const int32_t* work_t;   // query tile of each work item
  const int32_t* n_work;   // device count of work items
  const int32_t* cptr;     // cluster mode when non-null
  const int32_t* cusers;
  const int32_t* queries;  // judge mode: query list (NULL = 0..n_queries-1)
  int32_t n_queries, n_users;
  int32_t *out_id, *out_in, *out_un;
  const int64_t* gofs;     // per-cluster offset into gram (elements), -1 = brute force
  uint16_t* gram;
  DevHeader* hdr;
  unsigned* counter;
};

// Count of query j from the 16-bit counters (see flush()).
__device__ __forceinline__ int creg(int j) {
  const int w = j >> 5, q = j & 31, j4 = q & 3, p = q >> 2;
  return 16 * w + (p & 1) * 8 + 2 * j4 + ((p >> 1) & 1);
}
__device__ __forceinline__ int chalf(int j) { return ((j & 31) >> 4) & 1; }

// 4-bit lanes: acc[j4] nibble p counts query 4p+j4 of this word.
__device__ __forceinline__ void add_mask(uint32_t* acc, uint32_t m) {
  acc[0] += m & 0x11111111u;
  acc[1] += (m >> 1) & 0x11111111u;
  acc[2] += (m >> 2) & 0x11111111u;
  acc[3] += (m >> 3) & 0x11111111u;
}

// Nibbles -> 16-bit counters.  For nibble accumulator j4: even nibbles 2b sit
// in byte b of lo, odd nibbles 2b+1 in byte b of hi; bytes 0/2 and 1/3 go to
// the two halves of consecutive counters.
__device__ __forceinline__ void flush(uint32_t* acc, uint32_t* C) {
#pragma unroll
  for (int j4 = 0; j4 < 4; ++j4) {
    const uint32_t lo = acc[j4] & 0x0F0F0F0Fu;
    const uint32_t hi = (acc[j4] >> 4) & 0x0F0F0F0Fu;
    C[2 * j4] += lo & 0x00FF00FFu;
    C[2 * j4 + 1] += (lo >> 8) & 0x00FF00FFu;
    C[8 + 2 * j4] += hi & 0x00FF00FFu;
    C[8 + 2 * j4 + 1] += (hi >> 8) & 0x00FF00FFu;
    acc[j4] = 0;
  }
}

template <int W>
__device__ __forceinline__ void count_profile(const int32_t* __restrict__ row, int len,
                                              const uint32_t* __restrict__ T, uint32_t* C) {
  uint32_t acc[4 * W];
#pragma unroll
  for (int i = 0; i < 4 * W; ++i) acc[i] = 0;
  for (int e0 = 0; e0 < len; e0 += 15) {
    const int e1 = min(len, e0 + 15);
    for (int e = e0; e < e1; ++e) {
      const int x = __ldg(row + e);
      if (W == 1) {
        add_mask(acc, T[x]);
      } else {
        const uint2 m = reinterpret_cast<const uint2*>(T)[x];
        add_mask(acc, m.x);
        add_mask(acc + 4, m.y);
      }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) flush(acc + 4 * w, C + 16 * w);
  }
}

template <int W>
__global__ void __launch_bounds__(kNT) k_table(TableArgs a) {
  constexpr int Q = 32 * W, QPW = Q / 8;
  extern __shared__ __align__(16) uint32_t T[];
  __shared__ uint32_t cntw[16 * W][kNT];
  __shared__ int32_t cand_id[kNT], cand_len[kNT];
  __shared__ int32_t q_id[Q], q_len[Q];
  __shared__ int s_work;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k;
  for (int i = tid; i < a.n_items * W; i += kNT) T[i] = 0;
  const int nwork = *a.n_work;
  unsigned long long visits = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) s_work = dev_failed(a.hdr) ? nwork : (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int wi = s_work;
    if (wi >= nwork) break;
    const bool judge = a.cptr == nullptr;
    int qbase, nq, M, cbase, tq;
    int64_t gofs = -1;
    const int32_t* qlist;
    const int32_t* clist;
    if (!judge) {
      const int c = a.work_c[wi];
      tq = a.work_t[wi];
      cbase = a.cptr[c];
      M = a.cptr[c + 1] - cbase;
      qbase = cbase + tq * Q;
      nq = min(Q, M - tq * Q);
      if (a.gofs) gofs = a.gofs[c];
      qlist = a.cusers;
      clist = a.cusers;
    } else {
      tq = wi;
      qbase = tq * Q;
      nq = min(Q, a.n_queries - qbase);
      M = a.n_users;
      cbase = 0;
      qlist = a.queries;
      clist = nullptr;
    }
    if (tid < Q) {
      int id = -1, len = 0;
      if (tid < nq) {
        id = qlist ? qlist[qbase + tid] : qbase + tid;
        len = a.ptr[id + 1] - a.ptr[id];
      }
      q_id[tid] = id;
      q_len[tid] = len;
    }
    __syncthreads();
    for (int j = warp; j < nq; j += 8) {
      const int u = q_id[j];
      for (int e = a.ptr[u] + lane; e < a.ptr[u + 1]; e += 32)
        atomicOr(&T[a.items[e] * W + (j >> 5)], 1u << (j & 31));
    }
    __syncthreads();
    WarpList L[QPW];
#pragma unroll
    for (int s = 0; s < QPW; ++s) { L[s].id = -1; L[s].c = 0; L[s].u = 0; }
    for (int cb = 0; cb < M; cb += kNT) {
      const int vl = cb + tid;
      const bool act = vl < M;
      const int v = act ? (clist ? clist[cbase + vl] : vl) : -1;
      const int len = act ? a.ptr[v + 1] - a.ptr[v] : 0;
      uint32_t C[16 * W];
#pragma unroll
      for (int r = 0; r < 16 * W; ++r) C[r] = 0;
      if (act) count_profile<W>(a.items + a.ptr[v], len, T, C);
      visits += (unsigned)len;
      if (gofs >= 0) {
        // greedy cluster: keep every count (row = query, column = candidate)
        uint16_t* G = a.gram + gofs + (int64_t)(tq * Q) * M + vl;
        if (act) {
#pragma unroll
          for (int j = 0; j < Q; ++j)
            if (j < nq) G[(int64_t)j * M] = (uint16_t)((C[creg(j)] >> (16 * chalf(j))) & 0xFFFFu);
        }
        continue;
      }
#pragma unroll
      for (int r = 0; r < 16 * W; ++r) cntw[r][tid] = C[r];
      cand_id[tid] = v;
      cand_len[tid] = len;
      __syncthreads();
      const int nc = min(kNT, M - cb);
#pragma unroll
      for (int s = 0; s < QPW; ++s) {
        const int j = warp + 8 * s;
        if (j < nq) {
          const int qid = q_id[j], qlen = q_len[j];
          const int r = creg(j), h = chalf(j);
          for (int i0 = 0; i0 < nc; i0 += 32) {
            WarpList kth;
            kth.id = __shfl_sync(0xffffffffu, L[s].id, k - 1);
            kth.c = __shfl_sync(0xffffffffu, L[s].c, k - 1);
            kth.u = __shfl_sync(0xffffffffu, L[s].u, k - 1);
            const int i = i0 + lane;
            bool pass = false;
            uint32_t cc = 0, uu = 0;
            int32_t vid = -1;
            if (i < nc) {
              cc = (cntw[r][i] >> (16 * h)) & 0xFFFFu;
              vid = cand_id[i];
              if (vid != qid && cc > 0) {
                uu = (uint32_t)(qlen + cand_len[i]) - cc;
                pass = beats(kth, vid, cc, uu);
              }
            }
            unsigned mask = __ballot_sync(0xffffffffu, pass);
            while (mask) {
              const int src = __ffs(mask) - 1;
              mask &= mask - 1;
              const int32_t bid = __shfl_sync(0xffffffffu, vid, src);
              const uint32_t bc = __shfl_sync(0xffffffffu, cc, src);
              const uint32_t bu = __shfl_sync(0xffffffffu, uu, src);
              warp_list_insert(L[s], k, bid, bc, bu);
            }
          }
        }
      }
      __syncthreads();
    }
    if (gofs < 0) {
#pragma unroll
      for (int s = 0; s < QPW; ++s) {
        const int j = warp + 8 * s;
        if (j < nq && lane < k) {
          const int64_t row = (int64_t)(qbase + j) * k + lane;
          const bool ok = L[s].id >= 0;
          a.out_id[row] = ok ? L[s].id : -1;
          a.out_in[row] = ok ? (int32_t)L[s].c : 0;
          a.out_un[row] = ok ? (int32_t)L[s].u : 0;
        }
      }
    }
    __syncthreads();
    for (int j = warp; j < nq; j += 8) {
      const int u = q_id[j];
      for (int e = a.ptr[u] + lane; e < a.ptr[u + 1]; e += 32) T[a.items[e] * W + (j >> 5)] = 0;
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) visits += __shfl_xor_sync(0xffffffffu, visits, o);
  if (lane == 0 && visits) atomicAdd(&a.hdr->item_visits[a.gofs ? 1 : 0], visits);
}

// ------------------------------------------------------------------ merge kernel
// One warp per query user; lane i compares the query with candidate i of a
// chunk of 32 by a two-pointer merge of the sorted profiles.
__device__ __forceinline__ uint32_t merge_count(const int32_t* __restrict__ a, int la,
                                                const int32_t* __restrict__ b, int lb) {
  int i = 0, j = 0;
  uint32_t c = 0;
  while (i < la && j < lb) {
    const int x = __ldg(a + i), y = __ldg(b + j);
    c += (x == y);
    i += (x <= y);
    j += (y <= x);
  }
  return c;
}

struct MergeArgs {
  const int32_t* ptr;
  const int32_t* items;
  int32_t k;
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* slot2c;
  int64_t n_rows;          // slots (cluster mode) or queries (judge mode)
  int32_t thr;             // brute force iff |C| < thr
  const int32_t* queries;  // judge mode when cptr == NULL
  int32_t n_users;
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

__global__ void __launch_bounds__(kNT) k_merge_knn(MergeArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= a.n_rows || dev_failed(a.hdr)) return;
  int u, M, cbase;
  const int32_t* clist;
  if (a.cptr) {
    const int c = a.slot2c[row];
    cbase = a.cptr[c];
    M = a.cptr[c + 1] - cbase;
    if (M < 2 || M >= a.thr) return;
    u = a.cusers[row];
    clist = a.cusers;
  } else {
    u = a.queries ? a.queries[row] : (int)row;
    M = a.n_users;
    cbase = 0;
    clist = nullptr;
  }
  const int k = a.k;
  const int32_t* ur = a.items + a.ptr[u];
  const int ul = a.ptr[u + 1] - a.ptr[u];
  WarpList L;
  L.id = -1; L.c = 0; L.u = 0;
  for (int cb = 0; cb < M; cb += 32) {
    const int vl = cb + lane;
    bool pass = false;
    uint32_t cc = 0, uu = 0;
    int v = -1;
    if (vl < M) {
      v = clist ? clist[cbase + vl] : vl;
      if (v != u) {
        const int vlen = a.ptr[v + 1] - a.ptr[v];
        cc = merge_count(ur, ul, a.items + a.ptr[v], vlen);
        uu = (uint32_t)(ul + vlen) - cc;
      }
    }
    WarpList kth;
    kth.id = __shfl_sync(0xffffffffu, L.id, k - 1);
    kth.c = __shfl_sync(0xffffffffu, L.c, k - 1);
    kth.u = __shfl_sync(0xffffffffu, L.u, k - 1);
    pass = v >= 0 && v != u && cc > 0 && beats(kth, v, cc, uu);
    unsigned mask = __ballot_sync(0xffffffffu, pass);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      warp_list_insert(L, k, __shfl_sync(0xffffffffu, v, src), __shfl_sync(0xffffffffu, cc, src),
                       __shfl_sync(0xffffffffu, uu, src));
    }
  }
  if (lane < k) {
    const int64_t o = row * k + lane;
    const bool ok = L.id >= 0;
    a.out_id[o] = ok ? L.id : -1;
    a.out_in[o] = ok ? (int32_t)L.c : 0;
    a.out_un[o] = ok ? (int32_t)L.u : 0;
  }
}

// ------------------------------------------------------------------ preparation
// Per cluster: brute-force tiles, greedy flag, pair count; singletons get an
// empty row (nobody else is in their cluster).
__global__ void k_prep(const int32_t* __restrict__ cptr, const int32_t* __restrict__ n_clusters,
                       int64_t S, int32_t thr, int32_t Q, int32_t k, int32_t* __restrict__ ntiles,
                       int32_t* __restrict__ gflag, int32_t* __restrict__ lid,
                       int32_t* __restrict__ lin, int32_t* __restrict__ lun, DevHeader* hdr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t L = *n_clusters;
  int32_t M = 0;
  if (c < S && c < L) M = cptr[c + 1] - cptr[c];
  const bool brute = M >= 2 && M < thr;
  const bool greedy = M >= 2 && M >= thr;
  if (c < S) {
    ntiles[c] = brute ? (M + Q - 1) / Q : 0;
    gflag[c] = greedy ? 1 : 0;
    if (M == 1) {
      const int64_t s = cptr[c];
      for (int j = 0; j < k; ++j) {
        lid[s * k + j] = -1;
        lin[s * k + j] = 0;
        lun[s * k + j] = 0;
      }
    }
  }
  unsigned long long p = brute ? (unsigned long long)M * (M - 1) / 2 : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  if ((threadIdx.x & 31) == 0 && p) atomicAdd(&hdr->pairs, p);
  if (c == 0) hdr->n_labels = L;
}

// slot -> cluster by binary search in cptr; slot -> profile length.
__global__ void k_slot_info(const int32_t* __restrict__ cptr, const int32_t* __restrict__ n_clusters,
                            const int32_t* __restrict__ cusers, const int32_t* __restrict__ ptr,
                            int64_t S, int32_t* __restrict__ slot2c, int32_t* __restrict__ slen) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  int lo = 0, hi = *n_clusters - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cptr[mid] <= s) lo = mid; else hi = mid - 1;
  }
  slot2c[s] = lo;
  const int u = cusers[s];
  slen[s] = ptr[u + 1] - ptr[u];
}

// Work items (cluster, tile) from per-cluster tile counts and their scan.
__global__ void k_fill_work(const int32_t* __restrict__ ntiles, const int32_t* __restrict__ toff,
                            const int32_t* __restrict__ list, int64_t count,
                            int32_t* __restrict__ work_c, int32_t* __restrict__ work_t,
                            int32_t* __restrict__ n_work) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) *n_work = toff[count];
  if (j >= count) return;
  const int32_t c = list ? list[j] : (int32_t)j;
  const int32_t o = toff[j];
  for (int q = 0; q < ntiles[j]; ++q) {
    work_c[o + q] = c;
    work_t[o + q] = q;
  }
}

__global__ void k_greedy_list(const int32_t* __restrict__ gflag, const int32_t* __restrict__ gidx,
                              const int32_t* __restrict__ cptr, int64_t S, int32_t* __restrict__ gcl,
                              int64_t* __restrict__ gsq, int32_t* __restrict__ gsz, DevHeader* hdr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) hdr->n_greedy = gidx[S];
  if (c >= S || !gflag[c]) return;
  const int g = gidx[c];
  const int32_t M = cptr[c + 1] - cptr[c];
  gcl[g] = (int32_t)c;
  gsq[g] = (int64_t)M * M;
  gsz[g] = M;
  atomicMax(&hdr->max_cluster, M);
  atomicAdd(&hdr->greedy_users, M);
}

__global__ void k_batch_setup(const int32_t* __restrict__ gcl, const int64_t* __restrict__ goff,
                              const int32_t* __restrict__ gsz, int32_t g0, int32_t g1, int32_t Q,
                              int64_t* __restrict__ gofs, int32_t* __restrict__ ntiles,
                              int32_t* __restrict__ nusers) {
  const int g = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= g1) return;
  gofs[gcl[g]] = goff[g] - goff[g0];
  ntiles[g - g0] = (gsz[g] + Q - 1) / Q;
  nusers[g - g0] = gsz[g];
}

__global__ void k_fill_users(const int32_t* __restrict__ gcl, const int32_t* __restrict__ cptr,
                             const int32_t* __restrict__ uoff, int32_t g0, int32_t ng,
                             int32_t* __restrict__ gu_slot, int32_t* __restrict__ gu_g) {
  const int gl = blockIdx.x;
  if (gl >= ng) return;
  const int c = gcl[g0 + gl];
  const int cs = cptr[c], M = cptr[c + 1] - cs;
  const int o = uoff[gl];
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    gu_slot[o + l] = cs + l;
    gu_g[o + l] = g0 + gl;
  }
}

__global__ void k_fill_i64(int64_t* p, int64_t n, int64_t v) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) p[j] = v;
}

// ------------------------------------------------------------------ greedy rounds
struct GreedyArgs {
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* slen;     // profile length per slot
  const int32_t* gcl;
  const int64_t* gofs;     // per cluster
  const uint16_t* gram;
  const int32_t* gu_slot;
  const int32_t* gu_g;
  const int32_t* n_users_dev;
  int32_t k, round, n_random;
  uint2 key;               // Philox key = run seed
  const int32_t* wl_in;    // [S][k] local indices
  int32_t* wl_out;
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

// Member of a cluster of size M other than l, from one Philox word.
__device__ __forceinline__ int draw_other(uint32_t r, int l, int M) {
  const int x = (int)(r % (uint32_t)(M - 1));
  return x + (x >= l ? 1 : 0);
}

// Round 0: k distinct random members per user (in draw order), then sorted.
__global__ void __launch_bounds__(kNT) k_greedy_init(GreedyArgs a) {
  __shared__ uint32_t bm_all[8][kBitmapWords];
  __shared__ int32_t drawn_all[8][kMaxK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* bm = bm_all[warp];
  int32_t* drawn = drawn_all[warp];
  for (int i = lane; i < kBitmapWords; i += 32) bm[i] = 0;
  __syncwarp();
  const int nu = *a.n_users_dev;
  const int nwarps = gridDim.x * 8;
  unsigned long long evals = 0;
  for (int w = blockIdx.x * 8 + warp; w < nu; w += nwarps) {
    if (dev_failed(a.hdr)) break;
    const int slot = a.gu_slot[w];
    const int c = a.gcl[a.gu_g[w]];
    const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, l = slot - cs;
    const uint16_t* G = a.gram + a.gofs[c] + (int64_t)l * M;
    const int k = a.k, k0 = min(k, M - 1);
    int cnt = 0;
    // rejection sampling of distinct members; bounded so that no warp can
    // loop forever (never reached for k0 <= M-1 with a uniform generator)
    for (int j0 = 0; cnt < k0; j0 += 32) {
      if (j0 >= (1 << 24)) {
        if (lane == 0) dev_fail(a.hdr, C2_ERR_TIMEOUT);
        break;
      }
      const uint4 r = philox10(make_uint4((uint32_t)c, (uint32_t)l, 0u, (uint32_t)(j0 + lane)), a.key);
      const int v = draw_other(r.x, l, M);
      const unsigned peers = __match_any_sync(0xffffffffu, v);
      const bool first = (peers & lanemask_lt()) == 0;
      const bool seen = (bm[v >> 5] >> (v & 31)) & 1u;
      const bool ok = first && !seen;
      const unsigned okm = __ballot_sync(0xffffffffu, ok);
      const int rank = __popc(okm & lanemask_lt());
      __syncwarp();
      if (ok && cnt + rank < k0) {
        atomicOr(&bm[v >> 5], 1u << (v & 31));
        drawn[cnt + rank] = v;
      }
      cnt = min(k0, cnt + __popc(okm));
      __syncwarp();
    }
    WarpList Lst;
    Lst.id = -1; Lst.c = 0; Lst.u = 0;
    const uint32_t my = (uint32_t)a.slen[slot];
    for (int q = 0; q < cnt; ++q) {
      const int v = drawn[q];
      const uint32_t cc = G[v];
      const uint32_t uu = my + (uint32_t)a.slen[cs + v] - cc;
      warp_list_insert(Lst, k, v, cc, uu);
    }
    if (lane < k) a.wl_out[(int64_t)slot * k + lane] = Lst.id;
    __syncwarp();
    for (int q = lane; q < cnt; q += 32) {
      const int v = drawn[q];
      atomicAnd(&bm[v >> 5], ~(1u << (v & 31)));
    }
    __syncwarp();
    evals += (unsigned long long)k0;
  }
  if (lane == 0 && evals) atomicAdd(&a.hdr->pairs, evals);
}

// One synchronous round: candidates = own list + neighbours' lists (+ random
// draws), deduplicated with a per-warp bitmap of the cluster.
__global__ void __launch_bounds__(kNT) k_greedy_round(GreedyArgs a) {
  __shared__ uint32_t bm_all[8][kBitmapWords];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* bm = bm_all[warp];
  for (int i = lane; i < kBitmapWords; i += 32) bm[i] = 0;
  __syncwarp();
  const int nu = *a.n_users_dev;
  const int nwarps = gridDim.x * 8;
  unsigned long long evals = 0;
  for (int w = blockIdx.x * 8 + warp; w < nu; w += nwarps) {
    if (dev_failed(a.hdr)) break;
    const int slot = a.gu_slot[w];
    const int c = a.gcl[a.gu_g[w]];
    const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, l = slot - cs;
    const uint16_t* G = a.gram + a.gofs[c] + (int64_t)l * M;
    const int k = a.k;
    const uint32_t my = (uint32_t)a.slen[slot];
    const int e = lane < k ? a.wl_in[(int64_t)slot * k + lane] : -1;
    WarpList Lst;
    Lst.id = e;
    Lst.c = 0;
    Lst.u = 0;
    if (e >= 0) {
      Lst.c = G[e];
      Lst.u = my + (uint32_t)a.slen[cs + e] - Lst.c;
      atomicOr(&bm[e >> 5], 1u << (e & 31));
    }
    if (lane == 0) atomicOr(&bm[l >> 5], 1u << (l & 31));
    __syncwarp();
    unsigned fresh = 0;
    const int nlist = __popc(__ballot_sync(0xffffffffu, e >= 0));
    const int nsrc = nlist + ((a.n_random + 31) / 32);
    for (int j = 0; j < nsrc; ++j) {
      int v = -1;
      if (j < nlist) {
        const int nb = __shfl_sync(0xffffffffu, e, j);
        if (lane < k) v = a.wl_in[(int64_t)(cs + nb) * k + lane];
      } else {
        const int d = (j - nlist) * 32 + lane;
        if (d < a.n_random) {
          const uint4 r = philox10(make_uint4((uint32_t)c, (uint32_t)l, (uint32_t)a.round, (uint32_t)d), a.key);
          v = draw_other(r.x, l, M);
        }
      }
      bool isnew = false;
      if (v >= 0) {
        const uint32_t bit = 1u << (v & 31);
        isnew = (atomicOr(&bm[v >> 5], bit) & bit) == 0;
      }
      uint32_t cc = 0, uu = 0;
      bool pass = false;
      if (isnew) {
        ++fresh;
        cc = G[v];
        uu = my + (uint32_t)a.slen[cs + v] - cc;
      }
      WarpList kth;
      kth.id = __shfl_sync(0xffffffffu, Lst.id, k - 1);
      kth.c = __shfl_sync(0xffffffffu, Lst.c, k - 1);
      kth.u = __shfl_sync(0xffffffffu, Lst.u, k - 1);
      if (isnew) pass = beats(kth, v, cc, uu);
      unsigned mask = __ballot_sync(0xffffffffu, pass);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        warp_list_insert(Lst, k, __shfl_sync(0xffffffffu, v, src), __shfl_sync(0xffffffffu, cc, src),
                         __shfl_sync(0xffffffffu, uu, src));
      }
    }
    if (lane < k) a.wl_out[(int64_t)slot * k + lane] = Lst.id;
    __syncwarp();
    for (int i = lane; i < (M + 31) / 32; i += 32) bm[i] = 0;
    __syncwarp();
    evals += fresh;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(&a.hdr->pairs, evals);
}

// Final rows: global ids, zero-similarity entries dropped (they sort last).
__global__ void __launch_bounds__(kNT) k_greedy_emit(GreedyArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_users_dev || dev_failed(a.hdr)) return;
  const int slot = a.gu_slot[w];
  const int c = a.gcl[a.gu_g[w]];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, l = slot - cs;
  const uint16_t* G = a.gram + a.gofs[c] + (int64_t)l * M;
  const int k = a.k;
  if (lane >= k) return;
  const int e = a.wl_in[(int64_t)slot * k + lane];
  const int64_t o = (int64_t)slot * k + lane;
  uint32_t cc = e >= 0 ? G[e] : 0u;
  if (e >= 0 && cc > 0) {
    a.out_id[o] = a.cusers[cs + e];
    a.out_in[o] = (int32_t)cc;
    a.out_un[o] = a.slen[slot] + a.slen[cs + e] - (int32_t)cc;
  } else {
    a.out_id[o] = -1;
    a.out_in[o] = 0;
    a.out_un[o] = 0;
  }
}

__global__ void k_gram_stats(const int64_t* __restrict__ goff, int32_t ng, DevHeader* hdr) {
  hdr->greedy_gram_elems = (unsigned long long)goff[ng];
  hdr->gram_pairs += (unsigned long long)goff[ng];
}

// ------------------------------------------------------------------ launch helpers
int table_smem_bytes(int W, int m) { return m * W * 4; }

bool table_fits(int W, int m) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int stat = 16 * W * kNT * 4 + 2 * kNT * 4 + 64 * W * 4 * 2 + 64;
  return table_smem_bytes(W, m) + stat <= optin;
}

template <int W>
c2_status launch_table(const TableArgs& a, cudaStream_t st) {
  const int smem = table_smem_bytes(W, a.n_items);
  C2_CUDA_TRY(cudaFuncSetAttribute(k_table<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_table<W>, kNT, smem));
  if (per_sm < 1) return C2_ERR_UNSUPPORTED;
  C2_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
  C2_LAUNCH(k_table<W>, num_sms() * per_sm, kNT, smem, st, a);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

int pick_w(int strategy, int m) {
  if (strategy == C2_STRATEGY_MERGE) return 0;
  if (strategy == C2_STRATEGY_TABLE32) return table_fits(1, m) ? 1 : 0;
  if (strategy == C2_STRATEGY_TABLE64) return table_fits(2, m) ? 2 : (table_fits(1, m) ? 1 : 0);
  // automatic: the widest table that fits
  if (table_fits(2, m)) return 2;
  if (table_fits(1, m)) return 1;
  return 0;
}

c2_status launch_table_w(int W, const TableArgs& a, cudaStream_t st) {
  return W == 2 ? launch_table<2>(a, st) : launch_table<1>(a, st);
}

}  // namespace

c2_status run_cluster_knn(const int32_t* ptr, const int32_t* items, const Sizes& s,
                          const int32_t* cptr, const int32_t* cusers, const int32_t* n_clusters,
                          uint64_t seed, const c2_options& opt, int32_t* lid, int32_t* lin,
                          int32_t* lun, KnnWs& w, cudaStream_t st) {
  const int64_t S = s.S;
  if (S == 0) return C2_OK;
  const int T = 256;
  const int k = s.k;
  const int thr = opt.greedy_threshold > 0 ? opt.greedy_threshold : 5 * k * k;
  const int rounds = opt.greedy_rounds >= 0 ? opt.greedy_rounds : 10;
  const int W = pick_w(opt.strategy, s.m);
  const int Q = W ? 32 * W : 32;

  Prof p_prep(st, "knn_prep");
  C2_LAUNCH(k_prep, div_up(S, T), T, 0, st, cptr, n_clusters, S, thr, Q, k, w.ntiles, w.gflag, lid, lin,
                                      lun, w.hdr);
  C2_LAUNCH(k_slot_info, div_up(S, T), T, 0, st, cptr, n_clusters, cusers, ptr, S, w.slot2c, w.slen);
  C2_CUDA_TRY(cudaGetLastError());

  p_prep.end();
  // ---- brute-force clusters
  Prof p_brute(st, W ? "brute_table" : "brute_merge");
  if (W) {
    C2_CUDA_TRY(scan_exclusive(w.ntiles, w.toff, S, w.scan_tmp, st));
    C2_LAUNCH(k_fill_work, div_up(S, T), T, 0, st, w.ntiles, w.toff, nullptr, S, w.work_c, w.work_t,
                                            &w.hdr->n_work);
    TableArgs a{};
    a.ptr = ptr; a.items = items; a.n_items = s.m; a.k = k;
    a.work_c = w.work_c; a.work_t = w.work_t; a.n_work = &w.hdr->n_work;
    a.cptr = cptr; a.cusers = cusers;
    a.out_id = lid; a.out_in = lin; a.out_un = lun;
    a.gofs = nullptr; a.gram = nullptr;
    a.hdr = w.hdr; a.counter = &w.hdr->work_counter[0];
    c2_status rc = launch_table_w(W, a, st);
    if (rc) return rc;
  } else {
    MergeArgs a{};
    a.ptr = ptr; a.items = items; a.k = k; a.cptr = cptr; a.cusers = cusers; a.slot2c = w.slot2c;
    a.n_rows = S; a.thr = thr; a.out_id = lid; a.out_in = lin; a.out_un = lun; a.hdr = w.hdr;
    C2_LAUNCH(k_merge_knn, div_up(S * 32, kNT), kNT, 0, st, a);
    C2_CUDA_TRY(cudaGetLastError());
  }

  p_brute.end();
  // ---- greedy clusters
  Prof p_gsetup(st, "greedy_setup");
  C2_CUDA_TRY(scan_exclusive(w.gflag, w.gidx, S, w.scan_tmp, st));
  C2_LAUNCH(k_greedy_list, div_up(S, T), T, 0, st, w.gflag, w.gidx, cptr, S, w.gcl, w.gsq, w.gsz, w.hdr);
  int32_t ng = 0;
  C2_CUDA_TRY(cudaMemcpyAsync(&ng, &w.hdr->n_greedy, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaStreamSynchronize(st));
  if (ng == 0) return C2_OK;
  if (W == 0) return C2_ERR_UNSUPPORTED;   // greedy needs the table kernel for its counts
  C2_CUDA_TRY(scan_exclusive64(w.gsq, w.goff, ng, w.scan_tmp64, st));
  C2_LAUNCH(k_gram_stats, 1, 1, 0, st, w.goff, ng, w.hdr);
  std::vector<int64_t> goff(ng + 1);
  std::vector<int32_t> gsz(ng);
  C2_CUDA_TRY(cudaMemcpyAsync(goff.data(), w.goff, (ng + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(gsz.data(), w.gsz, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t cap = s.gram_budget / (int64_t)sizeof(uint16_t);
  for (int g = 0; g < ng; ++g) {
    if (gsz[g] > kMaxGreedyM || goff[g + 1] - goff[g] > cap) return C2_ERR_UNSUPPORTED;
  }
  C2_LAUNCH(k_fill_i64, div_up(S, T), T, 0, st, w.gofs, S, -1);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  int g0 = 0;
  while (g0 < ng) {
    int g1 = g0;
    int64_t nu = 0;
    while (g1 < ng && goff[g1 + 1] - goff[g0] <= cap) nu += gsz[g1++];
    const int nb = g1 - g0;
    p_gsetup.end();
    Prof p_gram(st, "greedy_gram");
    // counts of the batch's greedy clusters into their intersection matrices
    C2_LAUNCH(k_batch_setup, div_up(nb, T), T, 0, st, w.gcl, w.goff, w.gsz, g0, g1, Q, w.gofs, w.bt_cnt,
                                               w.bu_cnt);
    C2_CUDA_TRY(scan_exclusive(w.bt_cnt, w.bt_off, nb, w.scan_tmp, st));
    C2_CUDA_TRY(scan_exclusive(w.bu_cnt, w.bu_off, nb, w.scan_tmp, st));
    C2_LAUNCH(k_fill_work, div_up(nb, T), T, 0, st, w.bt_cnt, w.bt_off, w.gcl + g0, nb, w.work_c,
                                             w.work_t, &w.hdr->n_work);
    TableArgs a{};
    a.ptr = ptr; a.items = items; a.n_items = s.m; a.k = k;
    a.work_c = w.work_c; a.work_t = w.work_t; a.n_work = &w.hdr->n_work;
    a.cptr = cptr; a.cusers = cusers;
    a.out_id = lid; a.out_in = lin; a.out_un = lun;
    a.gofs = w.gofs; a.gram = w.gram;
    a.hdr = w.hdr; a.counter = &w.hdr->work_counter[1];
    c2_status rc = launch_table_w(W, a, st);
    if (rc) return rc;
    p_gram.end();
    Prof p_init(st, "greedy_init");
    // greedy rounds over the batch's users
    C2_LAUNCH(k_fill_users, nb, 256, 0, st, w.gcl, cptr, w.bu_off, g0, nb, w.gu_slot, w.gu_g);
    GreedyArgs ga{};
    ga.cptr = cptr; ga.cusers = cusers; ga.slen = w.slen; ga.gcl = w.gcl; ga.gofs = w.gofs;
    ga.gram = w.gram; ga.gu_slot = w.gu_slot; ga.gu_g = w.gu_g; ga.n_users_dev = w.bu_off + nb;
    ga.k = k; ga.n_random = opt.greedy_random; ga.key = key;
    ga.out_id = lid; ga.out_in = lin; ga.out_un = lun; ga.hdr = w.hdr;
    const int grid = (int)std::min<int64_t>(div_up(nu, 8), (int64_t)num_sms() * 8);
    ga.round = 0;
    ga.wl_in = nullptr;
    ga.wl_out = w.wl0;
    C2_LAUNCH(k_greedy_init, grid, kNT, 0, st, ga);
    p_init.end();
    Prof p_rounds(st, "greedy_rounds");
    int32_t* cur = w.wl0;
    int32_t* nxt = w.wl1;
    for (int r = 1; r <= rounds; ++r) {
      ga.round = r;
      ga.wl_in = cur;
      ga.wl_out = nxt;
      C2_LAUNCH(k_greedy_round, grid, kNT, 0, st, ga);
      std::swap(cur, nxt);
    }
    p_rounds.end();
    Prof p_emit(st, "greedy_emit");
    ga.wl_in = cur;
    C2_LAUNCH(k_greedy_emit, div_up(nu * 32, kNT), kNT, 0, st, ga);
    C2_CUDA_TRY(cudaGetLastError());
    g0 = g1;
  }
  return C2_OK;
}

c2_status run_bruteforce(const int32_t* ptr, const int32_t* items, const Sizes& s,
                         const int32_t* queries, int32_t nq, int32_t* nid, int32_t* nin,
                         int32_t* nun, KnnWs& w, cudaStream_t st) {
  const int rows = queries ? nq : s.n;
  if (rows == 0) return C2_OK;
  const int W = pick_w(C2_STRATEGY_AUTO, s.m);
  if (W) {
    const int Q = 32 * W;
    const int nwork = div_up(rows, Q);
    C2_CUDA_TRY(cudaMemcpyAsync(&w.hdr->n_work, &nwork, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TableArgs a{};
    a.ptr = ptr; a.items = items; a.n_items = s.m; a.k = s.k;
    a.n_work = &w.hdr->n_work;
    a.cptr = nullptr; a.queries = queries; a.n_queries = rows; a.n_users = s.n;
    a.out_id = nid; a.out_in = nin; a.out_un = nun;
    a.hdr = w.hdr; a.counter = &w.hdr->work_counter[2];
    c2_status rc = launch_table_w(W, a, st);
    C2_CUDA_TRY(cudaStreamSynchronize(st));   // nwork lives on this host stack frame
    return rc;
  }
  MergeArgs a{};
  a.ptr = ptr; a.items = items; a.k = s.k; a.cptr = nullptr; a.n_rows = rows;
  a.queries = queries; a.n_users = s.n; a.out_id = nid; a.out_in = nin; a.out_un = nun;
  a.hdr = w.hdr;
  C2_LAUNCH(k_merge_knn, div_up((int64_t)rows * 32, kNT), kNT, 0, st, a);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
