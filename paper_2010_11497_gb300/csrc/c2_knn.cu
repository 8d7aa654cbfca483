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
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "c2_internal.cuh"

namespace c2 {

cudaError_t scan_exclusive64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* tmp,
                             cudaStream_t st);

namespace {

constexpr int kNT = 256;
constexpr int kMaxGreedyM = 10240;            // greedy cluster size limit (shared staging)
constexpr int kBitmapWords = kMaxGreedyM / 32;
constexpr int kGreedyUsersPerWarp = 4;
constexpr int kGreedySmallItemRounds = 2;      // rounds with one user per warp and work item
constexpr int kSmallCut = 9;     // brute clusters below this size: warp-per-cluster kernel (<= 33)
constexpr int kTcMinM = 128;     // smallest cluster for the tensor-core count matrix
constexpr int kDensityBuckets = 5;
// Density of a cluster for the strategy choice: the members' mean profile
// length over the items held by two members or more, in buckets below 1/64,
// 1/32, 1/16, 1/8 and from 1/8 on.
inline int density_bucket(int64_t sumlen, int M, int k2) {
  const double d = (double)sumlen / ((double)M * (double)std::max(k2, 1));
  return d < 1.0 / 64 ? 0 : (d < 1.0 / 32 ? 1 : (d < 1.0 / 16 ? 2 : (d < 1.0 / 8 ? 3 : 4)));
}
constexpr int kGreedyChunk = 8 * kGreedyUsersPerWarp;   // users per block work item


// ------------------------------------------------------------------ table kernel
struct TableArgs {
  const int32_t* ptr;      // CSR (query items, profile lengths)
  const int32_t* items;
  const int32_t* pptr;     // padded CSR: rows start on 16-byte boundaries,
  const int32_t* pitems;   //   padded with the sentinel item n_items
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
  uint16_t* gram;          // rows of stride round_up(M, 8)
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
__device__ __forceinline__ void look4(const uint32_t* __restrict__ T, const int4 q, uint32_t* acc) {
  const int xs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (W == 1) {
      add_mask(acc, T[xs[i]]);
    } else {
      const uint2 m = reinterpret_cast<const uint2*>(T)[xs[i]];
      add_mask(acc, m.x);
      add_mask(acc + 4, m.y);
    }
  }
}

// Walks one padded profile (n4 int4 words) in groups of 12 items (3 loads),
// the next group's loads issued before the current group is counted.
template <int W>
__device__ __forceinline__ void count_row4(const int4* __restrict__ r4, int n4,
                                           const uint32_t* __restrict__ T, int sentinel,
                                           uint32_t* C) {
  const int4 pad = make_int4(sentinel, sentinel, sentinel, sentinel);
  int4 cur[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) cur[j] = j < n4 ? __ldg(r4 + j) : pad;
  uint32_t acc[4 * W];
#pragma unroll
  for (int i = 0; i < 4 * W; ++i) acc[i] = 0;
  for (int i = 0; i < n4; i += 3) {
    int4 nxt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) nxt[j] = (i + 3 + j < n4) ? __ldg(r4 + i + 3 + j) : pad;
#pragma unroll
    for (int j = 0; j < 3; ++j) look4<W>(T, cur[j], acc);
#pragma unroll
    for (int w = 0; w < W; ++w) flush(acc + 4 * w, C + 16 * w);
#pragma unroll
    for (int j = 0; j < 3; ++j) cur[j] = nxt[j];
  }
}

// Walks one 16-bit padded profile (n8 loads of 8 items) in steps of 24 items
// (three 16-byte loads, the next step's loads issued before the current step
// is counted), flushing the 4-bit lanes every 12 items.
template <int W>
__device__ __forceinline__ void count_row16(const uint4* __restrict__ r8, int n8,
                                            const uint32_t* __restrict__ T, int sentinel,
                                            uint32_t* C) {
  const uint32_t s2 = (uint32_t)sentinel * 0x10001u;
  const uint4 pad = make_uint4(s2, s2, s2, s2);
  uint4 cur[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) cur[j] = j < n8 ? __ldg(r8 + j) : pad;
  uint32_t acc[4 * W];
#pragma unroll
  for (int i = 0; i < 4 * W; ++i) acc[i] = 0;
  for (int i = 0; i < n8; i += 3) {
    uint4 nxt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) nxt[j] = (i + 3 + j < n8) ? __ldg(r8 + i + 3 + j) : pad;
    const uint32_t ws[12] = {cur[0].x, cur[0].y, cur[0].z, cur[0].w, cur[1].x, cur[1].y,
                             cur[1].z, cur[1].w, cur[2].x, cur[2].y, cur[2].z, cur[2].w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const uint32_t xs[2] = {ws[6 * h + q] & 0xFFFFu, ws[6 * h + q] >> 16};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (W == 1) {
            add_mask(acc, T[xs[e]]);
          } else {
            const uint2 mm = reinterpret_cast<const uint2*>(T)[xs[e]];
            add_mask(acc, mm.x);
            add_mask(acc + 4, mm.y);
          }
        }
      }
#pragma unroll
      for (int w = 0; w < W; ++w) flush(acc + 4 * w, C + 16 * w);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) cur[j] = nxt[j];
  }
}

// ---- bit-sliced counts (tables of one word: 32 queries)
// Each thread keeps its candidate's 32 counts as 16 bit planes: bit b of
// plane i is bit i of the count of the query marked with bit b.  Query j of a
// tile is marked with bit qbit(j), which puts queries 2h and 2h+1 at bits h
// and 16+h, so that transposing the planes as two 16 x 16 bit matrices (one
// per half word) leaves word h = count(2h) | count(2h+1) << 16: the row
// segment as it is stored.
__device__ __forceinline__ uint32_t qbit(int j) { return (uint32_t)((j >> 1) + 16 * (j & 1)); }

// Full adder on 32 one-bit lanes: a <- a ^ b ^ c, carry <- majority(a, b, c).
__device__ __forceinline__ void csa(uint32_t& a, uint32_t b, uint32_t c, uint32_t& carry) {
  carry = (a & b) | (a & c) | (b & c);
  a ^= b ^ c;
}

// Adds 16 masks to the planes A[0..B-1]: a carry-save tree (15 full adders)
// into the planes of weight 1, 2, 4 and 8, then the one carry of weight 16
// rippled through the planes above.  The counts stay below 2^B (B = 8 when
// every walked profile is shorter than 256 items).
template <int B>
__device__ __forceinline__ void add16(uint32_t* A, const uint32_t* m) {
  uint32_t t8[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t t4[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      uint32_t t2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) csa(A[0], m[8 * h + 4 * g + 2 * e], m[8 * h + 4 * g + 2 * e + 1], t2[e]);
      csa(A[1], t2[0], t2[1], t4[g]);
    }
    csa(A[2], t4[0], t4[1], t8[h]);
  }
  uint32_t t;
  csa(A[3], t8[0], t8[1], t);
#pragma unroll
  for (int b = 4; b < B; ++b) {
    const uint32_t c = A[b] & t;
    A[b] ^= t;
    t = c;
  }
}

// Two 16 x 16 bit transposes at once (one per half word) of the planes
// z[0..15]: z[h] bit i <-> z[i] bit h, and likewise bits 16+i / 16+h.
// Block swaps of 8 (byte permutes), 4, 2 and 1 rows.
__device__ __forceinline__ void transpose_halves16(uint32_t* z) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t a = z[k], b = z[k + 8];
    z[k] = __byte_perm(a, b, 0x6240);
    z[k + 8] = __byte_perm(a, b, 0x7351);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (!(k & 4)) {
      const uint32_t t = ((z[k] >> 4) ^ z[k + 4]) & 0x0F0F0F0Fu;
      z[k + 4] ^= t;
      z[k] ^= t << 4;
    }
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (!(k & 2)) {
      const uint32_t t = ((z[k] >> 2) ^ z[k + 2]) & 0x33333333u;
      z[k + 2] ^= t;
      z[k] ^= t << 2;
    }
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (!(k & 1)) {
      const uint32_t t = ((z[k] >> 1) ^ z[k + 1]) & 0x55555555u;
      z[k + 1] ^= t;
      z[k] ^= t << 1;
    }
}

// Walks one 16-bit padded profile (n8 loads of 8 items) 16 items at a time
// into the planes A, the next two loads issued before the current 16 items
// are counted.
template <int B>
__device__ __forceinline__ void count_row16_bs(const uint4* __restrict__ r8, int n8,
                                               const uint32_t* __restrict__ T, int sentinel,
                                               uint32_t* A) {
  const uint32_t s2 = (uint32_t)sentinel * 0x10001u;
  const uint4 pad = make_uint4(s2, s2, s2, s2);
  uint4 cur[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) cur[j] = j < n8 ? __ldg(r8 + j) : pad;
  for (int i = 0; i < n8; i += 2) {
    uint4 nxt[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) nxt[j] = (i + 2 + j < n8) ? __ldg(r8 + i + 2 + j) : pad;
    const uint32_t ws[8] = {cur[0].x, cur[0].y, cur[0].z, cur[0].w,
                            cur[1].x, cur[1].y, cur[1].z, cur[1].w};
    uint32_t m[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      m[2 * q] = T[ws[q] & 0xFFFFu];
      m[2 * q + 1] = T[ws[q] >> 16];
    }
    add16<B>(A, m);
#pragma unroll
    for (int j = 0; j < 2; ++j) cur[j] = nxt[j];
  }
}

// The same over the int32 padded profile (n4 loads of 4 items).
template <int B>
__device__ __forceinline__ void count_row4_bs(const int4* __restrict__ r4, int n4,
                                              const uint32_t* __restrict__ T, int sentinel,
                                              uint32_t* A) {
  const int4 pad = make_int4(sentinel, sentinel, sentinel, sentinel);
  int4 cur[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) cur[j] = j < n4 ? __ldg(r4 + j) : pad;
  for (int i = 0; i < n4; i += 4) {
    int4 nxt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) nxt[j] = (i + 4 + j < n4) ? __ldg(r4 + i + 4 + j) : pad;
    uint32_t m[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m[4 * j] = T[cur[j].x];
      m[4 * j + 1] = T[cur[j].y];
      m[4 * j + 2] = T[cur[j].z];
      m[4 * j + 3] = T[cur[j].w];
    }
    add16<B>(A, m);
#pragma unroll
    for (int j = 0; j < 4; ++j) cur[j] = nxt[j];
  }
}

template <int W, int NT>
__host__ __device__ constexpr int table_static_words() {
  return 16 * W * NT + 2 * NT;
}

__host__ __device__ inline int table_T_words(int W, int m) { return (((m + 1) * W) + 3) & ~3; }

template <int W, int NT>
__global__ void __launch_bounds__(NT) k_table(TableArgs a) {
  constexpr int Q = 32 * W, NWARP = NT / 32, QPW = (Q + NWARP - 1) / NWARP;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* T = smem;
  uint32_t* cntw = smem + table_T_words(W, a.n_items);      // [16W][NT]
  int32_t* cand_id = reinterpret_cast<int32_t*>(cntw + 16 * W * NT);
  int32_t* cand_len = cand_id + NT;
  __shared__ int32_t q_id[Q], q_len[Q];
  __shared__ int s_work;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k;
  for (int i = tid; i < (a.n_items + 1) * W; i += NT) T[i] = 0;
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
    for (int j = warp; j < nq; j += NWARP) {
      const int u = q_id[j];
      for (int e = a.ptr[u] + lane; e < a.ptr[u + 1]; e += 32)
        atomicOr(&T[a.items[e] * W + (j >> 5)], 1u << (j & 31));
    }
    __syncthreads();
    WarpList L[QPW];
#pragma unroll
    for (int s = 0; s < QPW; ++s) { L[s].id = -1; L[s].c = 0; L[s].u = 0; }
    const int Mp = (M + 7) & ~7;
    for (int cb = 0; cb < M; cb += NT) {
      const int vl = cb + tid;
      const bool act = vl < M;
      const int v = act ? (clist ? clist[cbase + vl] : vl) : -1;
      const int len = act ? a.ptr[v + 1] - a.ptr[v] : 0;
      uint32_t C[16 * W];
#pragma unroll
      for (int r = 0; r < 16 * W; ++r) C[r] = 0;
      if (act) {
        count_row4<W>(reinterpret_cast<const int4*>(a.pitems + a.pptr[v]), (len + 3) >> 2, T,
                      a.n_items, C);
        visits += (unsigned)len;
      }
      if (gofs >= 0) {
        // greedy cluster: keep every count (row = query, column = candidate)
        uint16_t* G = a.gram + gofs + (int64_t)(tq * Q) * Mp + vl;
        if (act) {
#pragma unroll
          for (int j = 0; j < Q; ++j)
            if (j < nq) G[(int64_t)j * Mp] = (uint16_t)((C[creg(j)] >> (16 * chalf(j))) & 0xFFFFu);
        }
        continue;
      }
#pragma unroll
      for (int r = 0; r < 16 * W; ++r) cntw[r * NT + tid] = C[r];
      cand_id[tid] = v;
      cand_len[tid] = len;
      __syncthreads();
      const int nc = min(NT, M - cb);
#pragma unroll
      for (int s = 0; s < QPW; ++s) {
        const int j = warp + NWARP * s;
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
              cc = (cntw[r * NT + i] >> (16 * h)) & 0xFFFFu;
              vid = cand_id[i];
              if (vid != qid && cc > 0) {
                uu = (uint32_t)(qlen + cand_len[i]) - cc;
                pass = beats(kth, vid, cc, uu);
              }
            }
            warp_list_add(L[s], k, pass, vid, cc, uu);
          }
        }
      }
      __syncthreads();
    }
    if (gofs < 0) {
#pragma unroll
      for (int s = 0; s < QPW; ++s) {
        const int j = warp + NWARP * s;
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
    for (int j = warp; j < nq; j += NWARP) {
      const int u = q_id[j];
      for (int e = a.ptr[u] + lane; e < a.ptr[u + 1]; e += 32) T[a.items[e] * W + (j >> 5)] = 0;
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) visits += __shfl_xor_sync(0xffffffffu, visits, o);
  if (lane == 0 && visits) atomicAdd(&a.hdr->item_visits[a.gofs ? 1 : 0], visits);
}

// ------------------------------------------------------------------ gram kernel
// Count matrix of one cluster, G[p][q] = |P_p n P_q| for members at internal
// positions p, q (the cluster's members by decreasing profile length), stored
// in rows of stride Mp = round_up(M, 8).  A work item is a tile of Q = 32*W
// query positions marked in the shared table; the candidates are the
// positions from the tile on (the matrix is symmetric), taken 32 at a time by
// whichever warp is free, so that the lanes of a warp walk profiles of
// similar length.  Each thread writes its candidate's counts against the
// tile's queries as one contiguous row segment and, for candidates past the
// tile, the mirrored column (32 consecutive positions per warp store).
struct GramArgs {
  const int32_t* ptr;
  const int32_t* items;
  const int32_t* pptr;
  const int32_t* pitems;
  int32_t n_items;
  const int32_t* work_c;
  const int32_t* work_t;
  const int32_t* work_begin;   // device: first and one-past-last work item of this launch
  const int32_t* work_end;
  const int32_t* cptr;
  const int32_t* cusers;
  const int2* iinfo;       // internal slot -> (local index, profile length)
  const int4* islot;       // internal slot -> (int32 offset, 16-bit offset, length, user)
  const int64_t* gofs;
  uint16_t* gram;
  DevHeader* hdr;
  unsigned* counter;
};

// Marks (bit) or clears (Clear) the table entries of the items of query q
// (its slot record: padded offsets and length), read
// from the padded copy the walk reads (eight 16-bit or four int32 items per
// 16-byte load, one load per lane and step): a query of up to 256 items is
// one step.  Padding positions are skipped, so the sentinel's entry stays 0.
template <int W, bool P16, bool Clear>
__device__ __forceinline__ void mark_query(uint32_t* T, int word, uint32_t bit, int4 q, int lane,
                                           const GramArgs& a,
                                           const uint16_t* __restrict__ pitems16) {
  const int len = q.z;
  if constexpr (P16) {
    const uint4* r8 = reinterpret_cast<const uint4*>(pitems16 + q.y);
    for (int g = lane; g < (len + 7) >> 3; g += 32) {
      const uint4 x8 = __ldg(r8 + g);
      const uint32_t ws[4] = {x8.x, x8.y, x8.z, x8.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint32_t x = (e & 1) ? ws[e >> 1] >> 16 : ws[e >> 1] & 0xFFFFu;
        if (8 * g + e < len) {
          if constexpr (Clear) T[x * W + word] = 0u;
          else atomicOr(&T[x * W + word], bit);
        }
      }
    }
  } else {
    const int4* r4 = reinterpret_cast<const int4*>(a.pitems + q.x);
    for (int g = lane; g < (len + 3) >> 2; g += 32) {
      const int4 x4 = __ldg(r4 + g);
      const int xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * g + e < len) {
          if constexpr (Clear) T[xs[e] * W + word] = 0u;
          else atomicOr(&T[xs[e] * W + word], bit);
        }
    }
  }
}

// P16: the candidates' profiles are walked in the 16-bit copy (pptr16,
// pitems16; item ids below 2^16), eight items per 16-byte load.
template <int W, int NT, int MB, bool P16>
__global__ void __launch_bounds__(NT, MB > 0 ? MB : 1)
    k_gram(GramArgs a, const int32_t* __restrict__ pptr16, const uint16_t* __restrict__ pitems16) {
  constexpr int Q = 32 * W, NWARP = NT / 32;
  extern __shared__ __align__(16) uint32_t T[];
  // Blocks of 16 warps or more keep two work-item buffers: the next tile
  // (work counter, cluster, its queries' slot records) is fetched by one warp
  // while the current tile is walked.  Smaller blocks, where that warp would
  // be missed in the walk and other resident blocks hide the latency, fetch
  // each tile when the previous one is done.
  constexpr bool kAhead = NWARP >= 16;
  __shared__ int4 q_slot[2][Q];
  __shared__ int s_wi[2], s_c[2], s_tq[2], s_cbase[2], s_M[2];
  __shared__ int s_next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < (a.n_items + 1) * W; i += NT) T[i] = 0;
  if (tid == 0) s_next = 0;
  const int wbeg = *a.work_begin, nwork = *a.work_end;
  unsigned long long visits = 0;
  auto fetch = [&](int buf) {   // one whole warp
    int wi = 0;
    if (lane == 0) wi = dev_failed(a.hdr) ? nwork : wbeg + (int)atomicAdd(a.counter, 1u);
    wi = __shfl_sync(0xffffffffu, wi, 0);
    int c = 0, tq = 0, cbase = 0, M = 0;
    if (wi < nwork) {
      c = a.work_c[wi];
      tq = a.work_t[wi];
      cbase = a.cptr[c];
      M = a.cptr[c + 1] - cbase;
    }
    const int nq = min(Q, M - tq * Q);
    for (int j = lane; j < Q; j += 32)
      q_slot[buf][j] = j < nq ? a.islot[cbase + tq * Q + j] : make_int4(0, 0, 0, -1);
    if (lane == 0) {
      s_wi[buf] = wi;
      s_c[buf] = c;
      s_tq[buf] = tq;
      s_cbase[buf] = cbase;
      s_M[buf] = M;
    }
  };
  if (kAhead) {
    if (warp == 0) fetch(0);
    __syncthreads();
  }
  for (int buf = 0;; buf ^= kAhead ? 1 : 0) {
    if (!kAhead) {
      if (warp == 0) fetch(0);
      __syncthreads();
    }
    const int wi = s_wi[buf];
    if (wi >= nwork) break;
    const int c = s_c[buf], tq = s_tq[buf];
    const int cbase = s_cbase[buf], M = s_M[buf], Mp = (M + 7) & ~7;
    const int nq = min(Q, M - tq * Q);
    for (int j = warp; j < nq; j += NWARP)
      mark_query<W, P16, false>(T, j >> 5, W == 1 ? 1u << qbit(j) : 1u << (j & 31),
                                q_slot[buf][j], lane, a, pitems16);
    __syncthreads();
    // the other buffer was last read before the previous tile's final barrier
    if (kAhead && warp == NWARP - 1) fetch(buf ^ 1);
    uint16_t* G0 = a.gram + a.gofs[c];
    uint16_t* Gc = G0 + tq * Q;
    for (;;) {
      int p0 = 0;
      if (lane == 0) p0 = atomicAdd(&s_next, 32);
      p0 = tq * Q + __shfl_sync(0xffffffffu, p0, 0);
      if (p0 >= M) break;
      const int p = p0 + lane;
      if constexpr (W == 1) {
        const unsigned act = __ballot_sync(0xffffffffu, p < M);
        if (p < M) {
          const int4 sl = a.islot[cbase + p];
          const int len = sl.z;
          uint32_t A[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) A[r] = 0;
          // eight planes while every profile of the warp is shorter than 256
          const bool wide = __any_sync(act, len > 255);
          if constexpr (P16) {
            const uint4* r8 = reinterpret_cast<const uint4*>(pitems16 + sl.y);
            if (wide) count_row16_bs<16>(r8, (len + 7) >> 3, T, a.n_items, A);
            else count_row16_bs<8>(r8, (len + 7) >> 3, T, a.n_items, A);
          } else {
            const int4* r4 = reinterpret_cast<const int4*>(a.pitems + sl.x);
            if (wide) count_row4_bs<16>(r4, (len + 3) >> 2, T, a.n_items, A);
            else count_row4_bs<8>(r4, (len + 3) >> 2, T, a.n_items, A);
          }
          visits += (unsigned)len;
          transpose_halves16(A);   // A[h] = count(2h) | count(2h + 1) << 16
          uint4* dst = reinterpret_cast<uint4*>(Gc + (int64_t)p * Mp);
#pragma unroll
          for (int g8 = 0; g8 < 4; ++g8)
            if (g8 * 8 < nq)
              __stcs(dst + g8, make_uint4(A[4 * g8], A[4 * g8 + 1], A[4 * g8 + 2], A[4 * g8 + 3]));
          if (p >= (tq + 1) * Q) {
            uint16_t* col = G0 + (int64_t)(tq * Q) * Mp + p;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nq)
                __stcs(reinterpret_cast<unsigned short*>(col + (int64_t)j * Mp),
                       (unsigned short)(A[j >> 1] >> (16 * (j & 1))));
          }
        }
        continue;
      }
      if (p < M) {
        const int4 sl = a.islot[cbase + p];
        const int len = sl.z;
        uint32_t C[16 * W];
#pragma unroll
        for (int r = 0; r < 16 * W; ++r) C[r] = 0;
        if constexpr (P16)
          count_row16<W>(reinterpret_cast<const uint4*>(pitems16 + sl.y), (len + 7) >> 3, T,
                         a.n_items, C);
        else
          count_row4<W>(reinterpret_cast<const int4*>(a.pitems + sl.x), (len + 3) >> 2, T,
                        a.n_items, C);
        visits += (unsigned)len;
        // row p, columns tq*Q .. tq*Q + nq (16-byte stores, padding columns allowed)
        uint4* dst = reinterpret_cast<uint4*>(Gc + (int64_t)p * Mp);
#pragma unroll
        for (int g8 = 0; g8 < Q / 8; ++g8) {
          if (g8 * 8 < nq) {
            uint32_t wv[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int j0 = g8 * 8 + 2 * h, j1 = j0 + 1;
              const uint32_t lo = (C[creg(j0)] >> (16 * chalf(j0))) & 0xFFFFu;
              const uint32_t hi = (C[creg(j1)] >> (16 * chalf(j1))) & 0xFFFFu;
              wv[h] = lo | (hi << 16);
            }
            __stcs(dst + g8, make_uint4(wv[0], wv[1], wv[2], wv[3]));
          }
        }
        // column p of the tile's rows (the tile's own block is computed whole)
        if (p >= (tq + 1) * Q) {
          uint16_t* col = G0 + (int64_t)(tq * Q) * Mp + p;
#pragma unroll
          for (int j = 0; j < Q; ++j)
            if (j < nq)
              __stcs(reinterpret_cast<unsigned short*>(col + (int64_t)j * Mp),
                     (unsigned short)((C[creg(j)] >> (16 * chalf(j))) & 0xFFFFu));
        }
      }
    }
    __syncthreads();
    for (int j = warp; j < nq; j += NWARP)
      mark_query<W, P16, true>(T, j >> 5, 0u, q_slot[buf][j], lane, a, pitems16);
    if (tid == 0) s_next = 0;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) visits += __shfl_xor_sync(0xffffffffu, visits, o);
  if (lane == 0 && visits) atomicAdd(&a.hdr->item_visits[1], visits);
}

// ------------------------------------------------------------------ hashed gram kernel
// k_gram for item universes too large for the shared table: the tile's query
// items go into a shared open-addressing hash table (item -> mask of the
// tile's queries holding it, linear probing, at most half full) behind a
// 64 Ki-bit presence filter, so most candidate items (absent from every
// query) cost one shared load.  A tile whose queries hold more items than
// half the table is processed in passes over consecutive query groups.
constexpr int kHashSlots = 8192;                 // keys + masks: 64 KiB
constexpr int kHashCap = kHashSlots / 2;         // items per pass (load factor 1/2)
constexpr int kHashFilterWords = 2048;           // 65,536-bit presence filter
constexpr uint32_t kHashEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t hash_mix(int32_t x) { return (uint32_t)x * 0x9E3779B1u; }

// Mask of the tile's queries holding item x (0 if none).
__device__ __forceinline__ uint32_t hash_find(const uint32_t* __restrict__ hkey,
                                              const uint32_t* __restrict__ hval,
                                              const uint32_t* __restrict__ filt, int32_t x) {
  const uint32_t h = hash_mix(x);
  const uint32_t fb = h >> 16;
  if (!((filt[fb >> 5] >> (fb & 31)) & 1u)) return 0u;
  uint32_t slot = (h >> 3) & (kHashSlots - 1);
  for (int probe = 0; probe < kHashSlots; ++probe) {   // ends at an empty slot (half full)
    const uint32_t kx = hkey[slot];
    if (kx == (uint32_t)x) return hval[slot];
    if (kx == kHashEmpty) return 0u;
    slot = (slot + 1) & (kHashSlots - 1);
  }
  return 0u;
}

__device__ __forceinline__ void hash_insert(uint32_t* hkey, uint32_t* hval, uint32_t* filt,
                                            int32_t x, uint32_t bit) {
  const uint32_t h = hash_mix(x);
  const uint32_t fb = h >> 16;
  atomicOr(&filt[fb >> 5], 1u << (fb & 31));
  uint32_t slot = (h >> 3) & (kHashSlots - 1);
  for (int probe = 0; probe < kHashSlots; ++probe) {
    const uint32_t old = atomicCAS(&hkey[slot], kHashEmpty, (uint32_t)x);
    if (old == kHashEmpty || old == (uint32_t)x) {
      atomicOr(&hval[slot], bit);
      return;
    }
    slot = (slot + 1) & (kHashSlots - 1);
  }
}

// count_row4 with the hashed table (W = 1).
__device__ __forceinline__ void count_row4_hash(const int4* __restrict__ r4, int n4,
                                                const uint32_t* __restrict__ hkey,
                                                const uint32_t* __restrict__ hval,
                                                const uint32_t* __restrict__ filt, int sentinel,
                                                uint32_t* C) {
  const int4 pad = make_int4(sentinel, sentinel, sentinel, sentinel);
  int4 cur[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) cur[j] = j < n4 ? __ldg(r4 + j) : pad;
  uint32_t acc[4] = {0u, 0u, 0u, 0u};
  for (int i = 0; i < n4; i += 3) {
    int4 nxt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) nxt[j] = (i + 3 + j < n4) ? __ldg(r4 + i + 3 + j) : pad;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int xs[4] = {cur[j].x, cur[j].y, cur[j].z, cur[j].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t m = hash_find(hkey, hval, filt, xs[q]);
        if (m) add_mask(acc, m);
      }
    }
    flush(acc, C);
#pragma unroll
    for (int j = 0; j < 3; ++j) cur[j] = nxt[j];
  }
}

size_t gram_hash_smem_bytes() { return (size_t)(2 * kHashSlots + kHashFilterWords) * 4; }

template <int NT, int MB>
__global__ void __launch_bounds__(NT, MB) k_gram_hash(GramArgs a) {
  constexpr int Q = 32, NWARP = NT / 32;
  extern __shared__ __align__(16) uint32_t hsm[];
  uint32_t* hkey = hsm;
  uint32_t* hval = hsm + kHashSlots;
  uint32_t* filt = hsm + 2 * kHashSlots;
  __shared__ int32_t q_id[Q], q_len[Q];
  __shared__ int s_work, s_next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kHashSlots; i += NT) { hkey[i] = kHashEmpty; hval[i] = 0u; }
  for (int i = tid; i < kHashFilterWords; i += NT) filt[i] = 0u;
  if (tid == 0) s_next = 0;
  const int wbeg = *a.work_begin, nwork = *a.work_end;
  unsigned long long visits = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) s_work = dev_failed(a.hdr) ? nwork : wbeg + (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int wi = s_work;
    if (wi >= nwork) break;
    const int c = a.work_c[wi], tq = a.work_t[wi];
    const int cbase = a.cptr[c], M = a.cptr[c + 1] - cbase, Mp = (M + 7) & ~7;
    const int nq = min(Q, M - tq * Q);
    if (tid < Q) {
      int id = -1, len = 0;
      if (tid < nq) {
        const int2 in = a.iinfo[cbase + tq * Q + tid];
        id = a.cusers[cbase + in.x];
        len = in.y;
      }
      q_id[tid] = id;
      q_len[tid] = len;
    }
    __syncthreads();
    uint16_t* G0 = a.gram + a.gofs[c];
    // passes over consecutive query groups of at most kHashCap items (every
    // profile fits: the host checks the longest against kHashCap)
    int j0 = 0;
    while (j0 < nq) {
      int j1 = j0, sum = 0;
      while (j1 < nq && sum + q_len[j1] <= kHashCap) sum += q_len[j1++];
      if (j1 == j0) j1 = j0 + 1;   // not reached when the host check holds
      for (int j = j0 + warp; j < j1; j += NWARP) {
        const int u = q_id[j];
        for (int e = a.ptr[u] + lane; e < a.ptr[u + 1]; e += 32)
          hash_insert(hkey, hval, filt, a.items[e], 1u << j);
      }
      __syncthreads();
      for (;;) {
        int p0 = 0;
        if (lane == 0) p0 = atomicAdd(&s_next, 32);
        p0 = tq * Q + __shfl_sync(0xffffffffu, p0, 0);
        if (p0 >= M) break;
        const int p = p0 + lane;
        if (p < M) {
          const int2 info = a.iinfo[cbase + p];
          const int v = a.cusers[cbase + info.x];
          const int len = info.y;
          uint32_t C[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) C[r] = 0;
          count_row4_hash(reinterpret_cast<const int4*>(a.pitems + a.pptr[v]), (len + 3) >> 2,
                          hkey, hval, filt, a.n_items, C);
          visits += (unsigned)len;
          // row p, columns tq*Q + j0 .. tq*Q + j1
          uint16_t* rowp = G0 + (int64_t)p * Mp + tq * Q;
#pragma unroll
          for (int j = 0; j < Q; ++j)
            if (j >= j0 && j < j1) rowp[j] = (uint16_t)((C[creg(j)] >> (16 * chalf(j))) & 0xFFFFu);
          // column p of the tile's rows (the tile's own block is computed whole)
          if (p >= (tq + 1) * Q) {
            uint16_t* col = G0 + (int64_t)(tq * Q) * Mp + p;
#pragma unroll
            for (int j = 0; j < Q; ++j)
              if (j >= j0 && j < j1)
                col[(int64_t)j * Mp] = (uint16_t)((C[creg(j)] >> (16 * chalf(j))) & 0xFFFFu);
          }
        }
      }
      __syncthreads();
      // empty the table for the next pass or tile
      for (int i = tid; i < kHashSlots; i += NT) { hkey[i] = kHashEmpty; hval[i] = 0u; }
      for (int i = tid; i < kHashFilterWords; i += NT) filt[i] = 0u;
      if (tid == 0) s_next = 0;
      __syncthreads();
      j0 = j1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) visits += __shfl_xor_sync(0xffffffffu, visits, o);
  if (lane == 0 && visits) atomicAdd(&a.hdr->item_visits[1], visits);
}

// Judge (exact global top-k of query users, Eq. 2's denominator) for item
// universes too large for the shared table: k_table's judge mode with the
// tile's items in the shared hash table, in passes over query groups of at
// most kHashCap items; each query's list is updated in its own pass.
template <int NT>
__global__ void __launch_bounds__(NT) k_table_hash(TableArgs a) {
  constexpr int Q = 32, NWARP = NT / 32, QPW = Q / NWARP;
  extern __shared__ __align__(16) uint32_t tsm[];
  uint32_t* hkey = tsm;
  uint32_t* hval = tsm + kHashSlots;
  uint32_t* filt = tsm + 2 * kHashSlots;
  uint32_t* cntw = filt + kHashFilterWords;                 // [16][NT]
  int32_t* cand_id = reinterpret_cast<int32_t*>(cntw + 16 * NT);
  int32_t* cand_len = cand_id + NT;
  __shared__ int32_t q_id[Q], q_len[Q];
  __shared__ int s_work;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k;
  for (int i = tid; i < kHashSlots; i += NT) { hkey[i] = kHashEmpty; hval[i] = 0u; }
  for (int i = tid; i < kHashFilterWords; i += NT) filt[i] = 0u;
  const int nwork = *a.n_work;
  unsigned long long visits = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) s_work = dev_failed(a.hdr) ? nwork : (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int wi = s_work;
    if (wi >= nwork) break;
    const int qbase = wi * Q, nq = min(Q, a.n_queries - qbase), M = a.n_users;
    if (tid < Q) {
      int id = -1, len = 0;
      if (tid < nq) {
        id = a.queries ? a.queries[qbase + tid] : qbase + tid;
        len = a.ptr[id + 1] - a.ptr[id];
      }
      q_id[tid] = id;
      q_len[tid] = len;
    }
    __syncthreads();
    WarpList L[QPW];
#pragma unroll
    for (int s2 = 0; s2 < QPW; ++s2) { L[s2].id = -1; L[s2].c = 0; L[s2].u = 0; }
    int j0 = 0;
    while (j0 < nq) {
      int j1 = j0, sum = 0;
      while (j1 < nq && sum + q_len[j1] <= kHashCap) sum += q_len[j1++];
      if (j1 == j0) j1 = j0 + 1;   // not reached: the host checks the longest profile
      for (int j = j0 + warp; j < j1; j += NWARP) {
        const int u = q_id[j];
        for (int e = a.ptr[u] + lane; e < a.ptr[u + 1]; e += 32)
          hash_insert(hkey, hval, filt, a.items[e], 1u << j);
      }
      __syncthreads();
      for (int cb = 0; cb < M; cb += NT) {
        const int v = cb + tid;
        const bool act = v < M;
        const int len = act ? a.ptr[v + 1] - a.ptr[v] : 0;
        uint32_t C[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) C[r] = 0;
        if (act) {
          count_row4_hash(reinterpret_cast<const int4*>(a.pitems + a.pptr[v]), (len + 3) >> 2,
                          hkey, hval, filt, a.n_items, C);
          visits += (unsigned)len;
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) cntw[r * NT + tid] = C[r];
        cand_id[tid] = act ? v : -1;
        cand_len[tid] = len;
        __syncthreads();
        const int nc = min(NT, M - cb);
#pragma unroll
        for (int s2 = 0; s2 < QPW; ++s2) {
          const int j = warp + NWARP * s2;
          if (j >= j0 && j < j1) {
            const int qid = q_id[j], qlen = q_len[j];
            const int r = creg(j), h = chalf(j);
            for (int i0 = 0; i0 < nc; i0 += 32) {
              WarpList kth;
              kth.id = __shfl_sync(0xffffffffu, L[s2].id, k - 1);
              kth.c = __shfl_sync(0xffffffffu, L[s2].c, k - 1);
              kth.u = __shfl_sync(0xffffffffu, L[s2].u, k - 1);
              const int i = i0 + lane;
              bool pass = false;
              uint32_t cc = 0, uu = 0;
              int32_t vid = -1;
              if (i < nc) {
                cc = (cntw[r * NT + i] >> (16 * h)) & 0xFFFFu;
                vid = cand_id[i];
                if (vid != qid && cc > 0) {
                  uu = (uint32_t)(qlen + cand_len[i]) - cc;
                  pass = beats(kth, vid, cc, uu);
                }
              }
              warp_list_add(L[s2], k, pass, vid, cc, uu);
            }
          }
        }
        __syncthreads();
      }
      for (int i = tid; i < kHashSlots; i += NT) { hkey[i] = kHashEmpty; hval[i] = 0u; }
      for (int i = tid; i < kHashFilterWords; i += NT) filt[i] = 0u;
      __syncthreads();
      j0 = j1;
    }
#pragma unroll
    for (int s2 = 0; s2 < QPW; ++s2) {
      const int j = warp + NWARP * s2;
      if (j < nq && lane < k) {
        const int64_t row = (int64_t)(qbase + j) * k + lane;
        const bool ok = L[s2].id >= 0;
        a.out_id[row] = ok ? L[s2].id : -1;
        a.out_in[row] = ok ? (int32_t)L[s2].c : 0;
        a.out_un[row] = ok ? (int32_t)L[s2].u : 0;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) visits += __shfl_xor_sync(0xffffffffu, visits, o);
  if (lane == 0 && visits) atomicAdd(&a.hdr->item_visits[0], visits);
}

__device__ __forceinline__ uint32_t merge_count(const int32_t* __restrict__ a, int la,
                                                const int32_t* __restrict__ b, int lb);

// Count-matrix rows by sorted-list merges, for item universes too large for
// the shared table: one warp per member (row), lane per candidate (column).
struct MergeGramArgs {
  const int32_t* ptr;
  const int32_t* items;
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* gcl;
  const int64_t* gofs;
  uint16_t* gram;
  const int32_t* u_slot;
  const int32_t* u_g;
  const int32_t* n_users_dev;
  const int32_t* ipos;
  const int2* iinfo;
  DevHeader* hdr;
};

// One warp per member (a slot in user-id order): its row at its internal
// position, columns in internal order.
__global__ void __launch_bounds__(256) k_merge_gram(MergeGramArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_users_dev || dev_failed(a.hdr)) return;
  const int slot = a.u_slot[w];
  const int c = a.gcl[a.u_g[w]];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, Mp = (M + 7) & ~7;
  const int u = a.cusers[slot];
  const int32_t* ur = a.items + a.ptr[u];
  const int ul = a.ptr[u + 1] - a.ptr[u];
  uint16_t* row = a.gram + a.gofs[c] + (int64_t)a.ipos[slot] * Mp;
  for (int p0 = 0; p0 < M; p0 += 32) {
    const int p = p0 + lane;
    if (p < M) {
      const int v = a.cusers[cs + a.iinfo[cs + p].x];
      row[p] = (uint16_t)merge_count(ur, ul, a.items + a.ptr[v], a.ptr[v + 1] - a.ptr[v]);
    }
  }
}

// Length bucket: exact below 4, then 4 buckets per octave (at most 63).
__device__ __forceinline__ int len_bucket(int len) {
  if (len < 4) return len;
  const int oct = 31 - __clz(len);                 // >= 2
  const int b = oct * 4 + ((len >> (oct - 2)) & 3);
  return min(b, 63);
}

// Internal order of a cluster with a count matrix: members by decreasing
// profile length (64 buckets, 4 per octave), stable within a bucket; one
// block per cluster, chunks of 256 members placed in order.
// ipos[slot] = internal position, iinfo[cluster start + position] = (local
// index, profile length).
__global__ void __launch_bounds__(256) k_order(const int32_t* __restrict__ gcl, int32_t g0,
                                               const int32_t* __restrict__ cptr,
                                               const int32_t* __restrict__ slen,
                                               int32_t* __restrict__ ipos,
                                               int2* __restrict__ iinfo,
                                               const int64_t* __restrict__ gofs,
                                               uint16_t* __restrict__ gram,
                                               const int32_t* __restrict__ cusers,
                                               const int32_t* __restrict__ pptr,
                                               const int32_t* __restrict__ pptr16,
                                               int4* __restrict__ islot) {
  __shared__ int32_t start[64];
  __shared__ int32_t wcnt[8][64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = gcl[g0 + blockIdx.x];
  const int cbase = cptr[c], M = cptr[c + 1] - cbase, Mp = (M + 7) & ~7;
  // the row after the M count rows: profile lengths in internal order
  uint16_t* lenrow = gram + gofs[c] + (int64_t)M * Mp;
  if (tid < 64) start[tid] = 0;
  if (tid < Mp - M) lenrow[M + tid] = 0;
  __syncthreads();
  for (int i = tid; i < M; i += 256) atomicAdd(&start[63 - len_bucket(slen[cbase + i])], 1);
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int b = 0; b < 64; ++b) {
      const int x = start[b];
      start[b] = acc;
      acc += x;
    }
  }
  __syncthreads();
  for (int base = 0; base < M; base += 256) {
    const int i = base + tid;
    const int len = i < M ? slen[cbase + i] : 0;
    const int bk = i < M ? 63 - len_bucket(len) : 64;
    const unsigned peers = __match_any_sync(0xffffffffu, bk);
    const int rank = __popc(peers & lanemask_lt());
    wcnt[warp][lane] = 0;
    wcnt[warp][lane + 32] = 0;
    __syncwarp();
    if (i < M && rank == 0) wcnt[warp][bk] = __popc(peers);
    __syncthreads();
    if (i < M) {
      int off = start[bk] + rank;
      for (int w2 = 0; w2 < warp; ++w2) off += wcnt[w2][bk];
      ipos[cbase + i] = off;
      iinfo[cbase + off] = make_int2(i, len);
      const int v = cusers[cbase + i];
      islot[cbase + off] = make_int4(pptr[v], pptr16 ? pptr16[v] : 0, len, v);
      lenrow[off] = (uint16_t)len;
    }
    __syncthreads();
    if (tid < 64) {
      int sum = 0;
      for (int w2 = 0; w2 < 8; ++w2) sum += wcnt[w2][tid];
      start[tid] += sum;
    }
    __syncthreads();
  }
}

// Brute-force top-k of one member from its row of the count matrix: warp per
// member, exact comparison, candidates with no common item skipped.
struct RowTopkArgs {
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* slen;
  const int32_t* gcl;
  const int64_t* gofs;
  const uint16_t* gram;
  const int32_t* u_slot;
  const int32_t* u_g;
  const int32_t* n_users_dev;
  const int32_t* ipos;
  const int2* iinfo;
  int32_t k;
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

// (common, union) counts of a member of the warp's cluster, by internal
// position, from the global row of counts and the internal (index, length).
struct GlobalCU {
  const uint16_t* row;
  const int2* info;        // internal (local index, length) from the cluster's start
  uint32_t my;
  __device__ __forceinline__ uint2 operator()(int32_t p) const {
    const uint32_t c = row[p];
    return make_uint2(c, my + (uint32_t)info[p].y - c);
  }
};

// One warp per user of a brute-force cluster: the top k of the user's row of
// intersection counts, 32 candidates per step (coalesced), staged and
// merged; `Keyed` (every union below 2^16) holds the list as exact 64-bit
// order keys.  Rows and columns are in internal order; candidates are
// ranked by local index (user-id order).
template <bool Keyed>
__device__ __forceinline__ void row_topk(const RowTopkArgs& a, int w, int32_t* sid, uint2* scu) {
  const int lane = threadIdx.x & 31;
  const int slot = a.u_slot[w];
  const int c = a.gcl[a.u_g[w]];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, Mp = (M + 7) & ~7;
  const int P = a.ipos[slot];
  const uint16_t* row = a.gram + a.gofs[c] + (int64_t)P * Mp;
  const int2* info = a.iinfo + cs;
  const uint32_t my = (uint32_t)a.slen[slot];
  const int k = a.k;
  typename std::conditional<Keyed, KeyTopk<GlobalCU>, WarpTopk>::type tk;
  if constexpr (Keyed) {
    tk.start(0ull, k, scu, GlobalCU{row, info, my});
    // first pass: each lane's best candidate; the k-th best of these 32
    // distinct candidates ranks no higher than the row's k-th best, so it
    // floors the filter of the second pass
    uint32_t bc = 0u, bu = 1u, bl = 0x7fffffffu;
    int bp = -1;
#pragma unroll 4
    for (int p = lane; p < M; p += 32) {   // unrolled: four candidates' loads in flight
      const uint32_t c = p != P ? (uint32_t)row[p] : 0u;
      const int2 in = info[p];
      if (c == 0u) continue;
      const uint32_t u = my + (uint32_t)in.y - c;
      const uint32_t l = c * bu, r = bc * u;
      if (l > r || (l == r && (uint32_t)in.x < bl)) { bc = c; bu = u; bl = (uint32_t)in.x; bp = p; }
    }
    const uint64_t bk = warp_sort32_keys(bp >= 0 ? nbr_key(bc, bu, (int32_t)bl, bp) : 0ull);
    tk.set_floor(__shfl_sync(0xffffffffu, bk, k - 1));
  } else {
    WarpList l0;
    l0.id = -1; l0.c = 0; l0.u = 0;
    tk.start(l0, k, sid, scu);
  }
  // steps of 32 candidates, through a ring of 4 steps of loads in flight (a
  // rolled loop keeps the kernel small enough for the instruction cache)
  auto fetch = [&](int j, uint32_t& cc, int2& in) {
    const int p = j * 32 + lane;
    cc = (p < M && p != P) ? (uint32_t)row[p] : 0u;
    in = p < M ? info[p] : make_int2(0, 0);
  };
  uint32_t c0, c1, c2, c3;
  int2 i0, i1, i2, i3;
  fetch(0, c0, i0); fetch(1, c1, i1); fetch(2, c2, i2); fetch(3, c3, i3);
  const int nsteps = (M + 31) >> 5;
#pragma unroll 1
  for (int j = 0; j < nsteps; ++j) {
    uint32_t cn;
    int2 in_;
    fetch(j + 4, cn, in_);
    const int p = j * 32 + lane;
    const uint32_t uu = my + (uint32_t)i0.y - c0;
    // local index order = user id order
    const bool pass = c0 > 0u && tk.filter(i0.x, c0, uu);
    if constexpr (Keyed) tk.stage(pass, p, i0.x, c0, uu);
    else tk.stage(pass, i0.x, c0, uu);
    c0 = c1; c1 = c2; c2 = c3; c3 = cn;
    i0 = i1; i1 = i2; i2 = i3; i3 = in_;
  }
  tk.finish();
  if (lane < k) {
    const int64_t o = (int64_t)slot * k + lane;
    int32_t id;
    uint32_t oc = 0, ou = 0;
    if constexpr (Keyed) {
      id = tk.id();
      if (id >= 0) {
        const uint2 x = GlobalCU{row, info, my}(tk.pos());
        oc = x.x; ou = x.y;
      }
    } else {
      id = tk.L.id; oc = tk.L.c; ou = tk.L.u;
    }
    a.out_id[o] = id >= 0 ? a.cusers[cs + id] : -1;
    a.out_in[o] = id >= 0 ? (int32_t)oc : 0;
    a.out_un[o] = id >= 0 ? (int32_t)ou : 0;
  }
}

template <bool Keyed>
__global__ void __launch_bounds__(kNT, 6) k_gram_topk(RowTopkArgs a) {
  __shared__ int32_t s_sid[Keyed ? 1 : kNT / 32][64];
  __shared__ uint2 s_scu[kNT / 32][64];
  const int warp = threadIdx.x >> 5;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_users_dev || dev_failed(a.hdr)) return;
  row_topk<Keyed>(a, w, s_sid[Keyed ? 0 : warp], s_scu[warp]);
}

// The keyed row path as a call, for the rows the select kernel hands back.
static __device__ __noinline__ void row_topk_keyed(const RowTopkArgs& a, int w, uint2* scu) {
  row_topk<true>(a, w, nullptr, scu);
}

// Exact floor(65536 c / u) for 0 < c <= u < 2^16, clamped to 65535.
__device__ __forceinline__ uint32_t jac_q16(uint32_t c, uint32_t u) {
  return min(udiv16(c << 16, u), 65535u);
}

// Brute-force rows by exact selection (keyed rows: unions below 2^16): warp
// per member.  q = floor(65536 J) is exact and monotone in J, so the k best
// candidates are among those whose q reaches the row's k-th largest q.
//  1. One pass over the count row (four candidates per lane and step, one
//     8-byte load of counts; the member itself and the padding are zeroed
//     per load) keeps each lane's two largest estimates of q (a float
//     quotient, at most one above the exact q).  T0 = the k-th largest of
//     these 64 estimates (a bitwise search, one warp sum per bit), minus one,
//     is at most the row's k-th largest q (k distinct candidates reach it).
//  2. A second pass stages every candidate with q >= T0 (tested exactly as
//     c * 2^16 >= T0 * u) -- typically a few more than k, at most kSelStage.
//  3. In shared memory, when more than 64 are staged: the staged q are
//     histogrammed in 256 buckets over [T0, 65535] (and the bucket of the k-th
//     largest again by its low bits when buckets are wider than one value),
//     giving the exact k-th largest q, qk; the staged candidates with q >= qk
//     are kept.  The (at most 64) remaining get exact order keys and are
//     sorted (one or two warp sorts and a bitonic merge).
// Rows with more than kSelStage candidates above T0, or more than 64 at or
// above qk, go through the general keyed path.
constexpr int kSelStage = 256;

// Bucket (largest first) holding the need-th largest of a 256-bucket
// histogram: lane l holds buckets 255 - 8l .. 248 - 8l.  Returns -1 when the
// histogram holds fewer than `need`; *above = entries in higher buckets.
__device__ __forceinline__ int hist_select(const uint32_t* hist, int need, uint32_t* above) {
  const int lane = threadIdx.x & 31;
  uint32_t v[8], sum = 0u;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = hist[255 - 8 * lane - i];
    sum += v[i];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned hit = __ballot_sync(0xffffffffu, incl >= (uint32_t)need);
  if (hit == 0u) {
    *above = 0u;
    return -1;
  }
  const int L = __ffs(hit) - 1;
  int b = -1;
  uint32_t run = __shfl_sync(0xffffffffu, incl - sum, L), ab = 0u;
  if (lane == L) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (b < 0 && run + v[i] >= (uint32_t)need) {
        b = 255 - 8 * lane - i;
        ab = run;
      }
      run += v[i];
    }
  }
  *above = __shfl_sync(0xffffffffu, ab, L);
  return __shfl_sync(0xffffffffu, b, L);
}

__global__ void __launch_bounds__(kNT, 6) k_gram_select(const __grid_constant__ RowTopkArgs a) {
  __shared__ uint2 s_stage[kNT / 32][kSelStage];   // (pos | lid << 16, c | u << 16)
  __shared__ uint32_t s_hist[kNT / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_users_dev || dev_failed(a.hdr)) return;
  uint2* stg = s_stage[warp];
  uint32_t* hist = s_hist[warp];
  const int slot = a.u_slot[w];
  const int c = a.gcl[a.u_g[w]];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, Mp = (M + 7) & ~7;
  const int P = a.ipos[slot];
  const uint16_t* row = a.gram + a.gofs[c] + (int64_t)P * Mp;
  // rows start on 16 bytes (matrices of M x Mp entries, Mp a multiple of 8)
  const uint2* row4 = reinterpret_cast<const uint2*>(row);
  const int M4 = (M + 3) >> 2;
  const int2* info = a.iinfo + cs;
  // the row after the count rows holds the members' lengths (same positions)
  const uint2* len4 = reinterpret_cast<const uint2*>(a.gram + a.gofs[c] + (int64_t)M * Mp);
  const uint32_t my = (uint32_t)a.slen[slot];
  const int k = a.k;
  // 1. each lane's two largest estimates of q.  Counts of the member itself
  // (position P) and of the padding past M are cleared per 8-byte load, so
  // that every position can be treated alike (a zero count estimates 0).
  const int gP = P >> 2, gL = M4 - 1;
  const uint32_t maskP = (P & 1) ? 0x0000FFFFu : 0xFFFF0000u;   // clears position P in its word
  const int rL = M - 4 * gL;                                     // positions of the last load
  const uint32_t tailx = rL >= 2 ? 0xFFFFFFFFu : 0x0000FFFFu;
  const uint32_t taily = rL >= 4 ? 0xFFFFFFFFu : (rL == 3 ? 0x0000FFFFu : 0u);
  auto load_counts = [&](int g) -> uint2 {
    uint2 cw = row4[g];
    if (g == gP) {
      if (P & 2) cw.y &= maskP;
      else cw.x &= maskP;
    }
    if (g == gL) {
      cw.x &= tailx;
      cw.y &= taily;
    }
    return cw;
  };
  uint32_t q1 = 0u, q2 = 0u;
#pragma unroll 2
  for (int g = lane; g < M4; g += 32) {
    const uint2 cw = load_counts(g), lw = len4[g];
    const uint32_t cq[4] = {cw.x & 0xFFFFu, cw.x >> 16, cw.y & 0xFFFFu, cw.y >> 16};
    const uint32_t lq[4] = {lw.x & 0xFFFFu, lw.x >> 16, lw.y & 0xFFFFu, lw.y >> 16};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t u = my + lq[q] - cq[q];
      // within one of the exact quotient (relative error below 2^-21); 0
      // for a zero count (0 / 0 converts to 0 as well)
      const uint32_t qe = __float2uint_rz(__fdividef((float)(cq[q] << 16), (float)u));
      q2 = max(q2, min(q1, qe));
      q1 = max(q1, qe);
    }
  }
  // the k-th largest of the 64 estimates (0: fewer than k reach 1), bit by bit
  uint32_t kth = 0u;
#pragma unroll
  for (int bit = 16; bit >= 0; --bit) {
    const uint32_t c = kth | (1u << bit);
    if (__reduce_add_sync(0xffffffffu, (uint32_t)(q1 >= c) + (uint32_t)(q2 >= c)) >= (uint32_t)k)
      kth = c;
  }
  const uint32_t T0 = kth ? kth - 1u : 0u;
  // 2. stage the candidates with q >= T0 (every candidate when T0 = 0)
  int n = 0;
  bool ok = true;
  for (int g0 = 0; g0 < M4; g0 += 32) {
    const int g = g0 + lane;
    uint2 cw = make_uint2(0u, 0u), lw = make_uint2(0u, 0u);
    if (g < M4) {
      cw = load_counts(g);
      lw = len4[g];
    }
    const uint32_t cq[4] = {cw.x & 0xFFFFu, cw.x >> 16, cw.y & 0xFFFFu, cw.y >> 16};
    const uint32_t lq[4] = {lw.x & 0xFFFFu, lw.x >> 16, lw.y & 0xFFFFu, lw.y >> 16};
    uint32_t uu[4];
    unsigned m[4];
    int tot = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uu[q] = my + lq[q] - cq[q];
      m[q] = __ballot_sync(0xffffffffu, cq[q] != 0u && (cq[q] << 16) >= T0 * uu[q]);
      tot += __popc(m[q]);
    }
    if (n + tot > kSelStage) {
      ok = false;
      break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if ((m[q] >> lane) & 1u) {   // the local index of a staged candidate only
        const int p = 4 * g + q;
        stg[n + __popc(m[q] & lanemask_lt())] =
            make_uint2((uint32_t)p | ((uint32_t)info[p].x << 16), cq[q] | (uu[q] << 16));
      }
      n += __popc(m[q]);
    }
  }
  if (!ok) {
    if (lane == 0) atomicAdd(&a.hdr->select_general, 1);
    row_topk_keyed(a, w, stg);
    return;
  }
  __syncwarp();
  // 3. the exact k-th largest q among the staged, when more than 64 are staged
  uint32_t qk = 0u;
  if (n > 64) {
    auto q_at = [&](int i) -> uint32_t {   // staged entry i's q (0xFFFFFFFF past the end)
      if (i >= n) return 0xFFFFFFFFu;
      const uint32_t x = stg[i].y;
      return jac_q16(x & 0xFFFFu, x >> 16);
    };
    const int sh = max(0, 32 - __clz((int)(65535u - T0)) - 8);
#pragma unroll
    for (int e = 0; e < 8; ++e) hist[lane + 32 * e] = 0u;
    __syncwarp();
    for (int i = lane; i < n; i += 32) atomicAdd(&hist[(q_at(i) - T0) >> sh], 1u);
    __syncwarp();
    uint32_t above = 0u;
    const int b1 = hist_select(hist, k, &above);   // n > 64 >= k: b1 >= 0
    if (sh == 0) {
      qk = T0 + (uint32_t)b1;
      ok = above + hist[b1] <= 64u;
    } else {
      const uint32_t lo = T0 + ((uint32_t)b1 << sh);
      __syncwarp();
#pragma unroll
      for (int e = 0; e < 8; ++e) hist[lane + 32 * e] = 0u;
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        const uint32_t q = q_at(i);
        if (q >= lo && q < lo + (1u << sh)) atomicAdd(&hist[q - lo], 1u);
      }
      __syncwarp();
      uint32_t above2 = 0u;
      const int b2 = hist_select(hist, k - (int)above, &above2);
      qk = lo + (uint32_t)(b2 < 0 ? 0 : b2);
      ok = b2 >= 0 && above + above2 + hist[b2] <= 64u;
    }
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicAdd(&a.hdr->select_general, 1);
      row_topk_keyed(a, w, stg);
      return;
    }
    // compact the staged with q >= qk to the front, in place: chunk e is read
    // before it is written, and writes never reach a later chunk
    int m_n = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const uint2 x = i < n ? stg[i] : make_uint2(0u, 0u);
      const bool pass = i < n && jac_q16(x.y & 0xFFFFu, x.y >> 16) >= qk;
      __syncwarp();
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) stg[m_n + __popc(m & lanemask_lt())] = x;
      m_n += __popc(m);
      __syncwarp();
    }
    n = m_n;
  }
  // exact order keys of the (at most 64) selected, sorted: one warp sort of
  // the first 32; up to 16 more are inserted one at a time, more than that
  // are sorted too and merged
  auto key_of = [&](int i) -> uint64_t {
    if (i >= n) return 0ull;
    const uint2 x = stg[i];
    return nbr_key(x.y & 0xFFFFu, x.y >> 16, (int32_t)(x.x >> 16), (int32_t)(x.x & 0xFFFFu));
  };
  uint64_t x = warp_sort32_keys(key_of(lane));
  if (n > 48) {
    const uint64_t y = warp_sort32_keys(key_of(lane + 32));
    const uint64_t r = __shfl_sync(0xffffffffu, y, 31 - lane);
    x = r > x ? r : x;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, x, j);
      const bool lower = (lane & j) == 0;
      x = lower ? (o > x ? o : x) : (o < x ? o : x);
    }
  } else if (n > 32) {
    const uint64_t y = key_of(lane + 32);
    for (int i = 0; i < n - 32; ++i) key_list_insert(x, k, __shfl_sync(0xffffffffu, y, i));
  }
  if (lane < k) {
    const int64_t o = (int64_t)slot * k + lane;
    const int32_t id = key_id(x);
    uint32_t oc = 0u, ou = 0u;
    if (id >= 0) {
      const int pos = key_pos(x);
      oc = (uint32_t)row[pos];
      ou = my + (uint32_t)reinterpret_cast<const uint16_t*>(len4)[pos] - oc;
    }
    a.out_id[o] = id >= 0 ? a.cusers[cs + id] : -1;
    a.out_in[o] = (int32_t)oc;
    a.out_un[o] = (int32_t)ou;
  }
}

// ------------------------------------------------------------------ padded CSR
// Rows padded to a multiple of 4 items with the sentinel item m, so that each
// row starts on a 16-byte boundary and is read with int4 loads.
__global__ void k_pad_len(const int32_t* __restrict__ ptr, int32_t n, int32_t* __restrict__ plen) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) plen[u] = ((ptr[u + 1] - ptr[u]) + 3) & ~3;
}

__global__ void k_pad_copy(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items,
                           const int32_t* __restrict__ pptr, int32_t n, int32_t m,
                           int64_t capacity, int32_t* __restrict__ pitems, DevHeader* hdr) {
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n || dev_failed(hdr)) return;
  if ((int64_t)pptr[n] > capacity || pptr[n] < 0) {
    if (lane == 0) dev_fail(hdr, C2_ERR_WORKSPACE);
    return;
  }
  const int32_t s = ptr[u], len = ptr[u + 1] - s, ps = pptr[u], plen = pptr[u + 1] - ps;
#pragma unroll 4
  for (int j = lane; j < plen; j += 32) pitems[ps + j] = j < len ? items[s + j] : m;
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
  int64_t n_rows;          // queries
  const int32_t* queries;  // NULL = 0 .. n_rows-1
  int32_t n_users;
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

// Top k of query `row` against every user, by sorted-list merges (lane i
// compares the query with candidate i of a chunk of 32).
__device__ __forceinline__ void merge_knn_row(const MergeArgs& a, int64_t row) {
  const int lane = threadIdx.x & 31;
  const int u = a.queries ? a.queries[row] : (int)row;
  const int M = a.n_users;
  const int k = a.k;
  const int32_t* ur = a.items + a.ptr[u];
  const int ul = a.ptr[u + 1] - a.ptr[u];
  WarpList L;
  L.id = -1; L.c = 0; L.u = 0;
  for (int cb = 0; cb < M; cb += 32) {
    const int v = cb + lane;
    uint32_t cc = 0, uu = 0;
    if (v < M && v != u) {
      const int vlen = a.ptr[v + 1] - a.ptr[v];
      cc = merge_count(ur, ul, a.items + a.ptr[v], vlen);
      uu = (uint32_t)(ul + vlen) - cc;
    }
    WarpList kth;
    kth.id = __shfl_sync(0xffffffffu, L.id, k - 1);
    kth.c = __shfl_sync(0xffffffffu, L.c, k - 1);
    kth.u = __shfl_sync(0xffffffffu, L.u, k - 1);
    const bool pass = v < M && v != u && cc > 0 && beats(kth, v, cc, uu);
    warp_list_add(L, k, pass, v, cc, uu);
  }
  if (lane < k) {
    const int64_t o = row * k + lane;
    const bool ok = L.id >= 0;
    a.out_id[o] = ok ? L.id : -1;
    a.out_in[o] = ok ? (int32_t)L.c : 0;
    a.out_un[o] = ok ? (int32_t)L.u : 0;
  }
}

// Judge mode: one warp per query against every user.
// The 16-bit copy of the profiles for item universes below 2^16: rows padded
// to a multiple of 8 items (one 16-byte load) with the sentinel item m.
__global__ void k_pad_len8(const int32_t* __restrict__ ptr, int32_t n, int32_t* __restrict__ plen) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) plen[u] = ((ptr[u + 1] - ptr[u]) + 7) & ~7;
}
__global__ void k_pad_copy16(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items,
                             const int32_t* __restrict__ pptr16, int32_t n, int32_t m,
                             int64_t capacity, uint16_t* __restrict__ p16, DevHeader* hdr) {
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n || dev_failed(hdr)) return;
  if ((int64_t)pptr16[n] > capacity || pptr16[n] < 0) {
    if (lane == 0) dev_fail(hdr, C2_ERR_WORKSPACE);
    return;
  }
  const int32_t s = ptr[u], len = ptr[u + 1] - s, ps = pptr16[u], plen = pptr16[u + 1] - ps;
#pragma unroll 4
  for (int j = lane; j < plen; j += 32) p16[ps + j] = (uint16_t)(j < len ? items[s + j] : m);
}

__global__ void __launch_bounds__(kNT) k_merge_knn(MergeArgs a) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.n_rows || dev_failed(a.hdr)) return;
  merge_knn_row(a, w);
}

// Small brute-force clusters (2 <= M <= 32 members, at most kSmallItems
// profile items in all): one warp per cluster (persistent grid over the
// listed clusters).  The members' profiles are staged in shared memory, the
// M(M-1)/2 intersections are counted by sorted-list merges spread over the
// lanes, and each member's row is one warp sort of its M-1 candidates (exact
// order, lower id first on ties; candidates with no common item dropped).
constexpr int kSmallItems = 2048;   // staged profile items per warp
constexpr int kSmallWarps = 4;      // warps per block

// merge_count for profiles that may sit in shared memory (generic loads).
__device__ __forceinline__ uint32_t merge_count_any(const int32_t* a, int la, const int32_t* b,
                                                    int lb) {
  int i = 0, j = 0;
  uint32_t c = 0;
  while (i < la && j < lb) {
    const int x = a[i], y = b[j];
    c += (x == y);
    i += (x <= y);
    j += (y <= x);
  }
  return c;
}

struct SmallArgs {
  const int32_t* ptr;
  const int32_t* items;
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* list;      // small clusters
  const int32_t* n_list;    // their device count
  int32_t k;
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

__global__ void __launch_bounds__(32 * kSmallWarps) k_small_knn(SmallArgs a) {
  __shared__ int32_t s_items[kSmallWarps][kSmallItems];
  __shared__ uint16_t s_cnt[kSmallWarps][32 * 32];
  __shared__ int32_t s_beg[kSmallWarps][32], s_len[kSmallWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t* sit = s_items[warp];
  uint16_t* cnt = s_cnt[warp];
  int32_t* mbeg = s_beg[warp];
  int32_t* mlen = s_len[warp];
  const int n = *a.n_list;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int k = a.k;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += nw) {
    if (dev_failed(a.hdr)) return;
    const int c = a.list[r];
    const int cbase = a.cptr[c], M = a.cptr[c + 1] - cbase;
    // member lane: its user, profile start and length; staged offsets
    const int u = lane < M ? a.cusers[cbase + lane] : 0;
    const int ps = lane < M ? a.ptr[u] : 0;
    const int len = lane < M ? a.ptr[u + 1] - ps : 0;
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const bool staged = total <= kSmallItems;
    const int32_t* base = staged ? sit : a.items;
    if (lane < M) {
      mbeg[lane] = staged ? incl - len : ps;
      mlen[lane] = len;
    }
    if (staged) {
      for (int m = 0; m < M; ++m) {
        const int s0 = __shfl_sync(0xffffffffu, ps, m), l0 = __shfl_sync(0xffffffffu, len, m);
        const int d0 = __shfl_sync(0xffffffffu, incl - len, m);
        for (int i = lane; i < l0; i += 32) sit[d0 + i] = a.items[s0 + i];
      }
    }
    __syncwarp();
    // pairs (i, j), i < j, in row order, spread over the lanes
    const int npairs = M * (M - 1) / 2;
    for (int q = lane; q < npairs; q += 32) {
      int i = 0, rem = q;
      while (rem >= M - 1 - i) { rem -= M - 1 - i; ++i; }
      const int j = i + 1 + rem;
      const uint32_t x = merge_count_any(base + mbeg[i], mlen[i], base + mbeg[j], mlen[j]);
      cnt[i * 32 + j] = (uint16_t)x;
      cnt[j * 32 + i] = (uint16_t)x;
    }
    __syncwarp();
    // rows: member i against the others, one warp sort each
    for (int i = 0; i < M; ++i) {
      WarpList e;
      e.id = -1; e.c = 0; e.u = 0;
      if (lane < M && lane != i) {
        const uint32_t x = cnt[i * 32 + lane];
        if (x > 0) {
          e.id = lane;                       // local index order = user id order
          e.c = x;
          e.u = (uint32_t)(mlen[i] + len) - x;
        }
      }
      warp_sort32(e);
      if (lane < k) {
        const int64_t o = (int64_t)(cbase + i) * k + lane;
        const bool ok = e.id >= 0;
        a.out_id[o] = ok ? a.cusers[cbase + e.id] : -1;
        a.out_in[o] = ok ? (int32_t)e.c : 0;
        a.out_un[o] = ok ? (int32_t)e.u : 0;
      }
    }
    __syncwarp();
  }
}

// Clusters that the small-cluster kernel computes (flag set), listed.
__global__ void k_fill_small(const int32_t* __restrict__ flag, const int32_t* __restrict__ off,
                             int64_t S, int32_t* __restrict__ list) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < S && flag[c]) list[off[c]] = (int32_t)c;
}

// ------------------------------------------------------------------ preparation
// Per cluster: does it get a count matrix (greedy clusters up to kMaxGreedyM
// members whose matrix fits the budget of cap elements, and brute-force
// clusters of at least small_cut members), is it greedy (1 with a count
// matrix, 2 without), pair count; singletons get an empty row (nobody else is
// in their cluster).
__global__ void k_prep(const int32_t* __restrict__ cptr, const int32_t* __restrict__ n_clusters,
                       const int32_t* __restrict__ cusers, const int32_t* __restrict__ ptr,
                       int64_t S, int32_t thr, int32_t small_cut, int32_t small_items, int32_t k,
                       int64_t cap, int32_t* __restrict__ gflag, int32_t* __restrict__ gkind,
                       int32_t* __restrict__ small_cnt,
                       int32_t* __restrict__ lid, int32_t* __restrict__ lin,
                       int32_t* __restrict__ lun, DevHeader* hdr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t L = *n_clusters;
  int32_t M = 0;
  if (c < S && c < L) M = cptr[c + 1] - cptr[c];
  const bool brute = M >= 2 && M < thr;
  const bool greedy = M >= 2 && M >= thr;
  const bool direct =
      greedy && (M > kMaxGreedyM || ((int64_t)M + 1) * (((int64_t)M + 7) & ~int64_t(7)) > cap);
  // small brute-force clusters whose profiles fit the per-warp stage go to
  // the warp-per-cluster kernel
  bool small = false;
  if (brute && M < small_cut) {
    int64_t tot = 0;
    for (int j = 0; j < M; ++j) {
      const int u = cusers[cptr[c] + j];
      tot += ptr[u + 1] - ptr[u];
    }
    small = tot <= small_items;
  }
  // counts are 16-bit: profiles of more than 65535 items are unsupported
  if (c == 0 && hdr->knn_max_len > 65535) dev_fail(hdr, C2_ERR_UNSUPPORTED);
  if (c < S) {
    gflag[c] = ((greedy && !direct) || (brute && !small)) ? 1 : 0;
    gkind[c] = direct ? 2 : (greedy ? 1 : 0);
    if (direct) {
      atomicMax(&hdr->max_cluster, M);
      atomicAdd(&hdr->greedy_users, M);
      atomicAdd(&hdr->n_greedy, 1);
      atomicAdd(&hdr->direct_users, M);
    }
    small_cnt[c] = small ? 1 : 0;
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
  unsigned long long pg = greedy ? (unsigned long long)M * (M - 1) / 2 : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    p += __shfl_xor_sync(0xffffffffu, p, o);
    pg += __shfl_xor_sync(0xffffffffu, pg, o);
  }
  if ((threadIdx.x & 31) == 0 && p) {
    atomicAdd(&hdr->pairs, p);
    atomicAdd(&hdr->brute_pairs, p);
  }
  if ((threadIdx.x & 31) == 0 && pg) atomicAdd(&hdr->greedy_pairs, pg);
  if (c == 0) hdr->n_labels = L;
}

// slot -> cluster by binary search in cptr; slot -> profile length; the
// longest profile.
__global__ void k_slot_info(const int32_t* __restrict__ cptr, const int32_t* __restrict__ n_clusters,
                            const int32_t* __restrict__ cusers, const int32_t* __restrict__ ptr,
                            int64_t S, int32_t* __restrict__ slot2c, int32_t* __restrict__ slen,
                            DevHeader* hdr) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int len = 0;
  if (s < S) {
    int lo = 0, hi = *n_clusters - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cptr[mid] <= s) lo = mid; else hi = mid - 1;
    }
    slot2c[s] = lo;
    const int u = cusers[s];
    len = ptr[u + 1] - ptr[u];
    slen[s] = len;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
  if ((threadIdx.x & 31) == 0 && len > 0) atomicMax(&hdr->knn_max_len, len);
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
                              const int32_t* __restrict__ gkind_c, const int32_t* __restrict__ cptr,
                              int64_t S, int32_t* __restrict__ gcl, int64_t* __restrict__ gsq,
                              int32_t* __restrict__ gsz, int32_t* __restrict__ gkind,
                              DevHeader* hdr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) hdr->n_work = gidx[S];   // count-matrix clusters
  if (c >= S || !gflag[c]) return;
  const int g = gidx[c];
  const int32_t M = cptr[c + 1] - cptr[c];
  gcl[g] = (int32_t)c;
  // M rows of counts, then one row of the members' profile lengths (uint16,
  // internal order); rows padded to 16 bytes
  const int64_t Mp = (M + 7) & ~7;
  gsq[g] = ((int64_t)M + 1) * Mp;
  gsz[g] = M;
  gkind[g] = gkind_c[c];
  atomicAdd(&hdr->gram_len_elems, (unsigned long long)Mp);
  if (gkind_c[c]) {
    atomicMax(&hdr->max_cluster, M);
    atomicAdd(&hdr->greedy_users, M);
    atomicAdd(&hdr->n_greedy, 1);
  } else {
    atomicAdd(&hdr->brute_gram_elems, (unsigned long long)(M * Mp));
    atomicAdd(&hdr->brute_rows, M);
  }
}

// Size buckets of count-matrix clusters (each gets its own table shape).
constexpr int kBuckets = 4;
__host__ __device__ inline int size_bucket(int M) {
  return M < 128 ? 0 : (M < 512 ? 1 : (M < 2048 ? 2 : 3));
}

// Per count-matrix cluster of a batch: its matrix offset and its members as
// greedy users / brute-force users / greedy work chunks.
__global__ void k_batch_setup(const int32_t* __restrict__ gcl, const int64_t* __restrict__ goff,
                              const int32_t* __restrict__ gsz, const int32_t* __restrict__ gkind,
                              int32_t g0, int32_t g1, int64_t* __restrict__ gofs,
                              int32_t* __restrict__ ngu, int32_t* __restrict__ nbu,
                              int32_t* __restrict__ ngw) {
  const int g = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= g1) return;
  const int M = gsz[g], j = g - g0;
  gofs[gcl[g]] = goff[g] - goff[g0];
  ngu[j] = gkind[g] ? M : 0;
  nbu[j] = gkind[g] ? 0 : M;
  ngw[j] = gkind[g] ? (M + kGreedyChunk - 1) / kGreedyChunk : 0;
}

// Query tiles of the batch clusters of one size bucket (tile = q members).
// bucket < 0 selects every cluster of the batch; clusters routed elsewhere
// (route[g] != 0: tensor cores, or not in this launch) get none.
__global__ void k_bucket_tiles(const int32_t* __restrict__ gsz, int32_t g0, int32_t nb,
                               int32_t bucket, int32_t q, const int32_t* __restrict__ route,
                               int32_t* __restrict__ cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int M = gsz[g0 + j];
  const bool in = (bucket < 0 || size_bucket(M) == bucket) && (!route || route[g0 + j] == 0);
  cnt[j] = in ? (M + q - 1) / q : 0;
}

// Adds the host-counted tensor-core work of a batch to the statistics.
__global__ void k_tc_stats(DevHeader* hdr, unsigned long long macs, int32_t clusters,
                           int32_t tiles) {
  hdr->tc_macs += macs;
  hdr->tc_clusters += clusters;
  hdr->tc_tiles += tiles;
}

// Members of the batch's clusters of one kind, as (slot, count-matrix index).
__global__ void k_fill_users(const int32_t* __restrict__ gcl, const int32_t* __restrict__ cptr,
                             const int32_t* __restrict__ gkind, int32_t want,
                             const int32_t* __restrict__ uoff, int32_t g0, int32_t ng,
                             int32_t* __restrict__ u_slot, int32_t* __restrict__ u_g) {
  const int gl = blockIdx.x;
  if (gl >= ng || gkind[g0 + gl] != want) return;
  const int c = gcl[g0 + gl];
  const int cs = cptr[c], M = cptr[c + 1] - cs;
  const int o = uoff[gl];
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    u_slot[o + l] = cs + l;
    u_g[o + l] = g0 + gl;
  }
}

__global__ void k_set_count(int32_t* p, int32_t v) { *p = v; }

__global__ void k_iota(int32_t* p, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) p[j] = (int32_t)j;
}


// ------------------------------------------------------------------ greedy rounds
struct GreedyArgs {
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* slen;     // profile length per slot
  const int32_t* gcl;
  const int64_t* gofs;     // per cluster
  const uint16_t* gram;    // count rows of stride round_up(M, 8)
  const int32_t* gu_slot;  // per-user launches: internal slot and greedy index
  const int32_t* gu_g;
  const int32_t* n_users_dev;
  const int32_t* gw_g;     // per-block launches: greedy index and user chunk
  const int32_t* gw_t;
  const int32_t* n_gwork;
  unsigned* counter;
  int32_t k, round, n_random, mcap;
  int32_t max_draws;       // bound on the round-0 draws per member
  uint32_t cluster_base;   // the run's number of cluster 0 (Philox counter word 0)
  uint2 key;               // Philox key = run seed
  const int32_t* ipos;     // slot -> internal position
  const int2* iinfo;       // internal slot -> (local index, profile length)
  const int32_t* wl_in;    // [S][k] internal positions, by internal slot
  int32_t* wl_out;
  const int32_t* chg_in;   // per slot: list changed in the previous round (NULL = no skipping)
  int32_t* chg_out;
  int32_t* fresh;          // per slot: evaluations of the last computed round
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

// Member of a cluster of size M other than l, from one Philox word.
__device__ __forceinline__ int draw_other(uint32_t r, int l, int M) {
  const int x = (int)(r % (uint32_t)(M - 1));
  return x + (x >= l ? 1 : 0);
}

// Round 0: k distinct random members per user (in draw order), then sorted.
// Draws are local indices (user-id order); lists hold internal positions.
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
    const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, p = slot - cs;
    const int2 me = a.iinfo[slot];
    const int l = me.x;
    const uint16_t* G = a.gram + a.gofs[c] + (int64_t)p * ((M + 7) & ~7);
    const int k = a.k, k0 = min(k, M - 1);
    int cnt = 0;
    // rejection sampling of distinct members; bounded so that no warp can
    // loop forever (the default bound is never reached for k0 <= M-1 with a
    // uniform generator)
    for (int j0 = 0; cnt < k0; j0 += 32) {
      if (j0 + 32 > a.max_draws) {   // draws come 32 at a time
        if (lane == 0) dev_fail(a.hdr, C2_ERR_TIMEOUT);
        break;
      }
      const uint4 r = philox10(
          make_uint4((uint32_t)c + a.cluster_base, (uint32_t)l, 0u, (uint32_t)(j0 + lane)), a.key);
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
    // the cnt <= k drawn members, one per lane, sorted best first
    __syncwarp();
    WarpList Lst;
    Lst.id = -1; Lst.c = 0; Lst.u = 0;
    if (lane < cnt) {
      const int v = drawn[lane];
      Lst.id = v;
      Lst.c = G[a.ipos[cs + v]];
      Lst.u = (uint32_t)me.y + (uint32_t)a.slen[cs + v] - Lst.c;
    }
    warp_sort32(Lst);
    if (lane < k) a.wl_out[(int64_t)slot * k + lane] = Lst.id >= 0 ? a.ipos[cs + Lst.id] : -1;
    if (lane == 0 && a.chg_out) a.chg_out[slot] = 1;
    __syncwarp();
    for (int q = lane; q < cnt; q += 32) {
      const int v = drawn[q];
      atomicAnd(&bm[v >> 5], ~(1u << (v & 31)));
    }
    __syncwarp();
    evals += (unsigned long long)cnt;
  }
  if (lane == 0 && evals) atomicAdd(&a.hdr->pairs, evals);
}

// (common, union) counts of a member of the warp's cluster, by internal
// position, from the staged row of counts and the packed (local index,
// length) words (shared memory).
struct SmemCU {
  const uint16_t* row;
  const uint32_t* info;
  uint32_t my;
  __device__ __forceinline__ uint2 operator()(int32_t p) const {
    const uint32_t c = row[p];
    return make_uint2(c, my + (info[p] & 0xffffu) - c);
  }
};

// One synchronous round.  A block takes a chunk of users of one cluster: the
// cluster's (local index, profile length) words are staged in shared memory
// once, and every warp stages its user's row of intersection counts before
// walking the candidates (own list, neighbours' lists, optional random
// draws), deduplicated with a per-warp bitmap of the cluster.  Candidates
// that beat the current k-th neighbour are staged and merged 32 at a time;
// `Keyed` (every union below 2^16) holds the list as exact 64-bit order keys.
// Users, lists and rows are in internal order; candidates are ranked by
// local index (user-id order).
//
// Without random draws, from round 2 on, the list of a neighbour v is known
// not to contribute when v was already in the user's list two rounds back and
// v's list did not change last round: then all of v's list was a candidate
// last round, and each such candidate is in the current list or ranks below
// all k of its entries (the current list is the top k of last round's
// candidates).  Those lists are only deduplicated, so that the count of
// evaluated pairs stays that of the method.
template <bool Keyed, int UPW>
__global__ void __launch_bounds__(kNT, 4) k_greedy_round(GreedyArgs a) {
  extern __shared__ __align__(16) uint32_t gsm[];
  __shared__ int32_t s_sid[Keyed ? 1 : 8][64];
  __shared__ uint2 s_scu[8][64];
  const int mcap = a.mcap;                               // multiple of 32
  // keyed: local index << 16 | length; otherwise the length alone
  uint32_t* s_info = gsm;                                // [mcap]
  uint16_t* s_rows = reinterpret_cast<uint16_t*>(gsm + mcap);   // [8][mcap]
  uint32_t* s_bm = gsm + mcap + 4 * mcap;                // [8][mcap/32]
  __shared__ int s_work;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint16_t* row = s_rows + warp * mcap;
  uint32_t* bm = s_bm + warp * (mcap >> 5);
  const int nwork = *a.n_gwork;
  const int k = a.k;
  const bool prune = a.chg_in != nullptr && a.round >= 2 && a.n_random == 0;
  // a work item of the list is a chunk of kGreedyChunk users; a round splits
  // it into nsub items of 8 * UPW users (UPW per warp)
  constexpr int nsub = kGreedyUsersPerWarp / UPW;
  const int nitems = nwork * nsub;
  unsigned long long evals = 0, visits = 0, computed = 0, evaluated = 0;
  for (;;) {
    if (threadIdx.x == 0) s_work = dev_failed(a.hdr) ? nitems : (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int wi = s_work;
    if (wi >= nitems) break;
    const int g = a.gw_g[wi / nsub];
    const int u0 = a.gw_t[wi / nsub] * kGreedyChunk + (wi % nsub) * 8 * UPW;   // first user
    const int c = a.gcl[g];
    const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, Mp = (M + 7) & ~7;
    const int2* info_g = a.iinfo + cs;
    for (int v = threadIdx.x; v < M; v += kNT) {
      const int2 x = info_g[v];
      s_info[v] = Keyed ? (((uint32_t)x.x << 16) | (uint32_t)x.y) : (uint32_t)x.y;
    }
    __syncthreads();
    const uint16_t* Gc = a.gram + a.gofs[c];
    const int32_t* wl_c = a.wl_in + (int64_t)cs * k + lane;
    // local index and length of the member at internal position x
    auto lid_of = [&](int x) -> int {
      if constexpr (Keyed) return (int)(s_info[x] >> 16);
      else return info_g[x].x;
    };
    auto len_of = [&](int x) -> uint32_t {
      if constexpr (Keyed) return s_info[x] & 0xffffu;
      else return s_info[x];
    };
    for (int uu = 0; uu < UPW; ++uu) {
      const int l = u0 + uu * 8 + warp;
      if (l >= M) break;
      const int slot = cs + l;
      const int e = lane < k ? a.wl_in[(int64_t)slot * k + lane] : -1;
      bool e_moved = false;
      if (a.chg_in) {
        // Unchanged list and unchanged neighbour lists: the candidate set,
        // hence the new list and its evaluation count, repeat the last round.
        e_moved = e >= 0 && a.chg_in[cs + e] != 0;
        const bool moved = a.chg_in[slot] != 0 || e_moved;
        if (!__any_sync(0xffffffffu, moved)) {
          if (lane < k) a.wl_out[(int64_t)slot * k + lane] = e;
          if (lane == 0) {
            a.chg_out[slot] = 0;
            evals += (unsigned)a.fresh[slot];
          }
          continue;
        }
      }
      // stage my row of counts (16-byte aligned rows) and clear my bitmap
      const uint4* g4 = reinterpret_cast<const uint4*>(Gc + (int64_t)l * Mp);
      uint4* r4 = reinterpret_cast<uint4*>(row);
      for (int i = lane; i < (Mp >> 3); i += 32) r4[i] = g4[i];
      for (int i = lane; i < ((M + 31) >> 5); i += 32) bm[i] = 0;
      __syncwarp();
      // neighbour lists to deduplicate only (see above); the list of two
      // rounds back is the row this warp is about to overwrite
      unsigned dedupe_only = 0u;
      if (prune) {
        const int p = lane < k ? a.wl_out[(int64_t)slot * k + lane] : -1;
        if (p >= 0) atomicOr(&bm[p >> 5], 1u << (p & 31));
        __syncwarp();
        const bool was = e >= 0 && ((bm[e >> 5] >> (e & 31)) & 1u) != 0u;
        dedupe_only = __ballot_sync(0xffffffffu, was && !e_moved);
        __syncwarp();
        if (p >= 0) bm[p >> 5] = 0u;     // only these bits are set
        __syncwarp();
      }
      const uint32_t my = len_of(l);
      const int lid_me = lid_of(l);
      const uint32_t c0 = e >= 0 ? row[e] : 0u;
      const uint32_t u0 = e >= 0 ? my + len_of(e) - c0 : 0u;
      const int lid0 = e >= 0 ? lid_of(e) : -1;
      if (e >= 0) atomicOr(&bm[e >> 5], 1u << (e & 31));
      if (lane == 0) atomicOr(&bm[l >> 5], 1u << (l & 31));
      const int nlist = __popc(__ballot_sync(0xffffffffu, e >= 0));
      __syncwarp();
      typename std::conditional<Keyed, KeyTopk<SmemCU>, WarpTopk>::type tk;
      if constexpr (Keyed) {
        tk.start(e >= 0 ? nbr_key(c0, u0, lid0, e) : 0ull, k, s_scu[warp],
                 SmemCU{row, s_info, my});
      } else {
        WarpList l0;
        l0.id = lid0; l0.c = c0; l0.u = u0;
        tk.start(l0, k, s_sid[warp], s_scu[warp]);
      }
      unsigned fresh = 0, looked = 0;
      if (lane == 0) {
        visits += (unsigned long long)nlist * (unsigned long long)k + (unsigned)a.n_random;
        computed += 1;
      }
      // one candidate per lane: dedupe, count lookup, filter, stage; an
      // absent candidate reads as the user itself, whose bit is set
      auto consider = [&](int v) {
        const int x = v >= 0 ? v : l;
        const uint32_t bit = 1u << (x & 31);
        const bool isnew = (atomicOr(&bm[x >> 5], bit) & bit) == 0u;
        const uint32_t cc = row[x];
        uint32_t uu2;
        int lx;
        if constexpr (Keyed) {
          const uint32_t inf = s_info[x];
          uu2 = my + (inf & 0xffffu) - cc;
          lx = (int)(inf >> 16);
        } else {
          uu2 = my + s_info[x] - cc;
          lx = info_g[x].x;
        }
        fresh += isnew ? 1u : 0u;
        looked += isnew ? 1u : 0u;
        const bool pass = isnew && tk.filter(lx, cc, uu2);
        if constexpr (Keyed) tk.stage(pass, x, lx, cc, uu2);
        else tk.stage(pass, lx, cc, uu2);
      };
      auto mark = [&](int v) {
        const int x = v >= 0 ? v : l;
        const uint32_t bit = 1u << (x & 31);
        fresh += (atomicOr(&bm[x >> 5], bit) & bit) == 0u ? 1u : 0u;
      };
      // neighbour lists in order, 8 loads in flight: neighbour j's entries sit
      // in q[j % 8], reloaded with neighbour j + 8's right after use (the
      // group of 8 is unrolled, so the registers never move)
      auto fetch = [&](int j) -> int {
        const int nb = __shfl_sync(0xffffffffu, e, j & 31);
        return (j < nlist && lane < k) ? wl_c[nb * k] : -1;
      };
      int q[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) q[r] = fetch(r);
#pragma unroll 1
      for (int j0 = 0; j0 < nlist; j0 += 8) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int j = j0 + r;
          if (j < nlist) {   // warp-uniform
            if ((dedupe_only >> j) & 1u) mark(q[r]);
            else consider(q[r]);
            q[r] = fetch(j + 8);
          }
        }
      }
      for (int d0 = 0; d0 < a.n_random; d0 += 32) {
        int v = -1;
        if (d0 + lane < a.n_random) {
          const uint4 r = philox10(make_uint4((uint32_t)c + a.cluster_base, (uint32_t)lid_me,
                                              (uint32_t)a.round,
                                              (uint32_t)(d0 + lane)), a.key);
          v = a.ipos[cs + draw_other(r.x, lid_me, M)];
        }
        consider(v);
      }
      tk.finish();
      int32_t nid;
      if constexpr (Keyed) {
        nid = tk.pos();
      } else {
        nid = tk.L.id >= 0 ? a.ipos[cs + tk.L.id] : -1;
      }
      if (lane < k) a.wl_out[(int64_t)slot * k + lane] = nid;
      if (a.chg_out) {
        const bool moved = __any_sync(0xffffffffu, lane < k && nid != e);
        unsigned f = fresh;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0) {
          a.chg_out[slot] = moved ? 1 : 0;
          a.fresh[slot] = (int32_t)f;
        }
      }
      evals += fresh;
      evaluated += looked;
      __syncwarp();
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(&a.hdr->pairs, evals);
  if (lane == 0 && visits) atomicAdd(&a.hdr->greedy_visits, visits);
  if (lane == 0 && computed) atomicAdd(&a.hdr->greedy_computed, computed);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
  if (lane == 0 && evaluated) atomicAdd(&a.hdr->greedy_evaluated, evaluated);
}

// Final rows: global ids, zero-similarity entries dropped (they sort last);
// the row of internal slot cs + p is written at its user's slot.
__global__ void __launch_bounds__(kNT) k_greedy_emit(GreedyArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_users_dev || dev_failed(a.hdr)) return;
  const int slot = a.gu_slot[w];
  const int c = a.gcl[a.gu_g[w]];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, p = slot - cs;
  const uint16_t* G = a.gram + a.gofs[c] + (int64_t)p * ((M + 7) & ~7);
  const int k = a.k;
  if (lane >= k) return;
  const int2 me = a.iinfo[slot];
  const int e = a.wl_in[(int64_t)slot * k + lane];
  const int64_t o = (int64_t)(cs + me.x) * k + lane;
  uint32_t cc = e >= 0 ? G[e] : 0u;
  if (e >= 0 && cc > 0) {
    const int2 x = a.iinfo[cs + e];
    a.out_id[o] = a.cusers[cs + x.x];
    a.out_in[o] = (int32_t)cc;
    a.out_un[o] = me.y + x.y - (int32_t)cc;
  } else {
    a.out_id[o] = -1;
    a.out_in[o] = 0;
    a.out_un[o] = 0;
  }
}

__global__ void k_gram_stats(const int64_t* __restrict__ goff, int32_t ng, DevHeader* hdr) {
  // count elements, without the length rows
  const unsigned long long e = (unsigned long long)goff[ng] - hdr->gram_len_elems;
  hdr->greedy_gram_elems = e;
  hdr->gram_pairs += e;
}

// ------------------------------------------------------------------ launch helpers
struct TableCfg {
  int W, NT;
  int MB;   // k_gram: minimum resident blocks per SM (register cap), 0 = none
  int P16;  // k_gram: walk the 16-bit copy of the profiles (item ids below 2^16)
};

int smem_optin() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return v;
}

int table_smem_bytes(TableCfg c, int m) {
  return 4 * (table_T_words(c.W, m) + 16 * c.W * c.NT + 2 * c.NT);
}

bool table_fits(TableCfg c, int m) {
  const int stat = 4 * (2 * 32 * c.W + 1) + 64;
  return table_smem_bytes(c, m) + stat <= smem_optin();
}

template <int W, int NT>
c2_status launch_table_t(const TableArgs& a, cudaStream_t st) {
  const int smem = table_smem_bytes(TableCfg{W, NT}, a.n_items);
  C2_CUDA_TRY(cudaFuncSetAttribute(k_table<W, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_table<W, NT>, NT, smem));
  if (per_sm < 1) return C2_ERR_UNSUPPORTED;
  C2_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
  C2_LAUNCH(k_table<W COMMA NT>, num_sms() * per_sm, NT, smem, st, a);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status launch_table(TableCfg c, const TableArgs& a, cudaStream_t st) {
  if (c.W == 1 && c.NT == 256) return launch_table_t<1, 256>(a, st);
  if (c.W == 1 && c.NT == 512) return launch_table_t<1, 512>(a, st);
  if (c.W == 1 && c.NT == 1024) return launch_table_t<1, 1024>(a, st);
  if (c.W == 2 && c.NT == 256) return launch_table_t<2, 256>(a, st);
  if (c.W == 2 && c.NT == 512) return launch_table_t<2, 512>(a, st);
  return C2_ERR_UNSUPPORTED;
}

// Table shapes in order of preference when nothing is forced; W = 0 means
// the sorted-merge kernel.
TableCfg pick_table(int strategy, int m) {
  static const TableCfg wide[] = {{2, 512}, {2, 256}};
  static const TableCfg narrow[] = {{1, 1024}, {1, 512}, {1, 256}};
  if (strategy == C2_STRATEGY_MERGE) return {0, 0};
  if (strategy != C2_STRATEGY_TABLE32) {
    for (const TableCfg& c : wide)
      if (table_fits(c, m)) return c;
  }
  for (const TableCfg& c : narrow)
    if (table_fits(c, m)) return c;
  return {0, 0};
}

int gram_smem_bytes(TableCfg c, int m) { return 4 * table_T_words(c.W, m); }

template <int W, int NT, int MB, bool P16>
c2_status launch_gram_t(const GramArgs& a, const int32_t* pptr16, const uint16_t* pitems16,
                        cudaStream_t st) {
  const int smem = gram_smem_bytes(TableCfg{W, NT, MB}, a.n_items);
  auto kern = k_gram<W, NT, MB, P16>;
  C2_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return C2_ERR_UNSUPPORTED;
  C2_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
  C2_LAUNCH(kern, num_sms() * per_sm, NT, smem, st, a, pptr16, pitems16);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status launch_gram_hash(const GramArgs& a, cudaStream_t st) {
  constexpr int NT = 256, MB = 3;
  const int smem = (int)gram_hash_smem_bytes();
  C2_CUDA_TRY(cudaFuncSetAttribute(k_gram_hash<NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_hash<NT, MB>, NT, smem));
  if (per_sm < 1) return C2_ERR_UNSUPPORTED;
  C2_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
  C2_LAUNCH(k_gram_hash<NT COMMA MB>, num_sms() * per_sm, NT, smem, st, a);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

// pptr16 / pitems16: the 16-bit profile copy (null when not built); the
// shapes with P16 walk it when it is there.
c2_status launch_gram(TableCfg c, const GramArgs& a, const int32_t* pptr16,
                      const uint16_t* pitems16, cudaStream_t st) {
  if (c.P16 && !pitems16) c.P16 = 0;   // no copy (workspace too small): the int32 rows
  if (c.P16) {
    if (c.W == 1 && c.NT == 512 && c.MB == 2) return launch_gram_t<1, 512, 2, true>(a, pptr16, pitems16, st);
    if (c.W == 1 && c.NT == 512 && c.MB == 0) return launch_gram_t<1, 512, 0, true>(a, pptr16, pitems16, st);
    if (c.W == 1 && c.NT == 256 && c.MB == 3) return launch_gram_t<1, 256, 3, true>(a, pptr16, pitems16, st);
    if (c.W == 1 && c.NT == 256 && c.MB == 4) return launch_gram_t<1, 256, 4, true>(a, pptr16, pitems16, st);
    if (c.W == 1 && c.NT == 256 && c.MB == 5) return launch_gram_t<1, 256, 5, true>(a, pptr16, pitems16, st);
    return C2_ERR_UNSUPPORTED;
  }
  if (c.W == 1 && c.NT == 128 && c.MB == 0) return launch_gram_t<1, 128, 0, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 128 && c.MB == 5) return launch_gram_t<1, 128, 5, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 256 && c.MB == 0) return launch_gram_t<1, 256, 0, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 256 && c.MB == 3) return launch_gram_t<1, 256, 3, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 256 && c.MB == 4) return launch_gram_t<1, 256, 4, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 256 && c.MB == 5) return launch_gram_t<1, 256, 5, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 512 && c.MB == 0) return launch_gram_t<1, 512, 0, false>(a, nullptr, nullptr, st);
  if (c.W == 1 && c.NT == 512 && c.MB == 2) return launch_gram_t<1, 512, 2, false>(a, nullptr, nullptr, st);
  if (c.W == 2 && c.NT == 128 && c.MB == 0) return launch_gram_t<2, 128, 0, false>(a, nullptr, nullptr, st);
  if (c.W == 2 && c.NT == 256 && c.MB == 0) return launch_gram_t<2, 256, 0, false>(a, nullptr, nullptr, st);
  if (c.W == 2 && c.NT == 512 && c.MB == 0) return launch_gram_t<2, 512, 0, false>(a, nullptr, nullptr, st);
  return C2_ERR_UNSUPPORTED;
}

// ---- autotuner: per size bucket, the table shape measured fastest; cached by
// problem sizes (a performance choice only: every shape gives the same counts)
struct TuneKey {
  int64_t n, m, t, b, N, k, thr;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, m, t, b, N, k, thr) < std::tie(o.n, o.m, o.t, o.b, o.N, o.k, o.thr);
  }
};
struct TuneEntry {
  bool unified;            // one launch over all buckets with cfg[0]
  bool shapes_done;        // table shapes measured
  bool tc_done;            // the strategy of the tensor-core candidates measured
  TableCfg cfg[kBuckets];
  float ms[kBuckets];
  // per (size bucket, density bucket): -1 not measured, 0 table, 1 tensor cores,
  // with the two times measured
  int8_t route[kBuckets * kDensityBuckets];
  float table_ms[kBuckets * kDensityBuckets];
  float tc_ms[kBuckets * kDensityBuckets];
  TuneEntry() : unified(true), shapes_done(false), tc_done(false) {
    for (int i = 0; i < kBuckets * kDensityBuckets; ++i) {
      route[i] = -1;
      table_ms[i] = tc_ms[i] = 0.f;
    }
    for (int q = 0; q < kBuckets; ++q) ms[q] = 0.f;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;

const TableCfg kGramShapes[] = {{2, 256, 0},    {2, 512, 0},    {2, 128, 0},    {1, 512, 0},
                                 {1, 256, 0},    {1, 128, 0},    {1, 256, 3},    {1, 256, 4},
                                 {1, 256, 5},    {1, 512, 2},    {1, 128, 5},    {1, 512, 2, 1},
                                 {1, 256, 3, 1}, {1, 256, 4, 1}, {1, 256, 5, 1}, {1, 512, 0, 1}};

bool gram_fits(TableCfg c, int m) { return gram_smem_bytes(c, m) + 1024 <= smem_optin(); }

TableCfg pick_gram(int strategy, int m) {
  static const TableCfg wide[] = {{2, 256}, {2, 512}};
  static const TableCfg narrow[] = {{1, 512}, {1, 256}};
  if (strategy == C2_STRATEGY_MERGE) return {0, 0};
  if (strategy != C2_STRATEGY_TABLE32) {
    for (const TableCfg& c : wide)
      if (gram_fits(c, m)) return c;
  }
  for (const TableCfg& c : narrow)
    if (gram_fits(c, m)) return c;
  return {0, 0};
}

// A second stream per device for work that is independent of the main
// stream's next kernels (brute-force clusters while the count matrices and the
// greedy rounds run): latency-bound kernels fill the SMs the main stream's
// persistent kernels leave idle at their tails.  Created once, never destroyed.
cudaStream_t side_stream() {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t sst = nullptr;
  if (cudaStreamCreateWithFlags(&sst, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  streams[dev] = sst;
  return sst;
}

// Work on `to` after everything issued so far on `from`.
cudaError_t stream_after(cudaStream_t to, cudaStream_t from) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev, from);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
  cudaEventDestroy(ev);   // released once the wait is satisfied
  return e;
}

// Joins the side stream back into the main stream when it goes out of scope
// (every return path of the local-KNN step).
struct SideJoin {
  cudaStream_t st, side;
  bool used = false;
  c2_status fork() {
    used = true;
    return stream_after(side, st) == cudaSuccess ? C2_OK : C2_ERR_CUDA;
  }
  c2_status join() {
    if (!used) return C2_OK;
    used = false;
    return stream_after(st, side) == cudaSuccess ? C2_OK : C2_ERR_CUDA;
  }
  ~SideJoin() { join(); }
};

c2_status build_padded_csr(const int32_t* ptr, const int32_t* items, const Sizes& s, KnnWs& w,
                           cudaStream_t st) {
  if (s.n == 0) return C2_OK;
  C2_LAUNCH(k_pad_len, div_up(s.n, 256), 256, 0, st, ptr, s.n, w.pptr);
  C2_CUDA_TRY(scan_exclusive(w.pptr, w.pptr, s.n, w.scan_tmp, st));
  C2_LAUNCH(k_pad_copy, div_up((int64_t)s.n * 32, 256), 256, 0, st, ptr, items, w.pptr, s.n, s.m,
            w.pitems_cap, w.pitems, w.hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
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
  const TableCfg tc = pick_gram(opt.strategy, s.m);
  // brute-force clusters smaller than small_cut (at most 33) go to the
  // warp-per-cluster kernel; larger ones and every greedy cluster get a count
  // matrix
  const int small_cut = kSmallCut;

  Prof p_prep(st, "knn_prep");
  C2_LAUNCH(k_set_count, 1, 1, 0, st, &w.hdr->knn_max_len, 0);
  C2_LAUNCH(k_slot_info, div_up(S, T), T, 0, st, cptr, n_clusters, cusers, ptr, S, w.slot2c,
            w.slen, w.hdr);
  const int64_t cap = s.gram_budget / (int64_t)sizeof(uint16_t);
  C2_LAUNCH(k_set_count, 1, 1, 0, st, &w.hdr->direct_users, 0);
  C2_LAUNCH(k_prep, div_up(S, T), T, 0, st, cptr, n_clusters, cusers, ptr, S, thr, small_cut,
            kSmallItems, k, cap, w.gflag, w.gkind_c, w.small_cnt, lid, lin, lun, w.hdr);
  C2_CUDA_TRY(cudaGetLastError());
  // the hashed count-matrix kernel is the candidate when no item table fits
  const bool hash_ok = !tc.W && opt.strategy != C2_STRATEGY_MERGE &&
                       (int)gram_hash_smem_bytes() + 1024 <= smem_optin();
  // the tensor-core count matrices (allowed by the strategy and the item
  // universe; their remapped lists need room in the workspace tail, checked
  // once nnz is read)
  const bool tc_allowed = s.tc && w.gt_work_cap > 0 && s.m <= kGramTcMaxItems &&
                          (opt.strategy == C2_STRATEGY_AUTO || opt.strategy == C2_STRATEGY_MMA);
  if (tc.W || hash_ok || tc_allowed) {
    c2_status rc = build_padded_csr(ptr, items, s, w, st);
    if (rc) return rc;
  }
  p_prep.end();

  // small brute-force clusters on the side stream, beside the count matrices
  cudaStream_t side = side_stream();
  if (!side) return C2_ERR_CUDA;
  SideJoin sj{st, side};
  {
    c2_status rc = sj.fork();
    if (rc) return rc;
    Prof p_small(side, "brute_merge");
    C2_CUDA_TRY(scan_exclusive(w.small_cnt, w.small_off, S, w.scan_tmp2, side));
    C2_LAUNCH(k_fill_small, div_up(S, T), T, 0, side, w.small_cnt, w.small_off, S, w.small_slot);
    SmallArgs sa{};
    sa.ptr = ptr; sa.items = items; sa.cptr = cptr; sa.cusers = cusers; sa.list = w.small_slot;
    sa.n_list = w.small_off + S; sa.k = k; sa.out_id = lid; sa.out_in = lin; sa.out_un = lun;
    sa.hdr = w.hdr;
    C2_LAUNCH(k_small_knn, (int)std::min<int64_t>(div_up(S, kSmallWarps), (int64_t)num_sms() * 5),
              32 * kSmallWarps, 0, side, sa);
    C2_CUDA_TRY(cudaGetLastError());
  }

  // ---- clusters with a count matrix
  Prof p_gsetup(st, "gram_setup");
  C2_CUDA_TRY(scan_exclusive(w.gflag, w.gidx, S, w.scan_tmp, st));
  C2_LAUNCH(k_greedy_list, div_up(S, T), T, 0, st, w.gflag, w.gidx, w.gkind_c, cptr, S, w.gcl,
            w.gsq, w.gsz, w.gkind, w.hdr);
  int32_t ng = 0, max_len = 0, nnz32 = 0, n_direct = 0;
  C2_CUDA_TRY(cudaMemcpyAsync(&ng, &w.hdr->n_work, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(&n_direct, &w.hdr->direct_users, sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(&max_len, &w.hdr->knn_max_len, sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(&nnz32, ptr + s.n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaStreamSynchronize(st));
  // greedy clusters without a count matrix: counts from the profiles, one
  // warp per member (the working lists are free again before the batches)
  p_gsetup.end();
  if (n_direct > 0) {
    Prof p_direct(st, "greedy_direct");
    const uint2 dkey = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    c2_status rc = run_big_greedy(
        ptr, items, s.m, cptr, cusers, w.slot2c, w.gkind_c, S, n_direct, k, rounds,
        opt.greedy_random, opt.greedy_max_draws > 0 ? opt.greedy_max_draws : (1 << 24),
        (uint32_t)opt.cluster_base, dkey, w.bg_flag, w.bg_off, w.bg_slot, w.scan_tmp, w.wl0,
        w.wl1, lid, lin, lun, w.hdr, st);
    if (rc) return rc;
  }
  if (ng == 0) return C2_OK;
  Prof p_gsetup2(st, "gram_setup");
  const TuneKey tkey{s.n, s.m, s.t, s.b, s.N, k, thr};
  TuneEntry tune;
  if (opt.strategy == C2_STRATEGY_AUTO) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tkey);
    if (it != g_tune.end()) tune = it->second;
  }
  // once measured for these sizes with no bucket faster on the tensor cores,
  // the autotuned build skips the candidates' density count
  bool tc_wanted = opt.strategy == C2_STRATEGY_MMA || !tune.tc_done;
  for (int i = 0; i < kBuckets * kDensityBuckets; ++i) tc_wanted = tc_wanted || tune.route[i] == 1;
  bool tc_possible = false;
  // bits mode: the operand rows are the caller's packed bit rows (whole rows,
  // no remap, no remapped-list area)
  const bool tc_bits = opt.d_sim_bits != nullptr && s.m % 128 == 0;
  if (tc_allowed && tc_wanted && tc_bits) {
    tc_possible = true;
  } else if (tc_allowed && tc_wanted && nnz32 > 0) {
    const size_t off = rl_offset(nnz32, s.n);
    const int64_t pn = rl_stride(nnz32, s.n);
    if ((int64_t)(off + (size_t)s.t * pn * 2) <= w.tail_bytes) {
      w.rl = reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(w.pitems) + off);
      w.rl_pn = pn;
      tc_possible = true;
    }
  }
  // tensor-core candidates: for every cluster of kTcMinM members or more, the
  // items held by two members or more (the width of its 0/1 operand) and the
  // members' total profile length (its density)
  if (tc_possible) {
    c2_status rc = gram_tc_count(nullptr, ng, kTcMinM, w.gsz, w.gcl, cptr, cusers, ptr, items,
                                 s.m, tc_bits, w.gk2, w.gsum, w.hdr, st);
    if (rc) return rc;
  }
  C2_CUDA_TRY(scan_exclusive64(w.gsq, w.goff, ng, w.scan_tmp64, st));
  C2_LAUNCH(k_gram_stats, 1, 1, 0, st, w.goff, ng, w.hdr);
  std::vector<int64_t> goff(ng + 1), gsum;
  std::vector<int32_t> gsz(ng), gkind(ng), gk2, gclh;
  C2_CUDA_TRY(cudaMemcpyAsync(goff.data(), w.goff, (ng + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(gsz.data(), w.gsz, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(gkind.data(), w.gkind, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (tc_possible) {
    gk2.resize(ng);
    gsum.resize(ng);
    gclh.resize(ng);
    C2_CUDA_TRY(cudaMemcpyAsync(gk2.data(), w.gk2, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    C2_CUDA_TRY(cudaMemcpyAsync(gsum.data(), w.gsum, ng * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    C2_CUDA_TRY(cudaMemcpyAsync(gclh.data(), w.gcl, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  }
  C2_CUDA_TRY(cudaStreamSynchronize(st));
  // exact 64-bit order keys need unions below 2^16 and clusters below 2^14
  bool keyed = max_len <= 32767;
  // hashed count matrices when every profile fits one pass of the hash table
  const bool use_hash = hash_ok && max_len <= kHashCap;
  for (int g = 0; g < ng; ++g) {
    if (goff[g + 1] - goff[g] > cap) return C2_ERR_UNSUPPORTED;   // brute force only
    if (gsz[g] > 16383) keyed = false;
  }
  C2_LAUNCH(k_iota, div_up(ng, T), T, 0, st, w.gseq, (int64_t)ng);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  // tensor-core eligibility and strategy bucket of each count-matrix cluster
  auto tc_eligible = [&](int g) {
    return tc_possible && gsz[g] >= kTcMinM && gk2[g] >= 1 && gk2[g] <= 65536;
  };
  auto tc_bucket = [&](int g) {
    return size_bucket(gsz[g]) * kDensityBuckets + density_bucket(gsum[g], gsz[g], gk2[g]);
  };
  p_gsetup2.end();

  GramArgs ga0{};
  // the table kernel walks a 16-bit copy of the profiles when item ids fit
  // 16 bits (half the load instructions of the int32 rows)
  w.pitems16 = nullptr;
  // needed by the autotuner's trials, or when a tuned shape walks it
  bool want16 = opt.strategy == C2_STRATEGY_AUTO && !tune.shapes_done;
  for (int q = 0; q < kBuckets; ++q)
    want16 = want16 || (opt.strategy == C2_STRATEGY_AUTO && tune.shapes_done && tune.cfg[q].P16);
  if (want16 && tc.W > 0 && s.m <= 65535 && nnz32 > 0 &&
      (int64_t)(p16_offset(nnz32, s.n) + p16_bytes(nnz32, s.n)) <= w.tail_bytes) {
    w.pitems16 = reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(w.pitems) +
                                             p16_offset(nnz32, s.n));
    C2_LAUNCH(k_pad_len8, div_up(s.n, T), T, 0, st, ptr, s.n, w.pptr16);
    C2_CUDA_TRY(scan_exclusive(w.pptr16, w.pptr16, s.n, w.scan_tmp, st));
    C2_LAUNCH(k_pad_copy16, div_up((int64_t)s.n * 32, T), T, 0, st, ptr, items, w.pptr16, s.n,
              s.m, (int64_t)(p16_bytes(nnz32, s.n) / 2), w.pitems16, w.hdr);
  }
  ga0.ptr = ptr; ga0.items = items; ga0.pptr = w.pptr; ga0.pitems = w.pitems;
  ga0.n_items = s.m; ga0.work_c = w.work_c; ga0.work_t = w.work_t;
  ga0.cptr = cptr; ga0.cusers = cusers; ga0.iinfo = w.iinfo; ga0.islot = w.islot;
  ga0.gofs = w.gofs; ga0.gram = w.gram;
  ga0.hdr = w.hdr; ga0.counter = &w.hdr->work_counter[1];

  // host -> device copy of small per-batch tables; the host buffer is reused
  // after it, and the stream's earlier kernels have read the old contents
  auto upload = [&](void* dst, const void* src, size_t bytes) -> c2_status {
    if (!bytes) return C2_OK;
    C2_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    C2_CUDA_TRY(cudaStreamSynchronize(st));
    return C2_OK;
  };
  cudaEvent_t te0 = nullptr, te1 = nullptr;
  // autotuner trials: the faster of two runs of fn (the first also warms the
  // caches), so that one slow run does not decide a shape or a route
  auto timed = [&](auto&& fn, float* ms) -> c2_status {
    if (!te0) {
      C2_CUDA_TRY(cudaEventCreate(&te0));
      C2_CUDA_TRY(cudaEventCreate(&te1));
    }
    float best = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      C2_CUDA_TRY(cudaEventRecord(te0, st));
      c2_status rc = fn();
      if (rc) return rc;
      C2_CUDA_TRY(cudaEventRecord(te1, st));
      C2_CUDA_TRY(cudaEventSynchronize(te1));
      float t = 0.f;
      C2_CUDA_TRY(cudaEventElapsedTime(&t, te0, te1));
      best = rep == 0 ? t : std::min(best, t);
    }
    *ms = best;
    return C2_OK;
  };
  struct EventGuard {
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~EventGuard() {
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } evg{&te0, &te1};

  // count matrices of the clusters `gs` on the tensor cores: remapped lists,
  // then the tiles, largest clusters first
  std::vector<int4> work_h;
  auto run_tc = [&](const std::vector<int32_t>& gs, bool count_stats) -> c2_status {
    if (gs.empty()) return C2_OK;
    const int BM = gram_tc_tile_rows(), BN = gram_tc_tile_cols(), BK = gram_tc_stage_cols();
    auto tiles_of = [&](int g) {
      const int TR = div_up(gsz[g], BM), TC = div_up(gsz[g], BN);
      int64_t nt = 0;
      for (int i = 0; i < TR; ++i) nt += TC - i / 2;
      return nt;
    };
    std::vector<int32_t> ord(gs);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      return tiles_of(a) * div_up(gk2[a], BK) > tiles_of(b) * div_up(gk2[b], BK);
    });
    work_h.clear();
    unsigned long long macs = 0;
    for (int g : ord) {
      const int c = gclh[g], TR = div_up(gsz[g], BM), TC = div_up(gsz[g], BN);
      const int nk = div_up(gk2[g], BK);
      for (int i = 0; i < TR; ++i)
        for (int j = i / 2; j < TC; ++j) work_h.push_back(make_int4(c, i, j, nk));
      macs += (unsigned long long)tiles_of(g) * nk * BM * BN * BK;
    }
    if ((int64_t)work_h.size() > w.gt_work_cap) return C2_ERR_WORKSPACE;
    c2_status rc = upload(w.gt_list, ord.data(), ord.size() * sizeof(int32_t));
    if (rc) return rc;
    rc = upload(w.gt_work, work_h.data(), work_h.size() * sizeof(int4));
    if (rc) return rc;
    if (!tc_bits) {
      Prof p_rm(st, "gram_tc_remap");
      rc = gram_tc_remap(w.gt_list, (int)ord.size(), w.gcl, cptr, cusers, ptr, items, s.m, w.pptr,
                         w.rl_pn, s.n, w.rl, w.rl_len, w.hdr, st);
      if (rc) return rc;
    }
    {
      Prof p_tc(st, "gram_tc");
      rc = gram_tc_run(w.gt_work, (int)work_h.size(), cptr, cusers, w.iinfo, w.pptr,
                       tc_bits ? nullptr : w.rl, w.rl_pn, s.n, w.rl_len, w.gofs, w.gram,
                       tc_bits ? opt.d_sim_bits : nullptr, s.m / 32, w.hdr, st);
      if (rc) return rc;
    }
    if (count_stats)
      C2_LAUNCH(k_tc_stats, 1, 1, 0, st, w.hdr, macs, (int32_t)ord.size(), (int32_t)work_h.size());
    return C2_OK;
  };

  int g0 = 0;
  while (g0 < ng) {
    int g1 = g0;
    int64_t n_greedy_users = 0, n_brute_users = 0;
    int mmax = 0;
    while (g1 < ng && goff[g1 + 1] - goff[g0] <= cap) {
      if (gkind[g1]) {
        mmax = std::max(mmax, gsz[g1]);
        n_greedy_users += gsz[g1];
      } else {
        n_brute_users += gsz[g1];
      }
      ++g1;
    }
    const int nb = g1 - g0;
    {
      Prof p_gram(st, "gram");
      C2_LAUNCH(k_batch_setup, div_up(nb, T), T, 0, st, w.gcl, w.goff, w.gsz, w.gkind, g0, g1,
                w.gofs, w.bu_cnt, w.bb_cnt, w.bw_cnt);
      // internal order (members by decreasing profile length) of every
      // count-matrix cluster of the batch
      C2_LAUNCH(k_order, nb, 256, 0, st, w.gcl, g0, cptr, w.slen, w.ipos, w.iinfo, w.gofs, w.gram,
                cusers, w.pptr, w.pitems16 ? w.pptr16 : nullptr, w.islot);
      // strategy of each cluster of the batch: 0 table, 1 tensor cores
      std::vector<int32_t> route(nb, 0);
      if (tc_possible && (tc.W || use_hash) && opt.strategy == C2_STRATEGY_AUTO) {
        // first call for these sizes: every (size, density) bucket with
        // tensor-core candidates is timed both ways on its clusters
        std::vector<std::vector<int32_t>> members(kBuckets * kDensityBuckets);
        for (int g = g0; g < g1; ++g)
          if (tc_eligible(g) && tune.route[tc_bucket(g)] < 0) members[tc_bucket(g)].push_back(g);
        for (int bk = 0; bk < kBuckets * kDensityBuckets; ++bk) {
          if (members[bk].empty()) continue;
          std::vector<int32_t> only(nb, 2);   // 2: in neither launch
          for (int g : members[bk]) only[g - g0] = 0;
          c2_status rc = upload(w.groute + g0, only.data(), nb * sizeof(int32_t));
          if (rc) return rc;
          float t_tab = 0.f, t_tc = 0.f;
          rc = timed([&]() -> c2_status {
            C2_LAUNCH(k_bucket_tiles, div_up(nb, T), T, 0, st, w.gsz, g0, nb, -1,
                      tc.W ? 32 * tc.W : 32, w.groute, w.bt_cnt);
            C2_CUDA_TRY(scan_exclusive(w.bt_cnt, w.bt_off, nb, w.scan_tmp, st));
            C2_LAUNCH(k_fill_work, div_up(nb, T), T, 0, st, w.bt_cnt, w.bt_off, w.gcl + g0, nb,
                      w.work_c, w.work_t, &w.hdr->n_work);
            GramArgs ga = ga0;
            ga.work_begin = w.bt_off;
            ga.work_end = w.bt_off + nb;
            return tc.W ? launch_gram(tc, ga, w.pptr16, w.pitems16, st) : launch_gram_hash(ga, st);
          }, &t_tab);
          if (rc) return rc;
          rc = timed([&]() { return run_tc(members[bk], false); }, &t_tc);
          if (rc) return rc;
          // the tensor cores must win clearly: routing any bucket to them adds the
          // density count of every candidate cluster to each later build
          tune.route[bk] = t_tc < 0.8f * t_tab ? 1 : 0;
          tune.table_ms[bk] = t_tab;
          tune.tc_ms[bk] = t_tc;
        }
        tune.tc_done = true;
      }
      for (int g = g0; g < g1; ++g) {
        if (!tc_eligible(g)) continue;
        if (opt.strategy == C2_STRATEGY_MMA) route[g - g0] = 1;
        else if (opt.strategy == C2_STRATEGY_AUTO && tune.route[tc_bucket(g)] == 1) route[g - g0] = 1;
      }
      std::vector<int32_t> tc_list;
      bool any_table = false;
      for (int g = g0; g < g1; ++g) {
        if (route[g - g0]) tc_list.push_back(g);
        else any_table = true;
      }
      if (tc_possible) {
        c2_status rc = upload(w.groute + g0, route.data(), nb * sizeof(int32_t));
        if (rc) return rc;
      }
      const int32_t* groute = tc_possible ? w.groute : nullptr;
      if (!any_table) {
        // every count matrix of the batch comes from the tensor cores
      } else if (tc.W) {
        bool present[kBuckets] = {false, false, false, false};
        for (int g = g0; g < g1; ++g)
          if (!route[g - g0]) present[size_bucket(gsz[g])] = true;
        // one launch per size bucket, over that bucket's query tiles
        auto run_bucket = [&](int bkt, TableCfg shape) -> c2_status {
          C2_LAUNCH(k_bucket_tiles, div_up(nb, T), T, 0, st, w.gsz, g0, nb, bkt, 32 * shape.W,
                    groute, w.bt_cnt);
          C2_CUDA_TRY(scan_exclusive(w.bt_cnt, w.bt_off, nb, w.scan_tmp, st));
          C2_LAUNCH(k_fill_work, div_up(nb, T), T, 0, st, w.bt_cnt, w.bt_off, w.gcl + g0, nb,
                    w.work_c, w.work_t, &w.hdr->n_work);
          GramArgs ga = ga0;
          ga.work_begin = w.bt_off;
          ga.work_end = w.bt_off + nb;
          return launch_gram(shape, ga, w.pptr16, w.pitems16, st);
        };
        if (opt.strategy == C2_STRATEGY_AUTO && !tune.shapes_done) {
          // first call for these sizes: time every shape that fits, on each
          // bucket alone and as one launch over all buckets; keep the faster plan
          tune.unified = true;
          for (int q = 0; q < kBuckets; ++q) { tune.cfg[q] = tc; tune.ms[q] = 0.f; }
          float split_total = 0.f;
          TableCfg best_cfg[kBuckets] = {tc, tc, tc, tc};
          float best_ms[kBuckets] = {0.f, 0.f, 0.f, 0.f};
          for (int q = 0; q < kBuckets; ++q) {
            if (!present[q]) continue;
            float best = 1e30f;
            for (const TableCfg& shape : kGramShapes) {
              if (!gram_fits(shape, s.m) || (shape.P16 && !w.pitems16)) continue;
              float ms = 0.f;
              c2_status rc = timed([&]() { return run_bucket(q, shape); }, &ms);
              if (rc) return rc;
              if (ms < best) { best = ms; best_cfg[q] = shape; best_ms[q] = ms; }
            }
            split_total += best;
          }
          float uni_best = 1e30f;
          TableCfg uni_cfg = tc;
          for (const TableCfg& shape : kGramShapes) {
            if (!gram_fits(shape, s.m) || (shape.P16 && !w.pitems16)) continue;
            float ms = 0.f;
            c2_status rc = timed([&]() { return run_bucket(-1, shape); }, &ms);
            if (rc) return rc;
            if (ms < uni_best) { uni_best = ms; uni_cfg = shape; }
          }
          if (uni_best <= split_total) {
            tune.unified = true;
            for (int q = 0; q < kBuckets; ++q) { tune.cfg[q] = uni_cfg; tune.ms[q] = q ? 0.f : uni_best; }
          } else {
            tune.unified = false;
            for (int q = 0; q < kBuckets; ++q) { tune.cfg[q] = best_cfg[q]; tune.ms[q] = best_ms[q]; }
          }
          tune.shapes_done = true;
          // every timed launch wrote the same counts: the matrices are complete
        } else {
          const bool auto_shapes = opt.strategy == C2_STRATEGY_AUTO && tune.shapes_done;
          if (!auto_shapes || tune.unified) {
            c2_status rc = run_bucket(-1, auto_shapes ? tune.cfg[0] : tc);
            if (rc) return rc;
          } else {
            for (int q = 0; q < kBuckets; ++q) {
              if (!present[q]) continue;
              c2_status rc = run_bucket(q, tune.cfg[q]);
              if (rc) return rc;
            }
          }
        }
      } else if (use_hash) {
        // no item table fits shared memory: the tiles' items in a shared hash
        // table, one launch over all count-matrix clusters of the batch
        C2_LAUNCH(k_bucket_tiles, div_up(nb, T), T, 0, st, w.gsz, g0, nb, -1, 32, groute, w.bt_cnt);
        C2_CUDA_TRY(scan_exclusive(w.bt_cnt, w.bt_off, nb, w.scan_tmp, st));
        C2_LAUNCH(k_fill_work, div_up(nb, T), T, 0, st, w.bt_cnt, w.bt_off, w.gcl + g0, nb,
                  w.work_c, w.work_t, &w.hdr->n_work);
        GramArgs ga = ga0;
        ga.work_begin = w.bt_off;
        ga.work_end = w.bt_off + nb;
        c2_status rc = launch_gram_hash(ga, st);
        if (rc) return rc;
      } else {
        // no item table fits shared memory and a profile is too long for the
        // hash table: rows by merges, greedy clusters' members then
        // brute-force clusters' members
        MergeGramArgs ma{};
        ma.ptr = ptr; ma.items = items; ma.cptr = cptr; ma.cusers = cusers; ma.gcl = w.gcl;
        ma.gofs = w.gofs; ma.gram = w.gram; ma.ipos = w.ipos; ma.iinfo = w.iinfo; ma.hdr = w.hdr;
        if (n_greedy_users) {
          C2_CUDA_TRY(scan_exclusive(w.bu_cnt, w.bu_off, nb, w.scan_tmp, st));
          C2_LAUNCH(k_fill_users, nb, 256, 0, st, w.gcl, cptr, w.gkind, 1, w.bu_off, g0, nb,
                    w.gu_slot, w.gu_g);
          ma.u_slot = w.gu_slot; ma.u_g = w.gu_g; ma.n_users_dev = w.bu_off + nb;
          C2_LAUNCH(k_merge_gram, div_up(n_greedy_users * 32, 256), 256, 0, st, ma);
        }
        if (n_brute_users) {
          C2_CUDA_TRY(scan_exclusive(w.bb_cnt, w.bb_off, nb, w.scan_tmp, st));
          C2_LAUNCH(k_fill_users, nb, 256, 0, st, w.gcl, cptr, w.gkind, 0, w.bb_off, g0, nb,
                    w.ub_slot, w.ub_g);
          ma.u_slot = w.ub_slot; ma.u_g = w.ub_g; ma.n_users_dev = w.bb_off + nb;
          C2_LAUNCH(k_merge_gram, div_up(n_brute_users * 32, 256), 256, 0, st, ma);
        }
      }
      p_gram.end();
      // the tensor-core clusters of the batch
      c2_status rc = run_tc(tc_list, true);
      if (rc) return rc;
      if (opt.strategy == C2_STRATEGY_AUTO) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tkey] = tune;
      }
    }
    // brute-force rows on the side stream (they and the greedy phase only read
    // this batch's count matrices): beside the greedy start when the round
    // kernel fills the SMs, beside the rounds when it leaves room for them
    // (large greedy clusters: at most two round blocks per SM)
    auto launch_brute_rows = [&]() -> c2_status {
      c2_status rc = sj.fork();
      if (rc) return rc;
      Prof p_bt(side, "brute_rows");
      C2_CUDA_TRY(scan_exclusive(w.bb_cnt, w.bb_off, nb, w.scan_tmp2, side));
      C2_LAUNCH(k_fill_users, nb, 256, 0, side, w.gcl, cptr, w.gkind, 0, w.bb_off, g0, nb,
                w.ub_slot, w.ub_g);
      RowTopkArgs ra{};
      ra.cptr = cptr; ra.cusers = cusers; ra.slen = w.slen; ra.gcl = w.gcl; ra.gofs = w.gofs;
      ra.gram = w.gram; ra.u_slot = w.ub_slot; ra.u_g = w.ub_g; ra.n_users_dev = w.bb_off + nb;
      ra.ipos = w.ipos; ra.iinfo = w.iinfo;
      ra.k = k; ra.out_id = lid; ra.out_in = lin; ra.out_un = lun; ra.hdr = w.hdr;
      if (keyed) C2_LAUNCH(k_gram_select, div_up(n_brute_users * 32, kNT), kNT, 0, side, ra);
      else C2_LAUNCH(k_gram_topk<false>, div_up(n_brute_users * 32, kNT), kNT, 0, side, ra);
      C2_CUDA_TRY(cudaGetLastError());
      return C2_OK;
    };
    bool brute_beside_rounds = false;
    if (n_brute_users && n_greedy_users) {
      const int smem_r = 21 * ((mmax + 31) & ~31);
      auto kr = keyed ? k_greedy_round<true, kGreedyUsersPerWarp>
                      : k_greedy_round<false, kGreedyUsersPerWarp>;
      C2_CUDA_TRY(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_r));
      int ps = 0;
      C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kr, kNT, smem_r));
      brute_beside_rounds = ps <= 2;
    }
    if (n_brute_users && !brute_beside_rounds) {
      c2_status rc = launch_brute_rows();
      if (rc) return rc;
    }
    if (n_greedy_users) {
      GreedyArgs ga{};
      ga.cptr = cptr; ga.cusers = cusers; ga.slen = w.slen; ga.gcl = w.gcl; ga.gofs = w.gofs;
      ga.gram = w.gram; ga.gu_slot = w.gu_slot; ga.gu_g = w.gu_g; ga.n_users_dev = w.bu_off + nb;
      ga.gw_g = w.gw_g; ga.gw_t = w.gw_t; ga.n_gwork = &w.hdr->n_gwork;
      ga.counter = &w.hdr->work_counter[2];
      ga.ipos = w.ipos; ga.iinfo = w.iinfo;
      ga.k = k; ga.n_random = opt.greedy_random; ga.key = key;
      ga.max_draws = opt.greedy_max_draws > 0 ? opt.greedy_max_draws : (1 << 24);
      ga.cluster_base = (uint32_t)opt.cluster_base;
      ga.out_id = lid; ga.out_in = lin; ga.out_un = lun; ga.hdr = w.hdr;
      ga.mcap = (mmax + 31) & ~31;
      {
        Prof p_init(st, "greedy_init");
        C2_CUDA_TRY(scan_exclusive(w.bu_cnt, w.bu_off, nb, w.scan_tmp, st));
        C2_CUDA_TRY(scan_exclusive(w.bw_cnt, w.bw_off, nb, w.scan_tmp, st));
        C2_LAUNCH(k_fill_users, nb, 256, 0, st, w.gcl, cptr, w.gkind, 1, w.bu_off, g0, nb,
                  w.gu_slot, w.gu_g);
        C2_LAUNCH(k_fill_work, div_up(nb, T), T, 0, st, w.bw_cnt, w.bw_off, w.gseq + g0, nb,
                  w.gw_g, w.gw_t, &w.hdr->n_gwork);
        const int grid = (int)std::min<int64_t>(div_up(n_greedy_users, 8), (int64_t)num_sms() * 8);
        ga.round = 0;
        ga.wl_in = nullptr;
        ga.wl_out = w.wl0;
        ga.chg_out = opt.greedy_random == 0 ? w.chg0 : nullptr;
        C2_LAUNCH(k_greedy_init, grid, kNT, 0, st, ga);
      }
      if (brute_beside_rounds) {
        c2_status rc = launch_brute_rows();
        if (rc) return rc;
      }
      int32_t* cur = w.wl0;
      int32_t* nxt = w.wl1;
      int32_t* chg_cur = w.chg0;
      int32_t* chg_nxt = w.chg1;
      const bool skipping = opt.greedy_random == 0;
      ga.fresh = w.gfresh;
      {
        Prof p_rounds(st, "greedy_rounds");
        const int smem = 21 * ga.mcap;
        // the first rounds compute (nearly) every user: work items of one user
        // per warp even out the round's tail; later rounds settle most users
        // by the skip test, where larger items cost less to schedule
        auto kbig = keyed ? k_greedy_round<true, kGreedyUsersPerWarp>
                          : k_greedy_round<false, kGreedyUsersPerWarp>;
        auto ksmall = keyed ? k_greedy_round<true, 1> : k_greedy_round<false, 1>;
        int per_sm = 0;
        for (auto kf : {kbig, ksmall}) {
          C2_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
          int ps = 0;
          C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kf, kNT, smem));
          if (ps < 1) return C2_ERR_UNSUPPORTED;
          per_sm = per_sm ? std::min(per_sm, ps) : ps;
        }
        static const char* kRoundName[] = {"round_01", "round_02", "round_03", "round_04",
                                           "round_05", "round_06", "round_07", "round_08",
                                           "round_09", "round_10", "round_11+"};
        for (int r = 1; r <= rounds; ++r) {
          Prof p_r(st, kRoundName[std::min(r, 11) - 1]);
          ga.round = r;
          ga.wl_in = cur;
          ga.wl_out = nxt;
          // round 1 computes every user (no previous round to repeat)
          ga.chg_in = (skipping && r > 1) ? chg_cur : nullptr;
          ga.chg_out = skipping ? chg_nxt : nullptr;
          std::swap(chg_cur, chg_nxt);
          C2_CUDA_TRY(cudaMemsetAsync(ga.counter, 0, sizeof(unsigned), st));
          auto kround = r <= kGreedySmallItemRounds ? ksmall : kbig;
          C2_LAUNCH(kround, num_sms() * per_sm, kNT, smem, st, ga);
          std::swap(cur, nxt);
        }
      }
      {
        Prof p_emit(st, "greedy_emit");
        ga.wl_in = cur;
        C2_LAUNCH(k_greedy_emit, div_up(n_greedy_users * 32, kNT), kNT, 0, st, ga);
      }
    }
    C2_CUDA_TRY(cudaGetLastError());
    if (g1 < ng) {
      // the next batch rewrites the count matrices the side stream reads
      c2_status rc = sj.join();
      if (rc) return rc;
    }
    g0 = g1;
  }
  return sj.join();
}

c2_status run_bruteforce(const int32_t* ptr, const int32_t* items, const Sizes& s,
                         const int32_t* queries, int32_t nq, int32_t* nid, int32_t* nin,
                         int32_t* nun, KnnWs& w, cudaStream_t st) {
  const int rows = queries ? nq : s.n;
  if (rows == 0) return C2_OK;
  const TableCfg tc = pick_table(C2_STRATEGY_AUTO, s.m);
  if (tc.W) {
    c2_status rc = build_padded_csr(ptr, items, s, w, st);
    if (rc) return rc;
    const int Q = 32 * tc.W;
    C2_LAUNCH(k_set_count, 1, 1, 0, st, &w.hdr->n_work, div_up(rows, Q));
    TableArgs a{};
    a.ptr = ptr; a.items = items; a.pptr = w.pptr; a.pitems = w.pitems;
    a.n_items = s.m; a.k = s.k;
    a.n_work = &w.hdr->n_work;
    a.cptr = nullptr; a.queries = queries; a.n_queries = rows; a.n_users = s.n;
    a.out_id = nid; a.out_in = nin; a.out_un = nun;
    a.hdr = w.hdr; a.counter = &w.hdr->work_counter[3];
    return launch_table(tc, a, st);
  }
  // no item table fits: the hashed judge when every profile fits one pass
  int32_t max_len = 0;
  C2_CUDA_TRY(cudaMemcpyAsync(&max_len, &w.hdr->max_profile, sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaStreamSynchronize(st));
  constexpr int NT = 256;
  const int hsmem = (int)(gram_hash_smem_bytes() + (16 * NT + 2 * NT) * sizeof(uint32_t));
  if (max_len <= kHashCap && hsmem + 1024 <= smem_optin()) {
    c2_status rc = build_padded_csr(ptr, items, s, w, st);
    if (rc) return rc;
    C2_LAUNCH(k_set_count, 1, 1, 0, st, &w.hdr->n_work, div_up(rows, 32));
    TableArgs a{};
    a.ptr = ptr; a.items = items; a.pptr = w.pptr; a.pitems = w.pitems;
    a.n_items = s.m; a.k = s.k;
    a.n_work = &w.hdr->n_work;
    a.cptr = nullptr; a.queries = queries; a.n_queries = rows; a.n_users = s.n;
    a.out_id = nid; a.out_in = nin; a.out_un = nun;
    a.hdr = w.hdr; a.counter = &w.hdr->work_counter[3];
    C2_CUDA_TRY(cudaFuncSetAttribute(k_table_hash<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     hsmem));
    int per_sm = 0;
    C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_table_hash<NT>, NT, hsmem));
    if (per_sm < 1) return C2_ERR_UNSUPPORTED;
    C2_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
    C2_LAUNCH(k_table_hash<NT>, num_sms() * per_sm, NT, hsmem, st, a);
    C2_CUDA_TRY(cudaGetLastError());
    return C2_OK;
  }
  MergeArgs a{};
  a.ptr = ptr; a.items = items; a.k = s.k; a.n_rows = rows;
  a.queries = queries; a.n_users = s.n; a.out_id = nid; a.out_in = nin; a.out_un = nun;
  a.hdr = w.hdr;
  C2_LAUNCH(k_merge_knn, div_up((int64_t)rows * 32, kNT), kNT, 0, st, a);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

size_t autotune_report(char* buf, size_t len) {
  std::string out = "[";
  std::lock_guard<std::mutex> lk(g_tune_mu);
  bool first = true;
  for (const auto& kv : g_tune) {
    char tmp[512];
    snprintf(tmp, sizeof tmp,
             "%s{\"n\": %lld, \"m\": %lld, \"t\": %lld, \"b\": %lld, \"N\": %lld, \"k\": %lld, "
             "\"threshold\": %lld, \"one_launch\": %s, \"buckets\": [",
             first ? "" : ", ", (long long)kv.first.n, (long long)kv.first.m, (long long)kv.first.t,
             (long long)kv.first.b, (long long)kv.first.N, (long long)kv.first.k,
             (long long)kv.first.thr, kv.second.unified ? "true" : "false");
    out += tmp;
    static const char* names[kBuckets] = {"<128", "128-511", "512-2047", "2048+"};
    for (int q = 0; q < kBuckets; ++q) {
      snprintf(tmp, sizeof tmp,
               "%s{\"sizes\": \"%s\", \"words\": %d, \"threads\": %d, \"min_blocks\": %d, "
               "\"items16\": %s, \"ms\": %.4f}",
               q ? ", " : "", names[q], kv.second.cfg[q].W, kv.second.cfg[q].NT, kv.second.cfg[q].MB,
               kv.second.cfg[q].P16 ? "true" : "false", kv.second.ms[q]);
      out += tmp;
    }
    out += "], \"strategy\": [";
    static const char* dnames[kDensityBuckets] = {"<1/64", "1/64-1/32", "1/32-1/16", "1/16-1/8",
                                                  ">=1/8"};
    bool f2 = true;
    for (int q = 0; q < kBuckets; ++q)
      for (int d = 0; d < kDensityBuckets; ++d) {
        const int bk = q * kDensityBuckets + d;
        if (kv.second.route[bk] < 0) continue;
        snprintf(tmp, sizeof tmp,
                 "%s{\"sizes\": \"%s\", \"density\": \"%s\", \"use\": \"%s\", "
                 "\"table_ms\": %.4f, \"tensor_ms\": %.4f}",
                 f2 ? "" : ", ", names[q], dnames[d], kv.second.route[bk] ? "tensor" : "table",
                 kv.second.table_ms[bk], kv.second.tc_ms[bk]);
        out += tmp;
        f2 = false;
      }
    out += "]}";
    first = false;
  }
  out += "]";
  if (buf && len) {
    const size_t n = out.size() < len - 1 ? out.size() : len - 1;
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return out.size() + 1;
}

// Text form of the autotuner's table, one line per problem size:
//   n m t b N k thr unified shapes_done tc_done  (W NT MB P16 ms) x kBuckets
//   (route table_ms tc_ms) x (kBuckets * kDensityBuckets)
// after a first line "c2-autotune 2".
int autotune_save(const char* path) {
  FILE* f = fopen(path, "w");
  if (!f) return -1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  fprintf(f, "c2-autotune 2\n");
  for (const auto& kv : g_tune) {
    const TuneKey& k = kv.first;
    const TuneEntry& e = kv.second;
    fprintf(f, "%lld %lld %lld %lld %lld %lld %lld %d %d %d", (long long)k.n, (long long)k.m,
            (long long)k.t, (long long)k.b, (long long)k.N, (long long)k.k, (long long)k.thr,
            e.unified ? 1 : 0, e.shapes_done ? 1 : 0, e.tc_done ? 1 : 0);
    for (int q = 0; q < kBuckets; ++q)
      fprintf(f, " %d %d %d %d %.6g", e.cfg[q].W, e.cfg[q].NT, e.cfg[q].MB, e.cfg[q].P16, e.ms[q]);
    for (int i = 0; i < kBuckets * kDensityBuckets; ++i)
      fprintf(f, " %d %.6g %.6g", (int)e.route[i], e.table_ms[i], e.tc_ms[i]);
    fprintf(f, "\n");
  }
  const int rc = ferror(f) ? -1 : 0;
  fclose(f);
  return rc;
}

// Reads a table written by autotune_save and merges it into the process's
// table (its entries replace those of the same sizes).  Returns the number
// of entries read, or -1 when the file is missing or not such a table.
int autotune_load(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  char magic[32] = {0};
  int version = 0;
  if (fscanf(f, "%31s %d", magic, &version) != 2 || strcmp(magic, "c2-autotune") || version != 2) {
    fclose(f);
    return -1;
  }
  std::map<TuneKey, TuneEntry> got;
  for (;;) {
    long long v[7];
    int uni = 0, sd = 0, td = 0;
    if (fscanf(f, "%lld %lld %lld %lld %lld %lld %lld %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4],
               &v[5], &v[6], &uni, &sd, &td) != 10)
      break;
    TuneEntry e;
    e.unified = uni != 0;
    e.shapes_done = sd != 0;
    e.tc_done = td != 0;
    bool ok = true;
    for (int q = 0; q < kBuckets && ok; ++q)
      ok = fscanf(f, "%d %d %d %d %f", &e.cfg[q].W, &e.cfg[q].NT, &e.cfg[q].MB, &e.cfg[q].P16,
                  &e.ms[q]) == 5;
    for (int i = 0; i < kBuckets * kDensityBuckets && ok; ++i) {
      int r = -1;
      ok = fscanf(f, "%d %f %f", &r, &e.table_ms[i], &e.tc_ms[i]) == 3;
      e.route[i] = (int8_t)(r < -1 || r > 1 ? -1 : r);
    }
    if (!ok) break;
    // only shapes this build has are kept; anything else is measured again
    for (int q = 0; q < kBuckets; ++q) {
      bool known = false;
      for (const TableCfg& c : kGramShapes)
        known = known || (c.W == e.cfg[q].W && c.NT == e.cfg[q].NT && c.MB == e.cfg[q].MB &&
                          c.P16 == e.cfg[q].P16);
      if (!known) e.shapes_done = false;
    }
    got[TuneKey{v[0], v[1], v[2], v[3], v[4], v[5], v[6]}] = e;
  }
  fclose(f);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : got) g_tune[kv.first] = kv.second;
  return (int)got.size();
}

}  // namespace c2
