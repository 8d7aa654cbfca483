// Greedy refinement (Algorithm 2's second branch; R11) for clusters whose
// intersection-count matrix is not built: more than kMaxGreedyM members, or
// an M x round_up(M, 8) matrix beyond the count-matrix budget.  The method
// is the same as for the other greedy clusters -- a Philox-seeded random
// start, then synchronous rounds over the own list, the neighbours' lists and
// optional random draws -- but every similarity is counted when it is needed,
// from the two profiles, instead of being looked up.
//
// One warp per member.  Working lists hold local indices (the cluster's
// user-id order, so that a lower index is a lower id), double-buffered per
// round, best first, and keep zero-similarity entries for navigation; the
// emitted rows drop them (R9).  A round gathers its candidates into a
// per-warp open-addressing set in shared memory -- the own list first, so
// that a candidate counts among the method's evaluations (R13) exactly when
// the set did not already hold it -- compacts the set in place, scores the
// candidates one per lane and keeps the best k with the exact comparator.
// Scoring tests each of the candidate's items against a bitmap of the
// member's profile in shared memory when the item universe is small enough,
// else merges the two sorted profiles.
#include "c2_internal.cuh"

namespace c2 {
namespace {

constexpr int kBgWarps = 8;                  // warps per block
constexpr int kBgSet = 2048;                 // set slots per warp
constexpr int kBgMaxCand = 1536;             // candidates per member and round (load <= 3/4)
constexpr int kBgMaxWords = 2048;            // bitmap scoring up to 65,536 items

struct BigArgs {
  const int32_t* ptr;
  const int32_t* items;
  const int32_t* cptr;
  const int32_t* cusers;
  const int32_t* bslot;      // slots of the members of such clusters
  const int32_t* slot2c;     // slot -> cluster
  const int32_t* n_dev;      // device: number of such slots
  int32_t k, round, n_random, max_draws;
  int32_t words;             // bitmap words per warp (0 = merge scoring)
  uint32_t cluster_base;
  uint2 key;                 // Philox key = run seed
  const int32_t* wl_in;      // [S][k] local indices by slot
  int32_t* wl_out;
  int32_t *out_id, *out_in, *out_un;
  DevHeader* hdr;
};

// |P_u n P_v| of two sorted rows (one lane).
__device__ __forceinline__ uint32_t merge_count(const int32_t* __restrict__ items, int a, int ae,
                                                int b, int be) {
  uint32_t c = 0;
  while (a < ae && b < be) {
    const int32_t x = items[a], y = items[b];
    c += x == y;
    a += x <= y;
    b += y <= x;
  }
  return c;
}

// Bit x of the warp's bitmap of W words; 0 outside it (items are checked
// against the universe when the CSR is validated; this keeps a stray one in
// bounds).
__device__ __forceinline__ uint32_t bm_bit(const uint32_t* bm, uint32_t W, int32_t x) {
  const uint32_t w = (uint32_t)x >> 5;
  return w < W ? (bm[w] >> (x & 31)) & 1u : 0u;
}

// |P_u n P_v| with P_u held as a bitmap (one lane).
__device__ __forceinline__ uint32_t bitmap_count(const int32_t* __restrict__ items,
                                                 const uint32_t* bm, uint32_t W, int b, int be) {
  uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  for (; b + 4 <= be; b += 4) {
    const int32_t x0 = items[b], x1 = items[b + 1], x2 = items[b + 2], x3 = items[b + 3];
    c0 += bm_bit(bm, W, x0);
    c1 += bm_bit(bm, W, x1);
    c2 += bm_bit(bm, W, x2);
    c3 += bm_bit(bm, W, x3);
  }
  for (; b < be; ++b) c0 += bm_bit(bm, W, items[b]);
  return c0 + c1 + c2 + c3;
}

__device__ __forceinline__ int draw_member(uint32_t r, int l, int M) {
  const int x = (int)(r % (uint32_t)(M - 1));
  return x + (x >= l ? 1 : 0);
}

// Round 0: min(k, M-1) distinct random members in draw order, then sorted.
__global__ void __launch_bounds__(32 * kBgWarps) k_bgreedy_init(BigArgs a) {
  __shared__ int32_t s_drawn[kBgWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_dev || dev_failed(a.hdr)) return;
  int32_t* drawn = s_drawn[warp];
  const int slot = a.bslot[w], c = a.slot2c[slot];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, l = slot - cs;
  const int k = a.k, k0 = min(k, M - 1);
  int cnt = 0;
  // rejection sampling of distinct members, bounded like the other greedy path
  for (int j0 = 0; cnt < k0; j0 += 32) {
    if (j0 + 32 > a.max_draws) {   // draws come 32 at a time
      if (lane == 0) dev_fail(a.hdr, C2_ERR_TIMEOUT);
      return;
    }
    const uint4 r =
        philox10(make_uint4((uint32_t)c + a.cluster_base, (uint32_t)l, 0u, (uint32_t)(j0 + lane)),
                 a.key);
    const int v = draw_member(r.x, l, M);
    bool dup = (__match_any_sync(0xffffffffu, v) & lanemask_lt()) != 0u;
    for (int q = 0; q < cnt; ++q) dup = dup || drawn[q] == v;
    const unsigned okm = __ballot_sync(0xffffffffu, !dup);
    const int rank = __popc(okm & lanemask_lt());
    __syncwarp();
    if (!dup && cnt + rank < k0) drawn[cnt + rank] = v;
    cnt = min(k0, cnt + __popc(okm));
    __syncwarp();
  }
  const int u = a.cusers[slot];
  const int ua = a.ptr[u], ue = a.ptr[u + 1];
  WarpList L;
  L.id = -1; L.c = 0; L.u = 0;
  if (lane < cnt) {
    const int v = drawn[lane];
    const int vu = a.cusers[cs + v];
    const int va = a.ptr[vu], ve = a.ptr[vu + 1];
    L.id = v;
    L.c = merge_count(a.items, ua, ue, va, ve);
    L.u = (uint32_t)(ue - ua) + (uint32_t)(ve - va) - L.c;
  }
  warp_sort32(L);
  if (lane < k) a.wl_out[(int64_t)slot * k + lane] = L.id;
  if (lane == 0 && cnt) atomicAdd(&a.hdr->pairs, (unsigned long long)cnt);
}

// Inserts v into the warp's set; true iff it was not there.  The set never
// holds more than kBgMaxCand < kBgSet entries, so a free slot is always found.
__device__ __forceinline__ bool set_insert(int32_t* set, int32_t v) {
  uint32_t h = ((uint32_t)v * 2654435761u) >> 21;   // 11 bits: kBgSet slots
  for (int probe = 0; probe < kBgSet; ++probe) {
    const int32_t prev = atomicCAS(&set[h], -1, v);
    if (prev == -1) return true;
    if (prev == v) return false;
    h = (h + 1) & (kBgSet - 1);
  }
  return false;
}

// Bytes of dynamic shared memory per warp of k_bgreedy_round.
__host__ __device__ constexpr int bg_warp_bytes(int words) {
  return kBgSet * 4 + 64 * 4 + 64 * 8 + words * 4;
}

// One synchronous round.
__global__ void __launch_bounds__(32 * kBgWarps) k_bgreedy_round(BigArgs a) {
  extern __shared__ __align__(16) unsigned char bg_sh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_dev || dev_failed(a.hdr)) return;
  unsigned char* base = bg_sh + (size_t)warp * bg_warp_bytes(a.words);
  int32_t* set = reinterpret_cast<int32_t*>(base);
  uint2* scu = reinterpret_cast<uint2*>(base + kBgSet * 4);
  int32_t* sid = reinterpret_cast<int32_t*>(base + kBgSet * 4 + 64 * 8);
  uint32_t* bm = reinterpret_cast<uint32_t*>(base + kBgSet * 4 + 64 * 12);
  const int slot = a.bslot[w], c = a.slot2c[slot];
  const int cs = a.cptr[c], M = a.cptr[c + 1] - cs, l = slot - cs;
  const int k = a.k;
  const int u = a.cusers[slot];
  const int ua = a.ptr[u], ue = a.ptr[u + 1];
  for (int i = lane; i < kBgSet; i += 32) set[i] = -1;
  if (a.words) {
    for (int i = lane; i < a.words; i += 32) bm[i] = 0u;
    __syncwarp();
    for (int e = ua + lane; e < ue; e += 32) {
      const int32_t x = a.items[e];
      if (((uint32_t)x >> 5) < (uint32_t)a.words) atomicOr(&bm[x >> 5], 1u << (x & 31));
    }
  }
  __syncwarp();
  int n = 0;            // entries in the set (uniform)
  int fresh = 0;        // of them, not in the own list (uniform)
  const int32_t own = lane < k ? a.wl_in[(int64_t)slot * k + lane] : -1;
  {
    const bool add = own >= 0 && set_insert(set, own);
    n += __popc(__ballot_sync(0xffffffffu, add));
  }
  for (int j = 0; j < k; ++j) {
    const int32_t v = __shfl_sync(0xffffffffu, own, j);
    if (v < 0) break;   // uniform; the list is best first with empties last
    const int32_t x = lane < k ? a.wl_in[(int64_t)(cs + v) * k + lane] : -1;
    const bool add = x >= 0 && x != l && set_insert(set, x);
    const int got = __popc(__ballot_sync(0xffffffffu, add));
    n += got;
    fresh += got;
  }
  for (int d0 = 0; d0 < a.n_random; d0 += 32) {
    bool add = false;
    if (d0 + lane < a.n_random) {
      const uint4 r = philox10(make_uint4((uint32_t)c + a.cluster_base, (uint32_t)l,
                                          (uint32_t)a.round, (uint32_t)(d0 + lane)),
                               a.key);
      add = set_insert(set, draw_member(r.x, l, M));
    }
    const int got = __popc(__ballot_sync(0xffffffffu, add));
    n += got;
    fresh += got;
  }
  __syncwarp();
  // compact the set in place: the chunk read always lies at or after the
  // positions written
  {
    int o = 0;
    for (int i0 = 0; i0 < kBgSet; i0 += 32) {
      const int32_t v = set[i0 + lane];
      const unsigned m = __ballot_sync(0xffffffffu, v >= 0);
      __syncwarp();
      if (v >= 0) set[o + __popc(m & lanemask_lt())] = v;
      o += __popc(m);
      __syncwarp();
    }
  }
  // score every candidate (one per lane) and keep the best k
  WarpTopk tk;
  WarpList l0;
  l0.id = -1; l0.c = 0; l0.u = 0;
  tk.start(l0, k, sid, scu);
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    int32_t v = -1;
    uint32_t cc = 0u, uu = 0u;
    if (i < n) {
      v = set[i];
      const int vu = a.cusers[cs + v];
      const int va = a.ptr[vu], ve = a.ptr[vu + 1];
      cc = a.words ? bitmap_count(a.items, bm, (uint32_t)a.words, va, ve)
                   : merge_count(a.items, ua, ue, va, ve);
      uu = (uint32_t)(ue - ua) + (uint32_t)(ve - va) - cc;
    }
    const bool pass = i < n && tk.filter(v, cc, uu);
    tk.stage(pass, v, cc, uu);
  }
  tk.finish();
  if (lane < k) a.wl_out[(int64_t)slot * k + lane] = tk.L.id;
  if (lane == 0 && fresh) atomicAdd(&a.hdr->pairs, (unsigned long long)fresh);
}

// The emitted rows: the working list without zero-similarity entries, by
// global id.  Reads only the warp's own row before writing it, so the output
// rows may alias the working lists.
__global__ void __launch_bounds__(32 * kBgWarps) k_bgreedy_emit(BigArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= *a.n_dev || dev_failed(a.hdr)) return;
  const int slot = a.bslot[w], c = a.slot2c[slot];
  const int cs = a.cptr[c];
  const int k = a.k;
  const int32_t v = lane < k ? a.wl_in[(int64_t)slot * k + lane] : -1;
  uint32_t cc = 0u, uu = 0u;
  if (v >= 0) {
    const int u = a.cusers[slot], vu = a.cusers[cs + v];
    const int ua = a.ptr[u], ue = a.ptr[u + 1], va = a.ptr[vu], ve = a.ptr[vu + 1];
    cc = merge_count(a.items, ua, ue, va, ve);
    uu = (uint32_t)(ue - ua) + (uint32_t)(ve - va) - cc;
  }
  const bool keep = v >= 0 && cc > 0u;
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  const int pos = __popc(m & lanemask_lt());
  const int kept = __popc(m);
  const int64_t o = (int64_t)slot * k;
  if (keep) {
    a.out_id[o + pos] = a.cusers[cs + v];
    a.out_in[o + pos] = (int32_t)cc;
    a.out_un[o + pos] = (int32_t)uu;
  }
  if (lane >= kept && lane < k) {
    a.out_id[o + lane] = -1;
    a.out_in[o + lane] = 0;
    a.out_un[o + lane] = 0;
  }
}

// Members of clusters flagged 2 in gkind_c, listed by slot.
__global__ void k_bg_flag(const int32_t* __restrict__ slot2c, const int32_t* __restrict__ gkind_c,
                          int64_t S, int32_t* __restrict__ flag) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) flag[s] = gkind_c[slot2c[s]] == 2 ? 1 : 0;
}

__global__ void k_bg_fill(const int32_t* __restrict__ flag, const int32_t* __restrict__ off,
                          int64_t S, int32_t* __restrict__ list, int32_t* __restrict__ n_out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *n_out = off[S];
  if (s < S && flag[s]) list[off[s]] = (int32_t)s;
}

}  // namespace

bool big_greedy_supported(int32_t k, int32_t n_random) {
  return (int64_t)k + (int64_t)k * k + (int64_t)std::max(n_random, 0) <= kBgMaxCand;
}

c2_status run_big_greedy(const int32_t* ptr, const int32_t* items, int32_t m, const int32_t* cptr,
                         const int32_t* cusers, const int32_t* slot2c, const int32_t* gkind_c,
                         int64_t S, int64_t n_users, int32_t k, int32_t rounds, int32_t n_random,
                         int32_t max_draws, uint32_t cluster_base, uint2 key, int32_t* flag,
                         int32_t* off, int32_t* bslot, int32_t* scan_tmp, int32_t* wl0,
                         int32_t* wl1, int32_t* out_id, int32_t* out_in, int32_t* out_un,
                         DevHeader* hdr, cudaStream_t st) {
  if (n_users <= 0) return C2_OK;
  if (!big_greedy_supported(k, n_random)) return C2_ERR_UNSUPPORTED;
  C2_LAUNCH(k_bg_flag, div_up(S, 256), 256, 0, st, slot2c, gkind_c, S, flag);
  C2_CUDA_TRY(scan_exclusive(flag, off, S, scan_tmp, st));
  int32_t* n_dev = flag + S;   // the flag array has S + 1 elements
  C2_LAUNCH(k_bg_fill, div_up(S, 256), 256, 0, st, flag, off, S, bslot, n_dev);
  BigArgs a{};
  a.ptr = ptr; a.items = items; a.cptr = cptr; a.cusers = cusers;
  a.bslot = bslot; a.slot2c = slot2c; a.n_dev = n_dev;
  a.k = k; a.n_random = std::max(n_random, 0); a.max_draws = max_draws;
  a.cluster_base = cluster_base; a.key = key;
  a.out_id = out_id; a.out_in = out_in; a.out_un = out_un; a.hdr = hdr;
  const int words = (m + 31) / 32;
  a.words = words <= kBgMaxWords ? ((words + 3) & ~3) : 0;
  const int smem = kBgWarps * bg_warp_bytes(a.words);
  C2_CUDA_TRY(cudaFuncSetAttribute(k_bgreedy_round, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem));
  const int grid = (int)div_up(n_users * 32, 32 * kBgWarps);
  a.round = 0;
  a.wl_in = nullptr;
  a.wl_out = wl0;
  C2_LAUNCH(k_bgreedy_init, grid, 32 * kBgWarps, 0, st, a);
  int32_t* cur = wl0;
  int32_t* nxt = wl1;
  for (int r = 1; r <= rounds; ++r) {
    a.round = r;
    a.wl_in = cur;
    a.wl_out = nxt;
    C2_LAUNCH(k_bgreedy_round, grid, 32 * kBgWarps, smem, st, a);
    std::swap(cur, nxt);
  }
  a.wl_in = cur;
  a.wl_out = nullptr;
  C2_LAUNCH(k_bgreedy_emit, grid, 32 * kBgWarps, 0, st, a);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
