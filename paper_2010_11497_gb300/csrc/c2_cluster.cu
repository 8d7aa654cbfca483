// Step 1 of Cluster-and-Conquer on sm_103a: FastRandomHash clustering
// (Eq. 3, Algorithm 1) and recursive splitting of oversized clusters
// (Section II-D), producing the canonical cluster CSR.
//
// Layout: every (hash function i, user u) pair is a "slot" s = i*n + u.  A
// split level keeps one label per slot; labels are dense and ordered like the
// clusters' paths (function, key, split keys..., residual first), so the final
// labels are the canonical cluster numbers.
#include "c2_internal.cuh"

namespace c2 {

cudaError_t scan_exclusive64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* tmp,
                             cudaStream_t st);

namespace {

// ------------------------------------------------------------------ K0: CSR check
// Profiles must be sets (Section II-A): ptr non-decreasing from 0, items in
// range and strictly increasing per row.  One warp per row.
__global__ void __launch_bounds__(256) k_validate(const int32_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ items, int32_t n,
                                                  int32_t m, DevHeader* hdr) {
  __shared__ int32_t s_len[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int32_t len = 0;
  if (row < n) {
    if (row == 0 && lane == 0 && ptr[0] != 0) dev_fail(hdr, C2_ERR_INVALID_CSR);
    const int32_t s = ptr[row], e = ptr[row + 1];
    if (e < s) {
      if (lane == 0) dev_fail(hdr, C2_ERR_INVALID_CSR);
    } else if (e - s > kMaxProfile) {
      if (lane == 0) dev_fail(hdr, C2_ERR_UNSUPPORTED);
    } else {
      bool bad = false;
#pragma unroll 4
      for (int32_t j = s + lane; j < e; j += 32) {   // four items' loads in flight
        const int32_t x = items[j];
        bad |= x < 0 || x >= m;
        if (j > s) bad |= items[j - 1] >= x;
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) dev_fail(hdr, C2_ERR_INVALID_CSR);
      len = e - s;
      // padded rows (multiples of 4 items) must still be addressable with int32
      if (row == n - 1 && lane == 0 && (int64_t)e + 3 * (int64_t)n + 64 >= (int64_t(1) << 31))
        dev_fail(hdr, C2_ERR_UNSUPPORTED);
    }
  }
  // longest profile: one atomic per block (every update goes to one address)
  if (lane == 0) s_len[warp] = len;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t mx = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, s_len[w]);
    if (mx > 0) atomicMax(&hdr->max_profile, mx);
  }
}

// ------------------------------------------------------------------ A1: item hashes
// Generative hash functions h_i : items -> [0, b) (Section II-D).  The
// library's h_i(x) takes the high 32 bits of SplitMix64(key_i xor x*C) and
// scales them to [0, b); key_i is the (i+1)-th SplitMix64 output of the run
// seed.  Stored item-major as uint16 [m][tp] so one 16-byte load serves 8
// functions.
__global__ void k_build_htab(uint16_t* __restrict__ htab, int32_t m, int32_t t, int32_t tp,
                             int32_t b, uint64_t seed, int32_t fn_offset,
                             const int32_t* __restrict__ explicit_h, DevHeader* hdr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * tp) return;
  const int32_t x = (int32_t)(idx / tp), i = (int32_t)(idx % tp);
  uint32_t hv = 0;
  if (i < t) {
    if (explicit_h) {
      const int32_t v = explicit_h[(int64_t)i * m + x];
      if (v < 0 || v >= b) {
        dev_fail(hdr, C2_ERR_INVALID_ARG);
        return;
      }
      hv = (uint32_t)v;
    } else {
      // the run's function fn_offset + i (a shard of the functions)
      const uint64_t key =
          sm64_mix(seed + (uint64_t)(fn_offset + i + 1) * 0x9E3779B97F4A7C15ull);
      const uint64_t z = sm64_mix(key ^ ((uint64_t)(uint32_t)x * 0xC2B2AE3D27D4EB4Full));
      hv = (uint32_t)(((z >> 32) * (uint64_t)(uint32_t)b) >> 32);
    }
  }
  htab[idx] = (uint16_t)hv;
}

// ------------------------------------------------------------------ A2: FRH keys
// The hash rows of one user's items, walked by a warp: lane l takes the
// 16-byte chunks l, l + 32, ... of the row's items (one vector load for four
// items; the chunk holding the array's last item is read item by item), then
// loads the four items' rows of 8 hashes (16 bytes each) together, so a row
// of up to 128 items costs two dependent loads per lane.  fn(hv) sees the
// 8 hashes of functions c .. c + 7 of every item of [s, e) exactly once.
// `vec` is false when the items array is not 16-byte aligned.
template <class Fn>
__device__ __forceinline__ void walk_hash_rows(const int32_t* __restrict__ items, int64_t nnz,
                                               int32_t s, int32_t e, bool vec,
                                               const uint16_t* __restrict__ htab, int32_t tp,
                                               int32_t c, Fn&& fn) {
  const int lane = threadIdx.x & 31;
  if (!vec) {
#pragma unroll 4
    for (int32_t j = s + lane; j < e; j += 32)
      fn(__ldg(reinterpret_cast<const uint4*>(htab + (int64_t)items[j] * tp + c)));
    return;
  }
  for (int64_t j4 = (s >> 2) + lane; 4 * j4 < e; j4 += 32) {
    int32_t xs[4];
    if (4 * j4 + 4 <= nnz) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(items) + j4);
      xs[0] = v.x; xs[1] = v.y; xs[2] = v.z; xs[3] = v.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) xs[q] = 4 * j4 + q < nnz ? items[4 * j4 + q] : 0;
    }
    uint4 hv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = 4 * j4 + q;
      if (j >= s && j < e) hv[q] = __ldg(reinterpret_cast<const uint4*>(htab + (int64_t)xs[q] * tp + c));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = 4 * j4 + q;
      if (j >= s && j < e) fn(hv[q]);
    }
  }
}

// Minimum over the warp of each of the lanes' 8 values v[0..7], by halving
// exchanges (4 + 2 + 1 shuffles, then 2 more): value q's minimum ends in the
// four lanes with (lane >> 2) == q.
__device__ __forceinline__ uint32_t warp_min8(const uint32_t v[8]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  uint32_t r4[4], r2[2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {   // keep values 4*b4 + q
    const uint32_t keep = b4 ? v[q + 4] : v[q], send = b4 ? v[q] : v[q + 4];
    r4[q] = min(keep, __shfl_xor_sync(0xffffffffu, send, 16));
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {   // keep values 4*b4 + 2*b3 + q
    const uint32_t keep = b3 ? r4[q + 2] : r4[q], send = b3 ? r4[q] : r4[q + 2];
    r2[q] = min(keep, __shfl_xor_sync(0xffffffffu, send, 8));
  }
  const uint32_t keep = b2 ? r2[1] : r2[0], send = b2 ? r2[0] : r2[1];
  uint32_t r = min(keep, __shfl_xor_sync(0xffffffffu, send, 4));   // value lane >> 2
  r = min(r, __shfl_xor_sync(0xffffffffu, r, 2));
  return min(r, __shfl_xor_sync(0xffffffffu, r, 1));
}

// key[i][u] = min over u's items of h_i (Eq. 3); b for an empty profile.
// One warp per user (hash rows walked by walk_hash_rows).  Also counts the
// level-0 histogram of (function, key), and keeps key2[i][u] and key3[i][u],
// the second and third smallest distinct values of h_i over u's items (b when
// there is none): the keys of the first two splits of an oversized cluster
// (each split key is the smallest value above the cluster's key), so those
// levels need no second walk of the profiles.
__global__ void __launch_bounds__(256, 4) k_minhash(const int32_t* __restrict__ ptr,
                                                 const int32_t* __restrict__ items, int32_t vec,
                                                 const uint16_t* __restrict__ htab,
                                                 int32_t n, int32_t t, int32_t tp, int32_t b,
                                                 int32_t* __restrict__ key,
                                                 int32_t* __restrict__ key2,
                                                 int32_t* __restrict__ key3,
                                                 int32_t* __restrict__ hist, DevHeader* hdr) {
  if (dev_failed(hdr)) return;
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n) return;
  const int32_t s = ptr[u], e = ptr[u + 1];
  const int64_t nnz = ptr[n];   // validated: the items array holds ptr[n] entries
  for (int c = 0; c < tp; c += 8) {
    // the lane's three smallest distinct values per function, ascending
    uint32_t v0[8], v1[8], v2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v0[q] = v1[q] = v2[q] = (uint32_t)b;
    walk_hash_rows(items, nnz, s, e, vec != 0, htab, tp, c, [&](const uint4& hv) {
      const uint32_t w[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t h = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
        // insertion into the sorted three (a value already held changes nothing)
        const bool seen = h == v0[q] || h == v1[q];
        const uint32_t x = max(v0[q], h), y = max(v1[q], x);
        if (!seen) {
          v0[q] = min(v0[q], h);
          v1[q] = min(v1[q], x);
          v2[q] = min(v2[q], y);
        }
      }
    });
    const uint32_t r0 = warp_min8(v0);
    // each lane's smallest value above the warp's minimum, then above the
    // warp's second value
    uint32_t above[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) above[q] = v0[q] > __shfl_sync(0xffffffffu, r0, 4 * q) ? v0[q] : v1[q];
    const uint32_t r1 = warp_min8(above);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t m1 = __shfl_sync(0xffffffffu, r1, 4 * q);
      above[q] = v0[q] > m1 ? v0[q] : (v1[q] > m1 ? v1[q] : v2[q]);
    }
    const uint32_t r2 = warp_min8(above);
    const int i = c + (lane >> 2);
    if ((lane & 3) == 0 && i < t) {
      key[(int64_t)i * n + u] = (int32_t)r0;
      key2[(int64_t)i * n + u] = (int32_t)r1;
      key3[(int64_t)i * n + u] = (int32_t)r2;
      atomicAdd(&hist[(int64_t)i * (b + 1) + r0], 1);
    }
  }
}

// First-level keys given by the caller (a learned proposer): copy, check the
// range, count the level-0 histogram.
__global__ void k_keys_given(const int32_t* __restrict__ given, int64_t S, int32_t n, int32_t b,
                             int32_t* __restrict__ key, int32_t* __restrict__ hist,
                             DevHeader* hdr) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || dev_failed(hdr)) return;
  const int32_t kv = given[s];
  if (kv < 0 || kv >= b) {
    dev_fail(hdr, C2_ERR_INVALID_ARG);
    key[s] = 0;
    return;
  }
  key[s] = kv;
  atomicAdd(&hist[(s / n) * (b + 1) + kv], 1);
}

// ------------------------------------------------------------------ A3: level 0
__global__ void k_flag_nonzero(const int32_t* __restrict__ hist, int32_t* __restrict__ flag,
                               int64_t nbins) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nbins) flag[j] = hist[j] > 0 ? 1 : 0;
}

// One cluster per non-empty (function, key) bin, in (function, key) order.
__global__ void k_level0_meta(const int32_t* __restrict__ hist, const int32_t* __restrict__ binlab,
                              int64_t nbins, int32_t b, int32_t given_keys,
                              int32_t* __restrict__ lsize, int32_t* __restrict__ leta,
                              int32_t* __restrict__ lflag, DevHeader* hdr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) hdr->n_labels = binlab[nbins];
  if (j >= nbins || hist[j] == 0) return;
  const int32_t l = binlab[j];
  const int32_t i = (int32_t)(j / (b + 1)), kv = (int32_t)(j % (b + 1));
  lsize[l] = hist[j];
  // a learned first-level key carries no hash threshold: its split keys are
  // the plain FastRandomHash keys (every hash value counts)
  leta[l] = given_keys ? -1 : kv;
  // the empty-profile bucket b cannot be split: terminal, listed as a residual
  lflag[l] = lf_pack(kv == b, kv == b, i, 0);
}

__global__ void k_level0_labels(const int32_t* __restrict__ key, const int32_t* __restrict__ binlab,
                                int32_t n, int64_t S, int32_t b, int32_t* __restrict__ lab,
                                const DevHeader* hdr) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  if (dev_failed(hdr)) {   // keys were not computed: keep labels in range
    lab[s] = 0;
    return;
  }
  const int64_t i = s / n;
  lab[s] = binlab[i * (b + 1) + key[s]];
}

// ------------------------------------------------------------------ A4: split level
// Oversized = more than N users and not terminal (the residual of a split and
// the empty-profile bucket are terminal).
__global__ void k_mark_oversized(const int32_t* __restrict__ lsize, const int32_t* __restrict__ lflag,
                                 int64_t S, int32_t N, int32_t* __restrict__ ov,
                                 int32_t* __restrict__ nchild, const DevHeader* hdr) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= S) return;
  const int32_t L = hdr->n_labels;
  const bool live = l < L;
  ov[l] = (live && lsize[l] > N && !lf_terminal(lflag[l])) ? 1 : 0;
  nchild[l] = live ? 1 : 0;
}

// The first two split levels of FastRandomHash clusters: at level L every slot
// of an oversized cluster holds the cluster's key eta = its own (L+1)-th
// smallest distinct value (level 0: the minimum; the sub-clusters of a split
// carry their members' next value, and residuals never split again), so its
// next key (the smallest value above eta) is the (L+2)-th, which k_minhash
// kept (`next` = key2 or key3).  One thread per slot.
__global__ void k_split_keys_first(const int32_t* __restrict__ next, int64_t S, int32_t b,
                                   const int32_t* __restrict__ lab,
                                   const int32_t* __restrict__ ovscan,
                                   int32_t* __restrict__ nextkey, int32_t* __restrict__ subcnt,
                                   const DevHeader* hdr) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || dev_failed(hdr)) return;
  const int32_t l = lab[s];
  if (ovscan[l + 1] == ovscan[l]) return;
  const int32_t nk = next[s];
  nextkey[s] = nk;
  atomicAdd(&subcnt[(int64_t)ovscan[l] * (b + 1) + nk], 1);
}

// For every slot of an oversized cluster with last key eta:
//   next = min { h_i(x) : x in P_u, h_i(x) > eta }   (b when undefined)
// and count the sub-groups.  One warp per user: the user's oversized slots
// of a group of 8 functions are served by one walk over its profile, each
// item's 16-byte hash row giving all 8 functions' values.
__global__ void __launch_bounds__(256) k_split_keys(
    const int32_t* __restrict__ ptr, const int32_t* __restrict__ items, int32_t vec,
    const uint16_t* __restrict__ htab, int32_t n, int32_t t, int32_t tp, int32_t b,
    const int32_t* __restrict__ lab, const int32_t* __restrict__ ovscan,
    const int32_t* __restrict__ leta, int32_t* __restrict__ nextkey, int32_t* __restrict__ subcnt,
    const DevHeader* hdr) {
  if (dev_failed(hdr)) return;
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n) return;
  const int32_t s0 = ptr[u], e0 = ptr[u + 1];
  const int64_t nnz = ptr[n];   // validated: the items array holds ptr[n] entries
  for (int c = 0; c < t; c += 8) {
    // lane q < 8 looks up function c + q's slot: oversized?, its label and eta
    int32_t l = 0, eta = 0;
    bool ov = false;
    if (lane < 8 && c + lane < t) {
      l = lab[(int64_t)(c + lane) * n + u];
      ov = ovscan[l + 1] != ovscan[l];
      eta = leta[l];
    }
    const unsigned ovm = __ballot_sync(0xffffffffu, ov) & 0xFFu;
    if (ovm == 0u) continue;
    int32_t et[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) et[q] = __shfl_sync(0xffffffffu, eta, q);
    uint32_t best[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) best[q] = (uint32_t)b;
    walk_hash_rows(items, nnz, s0, e0, vec != 0, htab, tp, c, [&](const uint4& hv) {
      const uint32_t w[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t v = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
        if (((ovm >> q) & 1u) && (int32_t)v > et[q]) best[q] = min(best[q], v);
      }
    });
    const uint32_t r = warp_min8(best);
    // function c + q's result sits in lanes 4q .. 4q + 3; lane q < 8 holds
    // that slot's label
    const uint32_t mine = __shfl_sync(0xffffffffu, r, 4 * (lane & 7));
    if (lane < 8 && ov) {
      nextkey[(int64_t)(c + lane) * n + u] = (int32_t)mine;
      atomicAdd(&subcnt[(int64_t)ovscan[l] * (b + 1) + mine], 1);
    }
  }
}

// Per oversized cluster (one block): rank the sub-groups with >= 2 users in
// key order; users with an undefined key or alone in their group form the
// residual, which comes first.
__global__ void __launch_bounds__(256) k_split_plan(const int32_t* __restrict__ ovlist,
                                                    int32_t b, const int32_t* __restrict__ subcnt,
                                                    int32_t* __restrict__ subrank,
                                                    int32_t* __restrict__ sub_resid,
                                                    int32_t* __restrict__ nchild,
                                                    const DevHeader* hdr) {
  __shared__ int32_t wsum[8];
  __shared__ int32_t carry_s, resid_s;
  const int64_t o = blockIdx.x;
  const int32_t l = ovlist[o];
  const int32_t* cnt = subcnt + o * (b + 1);
  int32_t* rank = subrank + o * (b + 1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    carry_s = 0;
    resid_s = cnt[b];
  }
  __syncthreads();
  for (int32_t base = 0; base < b; base += 256) {
    const int32_t j = base + threadIdx.x;
    const int32_t c = j < b ? cnt[j] : 0;
    const int32_t g = c >= 2 ? 1 : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, g);
    const unsigned one = __ballot_sync(0xffffffffu, c == 1);
    if (lane == 0) {
      wsum[w] = __popc(bal);
      if (one) atomicAdd(&resid_s, __popc(one));
    }
    __syncthreads();
    int32_t before = carry_s;
    for (int q = 0; q < w; ++q) before += wsum[q];
    before += __popc(bal & lanemask_lt());
    if (j < b) rank[j] = before;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t tot = 0;
      for (int q = 0; q < 8; ++q) tot += wsum[q];
      carry_s += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sub_resid[o] = resid_s;
    nchild[l] = (resid_s > 0 ? 1 : 0) + carry_s;
  }
}

__global__ void k_relabel(const int32_t* __restrict__ lab, const int32_t* __restrict__ ovscan,
                          const int32_t* __restrict__ newbase, const int32_t* __restrict__ nextkey,
                          const int32_t* __restrict__ subcnt, const int32_t* __restrict__ subrank,
                          const int32_t* __restrict__ sub_resid, int64_t S, int32_t b,
                          int32_t* __restrict__ lab2) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int32_t l = lab[s];
  int32_t nl = newbase[l];
  if (ovscan[l + 1] != ovscan[l]) {
    const int64_t o = ovscan[l];
    const int32_t nk = nextkey[s];
    const bool resid = nk == b || subcnt[o * (b + 1) + nk] == 1;
    if (!resid) nl += (sub_resid[o] > 0 ? 1 : 0) + subrank[o * (b + 1) + nk];
  }
  lab2[s] = nl;
}

// Metadata of the next level: unsplit clusters are copied; a split cluster
// yields its residual (terminal) and one child per group of >= 2 users.
__global__ void k_newmeta_copy(const int32_t* __restrict__ ovscan, const int32_t* __restrict__ newbase,
                               const int32_t* __restrict__ lsize, const int32_t* __restrict__ leta,
                               const int32_t* __restrict__ lflag, int64_t S,
                               int32_t* __restrict__ lsize2, int32_t* __restrict__ leta2,
                               int32_t* __restrict__ lflag2, const DevHeader* hdr) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= S || l >= hdr->n_labels || ovscan[l + 1] != ovscan[l]) return;
  const int32_t nl = newbase[l];
  lsize2[nl] = lsize[l];
  leta2[nl] = leta[l];
  lflag2[nl] = lflag[l];
}

__global__ void __launch_bounds__(256) k_newmeta_split(
    const int32_t* __restrict__ ovlist, const int32_t* __restrict__ newbase,
    const int32_t* __restrict__ lflag, const int32_t* __restrict__ leta, int32_t b,
    const int32_t* __restrict__ subcnt, const int32_t* __restrict__ subrank,
    const int32_t* __restrict__ sub_resid, int32_t* __restrict__ lsize2,
    int32_t* __restrict__ leta2, int32_t* __restrict__ lflag2) {
  const int64_t o = blockIdx.x;
  const int32_t l = ovlist[o];
  const int32_t f = lflag[l];
  const int32_t res = sub_resid[o];
  const int32_t nb = newbase[l];
  if (threadIdx.x == 0 && res > 0) {
    lsize2[nb] = res;
    leta2[nb] = leta[l];
    lflag2[nb] = lf_pack(1, 1, lf_fn(f), lf_depth(f));
  }
  const int32_t first = nb + (res > 0 ? 1 : 0);
  for (int32_t j = threadIdx.x; j < b; j += blockDim.x) {
    const int32_t c = subcnt[o * (b + 1) + j];
    if (c >= 2) {
      const int32_t nl = first + subrank[o * (b + 1) + j];
      lsize2[nl] = c;
      leta2[nl] = j;
      lflag2[nl] = lf_pack(0, 0, lf_fn(f), lf_depth(f) + 1);
    }
  }
}

__global__ void k_set_nlabels(DevHeader* hdr, const int32_t* __restrict__ total) {
  hdr->n_labels = *total;
  hdr->split_levels += 1;
}

__global__ void k_ovlist(const int32_t* __restrict__ ovscan, int64_t S, int32_t* __restrict__ ovlist) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l < S && ovscan[l + 1] != ovscan[l]) ovlist[ovscan[l]] = (int32_t)l;
}

__global__ void k_copy_oversized(DevHeader* hdr, const int32_t* __restrict__ total) {
  hdr->n_oversized = *total;
}

// ------------------------------------------------------------------ final CSR
__global__ void k_sort_input(const int32_t* __restrict__ lab, int64_t S, int32_t n,
                             uint32_t* __restrict__ skey, int32_t* __restrict__ sval) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  skey[s] = (uint32_t)lab[s];
  sval[s] = (int32_t)(s % n);
}

__global__ void k_final_meta(const int32_t* __restrict__ lsize, const int32_t* __restrict__ leta,
                             const int32_t* __restrict__ lflag, int64_t S,
                             int32_t* __restrict__ cmeta, int32_t* __restrict__ n_clusters,
                             DevHeader* hdr) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t L = hdr->n_labels;
  if (l == 0) *n_clusters = L;
  if (l >= S || l >= L) return;
  atomicMax(&hdr->max_cluster, lsize[l]);
  if (cmeta) {
    const int32_t f = lflag[l];
    cmeta[4 * l + 0] = lf_fn(f);
    cmeta[4 * l + 1] = lf_depth(f);
    cmeta[4 * l + 2] = lf_residual(f);
    cmeta[4 * l + 3] = leta[l];
  }
}

__global__ void k_zero_tail(int32_t* __restrict__ lsize, int64_t S, const DevHeader* hdr) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l < S && l >= hdr->n_labels) lsize[l] = 0;
}

int bits_for(int64_t v) {
  int b = 0;
  while (b < 32 && (int64_t(1) << b) <= v) ++b;
  return b;
}

}  // namespace

c2_status run_validate(const int32_t* ptr, const int32_t* items, const Sizes& s, DevHeader* hdr,
                       cudaStream_t st) {
  if (s.n > 0) C2_LAUNCH(k_validate, div_up((int64_t)s.n * 32, 256), 256, 0, st, ptr, items, s.n, s.m, hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status run_frh_cluster(const int32_t* ptr, const int32_t* items, const Sizes& s, uint64_t seed,
                          const c2_options& opt, int32_t* cluster_of, int32_t* cptr,
                          int32_t* cusers, int32_t* n_clusters, int32_t* cmeta, ClusterWs& w,
                          cudaStream_t st) {
  const int64_t S = s.S;
  const int64_t nbins = (int64_t)s.t * (s.b + 1);
  const int T = 256;
  // 16-byte item loads need a 16-byte aligned items array
  const int32_t vec16 = ((uintptr_t)items & 15u) == 0 ? 1 : 0;
  c2_status rc;
  {
    Prof p(st, "validate");
    rc = run_validate(ptr, items, s, w.hdr, st);
  }
  if (rc) return rc;
  Prof p_hash(st, "hash_minhash_level0");
  if (s.m > 0)
    C2_LAUNCH(k_build_htab, div_up((int64_t)s.m * s.tp, T), T, 0, st, w.htab, s.m, s.t, s.tp, s.b, seed,
              opt.fn_offset, opt.d_hash_table, w.hdr);
  C2_CUDA_TRY(cudaMemsetAsync(w.hist, 0, (nbins + 1) * sizeof(int32_t), st));
  if (s.n > 0 && opt.d_keys)
    C2_LAUNCH(k_keys_given, div_up(S, T), T, 0, st, opt.d_keys, S, s.n, s.b, w.key, w.hist, w.hdr);
  else if (s.n > 0)
    C2_LAUNCH(k_minhash, div_up((int64_t)s.n * 32, T), T, 0, st, ptr, items, vec16, w.htab,
              s.n, s.t, s.tp, s.b, w.key, w.key2, w.key3, w.hist, w.hdr);
  C2_LAUNCH(k_flag_nonzero, div_up(nbins, T), T, 0, st, w.hist, w.binlab, nbins);
  C2_CUDA_TRY(scan_exclusive(w.binlab, w.binlab, nbins, w.scan_tmp, st));
  C2_CUDA_TRY(cudaMemsetAsync(w.lsize, 0, (S + 1) * sizeof(int32_t), st));
  C2_LAUNCH(k_level0_meta, div_up(nbins, T), T, 0, st, w.hist, w.binlab, nbins, s.b,
            opt.d_keys ? 1 : 0, w.lsize, w.leta, w.lflag, w.hdr);
  if (S > 0) C2_LAUNCH(k_level0_labels, div_up(S, T), T, 0, st, w.key, w.binlab, s.n, S, s.b, w.lab, w.hdr);
  C2_CUDA_TRY(cudaGetLastError());

  p_hash.end();
  // Recursive split, one level per iteration (at most b levels: keys grow).
  Prof p_split(st, "split");
  int32_t h_over = 0;
  c2_status out = C2_OK;
  for (int level = 0; level <= s.b + 1 && S > 0; ++level) {
    C2_LAUNCH(k_mark_oversized, div_up(S, T), T, 0, st, w.lsize, w.lflag, S, s.N, w.ovidx, w.nchild, w.hdr);
    if (scan_exclusive(w.ovidx, w.ovidx, S, w.scan_tmp, st) != cudaSuccess) { out = C2_ERR_CUDA; break; }
    C2_LAUNCH(k_copy_oversized, 1, 1, 0, st, w.hdr, w.ovidx + S);
    if (cudaMemcpyAsync(&h_over, &w.hdr->n_oversized, sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      out = C2_ERR_CUDA;
      break;
    }
    const int64_t O = h_over;
    if (O == 0) break;
    if (O > s.omax) { out = C2_ERR_UNSUPPORTED; break; }
    C2_LAUNCH(k_ovlist, div_up(S, T), T, 0, st, w.ovidx, S, w.ovlist);
    cudaMemsetAsync(w.subcnt, 0, O * (s.b + 1) * sizeof(int32_t), st);
    if (level < 2 && !opt.d_keys)   // first two splits of FastRandomHash keys: no walk
      C2_LAUNCH(k_split_keys_first, div_up(S, T), T, 0, st, level == 0 ? w.key2 : w.key3, S, s.b,
                w.lab, w.ovidx, w.key, w.subcnt, w.hdr);
    else
      C2_LAUNCH(k_split_keys, div_up((int64_t)s.n * 32, T), T, 0, st, ptr, items, vec16,
                w.htab, s.n, s.t, s.tp, s.b, w.lab, w.ovidx, w.leta, w.key, w.subcnt, w.hdr);
    C2_LAUNCH(k_split_plan, (unsigned)O, 256, 0, st, w.ovlist, s.b, w.subcnt, w.subrank, w.sub_resid,
                                               w.nchild, w.hdr);
    if (scan_exclusive(w.nchild, w.nchild, S, w.scan_tmp, st) != cudaSuccess) { out = C2_ERR_CUDA; break; }
    C2_LAUNCH(k_relabel, div_up(S, T), T, 0, st, w.lab, w.ovidx, w.nchild, w.key, w.subcnt, w.subrank,
                                          w.sub_resid, S, s.b, w.lab2);
    cudaMemsetAsync(w.lsize2, 0, (S + 1) * sizeof(int32_t), st);
    C2_LAUNCH(k_newmeta_copy, div_up(S, T), T, 0, st, w.ovidx, w.nchild, w.lsize, w.leta, w.lflag, S,
                                               w.lsize2, w.leta2, w.lflag2, w.hdr);
    C2_LAUNCH(k_newmeta_split, (unsigned)O, 256, 0, st, w.ovlist, w.nchild, w.lflag, w.leta, s.b,
                                                  w.subcnt, w.subrank, w.sub_resid, w.lsize2,
                                                  w.leta2, w.lflag2);
    C2_LAUNCH(k_set_nlabels, 1, 1, 0, st, w.hdr, w.nchild + S);
    std::swap(w.lab, w.lab2);
    std::swap(w.lsize, w.lsize2);
    std::swap(w.leta, w.leta2);
    std::swap(w.lflag, w.lflag2);
    if (cudaGetLastError() != cudaSuccess) { out = C2_ERR_CUDA; break; }
  }
  p_split.end();
  if (out) return out;

  // Canonical CSR: stable sort of slots (function-major, user-minor) by label.
  Prof p_csr(st, "cluster_csr");
  if (S > 0) {
    C2_LAUNCH(k_zero_tail, div_up(S, T), T, 0, st, w.lsize, S, w.hdr);
    C2_CUDA_TRY(scan_exclusive(w.lsize, cptr, S, w.scan_tmp, st));
    C2_LAUNCH(k_sort_input, div_up(S, T), T, 0, st, w.lab, S, s.n, w.skey, w.sval);
    C2_CUDA_TRY(radix_sort_pairs(w.skey, w.sval, w.skey2, w.sval2, S, bits_for(S), w.shist,
                                 w.scan_tmp, st));
    C2_CUDA_TRY(cudaMemcpyAsync(cusers, w.sval, S * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    C2_CUDA_TRY(cudaMemcpyAsync(cluster_of, w.lab, S * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    C2_LAUNCH(k_final_meta, div_up(S, T), T, 0, st, w.lsize, w.leta, w.lflag, S, cmeta, n_clusters, w.hdr);
  } else {
    C2_CUDA_TRY(cudaMemsetAsync(cptr, 0, sizeof(int32_t), st));
    C2_CUDA_TRY(cudaMemsetAsync(n_clusters, 0, sizeof(int32_t), st));
  }
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
