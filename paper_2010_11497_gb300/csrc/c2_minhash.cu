// First-level keys of the C^2/MinHash variant (Section V-C, Table 4; Section
// II-E compares MinHash with FastRandomHash): one cluster per item, no split.
#include "c2_internal.cuh"

namespace c2 {

// v_i(x) = SplitMix64(K_i xor x * 0xD6E8FEB86659FD93) with K_i the key of
// function i; key_i(u) = the item of P_u with the least v_i (ties to the lower
// item), m for an empty profile.  Warp per user, every function in turn.
namespace {
__global__ void k_minhash_items(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items,
                                int32_t n, int32_t m, int32_t t, uint64_t seed,
                                int32_t* __restrict__ keys, const DevHeader* hdr) {
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n || dev_failed(hdr)) return;
  const int32_t s = ptr[u], e = ptr[u + 1];
  for (int i = 0; i < t; ++i) {
    const uint64_t K = sm64_mix(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    uint64_t best = ~0ull;
    int32_t bx = m;
    for (int32_t j = s + lane; j < e; j += 32) {
      const int32_t x = items[j];
      const uint64_t v = sm64_mix(K ^ ((uint64_t)(uint32_t)x * 0xD6E8FEB86659FD93ull));
      if (bx == m || v < best || (v == best && x < bx)) { best = v; bx = x; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int32_t ox = __shfl_xor_sync(0xffffffffu, bx, o);
      if (ox != m && (bx == m || ov < best || (ov == best && ox < bx))) { best = ov; bx = ox; }
    }
    if (lane == 0) keys[(int64_t)i * n + u] = bx;
  }
}
}  // namespace

c2_status run_minhash_keys(const int32_t* ptr, const int32_t* items, const Sizes& s,
                           uint64_t seed, int32_t* keys, DevHeader* hdr, cudaStream_t st) {
  c2_status rc = run_validate(ptr, items, s, hdr, st);
  if (rc) return rc;
  if (s.n > 0)
    C2_LAUNCH(k_minhash_items, div_up((int64_t)s.n * 32, 256), 256, 0, st, ptr, items, s.n, s.m,
              s.t, seed, keys, hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
