// GoldFinger fingerprints (Section II-F): the compact profile summaries the
// paper's prototype estimates Jaccard similarities with (1024 bits in its
// experiments, Section IV-E).  Item x sets bit
//   fp(x) = floor((SplitMix64(K_g ^ x * 0xC2B2AE3D27D4EB4F) >> 32) * B / 2^32),
//   K_g = SplitMix64(seed ^ 0x474F4C4446494E47),
// of a B-bit vector, and the estimate of J(u, v) is the Jaccard similarity
// of the two users' bit sets; Steps 2-3 of the method then run unchanged on
// the fingerprints as profiles over an item universe of B "items".
//
// One warp per user builds the user's bit vector in its own shared-memory
// words (atomicOr per item), then either counts the bits or writes them out
// in increasing order (a warp prefix sum over 32 words at a time), plus the
// packed words when asked for.
#include "c2_internal.cuh"

namespace c2 {
namespace {

constexpr int kGfWarps = 8;
constexpr int kGfMaxBits = 8192;

__device__ __forceinline__ uint32_t gf_bit(uint64_t key, int32_t x, uint32_t bits) {
  const uint64_t z = sm64_mix(key ^ ((uint64_t)(uint32_t)x * 0xC2B2AE3D27D4EB4Full));
  return (uint32_t)(((z >> 32) * (uint64_t)bits) >> 32);
}

// Fills the warp's W words with the fingerprint of user u.
__device__ __forceinline__ void gf_build(const int32_t* __restrict__ ptr,
                                         const int32_t* __restrict__ items, int u, uint64_t key,
                                         uint32_t bits, int W, uint32_t* bm) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < W; i += 32) bm[i] = 0;
  __syncwarp();
  for (int e = ptr[u] + lane; e < ptr[u + 1]; e += 32) {
    const uint32_t b = gf_bit(key, items[e], bits);
    atomicOr(&bm[b >> 5], 1u << (b & 31));
  }
  __syncwarp();
}

__global__ void __launch_bounds__(32 * kGfWarps) k_gf_count(const int32_t* __restrict__ ptr,
                                                            const int32_t* __restrict__ items,
                                                            int32_t n, uint64_t key, uint32_t bits,
                                                            int32_t* __restrict__ cnt,
                                                            const DevHeader* hdr) {
  extern __shared__ uint32_t gf_sh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = (int)(bits / 32);
  uint32_t* bm = gf_sh + warp * W;
  if (dev_failed(hdr)) return;
  for (int u = blockIdx.x * kGfWarps + warp; u < n; u += gridDim.x * kGfWarps) {
    gf_build(ptr, items, u, key, bits, W, bm);
    int c = 0;
    for (int i = lane; i < W; i += 32) c += __popc(bm[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[u] = c;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * kGfWarps) k_gf_emit(
    const int32_t* __restrict__ ptr, const int32_t* __restrict__ items, int32_t n, uint64_t key,
    uint32_t bits, const int32_t* __restrict__ fptr, int32_t* __restrict__ fitems,
    uint32_t* __restrict__ fbits, const DevHeader* hdr) {
  extern __shared__ uint32_t gf_sh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = (int)(bits / 32);
  uint32_t* bm = gf_sh + warp * W;
  if (dev_failed(hdr)) return;
  for (int u = blockIdx.x * kGfWarps + warp; u < n; u += gridDim.x * kGfWarps) {
    gf_build(ptr, items, u, key, bits, W, bm);
    int run = fptr[u];
    for (int base = 0; base < W; base += 32) {
      const int wi = base + lane;
      const uint32_t word = wi < W ? bm[wi] : 0u;
      const int pc = __popc(word);
      int incl = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int o = run + incl - pc;
      for (uint32_t wv = word; wv; wv &= wv - 1) fitems[o++] = wi * 32 + (__ffs(wv) - 1);
      run += __shfl_sync(0xffffffffu, incl, 31);
      if (fbits && wi < W) fbits[(int64_t)u * W + wi] = word;
    }
    __syncwarp();
  }
}

// Exact |P_u n P_v| and |P_u u P_v| of given neighbour rows: warp per user,
// lane j merges the two sorted profiles of slot j.
__global__ void __launch_bounds__(256) k_exact_counts(const int32_t* __restrict__ ptr,
                                                      const int32_t* __restrict__ items, int32_t n,
                                                      int32_t k, const int32_t* __restrict__ nbr,
                                                      int32_t* __restrict__ out_in,
                                                      int32_t* __restrict__ out_un) {
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n || lane >= k) return;
  const int64_t e = u * k + lane;
  const int32_t v = nbr[e];
  if (v < 0 || v >= n) {
    out_in[e] = 0;
    out_un[e] = 0;
    return;
  }
  int a = ptr[u], ae = ptr[u + 1], b = ptr[v], be = ptr[v + 1], c = 0;
  while (a < ae && b < be) {
    const int32_t x = items[a], y = items[b];
    c += x == y;
    a += x <= y;
    b += y <= x;
  }
  out_in[e] = c;
  out_un[e] = (ptr[u + 1] - ptr[u]) + (be - ptr[v]) - c;
}

}  // namespace

c2_status run_exact_counts(const int32_t* ptr, const int32_t* items, int32_t n, int32_t k,
                           const int32_t* nbr, int32_t* out_in, int32_t* out_un, cudaStream_t st) {
  if (n == 0) return C2_OK;
  C2_LAUNCH(k_exact_counts, div_up((int64_t)n * 32, 256), 256, 0, st, ptr, items, n, k, nbr,
            out_in, out_un);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

size_t goldfinger_ws_bytes(int32_t n) {
  return 256 + ((scan_tmp_elems((int64_t)n + 1) * 4 + 255) & ~size_t(255));
}

c2_status run_goldfinger(const int32_t* ptr, const int32_t* items, int32_t n, int32_t m,
                         int32_t bits, uint64_t seed, int32_t* fptr, int32_t* fitems,
                         uint32_t* fbits, DevHeader* hdr, int32_t* scan_tmp, cudaStream_t st) {
  if (bits < 32 || bits > kGfMaxBits || bits % 32) return C2_ERR_UNSUPPORTED;
  if (n == 0) return C2_OK;
  const uint64_t key = sm64_mix(seed ^ 0x474F4C4446494E47ull);
  const int smem = kGfWarps * (bits / 32) * 4;
  const int grid = (int)std::min<int64_t>(div_up(n, kGfWarps), (int64_t)num_sms() * 8);
  Sizes s = make_sizes(n, 0, m, 1, 1, 2, 2, nullptr);
  c2_status rc = run_validate(ptr, items, s, hdr, st);
  if (rc) return rc;
  C2_LAUNCH(k_gf_count, grid, 32 * kGfWarps, smem, st, ptr, items, n, key, (uint32_t)bits, fptr,
            hdr);
  C2_CUDA_TRY(scan_exclusive(fptr, fptr, n, scan_tmp, st));
  C2_LAUNCH(k_gf_emit, grid, 32 * kGfWarps, smem, st, ptr, items, n, key, (uint32_t)bits, fptr,
            fitems, fbits, hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
