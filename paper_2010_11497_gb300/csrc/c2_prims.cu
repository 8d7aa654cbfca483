// Device-wide primitives: exclusive prefix sum and stable LSD radix sort.
#include "c2_internal.cuh"

namespace c2 {

namespace {

constexpr int kScanNT = 1024;
constexpr int kScanIPT = 4;
constexpr int kScanTile = kScanNT * kScanIPT;

// Block-local exclusive scan of one 4096-element tile; writes the tile total.
template <class T>
__global__ void __launch_bounds__(kScanNT) k_scan_tile(const T* in, T* out, int64_t n, T* bsum,
                                                       T* total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanIPT;
  T v[kScanIPT];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanIPT; ++i) {
    v[i] = (base + i < n) ? in[base + i] : T(0);
    s += v[i];
  }
  T x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    T tsum = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, tsum, o);
      if (lane >= o) tsum += y;
    }
    warp_tot[lane] = tsum;
  }
  __syncthreads();
  T excl = x - s + (w > 0 ? warp_tot[w - 1] : T(0));
#pragma unroll
  for (int i = 0; i < kScanIPT; ++i) {
    if (base + i < n) out[base + i] = excl;
    excl += v[i];
  }
  if (threadIdx.x == kScanNT - 1) {
    bsum[blockIdx.x] = warp_tot[31];
    if (total) *total = warp_tot[31];    // single-tile scans: out[n]
  }
}

// Second pass of a two-launch scan: each block adds the sum of the tile
// totals before it (a block reduction over at most kScanFlat values) to its
// tile; the last block writes out[n].
constexpr int kScanFlat = 8192;

template <class T>
__global__ void __launch_bounds__(256) k_scan_add_flat(T* out, int64_t n, const T* bsum, int nb) {
  __shared__ T red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T acc = 0;
  for (int j = threadIdx.x; j < (int)blockIdx.x; j += 256) acc += bsum[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  T add = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) add += red[w];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  constexpr int V = 16 / sizeof(T);   // elements per 16-byte access
  if (base + kScanTile <= n && (reinterpret_cast<uintptr_t>(out + base) & 15) == 0) {
    // a whole, aligned tile: 16-byte loads and stores
    uint4* o4 = reinterpret_cast<uint4*>(out + base);
    for (int i = threadIdx.x; i < kScanTile / V; i += 256) {
      uint4 q = o4[i];
      T* e = reinterpret_cast<T*>(&q);
#pragma unroll
      for (int v = 0; v < V; ++v) e[v] += add;
      o4[i] = q;
    }
  } else {
    for (int i = threadIdx.x; i < kScanTile; i += 256)
      if (base + i < n) out[base + i] += add;
  }
  if ((int)blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = add + bsum[nb - 1];
}

template <class T>
__global__ void k_scan_add(T* out, int64_t n, const T* boff) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const T add = boff[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
    if (base + i < n) out[base + i] += add;
}

template <class T>
__global__ void k_store_total(T* dst, const T* src) { *dst = *src; }

template <class T>
cudaError_t scan_impl(const T* in, T* out, int64_t n, T* tmp, cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(T), st);
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  T* bsum = tmp;
  // one tile: one launch; up to kScanFlat tiles: two launches
  C2_LAUNCH(k_scan_tile<T>, (unsigned)nb, kScanNT, 0, st, in, out, n, bsum,
            nb == 1 ? out + n : (T*)nullptr);
  if (nb == 1) return cudaGetLastError();
  if (nb <= kScanFlat) {
    C2_LAUNCH(k_scan_add_flat<T>, (unsigned)nb, 256, 0, st, out, n, (const T*)bsum, (int)nb);
    return cudaGetLastError();
  }
  {
    const int64_t used = ((nb + 1 + 63) / 64) * 64;
    cudaError_t e = scan_impl<T>(bsum, bsum, nb, tmp + used, st);
    if (e != cudaSuccess) return e;
    C2_LAUNCH(k_scan_add<T>, (unsigned)nb, 256, 0, st, out, n, bsum);
    C2_LAUNCH(k_store_total<T>, 1, 1, 0, st, out + n, bsum + nb);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
constexpr int kRsNT = 256;
constexpr int kRsIPT = 8;
constexpr int kRsTile = kRsNT * kRsIPT;   // 2048 keys per tile; warp w owns 256 consecutive

__global__ void __launch_bounds__(kRsNT) k_rs_upsweep(const uint32_t* keys, int64_t n, int shift,
                                                     int32_t* hist, int ntiles) {
  __shared__ int32_t h[256];
  for (int d = threadIdx.x; d < 256; d += kRsNT) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
  for (int r = 0; r < kRsIPT; ++r) {
    int64_t idx = base + r * kRsNT + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kRsNT) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: element order inside a tile is preserved per digit.
__global__ void __launch_bounds__(kRsNT) k_rs_downsweep(const uint32_t* kin, const int32_t* vin,
                                                       uint32_t* kout, int32_t* vout, int64_t n,
                                                       int shift, const int32_t* offs,
                                                       int ntiles) {
  __shared__ int32_t whist[8][257];
  __shared__ int32_t wbase[8][257];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < 8 * 257; d += kRsNT) (&whist[0][0])[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * (kRsTile / 8);
  uint32_t key[kRsIPT];
  int32_t val[kRsIPT], rank[kRsIPT], dig[kRsIPT];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kRsIPT; ++r) {
    const int64_t idx = base + r * 32 + lane;
    const bool ok = idx < n;
    key[r] = ok ? kin[idx] : 0u;
    val[r] = ok ? vin[idx] : 0;
    const int d = ok ? (int)((key[r] >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = __popc(peers & lt);
    const int old = whist[warp][d];
    __syncwarp();
    if (before == 0) whist[warp][d] = old + __popc(peers);
    __syncwarp();
    rank[r] = old + before;
    dig[r] = d;
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      wbase[w][threadIdx.x] = s;
      s += whist[w][threadIdx.x];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsIPT; ++r) {
    if (dig[r] < 256) {
      const int64_t pos = (int64_t)offs[(int64_t)dig[r] * ntiles + blockIdx.x] +
                          wbase[warp][dig[r]] + rank[r];
      kout[pos] = key[r];
      vout[pos] = val[r];
    }
  }
}

}  // namespace

size_t scan_tmp_elems(int64_t n) {
  size_t total = 64;
  while (n > kScanTile) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    total += ((nb + 1 + 63) / 64) * 64;
    n = nb;
  }
  return total + 64;
}

size_t sort_hist_elems(int64_t n) {
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  return (size_t)(256 * ntiles + 1);
}

cudaError_t scan_exclusive(const int32_t* d_in, int32_t* d_out, int64_t n, int32_t* tmp,
                           cudaStream_t st) {
  return scan_impl<int32_t>(d_in, d_out, n, tmp, st);
}

cudaError_t scan_exclusive64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* tmp,
                             cudaStream_t st) {
  return scan_impl<int64_t>(d_in, d_out, n, tmp, st);
}

cudaError_t radix_sort_pairs(uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int64_t n,
                             int bits, uint32_t* hist, int32_t* scan_tmp, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
  int32_t* h = reinterpret_cast<int32_t*>(hist);
  bool flipped = false;
  for (int shift = 0; shift < bits; shift += 8) {
    uint32_t* ki = flipped ? k1 : k0;
    int32_t* vi = flipped ? v1 : v0;
    uint32_t* ko = flipped ? k0 : k1;
    int32_t* vo = flipped ? v0 : v1;
    C2_LAUNCH(k_rs_upsweep, ntiles, kRsNT, 0, st, ki, n, shift, h, ntiles);
    cudaError_t e = scan_exclusive(h, h, (int64_t)256 * ntiles, scan_tmp, st);
    if (e != cudaSuccess) return e;
    C2_LAUNCH(k_rs_downsweep, ntiles, kRsNT, 0, st, ki, vi, ko, vo, n, shift, h, ntiles);
    flipped = !flipped;
  }
  if (flipped) {
    cudaMemcpyAsync(k0, k1, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v0, v1, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError();
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace c2
