// Count matrices of dense clusters on the 5th-generation tensor cores.
//
// For a cluster C of M members (internal order: decreasing profile length),
// G[p][q] = |P_p n P_q| is the (p, q) entry of A A^T, A the M x |I| 0/1 matrix
// of the members' profiles.  Only items held by at least two members change an
// entry off the diagonal, so A keeps those items' columns alone, renumbered
// 0 .. K2-1 in increasing item id (the cluster's "remap"), and the diagonal is
// written as the profile length.  0 and 1 are exact in FP8 E4M3 and every sum
// stays below 2^16, so tcgen05.mma.kind::f8f6f4 with FP32 accumulation gives
// the exact counts: the same uint16 matrices as the shared-memory table
// kernel, in the same internal order and row stride round_up(M, 8).
//
// Work item = (cluster, 128-row tile i, 256-column tile j) with 256(j+1) > 128 i
// (the matrix is symmetric: tiles wholly below the diagonal are skipped).
// One CTA per SM, persistent, items taken round-robin from a list sorted by
// decreasing cost.  Roles:
//   * 4 producer warps build the operands in shared memory from the remapped
//     lists: thread r owns row r of the A tile (128 rows) and rows r, r + 128
//     of the B tile (256 rows); per stage of 128 remapped columns it writes a
//     1.0 byte for each of its rows' entries in range, in the 128-byte swizzled
//     K-major layout the MMA descriptors describe, and records which 16-byte
//     chunks it touched; before refilling a stage it zeroes those chunks only,
//     so the cost follows the nonzeros, not the tile area;
//   * one thread issues tcgen05.mma (M = 128, N = 256, K = 32) into one of two
//     TMEM accumulators of 256 FP32 columns; a commit releases each stage;
//   * 8 epilogue warps (two per TMEM lane quadrant, one per 128-column half)
//     read the accumulator with tcgen05.ld, convert to uint16 and store the
//     row segment (16-byte stores) and, for columns past the row tile, the
//     mirrored column (32 consecutive rows per warp store).
// No TMA, no clusters: each CTA reads and writes only its own shared memory.
//
// Every mbarrier wait is bounded: after GT_WAIT_CYCLES, or once another role
// gave up, the kernel records C2_ERR_TIMEOUT, waits (again bounded) for the
// MMAs it issued, frees its TMEM and returns.
#include <algorithm>

#include "c2_internal.cuh"
#include "c2_tc.cuh"

namespace c2 {
namespace {

using namespace tc;

constexpr int GT_BM = 128;                       // rows per tile (TMEM lanes)
constexpr int GT_BN = 256;                       // columns per tile
constexpr int GT_BK = 128;                       // remapped columns per stage (128 B of FP8)
constexpr int GT_STAGES = 4;
constexpr int GT_A_BYTES = GT_BM * GT_BK;        // 16 KiB
constexpr int GT_B_BYTES = GT_BN * GT_BK;        // 32 KiB
constexpr int GT_STAGE_BYTES = GT_A_BYTES + GT_B_BYTES;
constexpr int GT_PROD_WARPS = 4;
constexpr int GT_MMA_WARP = GT_PROD_WARPS;       // warp 4
constexpr int GT_EPI_WARP0 = GT_MMA_WARP + 1;    // warps 5 .. 12
constexpr int GT_EPI_WARPS = 8;
constexpr int GT_THREADS = 32 * (GT_PROD_WARPS + 1 + GT_EPI_WARPS);
constexpr int GT_TMEM_COLS = 2 * GT_BN;
constexpr long long GT_WAIT_CYCLES = 4000000000LL;   // about 2 s
constexpr int GT_NBARS = 2 * GT_STAGES + 2 + 2 + 1;
constexpr size_t GT_SMEM = 1024 + (size_t)GT_STAGES * GT_STAGE_BYTES + GT_NBARS * 8;
constexpr uint8_t GT_ONE = 0x38;                 // 1.0 in FP8 E4M3

// Instruction descriptor, kind::f8f6f4: FP32 accumulator (bit 4), E4M3 A and
// B (format 0 at bits 7 and 10), both K-major, N >> 3 at bit 17, M >> 4 at 24.
constexpr uint32_t GT_IDESC =
    (1u << 4) | ((uint32_t)(GT_BN >> 3) << 17) | ((uint32_t)(GT_BM >> 4) << 24);

static_assert(GT_SMEM <= 232448, "stages must fit the shared memory of one CTA");

struct GtArgs {
  const int4* work;        // (cluster, row tile, column tile, stages of 128 columns)
  int32_t n_work;
  const int32_t* cptr;
  const int32_t* cusers;
  const int2* iinfo;       // internal slot -> (local index, profile length)
  const int32_t* pptr;     // padded CSR offsets: a user's list start within a function's area
  const uint16_t* rl;      // remapped lists [t][PN], ascending per (function, user)
  int64_t PN;
  int32_t n_users;
  const int32_t* rl_len;   // per slot: entries of its remapped list
  const int64_t* gofs;     // per cluster: offset of its count matrix
  uint16_t* gram;
  DevHeader* hdr;
  // bits mode (rl == NULL): the operand rows are the users' packed bit rows,
  // row_words 32-bit words each (bit b of word w = column 32w + b)
  const uint32_t* bits;
  int32_t row_words;
};

__device__ __forceinline__ bool gt_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                        bool check_abort) {
  return mbar_wait(bar, parity, abort_flag, check_abort, GT_WAIT_CYCLES);
}

__device__ __forceinline__ void gt_abort(volatile int* abort_flag, DevHeader* hdr) {
  *abort_flag = 1;
  dev_fail(hdr, C2_ERR_TIMEOUT);
}

// Byte offset of (row R, column c) in a K-major operand of 128-byte rows with
// the 128-byte swizzle: 8-row groups of 1024 bytes, the 16-byte chunk index
// XORed with the row's position in its group.
__device__ __forceinline__ uint32_t sw128_off(int R, int c) {
  return (uint32_t)((R >> 3) * 1024 + (R & 7) * 128 + ((((c >> 4) ^ R) & 7) << 4) + (c & 15));
}

// One operand row of the producer: its remapped list read four entries at a
// time (8-byte loads, the next four in flight).
struct RowList {
  const uint16_t* p;
  int n, cur, wb;
  uint2 w0, w1;
  __device__ __forceinline__ void start(const uint16_t* base, int len) {
    p = base;
    n = len;
    cur = 0;
    wb = 0;
    w0 = len > 0 ? __ldg(reinterpret_cast<const uint2*>(base)) : make_uint2(0, 0);
    w1 = len > 4 ? __ldg(reinterpret_cast<const uint2*>(base) + 1) : make_uint2(0, 0);
  }
  // Writes a 1.0 byte for every entry below `limit` (columns of this stage
  // start at limit - 128) into the row at `row_base` and returns the mask of
  // 16-byte chunks touched.
  __device__ __forceinline__ uint32_t fill(uint8_t* row_base, int R, int limit) {
    uint32_t mask = 0;
    while (cur < n) {
      if (cur >= wb + 4) {
        wb += 4;
        w0 = w1;
        w1 = wb + 4 < n ? __ldg(reinterpret_cast<const uint2*>(p + wb + 4)) : make_uint2(0, 0);
      }
      const int i = cur - wb;
      const uint32_t v = i < 2 ? w0.x : w0.y;
      const int x = (int)((i & 1) ? (v >> 16) : (v & 0xFFFFu));
      if (x >= limit) break;
      const int c = x & (GT_BK - 1);
      row_base[sw128_off(R, c)] = GT_ONE;
      mask |= 1u << (c >> 4);
      ++cur;
    }
    return mask;
  }
};

// One FP8 word of 0/1 values from 4 bits: byte i = 1.0 iff bit i (the four
// bits spread to bytes 0..3 by a multiply with no overlapping partial
// products, then scaled to 0x38).
__device__ __forceinline__ uint32_t nibble_fp8(uint32_t x) {
  return ((x * 0x00204081u) & 0x01010101u) * (uint32_t)GT_ONE;
}

// Writes the 128 columns of one stage of row R from 128 packed bits.
__device__ __forceinline__ void expand_row(uint8_t* tile, int R, uint4 b) {
  const uint32_t w[4] = {b.x, b.y, b.z, b.w};
  uint8_t* row = tile + (R >> 3) * 1024 + (R & 7) * 128;
#pragma unroll
  for (int j = 0; j < 8; ++j) {   // 16-byte chunk j = columns 16j .. 16j + 15
    const uint32_t v = w[j >> 1] >> (16 * (j & 1));
    *reinterpret_cast<uint4*>(row + (((j ^ R) & 7) << 4)) =
        make_uint4(nibble_fp8(v & 0xFu), nibble_fp8((v >> 4) & 0xFu), nibble_fp8((v >> 8) & 0xFu),
                   nibble_fp8((v >> 12) & 0xFu));
  }
}

// Zeroes the 16-byte chunks of row R named by `mask` (8 bits).
__device__ __forceinline__ void clear_chunks(uint8_t* tile, int R, uint32_t mask) {
  while (mask) {
    const int b = __ffs(mask) - 1;
    mask &= mask - 1;
    *reinterpret_cast<uint4*>(tile + (R >> 3) * 1024 + (R & 7) * 128 + (((b ^ R) & 7) << 4)) =
        make_uint4(0, 0, 0, 0);
  }
}

__global__ void __launch_bounds__(GT_THREADS, 1) k_gram_mma(GtArgs g) {
  extern __shared__ uint8_t gt_smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_sh, skip_sh;
  uint8_t* sm = (uint8_t*)(((uintptr_t)gt_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t s0 = su32(sm);
  const uint32_t bars = s0 + (uint32_t)GT_STAGES * GT_STAGE_BYTES;
  auto full = [&](int i) { return bars + 8u * i; };
  auto empty = [&](int i) { return bars + 8u * (GT_STAGES + i); };
  auto accfull = [&](int i) { return bars + 8u * (2 * GT_STAGES + i); };
  auto accempty = [&](int i) { return bars + 8u * (2 * GT_STAGES + 2 + i); };
  const uint32_t done = bars + 8u * (2 * GT_STAGES + 4);
  volatile int* abort_flag = &abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    skip_sh = dev_failed(g.hdr) ? 1 : 0;
    for (int i = 0; i < GT_STAGES; ++i) {
      mbar_init(full(i), GT_PROD_WARPS);
      mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(accfull(i), 1);
      mbar_init(accempty(i), GT_EPI_WARPS);
    }
    mbar_init(done, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // operands start at zero; producers only ever add and remove their bytes
  for (int i = threadIdx.x; i < GT_STAGES * GT_STAGE_BYTES / 16; i += GT_THREADS)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  if (skip_sh) return;   // a device error is already recorded: touch nothing
  if (warp == GT_MMA_WARP) tmem_alloc(su32(&tmem_slot), GT_TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp < GT_PROD_WARPS && !g.rl) {
    // ---------------- producers, bits mode: every stage of a row is 16 bytes
    // of its packed bits (the next stage's in flight), expanded in place
    const int r = threadIdx.x;   // A row r, B rows r and r + 128
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int idx = blockIdx.x; idx < g.n_work && ok; idx += gridDim.x) {
      const int4 wk = g.work[idx];
      const int c = wk.x, cbase = g.cptr[c], M = g.cptr[c + 1] - cbase;
      const uint4* src[3];
      const int pos[3] = {GT_BM * wk.y + r, GT_BN * wk.z + r, GT_BN * wk.z + GT_BM + r};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        src[q] = nullptr;
        if (pos[q] < M) {
          const int u = g.cusers[cbase + g.iinfo[cbase + pos[q]].x];
          src[q] = reinterpret_cast<const uint4*>(g.bits + (int64_t)u * g.row_words);
        }
      }
      uint4 cur[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) cur[q] = src[q] ? __ldg(src[q]) : make_uint4(0, 0, 0, 0);
      for (int kc = 0; kc < wk.w; ++kc) {
        uint4 nxt[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
          nxt[q] = (src[q] && kc + 1 < wk.w) ? __ldg(src[q] + kc + 1) : make_uint4(0, 0, 0, 0);
        const bool free_ok =
            __all_sync(0xffffffffu, gt_wait(empty(stage), phase ^ 1u, abort_flag, true));
        if (!free_ok) {
          if (lane == 0) gt_abort(abort_flag, g.hdr);
          ok = false;
          break;
        }
        uint8_t* A = sm + (size_t)stage * GT_STAGE_BYTES;
        uint8_t* B = A + GT_A_BYTES;
        expand_row(A, r, cur[0]);
        expand_row(B, r, cur[1]);
        expand_row(B, r + GT_BM, cur[2]);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(full(stage));
        if (++stage == GT_STAGES) stage = 0, phase ^= 1u;
#pragma unroll
        for (int q = 0; q < 3; ++q) cur[q] = nxt[q];
      }
    }
  } else if (warp < GT_PROD_WARPS) {
    // ---------------- producers, list mode
    const int r = threadIdx.x;   // A row r, B rows r and r + 128
    uint32_t masks[GT_STAGES];
#pragma unroll
    for (int i = 0; i < GT_STAGES; ++i) masks[i] = 0;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int idx = blockIdx.x; idx < g.n_work && ok; idx += gridDim.x) {
      const int4 wk = g.work[idx];
      const int c = wk.x, cbase = g.cptr[c], M = g.cptr[c + 1] - cbase;
      RowList rows[3];
      const int pos[3] = {GT_BM * wk.y + r, GT_BN * wk.z + r, GT_BN * wk.z + GT_BM + r};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (pos[q] < M) {
          const int slot = cbase + g.iinfo[cbase + pos[q]].x;
          const int u = g.cusers[slot];
          const int64_t f = slot / g.n_users;
          rows[q].start(g.rl + f * g.PN + g.pptr[u], g.rl_len[slot]);
        } else {
          rows[q].start(nullptr, 0);
        }
      }
      for (int kc = 0; kc < wk.w; ++kc) {
        const bool free_ok =
            __all_sync(0xffffffffu, gt_wait(empty(stage), phase ^ 1u, abort_flag, true));
        if (!free_ok) {
          if (lane == 0) gt_abort(abort_flag, g.hdr);
          ok = false;
          break;
        }
        uint8_t* A = sm + (size_t)stage * GT_STAGE_BYTES;
        uint8_t* B = A + GT_A_BYTES;
        // masks[i] belongs to the stage i steps ahead: masks[0] to this one
        const uint32_t m0 = masks[0];
        clear_chunks(A, r, m0 & 0xFFu);
        clear_chunks(B, r, (m0 >> 8) & 0xFFu);
        clear_chunks(B, r + GT_BM, (m0 >> 16) & 0xFFu);
        const int limit = (kc + 1) * GT_BK;
        uint32_t m1 = rows[0].fill(A, r, limit);
        m1 |= rows[1].fill(B, r, limit) << 8;
        m1 |= rows[2].fill(B, r + GT_BM, limit) << 16;
#pragma unroll
        for (int i = 0; i + 1 < GT_STAGES; ++i) masks[i] = masks[i + 1];
        masks[GT_STAGES - 1] = m1;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(full(stage));
        if (++stage == GT_STAGES) stage = 0, phase ^= 1u;
      }
    }
  } else if (warp == GT_MMA_WARP) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int t = 0;
      for (int idx = blockIdx.x; idx < g.n_work && ok; idx += gridDim.x, ++t) {
        const int nk = g.work[idx].w;
        const int a = t & 1;
        const uint32_t use = (uint32_t)(t >> 1);
        if (!gt_wait(accempty(a), (use & 1u) ^ 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(a * GT_BN);
        for (int kc = 0; kc < nk; ++kc) {
          if (!gt_wait(full(stage), phase, abort_flag, true)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t abase = s0 + (uint32_t)stage * GT_STAGE_BYTES;
          const uint32_t bbase = abase + GT_A_BYTES;
#pragma unroll
          for (int kk = 0; kk < GT_BK / 32; ++kk)
            umma_f8f6f4(d, sw128_desc(abase + kk * 32), sw128_desc(bbase + kk * 32), GT_IDESC,
                        (kc | kk) != 0 ? 1u : 0u);
          umma_commit(empty(stage));   // the stage is free once these MMAs finish
          if (++stage == GT_STAGES) stage = 0, phase ^= 1u;
        }
        if (!ok) break;
        umma_commit(accfull(a));
      }
      if (!ok) gt_abort(abort_flag, g.hdr);
      // every MMA issued by this thread has finished before TMEM is freed
      umma_commit(done);
      gt_wait(done, 0, abort_flag, false);
    }
  } else {
    // ---------------- epilogue: lane quadrant q (= warp % 4), column half h
    const int ew = warp - GT_EPI_WARP0;
    const int q = warp & 3, h = ew >> 2;
    int t = 0;
    for (int idx = blockIdx.x; idx < g.n_work; idx += gridDim.x, ++t) {
      const int a = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      // warp-uniform outcome: the TMEM loads below are warp-collective
      const bool ready =
          __all_sync(0xffffffffu, gt_wait(accfull(a), use & 1u, abort_flag, true));
      if (!ready) {
        if (lane == 0) gt_abort(abort_flag, g.hdr);
        break;
      }
      fence_after();
      const int4 wk = g.work[idx];
      const int c = wk.x, cbase = g.cptr[c], M = g.cptr[c + 1] - cbase, Mp = (M + 7) & ~7;
      uint16_t* G0 = g.gram + g.gofs[c];
      const int row = GT_BM * wk.y + 32 * q + lane;
      const bool row_ok = row < M;
      const uint32_t my_len = row_ok ? (uint32_t)g.iinfo[cbase + row].y : 0u;
      const int mirror_from = GT_BM * (wk.y + 1);   // columns past the row tile
      uint16_t* grow = G0 + (int64_t)row * Mp;
#pragma unroll 1
      for (int ch = 0; ch < 4; ++ch) {
        const int col0 = GT_BN * wk.z + 128 * h + 32 * ch;
        uint32_t v[32];
        tmem_ld32_async(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * GT_BN + 128 * h + 32 * ch), v);
        tmem_wait(v);
        if (col0 >= M) continue;   // warp-uniform
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          uint32_t x = (uint32_t)__float2uint_rn(__uint_as_float(v[e]));
          if (col0 + e == row) x = my_len;   // the diagonal: the profile length
          v[e] = x;
        }
        if (row_ok) {
#pragma unroll
          for (int g8 = 0; g8 < 4; ++g8)
            if (col0 + 8 * g8 < Mp)
              *reinterpret_cast<uint4*>(grow + col0 + 8 * g8) =
                  make_uint4(v[8 * g8] | (v[8 * g8 + 1] << 16), v[8 * g8 + 2] | (v[8 * g8 + 3] << 16),
                             v[8 * g8 + 4] | (v[8 * g8 + 5] << 16), v[8 * g8 + 6] | (v[8 * g8 + 7] << 16));
        }
        if (col0 + 32 > mirror_from && row_ok) {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int col = col0 + e;
            if (col >= mirror_from && col < M) G0[(int64_t)col * Mp + row] = (uint16_t)v[e];
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty(a));
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();   // every role is done with TMEM
  if (warp == GT_MMA_WARP) {
    fence_after();
    tmem_dealloc(tmem, GT_TMEM_COLS);
  }
}

// ---------------------------------------------------------------- remap
// Shared memory of the remap kernels: seen-once and seen-twice bitsets over
// the item universe, plus (k_remap) the rank of each bitset word.
__host__ __device__ inline int item_words(int m) { return (m + 31) / 32; }

// Marks the items of every member of cluster c: seen1 = held by one member or
// more, seen2 = held by two or more.
__device__ void mark_items(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items,
                           const int32_t* __restrict__ cusers, int cbase, int M, uint32_t* seen1,
                           uint32_t* seen2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = warp; l < M; l += nw) {
    const int u = cusers[cbase + l];
    for (int e = ptr[u] + lane; e < ptr[u + 1]; e += 32) {
      const int x = items[e];
      const uint32_t bit = 1u << (x & 31);
      if (atomicOr(&seen1[x >> 5], bit) & bit) atomicOr(&seen2[x >> 5], bit);
    }
  }
}

__device__ __forceinline__ int block_sum(int v, int* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int s = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Per candidate cluster (count-matrix index g of `list`): K2[g] = items held
// by at least two members, and the members' total profile length.
__global__ void __launch_bounds__(1024) k_remap_count(
    const int32_t* __restrict__ list, int32_t nlist, int32_t min_m, const int32_t* __restrict__ gsz,
    const int32_t* __restrict__ gcl, const int32_t* __restrict__ cptr,
    const int32_t* __restrict__ cusers, const int32_t* __restrict__ ptr,
    const int32_t* __restrict__ items, int32_t m, int32_t whole, int32_t* __restrict__ k2,
    int64_t* __restrict__ sumlen, DevHeader* hdr) {
  extern __shared__ uint32_t rm_sh[];
  __shared__ int red[32];
  if (blockIdx.x >= nlist || dev_failed(hdr)) return;
  const int gi = list ? list[blockIdx.x] : (int)blockIdx.x;
  if (gsz[gi] < min_m) {
    if (threadIdx.x == 0) {
      k2[gi] = -1;
      sumlen[gi] = 0;
    }
    return;
  }
  const int c = gcl[gi];
  const int cbase = cptr[c], M = cptr[c + 1] - cbase;
  int cnt = 0, len = 0;
  if (whole) {
    // whole rows (bits mode): every column is an operand column
    if (threadIdx.x == 0) cnt = m;
  } else {
    const int W = item_words(m);
    uint32_t* seen1 = rm_sh;
    uint32_t* seen2 = rm_sh + W;
    for (int i = threadIdx.x; i < 2 * W; i += blockDim.x) rm_sh[i] = 0;
    __syncthreads();
    mark_items(ptr, items, cusers, cbase, M, seen1, seen2);
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) cnt += __popc(seen2[i]);
  }
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    const int u = cusers[cbase + l];
    len += ptr[u + 1] - ptr[u];
  }
  cnt = block_sum(cnt, red);
  len = block_sum(len, red);
  if (threadIdx.x == 0) {
    k2[gi] = cnt;
    sumlen[gi] = len;
  }
}

// Remapped lists of the members of each cluster of `list`: for member slot s
// (user u, function f = s / n), rl[f * PN + pptr[u] + j] = the rank among the
// cluster's seen-twice items of u's j-th such item (ascending), rl_len[s] =
// their number.
__global__ void __launch_bounds__(1024) k_remap(
    const int32_t* __restrict__ list, int32_t nlist, const int32_t* __restrict__ gcl,
    const int32_t* __restrict__ cptr, const int32_t* __restrict__ cusers,
    const int32_t* __restrict__ ptr, const int32_t* __restrict__ items, int32_t m,
    const int32_t* __restrict__ pptr, int64_t PN, int32_t n, uint16_t* __restrict__ rl,
    int32_t* __restrict__ rl_len, DevHeader* hdr) {
  extern __shared__ uint32_t rm_sh[];
  __shared__ int wsum[32];
  if (blockIdx.x >= nlist || dev_failed(hdr)) return;
  const int gi = list[blockIdx.x], c = gcl[gi];
  const int cbase = cptr[c], M = cptr[c + 1] - cbase;
  const int W = item_words(m);
  uint32_t* seen1 = rm_sh;
  uint32_t* seen2 = rm_sh + W;
  int32_t* rank = reinterpret_cast<int32_t*>(rm_sh + 2 * W);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < 2 * W; i += blockDim.x) rm_sh[i] = 0;
  __syncthreads();
  mark_items(ptr, items, cusers, cbase, M, seen1, seen2);
  __syncthreads();
  // rank[w] = seen-twice items in words before w: each thread scans a
  // contiguous range of words, then the ranges' totals are scanned
  const int per = (W + blockDim.x - 1) / blockDim.x;
  const int w0 = tid * per, w1 = min(W, w0 + per);
  int loc = 0;
  for (int w = w0; w < w1; ++w) loc += __popc(seen2[w]);
  int incl = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) wsum[lane] = v;   // inclusive totals per warp
  }
  __syncthreads();
  int run = incl - loc + (warp > 0 ? wsum[warp - 1] : 0);
  for (int w = w0; w < w1; ++w) {
    rank[w] = run;
    run += __popc(seen2[w]);
  }
  __syncthreads();
  // one warp per member: 32 items at a time, seen-twice items compacted in order
  for (int l = warp; l < M; l += nw) {
    const int s = cbase + l, u = cusers[s];
    uint16_t* out = rl + (int64_t)(s / n) * PN + pptr[u];
    int cnt = 0;
    for (int e0 = ptr[u]; e0 < ptr[u + 1]; e0 += 32) {
      const int e = e0 + lane;
      int x = 0;
      bool keep = false;
      if (e < ptr[u + 1]) {
        x = items[e];
        keep = (seen2[x >> 5] >> (x & 31)) & 1u;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int r = rank[x >> 5] + __popc(seen2[x >> 5] & ((1u << (x & 31)) - 1u));
        out[cnt + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)r;
      }
      cnt += __popc(bal);
    }
    if (lane == 0) rl_len[s] = cnt;
  }
}

}  // namespace

static_assert(12 * (kGramTcMaxItems / 32) + 1024 <= 232448,
              "the remap bitsets and ranks must fit the shared memory of one CTA");

c2_status gram_tc_count(const int32_t* list, int nlist, int min_m, const int32_t* gsz,
                        const int32_t* gcl, const int32_t* cptr, const int32_t* cusers,
                        const int32_t* ptr, const int32_t* items, int m, bool whole, int32_t* k2,
                        int64_t* sumlen, DevHeader* hdr, cudaStream_t st) {
  if (nlist <= 0) return C2_OK;
  if (m > kGramTcMaxItems) return C2_ERR_UNSUPPORTED;
  const int smem = whole ? 0 : 8 * item_words(m);
  C2_CUDA_TRY(cudaFuncSetAttribute(k_remap_count, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  C2_LAUNCH(k_remap_count, nlist, whole ? 256 : 1024, smem, st, list, nlist, min_m, gsz, gcl, cptr,
            cusers, ptr, items, m, whole ? 1 : 0, k2, sumlen, hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status gram_tc_remap(const int32_t* list, int nlist, const int32_t* gcl, const int32_t* cptr,
                        const int32_t* cusers, const int32_t* ptr, const int32_t* items, int m,
                        const int32_t* pptr, int64_t PN, int n, uint16_t* rl, int32_t* rl_len,
                        DevHeader* hdr, cudaStream_t st) {
  if (nlist <= 0) return C2_OK;
  if (m > kGramTcMaxItems) return C2_ERR_UNSUPPORTED;
  const int smem = 12 * item_words(m);
  C2_CUDA_TRY(cudaFuncSetAttribute(k_remap, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  C2_LAUNCH(k_remap, nlist, 1024, smem, st, list, nlist, gcl, cptr, cusers, ptr, items, m, pptr,
            PN, n, rl, rl_len, hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status gram_tc_run(const int4* work, int n_work, const int32_t* cptr, const int32_t* cusers,
                      const int2* iinfo, const int32_t* pptr, const uint16_t* rl, int64_t PN,
                      int n, const int32_t* rl_len, const int64_t* gofs, uint16_t* gram,
                      const uint32_t* bits, int row_words, DevHeader* hdr, cudaStream_t st) {
  if (n_work <= 0) return C2_OK;
  if (rl && (((uintptr_t)rl & 7u) || (PN & 3))) return C2_ERR_INVALID_ARG;
  if (!rl && (!bits || ((uintptr_t)bits & 15u) || row_words % 4)) return C2_ERR_INVALID_ARG;
  GtArgs g;
  g.work = work;
  g.n_work = n_work;
  g.cptr = cptr;
  g.cusers = cusers;
  g.iinfo = iinfo;
  g.pptr = pptr;
  g.rl = rl;
  g.PN = PN;
  g.n_users = n;
  g.rl_len = rl_len;
  g.gofs = gofs;
  g.gram = gram;
  g.hdr = hdr;
  g.bits = bits;
  g.row_words = row_words;
  C2_CUDA_TRY(cudaFuncSetAttribute(k_gram_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)GT_SMEM));
  const int grid = std::min(num_sms(), n_work);
  C2_LAUNCH(k_gram_mma, grid, GT_THREADS, GT_SMEM, st, g);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

int gram_tc_tile_rows() { return GT_BM; }
int gram_tc_tile_cols() { return GT_BN; }
int gram_tc_stage_cols() { return GT_BK; }

}  // namespace c2
