// Logits GEMM of the learned proposer on the 5th-generation tensor cores,
// with the per-slice (max, argmax) fused into the epilogue.
//
// For rows r < M and column slices s of 128 columns:
//   part[r][s] = (max_j z[r][j], argmax_j z[r][j]),  j in [s*128, s*128 + 128),
//   z[r][j] = sum_k A[r][k] * Bt[j][k] + bias[j]
// with BF16 operands, FP32 accumulation and ties to the lower column.  A is
// the hidden layer h (row-major [M][K]) and Bt the transposed output weights
// (row-major [N][K]), so both operands are K-major.
//
// Structure (one CTA per SM, persistent, clusters of two CTAs): the two CTAs
// of a cluster walk the same contiguous range of (slice pair, row tile) work
// items, CTA rank r taking slice 2p + r of pair p.  A slice's 256 x K block of
// Bt stays resident in shared memory (loaded by TMA once per slice); 128-row
// tiles of A stream through a ring of stages of 128 x 64, each CTA loading
// 64 of the rows and multicasting them to both CTAs, so A crosses from L2
// once per pair of slices (A traffic, not the tensor pipe, bounds the
// single-CTA form of this kernel).  A stage is refilled once the MMAs of both
// CTAs have released it (their commits arrive on both CTAs' barriers).  One
// thread issues tcgen05.mma (M = 128, N = 256, K = 16) into one of two TMEM
// accumulators of 256 FP32 columns, so the epilogue of a tile overlaps the
// MMAs of the next.  Eight epilogue warps (two per 32-lane TMEM quadrant,
// one per 128-column half) read their rows with tcgen05.ld, add the bias and
// reduce each row's half to (max, argmax).
//
// Every mbarrier wait is bounded: after TC_WAIT_CYCLES, or once another role
// gave up, the kernel records C2_ERR_TIMEOUT in the status word, waits (again
// bounded) for its own copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "c2_internal.cuh"

namespace c2 {
namespace {

constexpr int TC_BM = 128;                     // rows per tile = TMEM lanes
constexpr int TC_BN = 256;                     // columns per slice
constexpr int TC_BK = 64;                      // K per TMA box: one 128-byte swizzle row
constexpr int TC_KMAX = 256;
constexpr int TC_STAGES = 6;
constexpr int TC_CLUSTER = 2;                  // CTAs sharing each A tile (multicast)
constexpr int TC_A_STAGE = TC_BM * TC_BK * 2;  // 16 KiB
constexpr int TC_B_CHUNK = TC_BN * TC_BK * 2;  // 32 KiB
constexpr int TC_EPI_WARPS = 8;                // two per TMEM lane quadrant
constexpr int TC_EPI_COLS = TC_BN / 2;         // columns per epilogue warp (one partial)
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;   // producer, MMA, epilogue warps
constexpr int TC_TMEM_COLS = 2 * TC_BN;        // two accumulators
constexpr long long TC_WAIT_CYCLES = 4000000000LL;   // about 2 s
constexpr int TC_NBARS = 2 * TC_STAGES + 2 + 2 + 2 + 1;
constexpr size_t TC_SMEM =
    1024 + (size_t)(TC_KMAX / TC_BK) * TC_B_CHUNK + (size_t)TC_STAGES * TC_A_STAGE + TC_NBARS * 8;

struct TcArgs {
  const float* bias;   // [N]
  float2* part;        // [M][2S]: one partial per half slice
  int32_t* status;     // device status word
  int M, K, S, MT;
  long long total;     // S * MT work items
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of `parity` to complete; false on timeout or when the
// CTA is aborting (check_abort).
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       bool check_abort) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (check_abort && *abort_flag) return false;
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void tc_abort(volatile int* abort_flag, int32_t* status) {
  *abort_flag = 1;
  atomicCAS(status, 0, (int32_t)C2_ERR_TIMEOUT);
}

// Multicast form: the box lands at the same offset in the shared memory of
// every CTA in `mask`, and complete_tx is signalled on each one's barrier at
// the offset of `bar`.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                               uint32_t bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3}], [%4], %5;\n" ::"r"(dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that TMA writes: rows of 128 bytes, 8-row groups 1024
// bytes apart (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   bar)
               : "memory");
}
// Arrives on the barrier at offset `bar` of every CTA in `mask` once this
// thread's MMAs so far have finished.
__device__ __forceinline__ void umma_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;\n" ::"r"(bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::
                   : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

#define TC_R32(r)                                                                              \
  "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), \
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),           \
      "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]),          \
      "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]),          \
      "r"(r[30]), "r"(r[31])

// Starts loading 32 consecutive FP32 columns of this warp's 32 TMEM lanes;
// the registers are valid after tmem_wait(r) on the same array.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// Waits for this thread's TMEM loads; the in/out operands keep every use of
// r after the wait.
__device__ __forceinline__ void tmem_wait(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Running (max, argmax) over 32 columns col..col+31 (ascending, so ties keep
// the lower column) with their bias.
__device__ __forceinline__ void tc_scan32(const uint32_t* r, const float* __restrict__ bias, int col,
                                          float& best, int& arg) {
  const float4* b4 = reinterpret_cast<const float4*>(bias + col);
#pragma unroll
  for (int j4 = 0; j4 < 8; ++j4) {
    const float4 bb = __ldg(b4 + j4);
    const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float z = __uint_as_float(r[4 * j4 + e]) + bv[e];
      if (z > best) {
        best = z;
        arg = col + 4 * j4 + e;
      }
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_logits_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                TcArgs g) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_sh;
  uint8_t* sm = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  const int KC = g.K / TC_BK;
  const uint32_t sB = su32(sm);
  const uint32_t sA = sB + (uint32_t)(TC_KMAX / TC_BK) * TC_B_CHUNK;
  const uint32_t bars = sA + (uint32_t)TC_STAGES * TC_A_STAGE;
  auto afull = [&](int i) { return bars + 8u * i; };
  auto aempty = [&](int i) { return bars + 8u * (TC_STAGES + i); };
  const uint32_t bfull = bars + 8u * (2 * TC_STAGES);
  const uint32_t bempty = bfull + 8;
  auto accfull = [&](int i) { return bempty + 8u + 8u * i; };
  auto accempty = [&](int i) { return bempty + 24u + 8u * i; };
  const uint32_t bdone = bempty + 40;
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int pair = blockIdx.x / TC_CLUSTER, npairs = gridDim.x / TC_CLUSTER;
  const long long lo = g.total * pair / npairs;
  const long long hi = g.total * (pair + 1) / npairs;
  constexpr uint16_t kMask = (1u << TC_CLUSTER) - 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_STAGES; ++i) {
      mbar_init(afull(i), 1);
      mbar_init(aempty(i), TC_CLUSTER);
    }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(accfull(i), 1);
      mbar_init(accempty(i), TC_EPI_WARPS);
    }
    mbar_init(bdone, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32(&tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  __syncwarp();
  tc_fence_before();
  cluster_sync_all();   // barriers of both CTAs initialised before any multicast
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int cur_s = -1, nb = 0, stage = 0;
    uint32_t phase = 0;
    int issued[TC_STAGES];
    uint32_t last_par[TC_STAGES];
    for (int i = 0; i < TC_STAGES; ++i) issued[i] = 0, last_par[i] = 0;
    bool ok = true;
    for (long long idx = lo; idx < hi && ok; ++idx) {
      const int s = TC_CLUSTER * (int)(idx / g.MT) + rank, m = (int)(idx % g.MT);
      if (s != cur_s) {
        if (nb > 0 && !mbar_wait(bempty, (uint32_t)(nb - 1) & 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        mbar_expect_tx(bfull, (uint32_t)(KC * TC_B_CHUNK));
        for (int kc = 0; kc < KC; ++kc)
          tma_load_2d(sB + (uint32_t)kc * TC_B_CHUNK, &tmB, kc * TC_BK, s * TC_BN, bfull);
        cur_s = s;
        ++nb;
      }
      for (int kc = 0; kc < KC; ++kc) {
        if (!mbar_wait(aempty(stage), phase ^ 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        // this CTA's rows of the tile, to both CTAs; the barrier counts both parts
        mbar_expect_tx(afull(stage), (uint32_t)TC_A_STAGE);
        tma_load_2d_mc(sA + (uint32_t)stage * TC_A_STAGE + (uint32_t)rank * (TC_A_STAGE / TC_CLUSTER),
                       &tmA, kc * TC_BK, m * TC_BM + rank * (TC_BM / TC_CLUSTER), afull(stage), kMask);
        issued[stage] = 1;
        last_par[stage] = phase;
        if (++stage == TC_STAGES) stage = 0, phase ^= 1u;
      }
    }
    if (!ok) {
      tc_abort(abort_flag, g.status);
      // let the copies already issued land before the CTA exits
      for (int i = 0; i < TC_STAGES; ++i)
        if (issued[i]) mbar_wait(afull(i), last_par[i], abort_flag, false);
      if (nb > 0) mbar_wait(bfull, (uint32_t)(nb - 1) & 1u, abort_flag, false);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int cur_s = -1, nb = 0, stage = 0;
    uint32_t phase = 0;
    long long t = 0;
    bool ok = true;
    for (long long idx = lo; idx < hi && ok; ++idx, ++t) {
      const int s = TC_CLUSTER * (int)(idx / g.MT) + rank;
      if (s != cur_s) {
        if (nb > 0) umma_commit(bempty);   // the old slice is free once its MMAs finish
        if (!mbar_wait(bfull, (uint32_t)nb & 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        tc_fence_after();
        cur_s = s;
        ++nb;
      }
      const int a = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      if (!mbar_wait(accempty(a), (use & 1u) ^ 1u, abort_flag, true)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(a * TC_BN);
      for (int kc = 0; kc < KC; ++kc) {
        if (!mbar_wait(afull(stage), phase, abort_flag, true)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t abase = sA + (uint32_t)stage * TC_A_STAGE;
        const uint32_t bbase = sB + (uint32_t)kc * TC_B_CHUNK;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)
          umma_bf16(d, sw128_desc(abase + kk * 32), sw128_desc(bbase + kk * 32),
                    (kc | kk) != 0 ? 1u : 0u);
        umma_commit_mc(aempty(stage), kMask);   // released in both CTAs once these MMAs finish
        if (++stage == TC_STAGES) stage = 0, phase ^= 1u;
      }
      if (!ok) break;
      umma_commit(accfull(a));
    }
    if (!ok) tc_abort(abort_flag, g.status);
    // every MMA issued by this thread has finished before TMEM is freed
    umma_commit(bdone);
    mbar_wait(bdone, 0, abort_flag, false);
  } else if (warp >= 2) {
    // ---------------- epilogue: rows 32q .. 32q + 31, columns h*128 .. h*128 + 127
    const int q = warp & 3, h = (warp - 2) >> 2;
    long long t = 0;
    for (long long idx = lo; idx < hi; ++idx, ++t) {
      const int s = TC_CLUSTER * (int)(idx / g.MT) + rank, m = (int)(idx % g.MT);
      const int a = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      // warp-uniform outcome: the TMEM loads below are warp-collective
      const bool ready = __all_sync(0xffffffffu, mbar_wait(accfull(a), use & 1u, abort_flag, true));
      if (!ready) {
        if (lane == 0) tc_abort(abort_flag, g.status);
        break;
      }
      tc_fence_after();
      float best = -INFINITY;
      int arg = 0x7fffffff;
      const int col0 = s * TC_BN + h * TC_EPI_COLS;
      const uint32_t tbase =
          tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * TC_BN + h * TC_EPI_COLS);
      uint32_t ra[32], rb[32];
      // four chunks of 32 columns, the next chunk's load in flight
      tmem_ld32_async(tbase, ra);
      tmem_wait(ra);
      tmem_ld32_async(tbase + 32, rb);
      tc_scan32(ra, g.bias, col0, best, arg);
      tmem_wait(rb);
      tmem_ld32_async(tbase + 64, ra);
      tc_scan32(rb, g.bias, col0 + 32, best, arg);
      tmem_wait(ra);
      tmem_ld32_async(tbase + 96, rb);
      tc_scan32(ra, g.bias, col0 + 64, best, arg);
      tmem_wait(rb);
      tc_scan32(rb, g.bias, col0 + 96, best, arg);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty(a));
      const int row = m * TC_BM + 32 * q + lane;
      if (row < g.M)
        g.part[(int64_t)row * (2 * g.S) + 2 * s + h] = make_float2(best, __int_as_float(arg));
    }
  }
  __syncwarp();          // lane 0 of the producer and MMA warps rejoins its warp
  tc_fence_before();
  cluster_sync_all();   // no multicast copy or commit of the peer still targets this CTA
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

// Bt[j][k] = B[k][j] (BF16), 32 x 32 tiles through shared memory.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ B, int K, int N,
                                 __nv_bfloat16* __restrict__ Bt) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int n0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, n = n0 + threadIdx.x;
    if (k < K && n < N) tile[r][threadIdx.x] = B[(int64_t)k * N + n];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, k = k0 + threadIdx.x;
    if (k < K && n < N) Bt[(int64_t)n * K + k] = tile[threadIdx.x][r];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D BF16 map over a row-major [rows][K] matrix, boxes of 64 x box_rows,
// 128-byte swizzle (the layout sw128_desc describes).
bool make_map(CUtensorMap* tm, const void* base, int K, int rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_logits_ok(int K, int N, int b) {
  return K >= TC_BK && K <= TC_KMAX && K % TC_BK == 0 && N % (TC_CLUSTER * TC_BN) == 0 &&
         b % TC_EPI_COLS == 0;
}
int tc_slice_width() { return TC_EPI_COLS; }

c2_status tc_transpose_bf16(const __nv_bfloat16* B, int K, int N, __nv_bfloat16* Bt,
                            cudaStream_t st) {
  dim3 grid(div_up(N, 32), div_up(K, 32)), block(32, 8);
  C2_LAUNCH(k_transpose_bf16, grid, block, 0, st, B, K, N, Bt);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status tc_logits_argmax(const __nv_bfloat16* A, int M, int K, const __nv_bfloat16* Bt, int N,
                           const float* bias, float2* part, int32_t* status, cudaStream_t st) {
  if (M <= 0) return C2_OK;
  if (K < TC_BK || K > TC_KMAX || K % TC_BK || N % (TC_CLUSTER * TC_BN)) return C2_ERR_UNSUPPORTED;
  if (((uintptr_t)A & 15u) || ((uintptr_t)Bt & 15u)) return C2_ERR_INVALID_ARG;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, A, K, M, TC_BM / TC_CLUSTER) || !make_map(&tmB, Bt, K, N, TC_BN))
    return C2_ERR_CUDA;
  TcArgs g;
  g.bias = bias;
  g.part = part;
  g.status = status;
  g.M = M;
  g.K = K;
  g.S = N / TC_BN;
  g.MT = div_up(M, TC_BM);
  g.total = (long long)(g.S / TC_CLUSTER) * g.MT;   // (slice pair, row tile) items
  C2_CUDA_TRY(cudaFuncSetAttribute(k_logits_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)TC_SMEM));
  const int pairs = (int)std::min<long long>(num_sms() / TC_CLUSTER, g.total);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pairs * TC_CLUSTER);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = TC_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = TC_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  C2_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_logits_tc, tmA, tmB, g));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return C2_OK;
}

}  // namespace c2
