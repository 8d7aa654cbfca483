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
// Structure (one CTA per SM, persistent, no clusters): each CTA walks a
// contiguous range of (256-column slice, 128-row tile) work items, slice
// major.  The slice's 256 x K block of Bt stays resident in shared memory
// (loaded by TMA once per slice); 128-row tiles of A stream through a ring of
// stages of 128 x 64, each CTA loading its own tiles.  A stage is refilled
// once the MMAs that read it have completed (their commit arrives on the
// stage's barrier).  One thread issues tcgen05.mma (M = 128, N = 256,
// K = 16) into one of two TMEM accumulators of 256 FP32 columns, so the
// epilogue of a tile overlaps the MMAs of the next.  Eight epilogue warps
// (two per 32-lane TMEM quadrant, one per 128-column half) read their rows
// with tcgen05.ld, add the bias and reduce each row's half to (max, argmax).
//
// Every mbarrier wait is bounded: after TC_WAIT_CYCLES, or once another role
// gave up, the kernel records C2_ERR_TIMEOUT in the status word, waits (again
// bounded) for its own copies and MMAs in flight, frees its TMEM and returns.
#include <algorithm>
#include <mutex>

#include "c2_internal.cuh"
#include "c2_tc.cuh"

namespace c2 {
namespace {

using namespace tc;

constexpr int TC_BM = 128;                     // rows per tile = TMEM lanes
constexpr int TC_BN = 256;                     // columns per slice
constexpr int TC_BK = 64;                      // K per TMA box: one 128-byte swizzle row
constexpr int TC_KMAX = 256;
constexpr int TC_STAGES = 6;
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

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                        bool check_abort) {
  return mbar_wait(bar, parity, abort_flag, check_abort, TC_WAIT_CYCLES);
}

__device__ __forceinline__ void tc_abort(volatile int* abort_flag, int32_t* status) {
  *abort_flag = 1;
  atomicCAS(status, 0, (int32_t)C2_ERR_TIMEOUT);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

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
  const long long lo = g.total * blockIdx.x / gridDim.x;
  const long long hi = g.total * (blockIdx.x + 1) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_STAGES; ++i) {
      mbar_init(afull(i), 1);
      mbar_init(aempty(i), 1);
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
    prefetch_map(&tmA);
    prefetch_map(&tmB);
  }
  if (warp == 1) tmem_alloc(su32(&tmem_slot), TC_TMEM_COLS);
  __syncwarp();
  fence_before();
  __syncthreads();   // barriers initialised and TMEM allocated before any role starts
  fence_after();
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
      const int s = (int)(idx / g.MT), m = (int)(idx % g.MT);
      if (s != cur_s) {
        if (nb > 0 && !tc_wait(bempty, (uint32_t)(nb - 1) & 1u, abort_flag, true)) {
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
        if (!tc_wait(aempty(stage), phase ^ 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        mbar_expect_tx(afull(stage), (uint32_t)TC_A_STAGE);
        tma_load_2d(sA + (uint32_t)stage * TC_A_STAGE, &tmA, kc * TC_BK, m * TC_BM, afull(stage));
        issued[stage] = 1;
        last_par[stage] = phase;
        if (++stage == TC_STAGES) stage = 0, phase ^= 1u;
      }
    }
    if (!ok) {
      tc_abort(abort_flag, g.status);
      // let the copies already issued land before the CTA exits
      for (int i = 0; i < TC_STAGES; ++i)
        if (issued[i]) tc_wait(afull(i), last_par[i], abort_flag, false);
      if (nb > 0) tc_wait(bfull, (uint32_t)(nb - 1) & 1u, abort_flag, false);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int cur_s = -1, nb = 0, stage = 0;
    uint32_t phase = 0;
    long long t = 0;
    bool ok = true;
    for (long long idx = lo; idx < hi && ok; ++idx, ++t) {
      const int s = (int)(idx / g.MT);
      if (s != cur_s) {
        if (nb > 0) umma_commit(bempty);   // the old slice is free once its MMAs finish
        if (!tc_wait(bfull, (uint32_t)nb & 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        fence_after();
        cur_s = s;
        ++nb;
      }
      const int a = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      if (!tc_wait(accempty(a), (use & 1u) ^ 1u, abort_flag, true)) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(a * TC_BN);
      for (int kc = 0; kc < KC; ++kc) {
        if (!tc_wait(afull(stage), phase, abort_flag, true)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t abase = sA + (uint32_t)stage * TC_A_STAGE;
        const uint32_t bbase = sB + (uint32_t)kc * TC_B_CHUNK;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)
          umma_f16(d, sw128_desc(abase + kk * 32), sw128_desc(bbase + kk * 32), TC_IDESC,
                   (kc | kk) != 0 ? 1u : 0u);
        umma_commit(aempty(stage));   // the stage is free once these MMAs finish
        if (++stage == TC_STAGES) stage = 0, phase ^= 1u;
      }
      if (!ok) break;
      umma_commit(accfull(a));
    }
    if (!ok) tc_abort(abort_flag, g.status);
    // every MMA issued by this thread has finished before TMEM is freed
    umma_commit(bdone);
    tc_wait(bdone, 0, abort_flag, false);
  } else if (warp >= 2) {
    // ---------------- epilogue: rows 32q .. 32q + 31, columns h*128 .. h*128 + 127
    const int q = warp & 3, h = (warp - 2) >> 2;
    long long t = 0;
    for (long long idx = lo; idx < hi; ++idx, ++t) {
      const int s = (int)(idx / g.MT), m = (int)(idx % g.MT);
      const int a = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      // warp-uniform outcome: the TMEM loads below are warp-collective
      const bool ready = __all_sync(0xffffffffu, tc_wait(accfull(a), use & 1u, abort_flag, true));
      if (!ready) {
        if (lane == 0) tc_abort(abort_flag, g.status);
        break;
      }
      fence_after();
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
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty(a));
      const int row = m * TC_BM + 32 * q + lane;
      if (row < g.M)
        g.part[(int64_t)row * (2 * g.S) + 2 * s + h] = make_float2(best, __int_as_float(arg));
    }
  }
  __syncwarp();          // lane 0 of the producer and MMA warps rejoins its warp
  fence_before();
  __syncthreads();   // every role is done with TMEM
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TC_TMEM_COLS);
  }
}

// ---------------------------------------------------------------- general GEMM
// C[M][N] (FP32, row stride ldc) = A[M][K] . B[N][K]^T (+ bias[N]), BF16
// operands, FP32 accumulation: the training GEMMs of the learned proposer
// (logits z = h W2, hidden gradient dh = dz W2^T, weight gradient
// dW2 = h^T dz with both operands transposed first, so that every operand is
// K-major).  Work item = (row tile of 128, column tile of 256, K chunk of
// kc_per blocks of 64); CTAs (one per SM, persistent) walk contiguous ranges
// of items.  A warp issues TMA loads of both operands (128-byte swizzle) into
// a ring of stages; one thread issues tcgen05.mma (M = 128, N = 256, K = 16)
// into one of two TMEM accumulators; eight epilogue warps read their rows
// with tcgen05.ld and store them (16-byte stores), or add them with FP32
// atomics when K is split over several items (C then starts at zero; the
// bias is added by the first K chunk).  Bounded waits as in k_logits_tc.
constexpr int GC_STAGES = 4;
constexpr int GC_A_STAGE = TC_BM * TC_BK * 2;          // 16 KiB
constexpr int GC_B_STAGE = TC_BN * TC_BK * 2;          // 32 KiB
constexpr int GC_STAGE = GC_A_STAGE + GC_B_STAGE;
constexpr int GC_NBARS = 2 * GC_STAGES + 2 + 2 + 1;
constexpr size_t GC_SMEM = 1024 + (size_t)GC_STAGES * GC_STAGE + GC_NBARS * 8;

struct GcArgs {
  float* C;
  const float* bias;   // [N] or null
  int32_t* status;
  int M, N, K, ldc;
  int MT, NT, KS, kc_per;   // row tiles, column tiles, K chunks, 64-blocks per chunk
  long long total;          // MT * NT * KS
  int atomic;               // K split: add into C
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              GcArgs g) {
  extern __shared__ uint8_t gc_smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_sh;
  uint8_t* sm = (uint8_t*)(((uintptr_t)gc_smem_raw + 1023) & ~(uintptr_t)1023);
  const int KB = g.K / TC_BK;   // 64-blocks of K
  const uint32_t sbase = su32(sm);
  const uint32_t bars = sbase + (uint32_t)GC_STAGES * GC_STAGE;
  auto sfull = [&](int i) { return bars + 8u * i; };
  auto sempty = [&](int i) { return bars + 8u * (GC_STAGES + i); };
  auto accfull = [&](int i) { return bars + 8u * (2 * GC_STAGES + i); };
  auto accempty = [&](int i) { return bars + 8u * (2 * GC_STAGES + 2 + i); };
  const uint32_t bdone = bars + 8u * (2 * GC_STAGES + 4);
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long lo = g.total * blockIdx.x / gridDim.x;
  const long long hi = g.total * (blockIdx.x + 1) / gridDim.x;
  // item -> (row tile, column tile, K chunk), K chunk fastest
  auto decode = [&](long long idx, int& mt, int& nt, int& ks) {
    ks = (int)(idx % g.KS);
    const long long r = idx / g.KS;
    nt = (int)(r % g.NT);
    mt = (int)(r / g.NT);
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < GC_STAGES; ++i) {
      mbar_init(sfull(i), 1);
      mbar_init(sempty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(accfull(i), 1);
      mbar_init(accempty(i), TC_EPI_WARPS);
    }
    mbar_init(bdone, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    prefetch_map(&tmA);
    prefetch_map(&tmB);
  }
  if (warp == 1) tmem_alloc(su32(&tmem_slot), TC_TMEM_COLS);
  __syncwarp();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int stage = 0;
    uint32_t phase = 0;
    int issued[GC_STAGES];
    uint32_t last_par[GC_STAGES];
    for (int i = 0; i < GC_STAGES; ++i) issued[i] = 0, last_par[i] = 0;
    bool ok = true;
    for (long long idx = lo; idx < hi && ok; ++idx) {
      int mt, nt, ks;
      decode(idx, mt, nt, ks);
      const int kb0 = ks * g.kc_per, kb1 = min(KB, kb0 + g.kc_per);
      for (int kb = kb0; kb < kb1; ++kb) {
        if (!tc_wait(sempty(stage), phase ^ 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        const uint32_t sa = sbase + (uint32_t)stage * GC_STAGE;
        mbar_expect_tx(sfull(stage), (uint32_t)GC_STAGE);
        tma_load_2d(sa, &tmA, kb * TC_BK, mt * TC_BM, sfull(stage));
        tma_load_2d(sa + GC_A_STAGE, &tmB, kb * TC_BK, nt * TC_BN, sfull(stage));
        issued[stage] = 1;
        last_par[stage] = phase;
        if (++stage == GC_STAGES) stage = 0, phase ^= 1u;
      }
    }
    if (!ok) {
      tc_abort(abort_flag, g.status);
      for (int i = 0; i < GC_STAGES; ++i)
        if (issued[i]) tc_wait(sfull(i), last_par[i], abort_flag, false);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int stage = 0;
    uint32_t phase = 0;
    long long t = 0;
    bool ok = true;
    for (long long idx = lo; idx < hi && ok; ++idx, ++t) {
      int mt, nt, ks;
      decode(idx, mt, nt, ks);
      const int kb0 = ks * g.kc_per, kb1 = min(KB, kb0 + g.kc_per);
      const int a = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      if (!tc_wait(accempty(a), (use & 1u) ^ 1u, abort_flag, true)) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(a * TC_BN);
      for (int kb = kb0; kb < kb1; ++kb) {
        if (!tc_wait(sfull(stage), phase, abort_flag, true)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t abase = sbase + (uint32_t)stage * GC_STAGE;
        const uint32_t bbase = abase + GC_A_STAGE;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)
          umma_f16(d, sw128_desc(abase + kk * 32), sw128_desc(bbase + kk * 32), TC_IDESC,
                   (kb > kb0 || kk > 0) ? 1u : 0u);
        umma_commit(sempty(stage));
        if (++stage == GC_STAGES) stage = 0, phase ^= 1u;
      }
      if (!ok) break;
      umma_commit(accfull(a));
    }
    if (!ok) tc_abort(abort_flag, g.status);
    umma_commit(bdone);
    tc_wait(bdone, 0, abort_flag, false);
  } else if (warp >= 2) {
    // ---------------- epilogue: rows 32q .. 32q + 31, columns h*128 .. h*128 + 127
    const int q = warp & 3, h = (warp - 2) >> 2;
    long long t = 0;
    for (long long idx = lo; idx < hi; ++idx, ++t) {
      int mt, nt, ks;
      decode(idx, mt, nt, ks);
      const int a = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      const bool ready = __all_sync(0xffffffffu, tc_wait(accfull(a), use & 1u, abort_flag, true));
      if (!ready) {
        if (lane == 0) tc_abort(abort_flag, g.status);
        break;
      }
      fence_after();
      const int row = mt * TC_BM + 32 * q + lane;
      const int col0 = nt * TC_BN + h * TC_EPI_COLS;
      const uint32_t tbase =
          tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * TC_BN + h * TC_EPI_COLS);
      const bool add_bias = g.bias && ks == 0;
      float* crow = g.C + (int64_t)row * g.ldc;
      const bool vec = !g.atomic && (g.ldc & 3) == 0;
#pragma unroll 1
      for (int c32 = 0; c32 < TC_EPI_COLS; c32 += 32) {
        uint32_t r[32];
        tmem_ld32_async(tbase + c32, r);
        tmem_wait(r);
        const int cb = col0 + c32;
        if (row < g.M) {
          if (vec && cb + 32 <= g.N) {
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4) {
              float4 v = make_float4(__uint_as_float(r[4 * j4]), __uint_as_float(r[4 * j4 + 1]),
                                     __uint_as_float(r[4 * j4 + 2]), __uint_as_float(r[4 * j4 + 3]));
              if (add_bias) {
                const float4 bb = __ldg(reinterpret_cast<const float4*>(g.bias + cb) + j4);
                v.x += bb.x; v.y += bb.y; v.z += bb.z; v.w += bb.w;
              }
              reinterpret_cast<float4*>(crow + cb)[j4] = v;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = cb + j;
              if (col < g.N) {
                float v = __uint_as_float(r[j]);
                if (add_bias) v += g.bias[col];
                if (g.atomic) atomicAdd(crow + col, v);
                else crow[col] = v;
              }
            }
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
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TC_TMEM_COLS);
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

PFN_cuTensorMapEncodeTiled_v12000 tc::encode_fn() {
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

bool tc_logits_ok(int K, int N, int b) {
  return K >= TC_BK && K <= TC_KMAX && K % TC_BK == 0 && N % TC_BN == 0 && b % TC_EPI_COLS == 0;
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
  if (K < TC_BK || K > TC_KMAX || K % TC_BK || N % TC_BN) return C2_ERR_UNSUPPORTED;
  if (((uintptr_t)A & 15u) || ((uintptr_t)Bt & 15u)) return C2_ERR_INVALID_ARG;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, A, K, M, TC_BM) || !make_map(&tmB, Bt, K, N, TC_BN)) return C2_ERR_CUDA;
  TcArgs g;
  g.bias = bias;
  g.part = part;
  g.status = status;
  g.M = M;
  g.K = K;
  g.S = N / TC_BN;
  g.MT = div_up(M, TC_BM);
  g.total = (long long)g.S * g.MT;   // (slice, row tile) items
  C2_CUDA_TRY(cudaFuncSetAttribute(k_logits_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)TC_SMEM));
  const int grid = (int)std::min<long long>(num_sms(), g.total);
  C2_LAUNCH(k_logits_tc, grid, TC_THREADS, TC_SMEM, st, tmA, tmB, g);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

bool tc_gemm_ok(int M, int N, int K) { return M > 0 && N > 0 && K >= TC_BK && K % TC_BK == 0; }

c2_status tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K,
                  const float* bias, float* C, int ldc, int32_t* status, cudaStream_t st) {
  if (M <= 0 || N <= 0) return C2_OK;
  if (!tc_gemm_ok(M, N, K) || ldc < N) return C2_ERR_UNSUPPORTED;
  if (((uintptr_t)A & 15u) || ((uintptr_t)B & 15u) || ((uintptr_t)C & 15u) ||
      (bias && ((uintptr_t)bias & 15u)))
    return C2_ERR_INVALID_ARG;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, A, K, M, TC_BM) || !make_map(&tmB, B, K, N, TC_BN)) return C2_ERR_CUDA;
  GcArgs g;
  g.C = C;
  g.bias = bias;
  g.status = status;
  g.M = M;
  g.N = N;
  g.K = K;
  g.ldc = ldc;
  g.MT = div_up(M, TC_BM);
  g.NT = div_up(N, TC_BN);
  const int KB = K / TC_BK;
  // split K when the output tiles leave SMs idle and each chunk keeps at
  // least 16 blocks of 64
  int KS = 1;
  while ((long long)g.MT * g.NT * KS * 2 <= num_sms() && KB / (KS * 2) >= 16) KS *= 2;
  g.kc_per = div_up(KB, KS);
  g.KS = div_up(KB, g.kc_per);
  g.atomic = g.KS > 1;
  g.total = (long long)g.MT * g.NT * g.KS;
  if (g.atomic) C2_CUDA_TRY(cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)N * 4, M, st));
  C2_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)GC_SMEM));
  const int grid = (int)std::min<long long>(num_sms(), g.total);
  C2_LAUNCH(k_gemm_tc, grid, TC_THREADS, GC_SMEM, st, tmA, tmB, g);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
