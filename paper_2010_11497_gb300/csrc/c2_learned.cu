// Learned cluster proposer (no counterpart in the paper: a stand-in for
// FastRandomHash as the source of first-level cluster keys).
//
// Network, for user u with profile P_u:
//   e_u = sum_{x in P_u} E[row(x)]                 (embedding bag; E in BF16, FP32 sums)
//   h_u = ReLU(W1^T e_u + b1)                       (D -> H)
//   z_u = W2^T h_u + b2                             (H -> t*b logits, t heads of b)
//   key_j(u) = argmax_c z_u[j*b + c]                (ties to the lower bucket)
// row(x) = SplitMix64(seed_e xor x) mod R.  GEMMs use BF16 operands on the
// tensor cores (mma.sync m16n8k16) with FP32 accumulation.
//
// Training (one Adam step per call) on positive pairs (u, v) -- neighbours in
// KNN graphs built by plain C^2 -- minimises, per pair and head j,
//   -log(sum_c p_u,jc p_v,jc + eps),   p = softmax of each head,
// plus lambda * sum_j KL(mean over the batch of p_j || uniform), which keeps
// the buckets in use.  Keys then feed the same split / local KNN / merge path
// as FastRandomHash keys.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "c2_internal.cuh"

namespace c2 {

// ---------------------------------------------------------------- layout
struct ModelDims {
  int D, H, T, t, b, rows;
  uint64_t seed;
};

struct ModelParams {   // pointers into the state buffer
  float *E, *W1, *b1, *W2, *b2;             // FP32 masters
  float *mE, *mW1, *mb1, *mW2, *mb2;        // Adam first moments
  float *vE, *vW1, *vb1, *vW2, *vb2;        // Adam second moments
  __nv_bfloat16 *E16, *W1_16, *W2_16;       // BF16 copies used by the forward pass
  int32_t* step;
};

ModelDims model_dims(const c2_model_config* c) {
  ModelDims d;
  d.D = c->dim;
  d.H = c->hidden;
  d.t = c->t;
  d.b = c->b;
  d.T = c->t * c->b;
  d.rows = 1 << c->rows_log2;
  d.seed = c->seed;
  return d;
}

size_t bind_model(char* base, const ModelDims& d, ModelParams* p) {
  Ws w;
  w.base = base;
  const size_t nE = (size_t)d.rows * d.D, nW1 = (size_t)d.D * d.H, nW2 = (size_t)d.H * d.T;
  ModelParams q;
  q.E = w.take<float>(nE); q.W1 = w.take<float>(nW1); q.b1 = w.take<float>(d.H);
  q.W2 = w.take<float>(nW2); q.b2 = w.take<float>(d.T);
  q.mE = w.take<float>(nE); q.mW1 = w.take<float>(nW1); q.mb1 = w.take<float>(d.H);
  q.mW2 = w.take<float>(nW2); q.mb2 = w.take<float>(d.T);
  q.vE = w.take<float>(nE); q.vW1 = w.take<float>(nW1); q.vb1 = w.take<float>(d.H);
  q.vW2 = w.take<float>(nW2); q.vb2 = w.take<float>(d.T);
  q.E16 = w.take<__nv_bfloat16>(nE); q.W1_16 = w.take<__nv_bfloat16>(nW1);
  q.W2_16 = w.take<__nv_bfloat16>(nW2);
  q.step = w.take<int32_t>(4);
  if (p) *p = q;
  return w.top + 256;
}

// Per-call scratch of a forward (+ backward) over `rows` users.
struct ModelScratch {
  float* e;              // [rows][D]
  __nv_bfloat16* e16;    // [rows][D]
  float* hpre;           // [rows][H]
  __nv_bfloat16* h16;    // [rows][H]
  float* z;              // [rows][T]  logits, then softmax, then dz
  __nv_bfloat16* dz16;   // [rows][T]
  float* dh;             // [rows][H]
  __nv_bfloat16* dh16;   // [rows][H]
  float* de;             // [rows][D]
  float *gE, *gW1, *gb1, *gW2, *gb2;   // gradients
  float* colmean;        // [T]
  float* loss;           // [4]
  int32_t* rowlist;      // [rows] user of each row
  float2* part;          // [rows][T / slice] (max, argmax) per column slice (proposals)
  __nv_bfloat16* w2t;    // [T][H] transposed W2 for the tcgen05 logits GEMMs
  __nv_bfloat16* hT;     // [H][rows] training: transposed operands of dW2 = h^T dz on the
  __nv_bfloat16* dzT;    // [T][rows]   tensor cores (both K-major)
};

// Training GEMMs on the tensor cores (tcgen05): logits z = h W2 + b2,
// dh = dz W2^T and dW2 = h^T dz need H and T multiples of 64 (and, per call,
// a multiple of 64 rows); the small GEMMs (K or N = D) stay on mma.sync.
bool tc_train_dims(const ModelDims& d) { return d.H % 64 == 0 && d.T % 64 == 0 && d.H <= 65536; }

// How a proposal computes the per-head argmax:
//   2: tcgen05 logits GEMM with the argmax of 256-column slices in its epilogue
//   1: mma.sync logits GEMM with the argmax of 128-column slices in its epilogue
//   0: logits written out, then an argmax kernel
int propose_kind(const ModelDims& d) {
  if (tc_logits_ok(d.H, d.T, d.b) && d.D % 32 == 0 && d.H % 128 == 0) return 2;
  if (d.H % 128 == 0 && d.D % 32 == 0 && d.T % 128 == 0 && d.H % 32 == 0 && d.b % 128 == 0) return 1;
  return 0;
}

size_t bind_scratch(char* base, const ModelDims& d, int rows, bool train, ModelScratch* s) {
  Ws w;
  w.base = base;
  ModelScratch q{};
  if (train) q.e = w.take<float>((size_t)rows * d.D);
  q.e16 = w.take<__nv_bfloat16>((size_t)rows * d.D);
  if (train) q.hpre = w.take<float>((size_t)rows * d.H);
  q.h16 = w.take<__nv_bfloat16>((size_t)rows * d.H);
  const int kind = train ? 0 : propose_kind(d);
  if (kind == 0) q.z = w.take<float>((size_t)rows * d.T);
  if (kind == 2) {
    q.part = w.take<float2>((size_t)rows * (d.T / tc_slice_width()));
    q.w2t = w.take<__nv_bfloat16>((size_t)d.T * d.H);
  }
  if (kind == 1) q.part = w.take<float2>((size_t)rows * (d.T / 128));
  q.rowlist = w.take<int32_t>(rows);
  q.loss = w.take<float>(4);
  if (train && tc_train_dims(d)) {
    q.w2t = w.take<__nv_bfloat16>((size_t)d.T * d.H);
    q.hT = w.take<__nv_bfloat16>((size_t)d.H * rows);
    q.dzT = w.take<__nv_bfloat16>((size_t)d.T * rows);
  }
  if (train) {
    q.dz16 = w.take<__nv_bfloat16>((size_t)rows * d.T);
    q.dh = w.take<float>((size_t)rows * d.H);
    q.dh16 = w.take<__nv_bfloat16>((size_t)rows * d.H);
    q.de = w.take<float>((size_t)rows * d.D);
    q.gE = w.take<float>((size_t)d.rows * d.D);
    q.gW1 = w.take<float>((size_t)d.D * d.H);
    q.gb1 = w.take<float>(d.H);
    q.gW2 = w.take<float>((size_t)d.H * d.T);
    q.gb2 = w.take<float>(d.T);
    q.colmean = w.take<float>(d.T);
  }
  if (s) *s = q;
  return w.top + 256;
}

namespace {

__device__ __forceinline__ uint32_t emb_row(uint64_t seed, int32_t x, int rows) {
  return (uint32_t)(sm64_mix(seed ^ (uint64_t)(uint32_t)x) & (uint64_t)(rows - 1));
}

// ---------------------------------------------------------------- init
// Uniform(-a, a) from Philox, keyed by (seed, tensor id, index).
__global__ void k_init_uniform(float* p, size_t n, float a, uint64_t seed, uint32_t tensor) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), tensor, 0x5EEDu),
                           make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u = (r.x >> 8) * (1.0f / 16777216.0f);   // [0, 1)
  p[i] = (2.0f * u - 1.0f) * a;
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// ---------------------------------------------------------------- embedding bag
// Warp per row, warps striding over the rows (a grid sized to the resident
// warps, so long and short profiles even out per warp).  The row's items are
// taken 32 at a time: lane l hashes item l of the batch (the next batch's ids
// are fetched meanwhile), then the warp's 32 / (D/8) groups of D/8 lanes
// gather the items' rows of E with 16-byte loads (8 dimensions per lane),
// group g taking items g, g + G, g + 2G, ... of the batch.  Each group sums
// its items in order and the groups are added by a fixed shuffle tree, so the
// summation order does not depend on timing.
template <int D>
__global__ void __launch_bounds__(256, D <= 64 ? 4 : 2) k_embbag_fwd(const int32_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ items,
                                                    const int32_t* __restrict__ rowlist, int nrows,
                                                    const __nv_bfloat16* __restrict__ E16, int R,
                                                    uint64_t seed, float* __restrict__ e,
                                                    __nv_bfloat16* __restrict__ e16) {
  constexpr int LPI = D / 8, G = 32 / LPI, PER = 32 / G;   // PER items per group and batch
  const int lane = threadIdx.x & 31;
  const int g = lane / LPI, sl = lane % LPI;
  const bool active = g < G;            // D = 96 leaves 8 lanes idle
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nwarps) {
    const int u = rowlist[r];
    const int beg = ptr[u], end = ptr[u + 1];
    float acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
    int nxt = beg + lane < end ? __ldg(items + beg + lane) : -1;
    for (int j0 = beg; j0 < end; j0 += 32) {
      const int cur = nxt;
      nxt = j0 + 32 + lane < end ? __ldg(items + j0 + 32 + lane) : -1;
      const uint32_t myrow = cur >= 0 ? emb_row(seed, cur, R) : 0xffffffffu;
#pragma unroll
      for (int q0 = 0; q0 < PER; q0 += 4) {   // four rows in flight per lane
        uint4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t row = __shfl_sync(0xffffffffu, myrow, (g + G * (q0 + q)) & 31);
          v[q] = make_uint4(0u, 0u, 0u, 0u);
          if (active && row != 0xffffffffu)
            v[q] = __ldg(reinterpret_cast<const uint4*>(E16 + (size_t)row * D) + sl);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t w[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
            acc[2 * i] += f.x;
            acc[2 * i + 1] += f.y;
          }
        }
      }
    }
#pragma unroll
    for (int off = (G / 2) * LPI; off >= LPI; off >>= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off);
    if (lane < LPI) {
      const size_t o = (size_t)r * D + 8 * lane;
      if (e) {
        *reinterpret_cast<float4*>(e + o) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        *reinterpret_cast<float4*>(e + o + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
      uint4 pk;
      __nv_bfloat162 h2[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) h2[i] = __floats2bfloat162_rn(acc[2 * i], acc[2 * i + 1]);
      pk.x = *reinterpret_cast<uint32_t*>(&h2[0]);
      pk.y = *reinterpret_cast<uint32_t*>(&h2[1]);
      pk.z = *reinterpret_cast<uint32_t*>(&h2[2]);
      pk.w = *reinterpret_cast<uint32_t*>(&h2[3]);
      *reinterpret_cast<uint4*>(e16 + o) = pk;
    }
  }
}

template <int D>
c2_status embbag_launch(const int32_t* ptr, const int32_t* items, const int32_t* rowlist,
                        int nrows, const __nv_bfloat16* E16, int R, uint64_t seed, float* e,
                        __nv_bfloat16* e16, cudaStream_t st) {
  int per_sm = 0;   // resident blocks per SM at this instance's register use
  C2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_embbag_fwd<D>, 256, 0));
  const int grid = std::min(div_up((int64_t)nrows * 32, 256), std::max(per_sm, 1) * num_sms());
  C2_LAUNCH(k_embbag_fwd<D>, grid, 256, 0, st, ptr, items, rowlist, nrows, E16, R, seed, e, e16);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status embbag_fwd(const int32_t* ptr, const int32_t* items, const int32_t* rowlist, int nrows,
                     const __nv_bfloat16* E16, int D, int R, uint64_t seed, float* e,
                     __nv_bfloat16* e16, cudaStream_t st) {
  if (nrows <= 0) return C2_OK;
  switch (D) {
    case 32: return embbag_launch<32>(ptr, items, rowlist, nrows, E16, R, seed, e, e16, st);
    case 64: return embbag_launch<64>(ptr, items, rowlist, nrows, E16, R, seed, e, e16, st);
    case 96: return embbag_launch<96>(ptr, items, rowlist, nrows, E16, R, seed, e, e16, st);
    case 128: return embbag_launch<128>(ptr, items, rowlist, nrows, E16, R, seed, e, e16, st);
    default: return C2_ERR_UNSUPPORTED;
  }
}

// dE[row(x)] += de[r] for every item x of the row's user (FP32 atomics).
__global__ void k_embbag_bwd(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items,
                             const int32_t* __restrict__ rowlist, int nrows,
                             const float* __restrict__ de, int D, int R, uint64_t seed,
                             float* __restrict__ gE) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nrows) return;
  const int u = rowlist[r];
  float g[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int d = lane + 32 * q;
    g[q] = d < D ? de[(size_t)r * D + d] : 0.f;
  }
  for (int j = ptr[u]; j < ptr[u + 1]; ++j) {
    const uint32_t row = emb_row(seed, items[j], R);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int d = lane + 32 * q;
      if (d < D) atomicAdd(&gE[(size_t)row * D + d], g[q]);
    }
  }
}

// ---------------------------------------------------------------- GEMM
// C[M][N] = sum_k A(m,k) B(k,n) (+ bias[n]) with BF16 operands and FP32
// accumulation on mma.sync.m16n8k16.  A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn] (any layout through the strides).  Block tile
// 64 x 64 x 32, four warps of 32 x 32.
constexpr int GBM = 64, GBN = 64, GBK = 32;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct GemmArgs {
  const __nv_bfloat16* A;
  int64_t sam, sak;
  const __nv_bfloat16* B;
  int64_t sbk, sbn;
  float* C;                 // FP32 output [M][N] row-major (ldc), may be NULL
  __nv_bfloat16* C16;       // optional BF16 copy
  int64_t ldc;
  const float* bias;        // optional [N]
  int relu;                 // apply max(0, .) to the BF16 copy only
  int M, N, K;
};

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  __shared__ __nv_bfloat16 As[GBM][GBK + 8];
  __shared__ __nv_bfloat16 Bs[GBK][GBN + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    for (int i = tid; i < GBM * GBK; i += 128) {
      const int m = i / GBK, kk = i % GBK;
      const int gm = m0 + m, gk = k0 + kk;
      As[m][kk] = (gm < g.M && gk < g.K) ? g.A[gm * g.sam + gk * g.sak] : zero;
    }
    for (int i = tid; i < GBK * GBN; i += 128) {
      const int kk = i / GBN, n = i % GBN;
      const int gk = k0 + kk, gn = n0 + n;
      Bs[kk][n] = (gk < g.K && gn < g.N) ? g.B[gk * g.sbk + gn * g.sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gq;
        af[i][0] = pack_bf16(As[r][ks + 2 * tq], As[r][ks + 2 * tq + 1]);
        af[i][1] = pack_bf16(As[r + 8][ks + 2 * tq], As[r + 8][ks + 2 * tq + 1]);
        af[i][2] = pack_bf16(As[r][ks + 2 * tq + 8], As[r][ks + 2 * tq + 9]);
        af[i][3] = pack_bf16(As[r + 8][ks + 2 * tq + 8], As[r + 8][ks + 2 * tq + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cidx = wn + j * 8 + gq;
        bf[j][0] = pack_bf16(Bs[ks + 2 * tq][cidx], Bs[ks + 2 * tq + 1][cidx]);
        bf[j][1] = pack_bf16(Bs[ks + 2 * tq + 8][cidx], Bs[ks + 2 * tq + 9][cidx]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gq + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tq + (q & 1);
        if (m < g.M && n < g.N) {
          float v = acc[i][j][q] + (g.bias ? g.bias[n] : 0.f);
          if (g.C) g.C[(int64_t)m * g.ldc + n] = v;
          if (g.C16) g.C16[(int64_t)m * g.ldc + n] = __float2bfloat16_rn(g.relu ? fmaxf(v, 0.f) : v);
        }
      }
}

// Faster GEMM for row-major operands: C[M][N] = A[M][K] B[K][N] (+ bias),
// N % 128 == 0, K % 32 == 0.  Block tile 128 x 128 x 32, eight warps of
// 64 x 32, cp.async double buffering, ldmatrix fragment loads (B transposed
// on load).  Epilogue: FP32 / BF16 outputs, or -- for proposals -- the
// (max, argmax) of every 128-column slice of each row, ties to the lower column.
constexpr int FBM = 128, FBN = 128, FBK = 32, FPAD = 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* smem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* smem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

struct FastGemmArgs {
  const __nv_bfloat16* A;  // [M][lda]
  int64_t lda;
  const __nv_bfloat16* B;  // [K][ldb]
  int64_t ldb;
  float* C;                // optional [M][ldc]
  __nv_bfloat16* C16;      // optional [M][ldc]
  int64_t ldc;
  const float* bias;       // optional [N]
  int relu;                // ReLU on the BF16 copy
  float2* part;            // optional [M][N/128]: (max, argmax column) per slice
  int M, N, K;
};

__global__ void __launch_bounds__(256) k_gemm_fast(FastGemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[2][FBM][FBK + FPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][FBK][FBN + FPAD];
  __shared__ float2 red[FBM][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * FBM, n0 = blockIdx.x * FBN;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  auto load = [&](int buf, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = tid + r * 256;            // 512 16-byte chunks per operand tile
      const int am = c >> 2, ak = (c & 3) * 8;
      const int gm = m0 + am;
      cp_async16(&As[buf][am][ak], g.A + (int64_t)min(gm, g.M - 1) * g.lda + k0 + ak, gm < g.M);
      const int bk = c >> 4, bn = (c & 15) * 8;
      cp_async16(&Bs[buf][bk][bn], g.B + (int64_t)(k0 + bk) * g.ldb + n0 + bn, true);
    }
    cp_async_commit();
  };
  const int nk = g.K / FBK;
  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      load(buf ^ 1, (kt + 1) * FBK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < FBK; ks += 16) {
      uint32_t af[4][4], bf[4][2];
      const int li = lane >> 3, lr = lane & 7;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = wm + i * 16 + lr + ((li & 1) ? 8 : 0);
        const int col = ks + ((li & 2) ? 8 : 0);
        ldsm_x4(af[i], &As[buf][row][col]);
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int krow = ks + lr + ((li & 1) ? 8 : 0);
        const int ncol = wn + jj * 16 + ((li & 2) ? 8 : 0);
        uint32_t r[4];
        ldsm_x4_t(r, &Bs[buf][krow][ncol]);
        bf[2 * jj][0] = r[0];
        bf[2 * jj][1] = r[1];
        bf[2 * jj + 1][0] = r[2];
        bf[2 * jj + 1][1] = r[3];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  const int gq = lane >> 2, tq = lane & 3;
  if (!g.part) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int m = m0 + wm + i * 16 + gq + (q >= 2 ? 8 : 0);
          const int n = n0 + wn + j * 8 + 2 * tq + (q & 1);
          if (m < g.M) {
            const float v = acc[i][j][q] + (g.bias ? g.bias[n] : 0.f);
            if (g.C) g.C[(int64_t)m * g.ldc + n] = v;
            if (g.C16) g.C16[(int64_t)m * g.ldc + n] = __float2bfloat16_rn(g.relu ? fmaxf(v, 0.f) : v);
          }
        }
    return;
  }
  // (max, argmax) per row over the block's 128 columns
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float best = -INFINITY;
      int arg = 0x7fffffff;
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int n = n0 + wn + j * 8 + 2 * tq + e;
          const float v = acc[i][j][2 * h + e] + (g.bias ? g.bias[n] : 0.f);
          if (v > best || (v == best && n < arg)) { best = v; arg = n; }
        }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ov > best || (ov == best && oa < arg)) { best = ov; arg = oa; }
      }
      if (tq == 0) red[wm + i * 16 + gq + 8 * h][warp & 3] = make_float2(best, __int_as_float(arg));
    }
  __syncthreads();
  if (tid < FBM && m0 + tid < g.M) {
    float2 b2 = red[tid][0];
#pragma unroll
    for (int w2 = 1; w2 < 4; ++w2) {
      const float2 o = red[tid][w2];
      if (o.x > b2.x || (o.x == b2.x && __float_as_int(o.y) < __float_as_int(b2.y))) b2 = o;
    }
    g.part[(int64_t)(m0 + tid) * (g.N / FBN) + blockIdx.x] = b2;
  }
}

// Key of every (row, head) from the per-slice partials (b % 128 == 0).
__global__ void k_argmax_parts(const float2* __restrict__ part, int nrows, int t, int b, int T,
                               int width, const int32_t* __restrict__ rowlist, int n_users,
                               int32_t* __restrict__ keys) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nrows * t) return;
  const int r = idx / t, j = idx % t;
  const int per = b / width, slices = T / width;
  float2 best = part[(int64_t)r * slices + j * per];
  for (int q = 1; q < per; ++q) {
    const float2 o = part[(int64_t)r * slices + j * per + q];
    if (o.x > best.x || (o.x == best.x && __float_as_int(o.y) < __float_as_int(best.y))) best = o;
  }
  keys[(int64_t)j * n_users + rowlist[r]] = __float_as_int(best.y) - j * b;
}

c2_status gemm_fast(const FastGemmArgs& g, cudaStream_t st) {
  if (g.M <= 0) return C2_OK;
  dim3 grid(g.N / FBN, div_up(g.M, FBM));
  C2_LAUNCH(k_gemm_fast, grid, 256, 0, st, g);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status gemm(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return C2_OK;
  dim3 grid(div_up(g.N, GBN), div_up(g.M, GBM));
  C2_LAUNCH(k_gemm_bf16, grid, 128, 0, st, g);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

// ---------------------------------------------------------------- heads
// Warp per (row, head): argmax of b logits, ties to the lower bucket.
__global__ void k_argmax(const float* __restrict__ z, int nrows, int t, int b, int T,
                         const int32_t* __restrict__ rowlist, int n_users,
                         int32_t* __restrict__ keys) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nrows * t) return;
  const int r = w / t, j = w % t;
  const float* zr = z + (size_t)r * T + (size_t)j * b;
  float best = -INFINITY;
  int arg = b;
  for (int c = lane; c < b; c += 32) {
    const float v = zr[c];
    if (v > best) { best = v; arg = c; }     // first (lowest) c per lane on ties
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ov > best || (ov == best && oa < arg)) { best = ov; arg = oa; }
  }
  if (lane == 0) keys[(size_t)j * n_users + rowlist[r]] = arg;
}

// Softmax of every head in place (row-major [rows][T]); warp per (row, head).
__global__ void k_softmax(float* __restrict__ z, int nrows, int t, int b, int T) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nrows * t) return;
  float* zr = z + (size_t)(w / t) * T + (size_t)(w % t) * b;
  float mx = -INFINITY;
  for (int c = lane; c < b; c += 32) mx = fmaxf(mx, zr[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sum = 0.f;
  for (int c = lane; c < b; c += 32) sum += __expf(zr[c] - mx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const float inv = 1.f / sum;
  for (int c = lane; c < b; c += 32) zr[c] = __expf(zr[c] - mx) * inv;
}

// Column means of the probabilities over the rows (balance term).
__global__ void k_colmean(const float* __restrict__ p, int nrows, int T, float* __restrict__ m) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= T) return;
  float s = 0.f;
  for (int r = 0; r < nrows; ++r) s += p[(size_t)r * T + c];
  m[c] = s / (float)nrows;
}

// Loss and gradient w.r.t. the logits.  Rows 0..P-1 are the pairs' first
// users, rows P..2P-1 the second.  Warp per (pair, head):
//   S = sum_c p_u p_v ;  L += -log(S + eps) / (P t)
//   dL/dp_u = -p_v / (S + eps) / (P t)     (and symmetrically for v)
// balance: dL/dp_r,c = lambda (log(b m_c) + 1) / (2P t)
// softmax: dz = p (g - sum_c p g).  dz overwrites nothing: written to dz16.
__global__ void k_pair_loss(const float* __restrict__ p, int P, int t, int b, int T,
                            const float* __restrict__ colmean, float lambda, float eps,
                            __nv_bfloat16* __restrict__ dz16, float* __restrict__ dzf,
                            float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= P * t) return;
  const int i = w / t, j = w % t;
  const float* pu = p + (size_t)i * T + (size_t)j * b;
  const float* pv = p + (size_t)(i + P) * T + (size_t)j * b;
  const float* mj = colmean + (size_t)j * b;
  float S = 0.f;
  for (int c = lane; c < b; c += 32) S += pu[c] * pv[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
  const float scale = 1.f / ((float)P * (float)t);
  const float bal = lambda / (2.f * (float)P * (float)t);
  // g for u and v, and the softmax correction sums
  float su = 0.f, sv = 0.f;
  for (int c = lane; c < b; c += 32) {
    const float gb = bal * (logf(fmaxf((float)b * mj[c], 1e-30f)) + 1.f);
    const float gu = -pv[c] / (S + eps) * scale + gb;
    const float gv = -pu[c] / (S + eps) * scale + gb;
    su += pu[c] * gu;
    sv += pv[c] * gv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_xor_sync(0xffffffffu, su, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  for (int c = lane; c < b; c += 32) {
    const float gb = bal * (logf(fmaxf((float)b * mj[c], 1e-30f)) + 1.f);
    const float gu = -pv[c] / (S + eps) * scale + gb;
    const float gv = -pu[c] / (S + eps) * scale + gb;
    const float du = pu[c] * (gu - su), dv = pv[c] * (gv - sv);
    const size_t iu = (size_t)i * T + (size_t)j * b + c, iv = (size_t)(i + P) * T + (size_t)j * b + c;
    dz16[iu] = __float2bfloat16_rn(du);
    dz16[iv] = __float2bfloat16_rn(dv);
    if (dzf) { dzf[iu] = du; dzf[iv] = dv; }
  }
  if (lane == 0) atomicAdd(&loss[0], -logf(S + eps) * scale);
}

__global__ void k_balance_loss(const float* __restrict__ colmean, int T, int t, int b,
                               float lambda, float* __restrict__ loss) {
  float s = 0.f;
  for (int c = threadIdx.x; c < T; c += blockDim.x) {
    const float m = colmean[c];
    if (m > 0.f) s += m * logf((float)b * m);
  }
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[1] = lambda * red[0] / (float)t;
}

// Column sums (bias gradients): out[c] = sum_r in[r][c] for BF16 or FP32 inputs.
__global__ void k_colsum_bf16(const __nv_bfloat16* __restrict__ a, int rows, int cols,
                              float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += __bfloat162float(a[(size_t)r * cols + c]);
  out[c] = s;
}

// dh (FP32, from GEMM) masked by the ReLU of the forward pre-activation.
__global__ void k_relu_bwd(float* __restrict__ dh, const float* __restrict__ hpre, size_t n,
                           __nv_bfloat16* __restrict__ dh16) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = hpre[i] > 0.f ? dh[i] : 0.f;
  dh[i] = v;
  dh16[i] = __float2bfloat16_rn(v);
}

// Adam (Kingma & Ba, 2015) on a dense tensor; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16* __restrict__ w16) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (w16) w16[i] = __float2bfloat16_rn(wi);
}

__global__ void k_rowlist_pairs(const int32_t* __restrict__ pairs, int P, int n,
                                int32_t* __restrict__ rowlist, DevHeader* hdr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int u = pairs[2 * i], v = pairs[2 * i + 1];
  if (u < 0 || u >= n || v < 0 || v >= n) {
    if (hdr) dev_fail(hdr, C2_ERR_INVALID_ARG);
    rowlist[i] = 0;
    rowlist[i + P] = 0;
    return;
  }
  rowlist[i] = u;
  rowlist[i + P] = v;
}

__global__ void k_gather_rows(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                              const int32_t* __restrict__ rows, int nr, int k,
                              int32_t* __restrict__ oa, int32_t* __restrict__ ob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr * k) return;
  const int r = i / k, j = i % k;
  oa[i] = a[(size_t)rows[r] * k + j];
  ob[i] = b[(size_t)rows[r] * k + j];
}

__global__ void k_rowlist_range(int32_t* __restrict__ rowlist, int start, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) rowlist[i] = start + i;
}

}  // namespace

// ---------------------------------------------------------------- drivers
// Forward pass over nrows rows of scratch (rowlist filled): e, h, z logits.
bool fast_ok(int N, int K) { return N % FBN == 0 && K % FBK == 0; }

// Forward pass over nrows rows; with `part` the second GEMM only leaves the
// per-slice (max, argmax) partials instead of the logits.
c2_status model_forward(const ModelDims& d, const ModelParams& p, const ModelScratch& s,
                        const int32_t* ptr, const int32_t* items, int nrows, cudaStream_t st,
                        float2* part = nullptr, int32_t* tc_status = nullptr) {
  c2_status rc0 = embbag_fwd(ptr, items, s.rowlist, nrows, p.E16, d.D, d.rows, d.seed, s.e, s.e16, st);
  if (rc0) return rc0;
  if (tc_status) {
    // hidden layer on mma.sync (K = D), logits on the tensor cores
    c2_status rc;
    if (fast_ok(d.H, d.D)) {
      FastGemmArgs f1{};
      f1.A = s.e16; f1.lda = d.D; f1.B = p.W1_16; f1.ldb = d.H;
      f1.C = s.hpre; f1.C16 = s.h16; f1.ldc = d.H; f1.bias = p.b1; f1.relu = 1;
      f1.M = nrows; f1.N = d.H; f1.K = d.D;
      rc = gemm_fast(f1, st);
    } else {
      GemmArgs g1{};
      g1.A = s.e16; g1.sam = d.D; g1.sak = 1;
      g1.B = p.W1_16; g1.sbk = d.H; g1.sbn = 1;
      g1.C = s.hpre; g1.C16 = s.h16; g1.ldc = d.H; g1.bias = p.b1; g1.relu = 1;
      g1.M = nrows; g1.N = d.H; g1.K = d.D;
      rc = gemm(g1, st);
    }
    if (rc) return rc;
    rc = tc_transpose_bf16(p.W2_16, d.H, d.T, s.w2t, st);
    if (rc) return rc;
    return tc_gemm(s.h16, s.w2t, nrows, d.T, d.H, p.b2, s.z, d.T, tc_status, st);
  }
  if (fast_ok(d.H, d.D) && fast_ok(d.T, d.H)) {
    FastGemmArgs f1{};
    f1.A = s.e16; f1.lda = d.D; f1.B = p.W1_16; f1.ldb = d.H;
    f1.C = s.hpre; f1.C16 = s.h16; f1.ldc = d.H; f1.bias = p.b1; f1.relu = 1;
    f1.M = nrows; f1.N = d.H; f1.K = d.D;
    c2_status rc = gemm_fast(f1, st);
    if (rc) return rc;
    FastGemmArgs f2{};
    f2.A = s.h16; f2.lda = d.H; f2.B = p.W2_16; f2.ldb = d.T;
    f2.C = part ? nullptr : s.z; f2.ldc = d.T; f2.bias = p.b2; f2.part = part;
    f2.M = nrows; f2.N = d.T; f2.K = d.H;
    return gemm_fast(f2, st);
  }
  GemmArgs g1{};
  g1.A = s.e16; g1.sam = d.D; g1.sak = 1;
  g1.B = p.W1_16; g1.sbk = d.H; g1.sbn = 1;
  g1.C = s.hpre; g1.C16 = s.h16; g1.ldc = d.H; g1.bias = p.b1; g1.relu = 1;
  g1.M = nrows; g1.N = d.H; g1.K = d.D;
  c2_status rc = gemm(g1, st);
  if (rc) return rc;
  GemmArgs g2{};
  g2.A = s.h16; g2.sam = d.H; g2.sak = 1;
  g2.B = p.W2_16; g2.sbk = d.T; g2.sbn = 1;
  g2.C = s.z; g2.ldc = d.T; g2.bias = p.b2;
  g2.M = nrows; g2.N = d.T; g2.K = d.H;
  return gemm(g2, st);
}

c2_status model_propose(const ModelDims& d, const ModelParams& p, const ModelScratch& s,
                        int chunk, const int32_t* ptr, const int32_t* items, int n,
                        int32_t* keys, DevHeader* hdr, cudaStream_t st) {
  const int kind = propose_kind(d);
  if (kind == 2) {
    c2_status rc = tc_transpose_bf16(p.W2_16, d.H, d.T, s.w2t, st);
    if (rc) return rc;
  }
  for (int start = 0; start < n; start += chunk) {
    const int rows = std::min(chunk, n - start);
    C2_LAUNCH(k_rowlist_range, div_up(rows, 256), 256, 0, st, s.rowlist, start, rows);
    if (kind == 2) {
      c2_status rc = embbag_fwd(ptr, items, s.rowlist, rows, p.E16, d.D, d.rows, d.seed, s.e,
                                s.e16, st);
      if (rc) return rc;
      FastGemmArgs f1{};
      f1.A = s.e16; f1.lda = d.D; f1.B = p.W1_16; f1.ldb = d.H;
      f1.C16 = s.h16; f1.ldc = d.H; f1.bias = p.b1; f1.relu = 1;
      f1.M = rows; f1.N = d.H; f1.K = d.D;
      rc = gemm_fast(f1, st);
      if (rc) return rc;
      rc = tc_logits_argmax(s.h16, rows, d.H, s.w2t, d.T, p.b2, s.part, &hdr->status, st);
      if (rc) return rc;
      C2_LAUNCH(k_argmax_parts, div_up((int64_t)rows * d.t, 256), 256, 0, st, s.part, rows, d.t,
                d.b, d.T, tc_slice_width(), s.rowlist, n, keys);
    } else if (kind == 1) {
      c2_status rc = model_forward(d, p, s, ptr, items, rows, st, s.part);
      if (rc) return rc;
      C2_LAUNCH(k_argmax_parts, div_up((int64_t)rows * d.t, 256), 256, 0, st, s.part, rows, d.t,
                d.b, d.T, FBN, s.rowlist, n, keys);
    } else {
      c2_status rc = model_forward(d, p, s, ptr, items, rows, st);
      if (rc) return rc;
      C2_LAUNCH(k_argmax, div_up((int64_t)rows * d.t * 32, 256), 256, 0, st, s.z, rows, d.t, d.b,
                d.T, s.rowlist, n, keys);
    }
  }
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

// Loss and all gradients of a batch of P pairs (rows = 2P).
c2_status model_grads(const ModelDims& d, const ModelParams& p, const ModelScratch& s,
                      const int32_t* ptr, const int32_t* items, int n, const int32_t* pairs, int P,
                      float lambda, float* dz_debug, DevHeader* hdr, cudaStream_t st) {
  const int rows = 2 * P;
  const bool tc = tc_train_dims(d) && rows % 64 == 0 && s.w2t;
  C2_LAUNCH(k_rowlist_pairs, div_up(P, 256), 256, 0, st, pairs, P, n, s.rowlist, hdr);
  c2_status rc = model_forward(d, p, s, ptr, items, rows, st, nullptr, tc ? &hdr->status : nullptr);
  if (rc) return rc;
  C2_LAUNCH(k_softmax, div_up((int64_t)rows * d.t * 32, 256), 256, 0, st, s.z, rows, d.t, d.b, d.T);
  C2_LAUNCH(k_colmean, div_up(d.T, 256), 256, 0, st, s.z, rows, d.T, s.colmean);
  C2_CUDA_TRY(cudaMemsetAsync(s.loss, 0, 4 * sizeof(float), st));
  C2_LAUNCH(k_pair_loss, div_up((int64_t)P * d.t * 32, 256), 256, 0, st, s.z, P, d.t, d.b, d.T,
            s.colmean, lambda, 1e-9f, s.dz16, dz_debug, s.loss);
  C2_LAUNCH(k_balance_loss, 1, 256, 0, st, s.colmean, d.T, d.t, d.b, lambda, s.loss);
  if (tc) {
    // dW2 = h^T dz [H][T] with both operands transposed (K = rows contiguous)
    rc = tc_transpose_bf16(s.h16, rows, d.H, s.hT, st);
    if (rc) return rc;
    rc = tc_transpose_bf16(s.dz16, rows, d.T, s.dzT, st);
    if (rc) return rc;
    rc = tc_gemm(s.hT, s.dzT, d.H, d.T, rows, nullptr, s.gW2, d.T, &hdr->status, st);
    if (rc) return rc;
    // dh = dz W2^T [rows][H]: W2 [H][T] is already K-major
    rc = tc_gemm(s.dz16, p.W2_16, rows, d.H, d.T, nullptr, s.dh, d.H, &hdr->status, st);
    if (rc) return rc;
  } else {
    // dW2 = h^T dz  [H][T]
    GemmArgs a{};
    a.A = s.h16; a.sam = 1; a.sak = d.H;        // A(m=h, k=r) = h16[r][h]
    a.B = s.dz16; a.sbk = d.T; a.sbn = 1;       // B(k=r, n=c) = dz[r][c]
    a.C = s.gW2; a.ldc = d.T; a.M = d.H; a.N = d.T; a.K = rows;
    rc = gemm(a, st);
    if (rc) return rc;
    // dh = dz W2^T  [rows][H]
    GemmArgs b{};
    b.A = s.dz16; b.sam = d.T; b.sak = 1;       // A(m=r, k=c) = dz[r][c]
    b.B = p.W2_16; b.sbk = 1; b.sbn = d.T;      // B(k=c, n=h) = W2[h][c]
    b.C = s.dh; b.ldc = d.H; b.M = rows; b.N = d.H; b.K = d.T;
    rc = gemm(b, st);
    if (rc) return rc;
  }
  // db2 = sum_r dz; dh is then masked by the ReLU
  C2_LAUNCH(k_colsum_bf16, div_up(d.T, 256), 256, 0, st, s.dz16, rows, d.T, s.gb2);
  C2_LAUNCH(k_relu_bwd, div_up((int64_t)rows * d.H, 256), 256, 0, st, s.dh, s.hpre,
            (size_t)rows * d.H, s.dh16);
  // dW1 = e^T dh  [D][H];  db1 = sum_r dh
  GemmArgs c{};
  c.A = s.e16; c.sam = 1; c.sak = d.D;
  c.B = s.dh16; c.sbk = d.H; c.sbn = 1;
  c.C = s.gW1; c.ldc = d.H; c.M = d.D; c.N = d.H; c.K = rows;
  rc = gemm(c, st);
  if (rc) return rc;
  C2_LAUNCH(k_colsum_bf16, div_up(d.H, 256), 256, 0, st, s.dh16, rows, d.H, s.gb1);
  // de = dh W1^T  [rows][D]
  GemmArgs e{};
  e.A = s.dh16; e.sam = d.H; e.sak = 1;
  e.B = p.W1_16; e.sbk = 1; e.sbn = d.H;
  e.C = s.de; e.ldc = d.D; e.M = rows; e.N = d.D; e.K = d.H;
  rc = gemm(e, st);
  if (rc) return rc;
  C2_CUDA_TRY(cudaMemsetAsync(s.gE, 0, sizeof(float) * (size_t)d.rows * d.D, st));
  C2_LAUNCH(k_embbag_bwd, div_up((int64_t)rows * 32, 256), 256, 0, st, ptr, items, s.rowlist,
            rows, s.de, d.D, d.rows, d.seed, s.gE);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status model_adam(const ModelDims& d, const ModelParams& p, const ModelScratch& s, int step,
                     float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  auto upd = [&](float* w, float* m, float* v, const float* g, size_t n, __nv_bfloat16* w16) {
    C2_LAUNCH(k_adam, div_up((int64_t)n, 256), 256, 0, st, w, m, v, g, n, lr, b1, b2, eps, c1, c2,
              w16);
  };
  upd(p.E, p.mE, p.vE, s.gE, (size_t)d.rows * d.D, p.E16);
  upd(p.W1, p.mW1, p.vW1, s.gW1, (size_t)d.D * d.H, p.W1_16);
  upd(p.b1, p.mb1, p.vb1, s.gb1, (size_t)d.H, nullptr);
  upd(p.W2, p.mW2, p.vW2, s.gW2, (size_t)d.H * d.T, p.W2_16);
  upd(p.b2, p.mb2, p.vb2, s.gb2, (size_t)d.T, nullptr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status model_init(const ModelDims& d, const ModelParams& p, cudaStream_t st) {
  const size_t nE = (size_t)d.rows * d.D, nW1 = (size_t)d.D * d.H, nW2 = (size_t)d.H * d.T;
  const float aE = 0.1f, aW1 = sqrtf(6.f / (float)(d.D + d.H)), aW2 = sqrtf(6.f / (float)(d.H + d.b));
  C2_LAUNCH(k_init_uniform, div_up((int64_t)nE, 256), 256, 0, st, p.E, nE, aE, d.seed, 1u);
  C2_LAUNCH(k_init_uniform, div_up((int64_t)nW1, 256), 256, 0, st, p.W1, nW1, aW1, d.seed, 2u);
  C2_LAUNCH(k_init_uniform, div_up((int64_t)nW2, 256), 256, 0, st, p.W2, nW2, aW2, d.seed, 3u);
  C2_CUDA_TRY(cudaMemsetAsync(p.b1, 0, d.H * sizeof(float), st));
  C2_CUDA_TRY(cudaMemsetAsync(p.b2, 0, d.T * sizeof(float), st));
  // Adam moments (contiguous after the masters) and the step counter
  C2_CUDA_TRY(cudaMemsetAsync(p.mE, 0, (size_t)((char*)p.E16 - (char*)p.mE), st));
  C2_CUDA_TRY(cudaMemsetAsync(p.step, 0, 4 * sizeof(int32_t), st));
  C2_LAUNCH(k_to_bf16, div_up((int64_t)nE, 256), 256, 0, st, p.E, p.E16, nE);
  C2_LAUNCH(k_to_bf16, div_up((int64_t)nW1, 256), 256, 0, st, p.W1, p.W1_16, nW1);
  C2_LAUNCH(k_to_bf16, div_up((int64_t)nW2, 256), 256, 0, st, p.W2, p.W2_16, nW2);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2

using namespace c2;

namespace {

// Users per proposal chunk inside the learned build: without the logits
// written out a row of scratch is under 1 KiB.
int32_t learned_chunk_rows(const c2_model_config* c) {
  return propose_kind(model_dims(c)) == 0 ? 8192 : 65536;
}

c2_status check_cfg(const c2_model_config* c) {
  if (!c) return C2_ERR_INVALID_ARG;
  if (c->t < 1 || c->t > kMaxT || c->b < 2 || c->b > kMaxB) return C2_ERR_UNSUPPORTED;
  if (c->dim < 32 || c->dim > 128 || c->dim % 32 || c->hidden < 16 || c->hidden > 4096 ||
      c->rows_log2 < 4 || c->rows_log2 > 26 || c->reserved0 != 0)
    return C2_ERR_UNSUPPORTED;
  if ((int64_t)c->t * c->b > (1 << 20)) return C2_ERR_UNSUPPORTED;
  return C2_OK;
}

}  // namespace

extern "C" {

size_t c2_model_state_bytes(const c2_model_config* cfg) {
  if (check_cfg(cfg)) return 0;
  return bind_model(nullptr, model_dims(cfg), nullptr);
}

size_t c2_model_workspace_size(const c2_model_config* cfg, int32_t max_rows, int32_t train) {
  if (check_cfg(cfg) || max_rows < 1) return 0;
  return 256 + bind_scratch(nullptr, model_dims(cfg), train ? 2 * max_rows : max_rows, train != 0,
                            nullptr);
}

c2_status c2_model_init(const c2_model_config* cfg, void* d_state, size_t state_bytes,
                        c2_stream_t stream) {
  c2_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!d_state || ((uintptr_t)d_state & 255u)) return C2_ERR_WORKSPACE;
  const ModelDims d = model_dims(cfg);
  ModelParams p;
  if (state_bytes < bind_model((char*)d_state, d, &p)) return C2_ERR_WORKSPACE;
  return model_init(d, p, (cudaStream_t)stream);
}

c2_status c2_model_propose(const c2_model_config* cfg, const void* d_state,
                           const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                           int32_t* d_keys, void* d_ws, size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!d_state || !d_csr_ptr || (!d_csr_items && n_users > 0) || !d_keys || n_users < 0)
    return C2_ERR_INVALID_ARG;
  if (!d_ws || ((uintptr_t)d_ws & 255u)) return C2_ERR_WORKSPACE;
  const ModelDims d = model_dims(cfg);
  ModelParams p;
  bind_model((char*)d_state, d, &p);
  // the largest row chunk whose scratch fits the workspace
  int chunk = 1;
  while (chunk < (1 << 20) && 256 + bind_scratch(nullptr, d, 2 * chunk, false, nullptr) <= ws_bytes)
    chunk *= 2;
  if (256 + bind_scratch(nullptr, d, chunk, false, nullptr) > ws_bytes) return C2_ERR_WORKSPACE;
  ModelScratch s;
  bind_scratch((char*)d_ws + 256, d, chunk, false, &s);
  C2_CUDA_TRY(cudaMemsetAsync(d_ws, 0, sizeof(DevHeader), (cudaStream_t)stream));
  return model_propose(d, p, s, chunk, d_csr_ptr, d_csr_items, n_users, d_keys,
                       reinterpret_cast<DevHeader*>(d_ws), (cudaStream_t)stream);
}

c2_status c2_model_train_step(const c2_model_config* cfg, void* d_state,
                              const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                              int32_t n_users, const int32_t* d_pairs, int32_t n_pairs, float lr,
                              float lambda, int32_t step, float* d_loss, void* d_ws,
                              size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!d_state || !d_csr_ptr || !d_csr_items || !d_pairs || n_pairs < 1 || step < 1 || !(lr > 0.f))
    return C2_ERR_INVALID_ARG;
  if (!d_ws || ((uintptr_t)d_ws & 255u)) return C2_ERR_WORKSPACE;
  const ModelDims d = model_dims(cfg);
  if (256 + bind_scratch(nullptr, d, 2 * n_pairs, true, nullptr) > ws_bytes) return C2_ERR_WORKSPACE;
  ModelParams p;
  bind_model((char*)d_state, d, &p);
  ModelScratch s;
  bind_scratch((char*)d_ws + 256, d, 2 * n_pairs, true, &s);
  DevHeader* hdr = reinterpret_cast<DevHeader*>(d_ws);
  cudaStream_t st = (cudaStream_t)stream;
  rc = model_grads(d, p, s, d_csr_ptr, d_csr_items, n_users, d_pairs, n_pairs, lambda, nullptr, hdr, st);
  if (rc) return rc;
  rc = model_adam(d, p, s, step, lr, st);
  if (rc) return rc;
  if (d_loss) C2_CUDA_TRY(cudaMemcpyAsync(d_loss, s.loss, 2 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return C2_OK;
}

c2_status c2_model_gradients(const c2_model_config* cfg, const void* d_state,
                             const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                             const int32_t* d_pairs, int32_t n_pairs, float lambda, float* d_loss,
                             float* d_gE, float* d_gW1, float* d_gb1, float* d_gW2, float* d_gb2,
                             void* d_ws, size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!d_state || !d_csr_ptr || !d_csr_items || !d_pairs || n_pairs < 1 || !d_loss || !d_gE ||
      !d_gW1 || !d_gb1 || !d_gW2 || !d_gb2)
    return C2_ERR_INVALID_ARG;
  if (!d_ws || ((uintptr_t)d_ws & 255u)) return C2_ERR_WORKSPACE;
  const ModelDims d = model_dims(cfg);
  if (256 + bind_scratch(nullptr, d, 2 * n_pairs, true, nullptr) > ws_bytes) return C2_ERR_WORKSPACE;
  ModelParams p;
  bind_model((char*)d_state, d, &p);
  ModelScratch s;
  bind_scratch((char*)d_ws + 256, d, 2 * n_pairs, true, &s);
  cudaStream_t st = (cudaStream_t)stream;
  rc = model_grads(d, p, s, d_csr_ptr, d_csr_items, n_users, d_pairs, n_pairs, lambda, nullptr,
                   reinterpret_cast<DevHeader*>(d_ws), st);
  if (rc) return rc;
  auto cp = [&](float* dst, const float* src, size_t n) {
    return cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  };
  C2_CUDA_TRY(cp(d_loss, s.loss, 2));
  C2_CUDA_TRY(cp(d_gE, s.gE, (size_t)d.rows * d.D));
  C2_CUDA_TRY(cp(d_gW1, s.gW1, (size_t)d.D * d.H));
  C2_CUDA_TRY(cp(d_gb1, s.gb1, (size_t)d.H));
  C2_CUDA_TRY(cp(d_gW2, s.gW2, (size_t)d.H * d.T));
  C2_CUDA_TRY(cp(d_gb2, s.gb2, (size_t)d.T));
  return C2_OK;
}

c2_status c2_model_params(const c2_model_config* cfg, const void* d_state, float** E, float** W1,
                          float** b1, float** W2, float** b2) {
  c2_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!d_state) return C2_ERR_INVALID_ARG;
  ModelParams p;
  bind_model((char*)d_state, model_dims(cfg), &p);
  if (E) *E = p.E;
  if (W1) *W1 = p.W1;
  if (b1) *b1 = p.b1;
  if (W2) *W2 = p.W2;
  if (b2) *b2 = p.b2;
  return C2_OK;
}

}  // extern "C"

extern "C" {

size_t c2_workspace_size_learned(const c2_model_config* cfg, int32_t n_users, int64_t nnz,
                                 int32_t n_items, int32_t k, int32_t N, int32_t n_probe,
                                 const c2_options* opt) {
  if (check_cfg(cfg) || n_probe < 1) return 0;
  const size_t base = c2_workspace_size(n_users, nnz, n_items, k, cfg->t, cfg->b, N, opt);
  if (!base) return 0;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t model = c2_model_workspace_size(cfg, learned_chunk_rows(cfg), 0);
  return up(base) + up(model) + up((size_t)cfg->t * n_users * 4) + up((size_t)n_probe * 4) +
         5 * up((size_t)n_probe * k * 4) + 2 * up(8);
}

c2_status c2_build_knn_graph_learned(const c2_model_config* cfg, const void* d_state,
                                     const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                                     int32_t n_users, int64_t nnz, int32_t n_items, int32_t k,
                                     int32_t N, uint64_t seed, const c2_options* opt,
                                     float quality_threshold, int32_t n_probe,
                                     int32_t* d_nbr_id, int32_t* d_nbr_inter,
                                     int32_t* d_nbr_union, void* d_ws, size_t ws_bytes,
                                     c2_stream_t stream, double* h_quality) {
  c2_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!d_state || !d_csr_ptr || !d_nbr_id || !d_nbr_inter || !d_nbr_union || n_users < 1)
    return C2_ERR_INVALID_ARG;
  n_probe = std::min(n_probe, n_users);
  const size_t need = c2_workspace_size_learned(cfg, n_users, nnz, n_items, k, N, n_probe, opt);
  if (!need) return C2_ERR_INVALID_ARG;
  if (!d_ws || ((uintptr_t)d_ws & 255u) || ws_bytes < need) return C2_ERR_WORKSPACE;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t base = c2_workspace_size(n_users, nnz, n_items, k, cfg->t, cfg->b, N, opt);
  const size_t model = c2_model_workspace_size(cfg, learned_chunk_rows(cfg), 0);
  char* p = (char*)d_ws + up(base);
  void* mws = p;
  p += up(model);
  int32_t* keys = (int32_t*)p;
  p += up((size_t)cfg->t * n_users * 4);
  int32_t* probe = (int32_t*)p;
  p += up((size_t)n_probe * 4);
  int32_t *jid = (int32_t*)p, *jin, *jun, *cin, *cun;
  p += up((size_t)n_probe * k * 4);
  jin = (int32_t*)p; p += up((size_t)n_probe * k * 4);
  jun = (int32_t*)p; p += up((size_t)n_probe * k * 4);
  cin = (int32_t*)p; p += up((size_t)n_probe * k * 4);
  cun = (int32_t*)p; p += up((size_t)n_probe * k * 4);
  double* sims = (double*)p;
  cudaStream_t st = (cudaStream_t)stream;
  rc = c2_model_propose(cfg, d_state, d_csr_ptr, d_csr_items, n_users, keys, mws, model, stream);
  if (rc) return rc;
  c2_options o;
  c2_default_options(&o);
  if (opt) o = *opt;
  o.d_keys = keys;
  rc = c2_build_knn_graph(d_csr_ptr, d_csr_items, n_users, n_items, k, cfg->t, cfg->b, N, seed,
                          &o, d_nbr_id, d_nbr_inter, d_nbr_union, d_ws, base, stream);
  if (rc) return rc;
  rc = c2_get_status(d_ws, stream);
  if (rc) return rc;
  rc = c2_get_status(mws, stream);   // the proposal's own device status (bounded waits)
  if (rc) return rc;
  // quality probe (Eq. 2) on every (n / n_probe)-th user against exact brute force
  std::vector<int32_t> hp(n_probe);
  for (int32_t i = 0; i < n_probe; ++i) hp[i] = (int32_t)((int64_t)i * n_users / n_probe);
  C2_CUDA_TRY(cudaMemcpyAsync(probe, hp.data(), n_probe * 4, cudaMemcpyHostToDevice, st));
  rc = c2_bruteforce_knn(d_csr_ptr, d_csr_items, n_users, n_items, k, probe, n_probe, jid, jin,
                         jun, d_ws, base, stream);
  if (rc) return rc;
  C2_LAUNCH(k_gather_rows, div_up((int64_t)n_probe * k, 256), 256, 0, st, d_nbr_inter,
            d_nbr_union, probe, n_probe, k, cin, cun);
  rc = c2_avg_sim(cin, cun, n_probe, k, sims, d_ws, base, stream);
  if (rc) return rc;
  rc = c2_avg_sim(jin, jun, n_probe, k, sims + 1, d_ws, base, stream);
  if (rc) return rc;
  double h[2] = {0, 0};
  C2_CUDA_TRY(cudaMemcpyAsync(h, sims, sizeof h, cudaMemcpyDeviceToHost, st));
  // the probe's judge reset the status header: a device error of the judge
  // or of the averages voids the probe (c2_get_status synchronises)
  rc = c2_get_status(d_ws, stream);
  if (rc) return rc;
  const double q = h[1] > 0 ? h[0] / h[1] : 1.0;
  if (h_quality) *h_quality = q;
  if (q >= (double)quality_threshold) return C2_OK;
  // below threshold: plain FastRandomHash clustering
  o.d_keys = nullptr;
  rc = c2_build_knn_graph(d_csr_ptr, d_csr_items, n_users, n_items, k, cfg->t, cfg->b, N, seed,
                          &o, d_nbr_id, d_nbr_inter, d_nbr_union, d_ws, base, stream);
  if (rc) return rc;
  // a device error of the fallback build takes precedence over the
  // informational fallback status
  rc = c2_get_status(d_ws, stream);
  if (rc) return rc;
  return C2_ERR_QUALITY_FALLBACK;
}

}  // extern "C"
