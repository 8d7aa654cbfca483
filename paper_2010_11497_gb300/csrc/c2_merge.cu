// Step 3 of Cluster-and-Conquer on sm_103a (Algorithm 3): every user's t
// cluster-local lists are folded into one list of the k best distinct
// neighbours, reusing the carried counts.  Also Eq. 1 (average similarity).
#include "c2_internal.cuh"

namespace c2 {

namespace {

// pos_of[i*n + u] = the slot of user u under function i.
__global__ void k_pos_of(const int32_t* __restrict__ cusers, int64_t S, int32_t n,
                         int32_t* __restrict__ pos_of) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int64_t i = s / n;
  pos_of[i * n + cusers[s]] = (int32_t)s;
}

// One warp per user; rows are folded 4 at a time (their slot and entry loads
// issued together).  The first row is the list; every later row drops the
// ids seen in an earlier row and is merged with the list by one bitonic merge
// (after compaction it stays sorted).  An id seen before carries the same
// counts (the similarity is exact), so it is in the list already or ranks
// below the list's k-th, which only improves: dropping it changes nothing.
// The ids seen so far sit in a per-warp open-addressing set in shared memory
// (one probe sequence per lane and row) when t * k <= 256, at most half of its
// 512 slots; larger products compare each row with the list by shuffles.
constexpr int kMergeSetLog = 9;
constexpr int kMergeSet = 1 << kMergeSetLog;

// Inserts id into the set; false when it was there already.  Ends within
// kMergeSet probes (the set never fills).
__device__ __forceinline__ bool merge_set_insert(int32_t* set, int32_t id) {
  uint32_t slot = ((uint32_t)id * 0x9E3779B1u) >> (32 - kMergeSetLog);
  for (int probe = 0; probe < kMergeSet; ++probe) {
    const int32_t old = atomicCAS(&set[slot], -1, id);
    if (old == -1) return true;
    if (old == id) return false;
    slot = (slot + 1) & (kMergeSet - 1);
  }
  return false;
}

__global__ void __launch_bounds__(256) k_merge(const int32_t* __restrict__ pos_of, int32_t n,
                                               int32_t t, int32_t k,
                                               const int32_t* __restrict__ lid,
                                               const int32_t* __restrict__ lin,
                                               const int32_t* __restrict__ lun,
                                               int32_t* __restrict__ nid,
                                               int32_t* __restrict__ nin,
                                               int32_t* __restrict__ nun, const DevHeader* hdr) {
  __shared__ int32_t s_id[8][32];
  __shared__ uint2 s_cu[8][32];
  __shared__ int32_t s_set[8][kMergeSet];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= n || dev_failed(hdr)) return;
  int32_t* set = s_set[warp];
  // rows beyond the set's half-full bound fall back to the shuffle scan
  const bool use_set = t * k <= kMergeSet / 2;
  if (use_set) {
    for (int i = lane; i < kMergeSet; i += 32) set[i] = -1;
    __syncwarp();
  }
  WarpList L;
  L.id = -1; L.c = 0; L.u = 0;
  for (int i0 = 0; i0 < t; i0 += 4) {
    WarpList R[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      R[r].id = -1; R[r].c = 0; R[r].u = 0;
      if (i0 + r < t && lane < k) {
        const int64_t s = pos_of[(int64_t)(i0 + r) * n + u];
        R[r].id = lid[s * k + lane];
        R[r].c = (uint32_t)lin[s * k + lane];
        R[r].u = (uint32_t)lun[s * k + lane];
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (i0 + r >= t) break;
      bool dup = false;
      if (use_set) {
        if (R[r].id >= 0) dup = !merge_set_insert(set, R[r].id);
      } else if (i0 + r > 0) {
        for (int j = 0; j < k; ++j) {
          const int32_t lj = __shfl_sync(0xffffffffu, L.id, j);   // every lane takes part
          dup |= R[r].id >= 0 && R[r].id == lj;
        }
      }
      if (i0 + r == 0) { L = R[0]; continue; }
      const unsigned keep = __ballot_sync(0xffffffffu, R[r].id >= 0 && !dup);
      if (keep == 0u) continue;
      // compact the survivors (still sorted) to the front
      if ((keep >> lane) & 1u) {
        const int d = __popc(keep & lanemask_lt());
        s_id[warp][d] = R[r].id;
        s_cu[warp][d] = make_uint2(R[r].c, R[r].u);
      }
      __syncwarp();
      WarpList b;
      b.id = -1; b.c = 0; b.u = 0;
      if (lane < __popc(keep)) {
        b.id = s_id[warp][lane];
        const uint2 cu = s_cu[warp][lane];
        b.c = cu.x; b.u = cu.y;
      }
      __syncwarp();
      L = warp_list_merge_sorted(L, k, b);
    }
  }
  if (lane < k) {
    const int64_t o = u * k + lane;
    nid[o] = L.id;
    nin[o] = L.id >= 0 ? (int32_t)L.c : 0;
    nun[o] = L.id >= 0 ? (int32_t)L.u : 0;
  }
}

// Eq. 1 in FP64: per-block partial sums over rows (fixed order), then one
// block adds the partials in block order.
constexpr int kAvgBlocks = 1024;

__global__ void k_avg_partial(const int32_t* __restrict__ nin, const int32_t* __restrict__ nun,
                              int64_t rows, int32_t k, double* __restrict__ partial) {
  __shared__ double red[256];
  const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
  double acc = 0.0;
  for (int64_t e = r0 * k + threadIdx.x; e < r1 * k; e += blockDim.x) {
    const int32_t U = nun[e];
    if (U > 0) acc += (double)nin[e] / (double)U;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_avg_final(const double* __restrict__ partial, int nb, double denom,
                            double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) acc += partial[j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / denom;
}

}  // namespace

c2_status run_merge(const int32_t* cusers, const Sizes& s, const int32_t* lid, const int32_t* lin,
                    const int32_t* lun, int32_t* nid, int32_t* nin, int32_t* nun, KnnWs& w,
                    cudaStream_t st) {
  if (s.n == 0) return C2_OK;
  Prof p(st, "merge");
  C2_LAUNCH(k_pos_of, div_up(s.S, 256), 256, 0, st, cusers, s.S, s.n, w.pos_of);
  C2_LAUNCH(k_merge, div_up((int64_t)s.n * 32, 256), 256, 0, st, w.pos_of, s.n, s.t, s.k, lid, lin, lun,
                                                          nid, nin, nun, w.hdr);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

c2_status run_avg_sim(const int32_t* nin, const int32_t* nun, int32_t rows, int32_t k, double* out,
                      DevHeader* hdr, double* partial, cudaStream_t st) {
  (void)hdr;
  if (rows <= 0) return C2_ERR_INVALID_ARG;
  const int nb = (int)std::min<int64_t>(kAvgBlocks, rows);
  C2_LAUNCH(k_avg_partial, nb, 256, 0, st, nin, nun, rows, k, partial);
  C2_LAUNCH(k_avg_final, 1, 256, 0, st, partial, nb, (double)k * (double)rows, out);
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // namespace c2
