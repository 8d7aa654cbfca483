// Step 3 (the per-user merge) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they merge: plug-ins
// whose host application owns every allocation, or real-time loops that forbid
// allocation after start-up.  They cannot provide the workspace the other
// entry points need.  c2_merge_topk_noalloc runs the same merge kernels with
// their scratch (the device status word and the slot index of every
// (function, user) pair) in a fixed array of this library instead.
#include <mutex>

#include "c2_internal.cuh"

namespace c2 {

namespace {

// Scratch shared by every call on a device: the status header, then
// pos_of[t * n_users].  Every GPU that loads the library holds these 8 MiB
// until the process exits.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
constexpr int64_t kStaticMaxSlots = (int64_t)((kStaticScratchBytes - 256) / sizeof(int32_t));

static __device__ __align__(256) unsigned char g_merge_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[256] = {nullptr};   // device address of g_merge_scratch, per device

// Device address of the scratch array on the current device.  Host code may
// not use &g_merge_scratch directly: on the host that name is only a stand-in
// for the device symbol.
c2_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return C2_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_merge_scratch) != cudaSuccess || !p) return C2_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return C2_OK;
}

}  // namespace

}  // namespace c2

using namespace c2;

extern "C" {

int64_t c2_merge_topk_noalloc_max_slots(void) { return kStaticMaxSlots; }

c2_status c2_merge_topk_noalloc(const int32_t* d_cusers, int32_t n_users, int32_t t, int32_t k,
                                const int32_t* d_loc_id, const int32_t* d_loc_inter,
                                const int32_t* d_loc_union, int32_t* d_nbr_id,
                                int32_t* d_nbr_inter, int32_t* d_nbr_union, c2_stream_t stream) {
  // the same argument checks and statuses as c2_merge_topk, then the cap of
  // the fixed scratch array
  c2_status rc = check_common(n_users, 0, k, t, 1, 2, nullptr);
  if (rc) return rc;
  if ((int64_t)t * n_users > kStaticMaxSlots) return C2_ERR_UNSUPPORTED;
  if (!d_cusers || !d_loc_id || !d_loc_inter || !d_loc_union || !d_nbr_id || !d_nbr_inter ||
      !d_nbr_union)
    return C2_ERR_INVALID_ARG;
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  KnnWs w{};
  w.hdr = reinterpret_cast<DevHeader*>(base);
  w.pos_of = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(base) + 256);
  // the status word must start at zero; pos_of is fully rewritten
  C2_CUDA_TRY(cudaMemsetAsync(w.hdr, 0, sizeof(DevHeader), st));
  Sizes s = make_sizes(n_users, 0, 0, k, t, 1, 2, nullptr);
  rc = run_merge(d_cusers, s, d_loc_id, d_loc_inter, d_loc_union, d_nbr_id, d_nbr_inter,
                 d_nbr_union, w, st);
  if (rc) return rc;
  C2_CUDA_TRY(cudaGetLastError());
  return C2_OK;
}

}  // extern "C"
