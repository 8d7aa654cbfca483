// C ABI entry points: argument checks, workspace layout, phase sequencing.
#include <string.h>

#include <algorithm>

#include "c2_internal.cuh"

namespace c2 {

// MinHash keys of the C^2/MinHash variant (c2_minhash.cu).
c2_status run_minhash_keys(const int32_t* ptr, const int32_t* items, const Sizes& s,
                           uint64_t seed, int32_t* keys, DevHeader* hdr, cudaStream_t st);

Sizes make_sizes(int32_t n, int64_t nnz, int32_t m, int32_t k, int32_t t, int32_t b, int32_t N,
                 const c2_options* opt) {
  Sizes s{};
  s.n = n; s.m = m; s.k = k; s.t = t; s.b = b; s.N = N; s.nnz = nnz;
  s.S = (int64_t)t * n;
  s.tp = (t + 7) / 8 * 8;
  s.omax = s.S / ((int64_t)N + 1) + 1;
  int64_t budget = (opt && opt->gram_budget_bytes > 0) ? opt->gram_budget_bytes : (int64_t(2) << 30);
  // sum over clusters of (M + 1) * round_up(M, 8) (the count rows and the row
  // of member lengths) <= S * (n + 15), two bytes each
  const int64_t worst = 2 * s.S * ((int64_t)std::max<int32_t>(n, 1) + 16);
  s.gram_budget = std::max<int64_t>(std::min(budget, worst), 2);
  // tensor-core count matrices, when the item universe and the strategy allow
  // that path; their remapped lists (one padded profile area per function)
  // live in the workspace tail, sized here when nnz is known
  const int strategy = opt ? opt->strategy : C2_STRATEGY_AUTO;
  const int32_t mk = (opt && opt->d_sim_ptr) ? opt->sim_n_items : m;   // local KNN universe
  s.tc = (strategy == C2_STRATEGY_AUTO || strategy == C2_STRATEGY_MMA) && mk >= 1 &&
         mk <= kGramTcMaxItems;
  s.rl_pn = s.tc && nnz > 0 ? rl_stride(nnz, n) : 0;
  return s;
}

void bind_cluster_ws(Ws& w, const Sizes& s, ClusterWs& c) {
  const int64_t S = s.S;
  const int64_t nbins = (int64_t)s.t * (s.b + 1);
  c.htab = w.take<uint16_t>((size_t)std::max<int64_t>(s.m, 1) * s.tp);
  c.key = w.take<int32_t>(S + 1);
  c.key2 = w.take<int32_t>(S + 1);
  c.key3 = w.take<int32_t>(S + 1);
  c.lab = w.take<int32_t>(S + 1);
  c.lab2 = w.take<int32_t>(S + 1);
  c.hist = w.take<int32_t>(nbins + 1);
  c.binlab = w.take<int32_t>(nbins + 1);
  c.ovlist = w.take<int32_t>(S + 1);
  c.lsize = w.take<int32_t>(S + 1);
  c.lsize2 = w.take<int32_t>(S + 1);
  c.leta = w.take<int32_t>(S + 1);
  c.leta2 = w.take<int32_t>(S + 1);
  c.lflag = w.take<int32_t>(S + 1);
  c.lflag2 = w.take<int32_t>(S + 1);
  c.ovidx = w.take<int32_t>(S + 1);
  c.nchild = w.take<int32_t>(S + 1);
  c.subcnt = w.take<int32_t>((size_t)s.omax * (s.b + 1));
  c.subrank = w.take<int32_t>((size_t)s.omax * (s.b + 1));
  c.sub_resid = w.take<int32_t>(s.omax);
  c.skey = w.take<uint32_t>(S + 1);
  c.skey2 = w.take<uint32_t>(S + 1);
  c.sval = w.take<int32_t>(S + 1);
  c.sval2 = w.take<int32_t>(S + 1);
  c.shist = w.take<uint32_t>(sort_hist_elems(S));
  c.scan_tmp = w.take<int32_t>(scan_tmp_elems(std::max<int64_t>({S, nbins, (int64_t)sort_hist_elems(S)})));
}

void bind_knn_ws(Ws& w, const Sizes& s, KnnWs& c) {
  const int64_t S = s.S;
  c.pptr16 = w.take<int32_t>((size_t)s.n + 1);
  c.slot2c = w.take<int32_t>(S + 1);
  c.slen = w.take<int32_t>(S + 1);
  c.small_cnt = w.take<int32_t>(S + 1);
  c.small_off = w.take<int32_t>(S + 1);
  c.small_slot = w.take<int32_t>(S + 1);
  c.gflag = w.take<int32_t>(S + 1);
  c.gidx = w.take<int32_t>(S + 1);
  c.work_c = w.take<int32_t>(S + 1);
  c.work_t = w.take<int32_t>(S + 1);
  c.gcl = w.take<int32_t>(S + 1);
  c.gsz = w.take<int32_t>(S + 1);
  c.gsq = w.take<int64_t>(S + 1);
  c.goff = w.take<int64_t>(S + 1);
  c.gofs = w.take<int64_t>(S + 1);
  c.bt_cnt = w.take<int32_t>(S + 1);
  c.bt_off = w.take<int32_t>(S + 1);
  c.bu_cnt = w.take<int32_t>(S + 1);
  c.bu_off = w.take<int32_t>(S + 1);
  c.gu_slot = w.take<int32_t>(S + 1);
  c.gu_g = w.take<int32_t>(S + 1);
  c.gw_g = w.take<int32_t>(S + 1);
  c.gw_t = w.take<int32_t>(S + 1);
  c.bw_cnt = w.take<int32_t>(S + 1);
  c.bw_off = w.take<int32_t>(S + 1);
  c.gseq = w.take<int32_t>(S + 1);
  c.gkind_c = w.take<int32_t>(S + 1);
  c.gkind = w.take<int32_t>(S + 1);
  c.bb_cnt = w.take<int32_t>(S + 1);
  c.bb_off = w.take<int32_t>(S + 1);
  c.ub_slot = w.take<int32_t>(S + 1);
  c.ub_g = w.take<int32_t>(S + 1);
  c.ipos = w.take<int32_t>(S + 1);
  c.iinfo = w.take<int2>(S + 1);
  c.islot = w.take<int4>(S + 1);
  c.chg0 = w.take<int32_t>(S + 1);
  c.chg1 = w.take<int32_t>(S + 1);
  c.gfresh = w.take<int32_t>(S + 1);
  c.pptr = w.take<int32_t>((int64_t)s.n + 1);
  c.wl0 = w.take<int32_t>((S + 1) * s.k);
  c.wl1 = w.take<int32_t>((S + 1) * s.k);
  c.gram = w.take<uint16_t>(s.gram_budget / 2);
  c.pos_of = w.take<int32_t>(S + 1);
  c.gk2 = w.take<int32_t>(S + 1);
  c.gsum = w.take<int64_t>(S + 1);
  c.groute = w.take<int32_t>(S + 1);
  c.gorder = w.take<int32_t>(S + 1);
  c.gt_list = w.take<int32_t>(S + 1);
  c.rl_len = w.take<int32_t>(S + 1);
  c.bg_flag = w.take<int32_t>(S + 1);
  c.bg_off = w.take<int32_t>(S + 1);
  c.bg_slot = w.take<int32_t>(S + 1);
  // tiles of one batch: at most 6 M^2 / (128 * 256) per cluster of M >= 128
  // members, and the batch's sum of M^2 is at most gram_budget / 2
  c.gt_work_cap = s.tc ? std::min<int64_t>(S + 64, 3 * s.gram_budget / 32768 + 64) : 0;
  c.gt_work = w.take<int4>((size_t)c.gt_work_cap + 1);
  c.rl_pn = 0;        // located in the tail once nnz is known (run_cluster_knn)
  c.rl = nullptr;
  c.partial = w.take<double>(1024);
  c.scan_tmp = w.take<int32_t>(scan_tmp_elems(S + 1));
  c.scan_tmp2 = w.take<int32_t>(scan_tmp_elems(S + 1));
  c.scan_tmp64 = w.take<int64_t>(scan_tmp_elems(S + 1));
}

// Build-owned intermediates of c2_build_knn_graph.
struct BuildBufs {
  int32_t *cluster_of, *cptr, *cusers, *ncl, *lid, *lin, *lun;
};

// Whole workspace: header, build intermediates, then the larger of the two
// phase scratch areas (they never live at the same time).
size_t layout(char* base, size_t ws_bytes, const Sizes& s, DevHeader** hdr, BuildBufs* bb,
              ClusterWs* cw, KnnWs* kw) {
  Ws w;
  w.base = base;
  DevHeader* h = w.take<DevHeader>(1);
  BuildBufs b{};
  b.cluster_of = w.take<int32_t>(s.S + 1);
  b.cptr = w.take<int32_t>(s.S + 1);
  b.cusers = w.take<int32_t>(s.S + 1);
  b.ncl = w.take<int32_t>(1);
  b.lid = w.take<int32_t>((s.S + 1) * s.k);
  b.lin = w.take<int32_t>((s.S + 1) * s.k);
  b.lun = w.take<int32_t>((s.S + 1) * s.k);
  const size_t phase = (w.top + 255) & ~size_t(255);
  Ws a = w;
  a.top = phase;
  ClusterWs c{};
  bind_cluster_ws(a, s, c);
  Ws k2 = w;
  k2.top = phase;
  KnnWs kk{};
  bind_knn_ws(k2, s, kk);
  c.hdr = h;
  kk.hdr = h;
  // the padded profiles take the rest of the workspace (sized by the caller
  // through c2_workspace_size, which knows nnz)
  const size_t fixed = (std::max(a.top, k2.top) + 255) & ~size_t(255);
  kk.pitems = reinterpret_cast<int32_t*>(base + fixed);
  kk.pitems_cap = ws_bytes > fixed ? (int64_t)((ws_bytes - fixed) / 4) : 0;
  kk.tail_bytes = ws_bytes > fixed ? (int64_t)(ws_bytes - fixed) : 0;
  if (hdr) *hdr = h;
  if (bb) *bb = b;
  if (cw) *cw = c;
  if (kw) *kw = kk;
  return fixed;
}

// Bytes of the tail before the remapped lists: the padded profiles (nnz
// entries over n rows) and their 16-bit copy.
size_t tail_bytes(int64_t nnz, int32_t n) { return rl_offset(nnz, n); }

bool sizes_ok(int32_t n, int32_t m, int32_t k, int32_t t, int32_t b, int32_t N) {
  return n >= 0 && m >= 0 && k >= 1 && k <= kMaxK && t >= 1 && t <= kMaxT && b >= 1 &&
         b <= kMaxB && N >= 2;
}

c2_status check_common(int32_t n, int32_t m, int32_t k, int32_t t, int32_t b, int32_t N,
                       const c2_options* opt) {
  if (n < 0 || m < 0 || k < 1 || t < 1 || b < 1 || N < 1) return C2_ERR_INVALID_ARG;
  if (!sizes_ok(n, m, k, t, b, N)) return C2_ERR_UNSUPPORTED;
  if ((int64_t)t * n >= (int64_t(1) << 31) - 1) return C2_ERR_UNSUPPORTED;
  if (opt) {
    if (opt->fn_offset < 0 || opt->cluster_base < 0) return C2_ERR_INVALID_ARG;
    if (opt->d_sim_ptr && (opt->sim_n_items < 1 || (!opt->d_sim_items && n > 0)))
      return C2_ERR_INVALID_ARG;
    if (opt->d_sim_bits && (opt->sim_n_items < 1 || opt->sim_n_items % 32))
      return C2_ERR_INVALID_ARG;
    if (opt->strategy < -1 || opt->strategy > 3) return C2_ERR_INVALID_ARG;
    if (opt->greedy_random < 0) return C2_ERR_INVALID_ARG;
  }
  return C2_OK;
}

c2_status check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (!ws || ((uintptr_t)ws & 255u)) return C2_ERR_WORKSPACE;
  if (ws_bytes < need) return C2_ERR_WORKSPACE;
  return C2_OK;
}

c2_options resolve(const c2_options* opt) {
  c2_options o;
  c2_default_options(&o);
  if (opt) o = *opt;
  return o;
}

}  // namespace c2

using namespace c2;

extern "C" {

void c2_default_options(c2_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->greedy_threshold = 0;
  opt->greedy_rounds = -1;
  opt->greedy_random = 0;
  opt->strategy = C2_STRATEGY_AUTO;
  opt->d_hash_table = nullptr;
  opt->gram_budget_bytes = 0;
  opt->d_keys = nullptr;
  opt->greedy_max_draws = 0;
  opt->sim_n_items = 0;
  opt->d_sim_ptr = nullptr;
  opt->d_sim_items = nullptr;
  opt->d_sim_bits = nullptr;
  opt->fn_offset = 0;
  opt->cluster_base = 0;
}

const char* c2_status_string(c2_status s) {
  switch (s) {
    case C2_OK: return "ok";
    case C2_ERR_INVALID_ARG: return "invalid argument";
    case C2_ERR_INVALID_CSR: return "invalid CSR profiles (not sorted sets of valid items)";
    case C2_ERR_UNSUPPORTED: return "size beyond the supported limits";
    case C2_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case C2_ERR_CUDA: return "CUDA runtime error";
    case C2_ERR_TIMEOUT: return "bounded device wait gave up";
    case C2_ERR_QUALITY_FALLBACK: return "learned proposer fell back to FastRandomHash";
  }
  return "unknown status";
}

size_t c2_workspace_size(int32_t n_users, int64_t nnz, int32_t n_items, int32_t k, int32_t t,
                         int32_t b, int32_t N, const c2_options* opt) {
  if (check_common(n_users, n_items, k, t, b, N, opt) != C2_OK || nnz < 0) return 0;
  Sizes s = make_sizes(n_users, nnz, n_items, k, t, b, N, opt);
  return layout(nullptr, 0, s, nullptr, nullptr, nullptr, nullptr) + tail_bytes(nnz, n_users) +
         (s.rl_pn ? rl_tail_bytes(nnz, n_users, t) : 0);
}

c2_status c2_reset_status(void* d_ws, c2_stream_t stream) {
  if (!d_ws) return C2_ERR_WORKSPACE;
  C2_CUDA_TRY(cudaMemsetAsync(d_ws, 0, sizeof(DevHeader), (cudaStream_t)stream));
  return C2_OK;
}

c2_status c2_get_status(const void* d_ws, c2_stream_t stream) {
  if (!d_ws) return C2_ERR_WORKSPACE;
  int32_t st = 0;
  C2_CUDA_TRY(cudaMemcpyAsync(&st, d_ws, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  C2_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return (c2_status)st;
}

c2_status c2_get_stats(const void* d_ws, c2_stream_t stream, c2_stats* out) {
  if (!d_ws || !out) return C2_ERR_INVALID_ARG;
  DevHeader h;
  C2_CUDA_TRY(cudaMemcpyAsync(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  C2_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  memset(out, 0, sizeof(*out));
  out->pairs = (int64_t)h.pairs;
  out->gram_pairs = (int64_t)h.gram_pairs;
  out->n_clusters = h.n_labels;
  out->split_levels = h.split_levels;
  out->n_greedy_clusters = h.n_greedy;
  out->max_cluster = h.max_cluster;
  out->max_profile = h.max_profile;
  out->greedy_users = h.greedy_users;
  out->item_visits_brute = (int64_t)h.item_visits[0];
  out->item_visits_greedy = (int64_t)h.item_visits[1];
  out->greedy_visits = (int64_t)h.greedy_visits;
  out->greedy_computed = (int64_t)h.greedy_computed;
  out->greedy_evaluated = (int64_t)h.greedy_evaluated;
  out->brute_gram_elems = (int64_t)h.brute_gram_elems;
  out->brute_rows = h.brute_rows;
  out->brute_pairs = (int64_t)h.brute_pairs;
  out->greedy_pairs = (int64_t)h.greedy_pairs;
  out->tc_macs = (int64_t)h.tc_macs;
  out->tc_clusters = h.tc_clusters;
  out->tc_tiles = h.tc_tiles;
  out->select_general = h.select_general;
  out->direct_users = h.direct_users;
  return C2_OK;
}

c2_status c2_frh_cluster(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                         int32_t n_items, int32_t t, int32_t b, int32_t N, uint64_t seed,
                         const c2_options* opt, int32_t* d_cluster_of, int32_t* d_cptr,
                         int32_t* d_cusers, int32_t* d_n_clusters, int32_t* d_cmeta, void* d_ws,
                         size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_common(n_users, n_items, 1, t, b, N, opt);
  if (rc) return rc;
  if (!d_csr_ptr || (!d_csr_items && n_users > 0) || !d_cluster_of || !d_cptr || !d_cusers ||
      !d_n_clusters)
    return C2_ERR_INVALID_ARG;
  Sizes s = make_sizes(n_users, 0, n_items, 1, t, b, N, opt);
  DevHeader* hdr;
  ClusterWs cw;
  size_t need = layout((char*)d_ws, ws_bytes, s, &hdr, nullptr, &cw, nullptr);
  rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  C2_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(DevHeader), st));
  c2_options o = resolve(opt);
  return run_frh_cluster(d_csr_ptr, d_csr_items, s, seed, o, d_cluster_of, d_cptr, d_cusers,
                         d_n_clusters, d_cmeta, cw, st);
}

c2_status c2_minhash_keys(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                          int32_t n_items, int32_t t, uint64_t seed, int32_t* d_keys, void* d_ws,
                          size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_common(n_users, n_items, 1, t, 2, 2, nullptr);
  if (rc) return rc;
  if (!d_csr_ptr || (!d_csr_items && n_users > 0) || !d_keys) return C2_ERR_INVALID_ARG;
  rc = check_ws(d_ws, ws_bytes, sizeof(DevHeader));
  if (rc) return rc;
  const Sizes s = make_sizes(n_users, 0, n_items, 1, t, 2, 2, nullptr);
  DevHeader* hdr = reinterpret_cast<DevHeader*>(d_ws);
  cudaStream_t st = (cudaStream_t)stream;
  C2_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(DevHeader), st));
  return run_minhash_keys(d_csr_ptr, d_csr_items, s, seed, d_keys, hdr, st);
}

c2_status c2_cluster_knn(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                         int32_t n_items, int32_t t, const int32_t* d_cptr,
                         const int32_t* d_cusers, const int32_t* d_n_clusters, int32_t k,
                         uint64_t seed, const c2_options* opt, int32_t* d_loc_id,
                         int32_t* d_loc_inter, int32_t* d_loc_union, void* d_ws,
                         size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_common(n_users, n_items, k, t, 1, 2, opt);
  if (rc) return rc;
  if (!d_csr_ptr || (!d_csr_items && n_users > 0) || !d_cptr || !d_cusers || !d_n_clusters ||
      !d_loc_id || !d_loc_inter || !d_loc_union)
    return C2_ERR_INVALID_ARG;
  Sizes s = make_sizes(n_users, 0, n_items, k, t, 1, 2, opt);
  DevHeader* hdr;
  KnnWs kw;
  size_t need = layout((char*)d_ws, ws_bytes, s, &hdr, nullptr, nullptr, &kw);
  rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  c2_options o = resolve(opt);
  return run_cluster_knn(d_csr_ptr, d_csr_items, s, d_cptr, d_cusers, d_n_clusters, seed, o,
                         d_loc_id, d_loc_inter, d_loc_union, kw, (cudaStream_t)stream);
}

c2_status c2_merge_topk(const int32_t* d_cusers, int32_t n_users, int32_t t, int32_t k,
                        const int32_t* d_loc_id, const int32_t* d_loc_inter,
                        const int32_t* d_loc_union, int32_t* d_nbr_id, int32_t* d_nbr_inter,
                        int32_t* d_nbr_union, void* d_ws, size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_common(n_users, 0, k, t, 1, 2, nullptr);
  if (rc) return rc;
  if (!d_cusers || !d_loc_id || !d_loc_inter || !d_loc_union || !d_nbr_id || !d_nbr_inter ||
      !d_nbr_union)
    return C2_ERR_INVALID_ARG;
  Sizes s = make_sizes(n_users, 0, 0, k, t, 1, 2, nullptr);
  DevHeader* hdr;
  KnnWs kw;
  size_t need = layout((char*)d_ws, ws_bytes, s, &hdr, nullptr, nullptr, &kw);
  rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  return run_merge(d_cusers, s, d_loc_id, d_loc_inter, d_loc_union, d_nbr_id, d_nbr_inter,
                   d_nbr_union, kw, (cudaStream_t)stream);
}

c2_status c2_build_knn_graph(const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                             int32_t n_users, int32_t n_items, int32_t k, int32_t t, int32_t b,
                             int32_t N, uint64_t seed, const c2_options* opt, int32_t* d_nbr_id,
                             int32_t* d_nbr_inter, int32_t* d_nbr_union, void* d_ws,
                             size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_common(n_users, n_items, k, t, b, N, opt);
  if (rc) return rc;
  if (!d_csr_ptr || (!d_csr_items && n_users > 0) || !d_nbr_id || !d_nbr_inter || !d_nbr_union)
    return C2_ERR_INVALID_ARG;
  Sizes s = make_sizes(n_users, 0, n_items, k, t, b, N, opt);
  DevHeader* hdr;
  BuildBufs bb;
  ClusterWs cw;
  KnnWs kw;
  size_t need = layout((char*)d_ws, ws_bytes, s, &hdr, &bb, &cw, &kw);
  rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  c2_options o = resolve(opt);
  C2_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(DevHeader), st));
  rc = run_frh_cluster(d_csr_ptr, d_csr_items, s, seed, o, bb.cluster_of, bb.cptr, bb.cusers,
                       bb.ncl, nullptr, cw, st);
  if (rc) return rc;
  // Steps 2-3 on the similarity profiles when given (Section II-F)
  const int32_t* kptr = o.d_sim_ptr ? o.d_sim_ptr : d_csr_ptr;
  const int32_t* kitems = o.d_sim_ptr ? o.d_sim_items : d_csr_items;
  Sizes sk = s;
  if (o.d_sim_ptr) {
    sk.m = o.sim_n_items;
    rc = run_validate(kptr, kitems, sk, hdr, st);
    if (rc) return rc;
  }
  rc = run_cluster_knn(kptr, kitems, sk, bb.cptr, bb.cusers, bb.ncl, seed, o, bb.lid, bb.lin,
                       bb.lun, kw, st);
  if (rc) return rc;
  return run_merge(bb.cusers, s, bb.lid, bb.lin, bb.lun, d_nbr_id, d_nbr_inter, d_nbr_union, kw,
                   st);
}

size_t c2_workspace_size_host(int32_t n_users, int64_t nnz, int32_t n_items, int32_t k,
                              int32_t t, int32_t b, int32_t N, const c2_options* opt) {
  size_t base = c2_workspace_size(n_users, nnz, n_items, k, t, b, N, opt);
  if (!base) return 0;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  return up(base) + up((size_t)(n_users + 1) * 4) + up((size_t)std::max<int64_t>(nnz, 1) * 4) +
         3 * up((size_t)n_users * k * 4);
}

c2_status c2_build_knn_graph_host(const int32_t* h_csr_ptr, const int32_t* h_csr_items,
                                  int32_t n_users, int32_t n_items, int32_t k, int32_t t,
                                  int32_t b, int32_t N, uint64_t seed, const c2_options* opt,
                                  int32_t* h_nbr_id, int32_t* h_nbr_inter, int32_t* h_nbr_union,
                                  void* d_ws, size_t ws_bytes, c2_stream_t stream) {
  if (!h_csr_ptr || n_users < 0) return C2_ERR_INVALID_ARG;
  const int64_t nnz = h_csr_ptr[n_users];
  if (nnz < 0) return C2_ERR_INVALID_CSR;
  size_t need = c2_workspace_size_host(n_users, nnz, n_items, k, t, b, N, opt);
  if (!need) return C2_ERR_INVALID_ARG;
  c2_status rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  if ((!h_csr_items && nnz > 0) || !h_nbr_id || !h_nbr_inter || !h_nbr_union)
    return C2_ERR_INVALID_ARG;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t base = c2_workspace_size(n_users, nnz, n_items, k, t, b, N, opt);
  char* p = (char*)d_ws + up(base);
  int32_t* d_ptr = (int32_t*)p;
  p += up((size_t)(n_users + 1) * 4);
  int32_t* d_items = (int32_t*)p;
  p += up((size_t)std::max<int64_t>(nnz, 1) * 4);
  const size_t rowb = (size_t)n_users * k * 4;
  int32_t* d_id = (int32_t*)p;
  p += up(rowb);
  int32_t* d_in = (int32_t*)p;
  p += up(rowb);
  int32_t* d_un = (int32_t*)p;
  cudaStream_t st = (cudaStream_t)stream;
  C2_CUDA_TRY(cudaMemcpyAsync(d_ptr, h_csr_ptr, (size_t)(n_users + 1) * 4, cudaMemcpyHostToDevice, st));
  if (nnz > 0)
    C2_CUDA_TRY(cudaMemcpyAsync(d_items, h_csr_items, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
  rc = c2_build_knn_graph(d_ptr, d_items, n_users, n_items, k, t, b, N, seed, opt, d_id, d_in,
                          d_un, d_ws, base, stream);
  if (rc) return rc;
  C2_CUDA_TRY(cudaMemcpyAsync(h_nbr_id, d_id, rowb, cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(h_nbr_inter, d_in, rowb, cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaMemcpyAsync(h_nbr_union, d_un, rowb, cudaMemcpyDeviceToHost, st));
  C2_CUDA_TRY(cudaStreamSynchronize(st));
  return c2_get_status(d_ws, stream);
}

c2_status c2_bruteforce_knn(const int32_t* d_csr_ptr, const int32_t* d_csr_items,
                            int32_t n_users, int32_t n_items, int32_t k,
                            const int32_t* d_queries, int32_t n_queries, int32_t* d_nbr_id,
                            int32_t* d_nbr_inter, int32_t* d_nbr_union, void* d_ws,
                            size_t ws_bytes, c2_stream_t stream) {
  c2_status rc = check_common(n_users, n_items, k, 1, 1, 2, nullptr);
  if (rc) return rc;
  if (!d_csr_ptr || !d_nbr_id || !d_nbr_inter || !d_nbr_union || (d_queries && n_queries < 0))
    return C2_ERR_INVALID_ARG;
  Sizes s = make_sizes(n_users, 0, n_items, k, 1, 1, 2, nullptr);
  DevHeader* hdr;
  KnnWs kw;
  size_t need = layout((char*)d_ws, ws_bytes, s, &hdr, nullptr, nullptr, &kw);
  rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  C2_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(DevHeader), st));
  rc = run_validate(d_csr_ptr, d_csr_items, s, hdr, st);
  if (rc) return rc;
  return run_bruteforce(d_csr_ptr, d_csr_items, s, d_queries, n_queries, d_nbr_id, d_nbr_inter,
                        d_nbr_union, kw, st);
}

c2_status c2_avg_sim(const int32_t* d_nbr_inter, const int32_t* d_nbr_union, int32_t rows,
                     int32_t k, double* d_out, void* d_ws, size_t ws_bytes, c2_stream_t stream) {
  if (!d_nbr_inter || !d_nbr_union || !d_out || rows <= 0 || k < 1 || k > kMaxK)
    return C2_ERR_INVALID_ARG;
  Sizes s = make_sizes(1, 0, 0, k, 1, 1, 2, nullptr);
  DevHeader* hdr;
  KnnWs kw;
  size_t need = layout((char*)d_ws, ws_bytes, s, &hdr, nullptr, nullptr, &kw);
  c2_status rc = check_ws(d_ws, ws_bytes, need);
  if (rc) return rc;
  return run_avg_sim(d_nbr_inter, d_nbr_union, rows, k, d_out, hdr, kw.partial,
                     (cudaStream_t)stream);
}

size_t c2_autotune_report(char* buf, size_t len) { return c2::autotune_report(buf, len); }
int32_t c2_autotune_save(const char* path) { return path ? c2::autotune_save(path) : -1; }
int32_t c2_autotune_load(const char* path) { return path ? c2::autotune_load(path) : -1; }

size_t c2_goldfinger_workspace_size(int32_t n_users) {
  if (n_users < 0) return 0;
  return goldfinger_ws_bytes(n_users);
}

c2_status c2_goldfinger(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                        int32_t n_items, int32_t bits, uint64_t seed, int32_t* d_fp_ptr,
                        int32_t* d_fp_items, uint32_t* d_fp_bits, void* d_ws, size_t ws_bytes,
                        c2_stream_t stream) {
  if (n_users < 0 || n_items < 0) return C2_ERR_INVALID_ARG;
  if (!d_csr_ptr || !d_fp_ptr || (n_users > 0 && (!d_csr_items || !d_fp_items)))
    return C2_ERR_INVALID_ARG;
  if (bits < 32 || bits > 8192 || bits % 32) return C2_ERR_UNSUPPORTED;
  c2_status rc = check_ws(d_ws, ws_bytes, goldfinger_ws_bytes(n_users));
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DevHeader* hdr = reinterpret_cast<DevHeader*>(d_ws);
  int32_t* scan_tmp = reinterpret_cast<int32_t*>((char*)d_ws + 256);
  C2_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(DevHeader), st));
  if (n_users == 0) {
    C2_CUDA_TRY(cudaMemsetAsync(d_fp_ptr, 0, sizeof(int32_t), st));
    return C2_OK;
  }
  return run_goldfinger(d_csr_ptr, d_csr_items, n_users, n_items, bits, seed, d_fp_ptr,
                        d_fp_items, d_fp_bits, hdr, scan_tmp, st);
}

c2_status c2_exact_counts(const int32_t* d_csr_ptr, const int32_t* d_csr_items, int32_t n_users,
                          int32_t k, const int32_t* d_nbr_id, int32_t* d_nbr_inter,
                          int32_t* d_nbr_union, c2_stream_t stream) {
  if (n_users < 0 || k < 1 || k > kMaxK) return k > kMaxK ? C2_ERR_UNSUPPORTED : C2_ERR_INVALID_ARG;
  if (!d_csr_ptr || (n_users > 0 && (!d_csr_items || !d_nbr_id || !d_nbr_inter || !d_nbr_union)))
    return C2_ERR_INVALID_ARG;
  return run_exact_counts(d_csr_ptr, d_csr_items, n_users, k, d_nbr_id, d_nbr_inter, d_nbr_union,
                          (cudaStream_t)stream);
}

}  // extern "C"
