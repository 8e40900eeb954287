// mpf_vit_api.cu -- host side of the P7Viterbi calls of the C ABI
// (mpf_vit_profile_create / _destroy, mpf_viterbi_scan, mpf_viterbi_rescore):
// profile tables, launch grouping and the MSV -> Viterbi hand-off.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/mpf.h"
#include "mpf_handles.h"
#include "mpf_internal.h"

using namespace mpf;
using namespace mpf::host;

struct mpf_vprofile {
  mpf_ctx *ctx = nullptr;
  int M = 0, K = 0, Mpad = 0;
  bool fast = false;            // every transition and special score <= 0
  int16_t *d_msc = nullptr;     // kVitRows x Mpad, striped
  int16_t *d_trans = nullptr;   // Mpad x kVitTrans, striped
  int sp[kVitSpecial] = {};
  int base = 0;
  float scale = 1.f;
};

namespace {

// Launch the Viterbi kernels over n_q queries: the general kernel for the
// profiles with a positive move, the fast kernel for the others, one launch
// per group of queries that share a kernel and launch shape (queries of one
// launch are scored one after the other by every block).  ranks /
// n_ranks (nullable) are [n_q][n_seqs] and [n_q] device arrays of selected
// length ranks.
int viterbi_enqueue(mpf_ctx *ctx, const mpf_vprofile *const *vps, int n_q, const mpf_db *db,
                    int16_t *score, uint8_t *flag, float *nat, const uint32_t *ranks,
                    const uint32_t *n_ranks) {
  const uint64_t n = db->n_seqs;
  // Group by kernel and launch shape (the key), then order by length.
  std::vector<std::tuple<int, int, int>> order;   // (key, Mpad, query)
  std::map<int, int> group_max;                    // key -> longest model of the group
  for (int q = 0; q < n_q; ++q) {
    const mpf_vprofile *v = vps[q];
    const int key = viterbi_shape_key(v->fast, v->Mpad, db->n_codes, ctx->max_smem, ctx->num_sms,
                                      ranks ? 0 : n);
    if (key < 0) return MPF_EUNSUPPORTED;
    order.emplace_back(key, v->Mpad, q);
    group_max[key] = std::max(group_max[key], v->Mpad);
  }
  // Groups with the longest models first (the launches are persistent and
  // fill the GPU in launch order, so the short-model groups finish last and
  // the final tail is short); within a group, longest models first.
  std::stable_sort(order.begin(), order.end(), [&](const std::tuple<int, int, int> &a,
                                                   const std::tuple<int, int, int> &b) {
    const int ga = group_max[std::get<0>(a)], gb = group_max[std::get<0>(b)];
    if (ga != gb) return ga > gb;
    if (std::get<0>(a) != std::get<0>(b)) return std::get<0>(a) < std::get<0>(b);
    return std::get<1>(a) > std::get<1>(b);
  });
  std::vector<VitQuery> qs;
  qs.reserve((size_t)n_q);
  for (const auto &o : order) {
    const int q = std::get<2>(o);
    const mpf_vprofile *v = vps[q];
    VitQuery d;
    memset(&d, 0, sizeof(d));
    d.msc = v->d_msc;
    d.trans = v->d_trans;
    for (int i = 0; i < kVitSpecial; ++i) d.sp[i] = v->sp[i];
    d.M = v->M;
    d.Mpad = v->Mpad;
    d.base = v->base;
    d.scale = v->scale;
    d.score = score + (uint64_t)q * n;
    d.flag = flag + (uint64_t)q * n;
    d.nat = nat ? nat + (uint64_t)q * n : nullptr;
    d.ranks = ranks ? ranks + (uint64_t)q * n : nullptr;
    d.n_ranks = n_ranks ? n_ranks + q : nullptr;
    d.team_max = viterbi_team_max(std::get<0>(o), v->Mpad, db->n_codes, ctx->max_smem, ctx->num_sms);
    qs.push_back(d);
  }
  // Groups run concurrently on the context's fork streams, so that one
  // group's tail overlaps the others' work.  Groups of models longer than
  // the shared-memory rows hold get their own slice of device scratch.
  std::vector<std::pair<int, int>> groups;
  std::vector<size_t> state_off, state_len;
  const size_t desc_bytes = sizeof(VitQuery) * (size_t)n_q;
  size_t total = (desc_bytes + 4 * (size_t)n_q + 255) & ~(size_t)255;
  for (int first = 0; first < n_q;) {
    int last = first;
    int max_Mpad = 32;
    while (last < n_q && std::get<0>(order[(size_t)last]) == std::get<0>(order[(size_t)first])) {
      max_Mpad = std::max(max_Mpad, std::get<1>(order[(size_t)last]));
      ++last;
    }
    const mpf_vprofile *v0 = vps[std::get<2>(order[(size_t)first])];
    const size_t len = vit_key_device_rows(std::get<0>(order[(size_t)first]))
                           ? viterbi_state_bytes(v0->fast, max_Mpad, ctx->num_sms)
                           : 0;
    groups.emplace_back(first, last);
    state_off.push_back(total);
    state_len.push_back(len);
    total += (len + 255) & ~(size_t)255;
    first = last;
  }
  uint8_t *dev = nullptr;
  MPF_CUDA(cudaMallocAsync((void **)&dev, total, ctx->stream));
  cudaError_t e = cudaMemcpyAsync(dev, qs.data(), desc_bytes, cudaMemcpyHostToDevice, ctx->stream);
  uint32_t *counters = reinterpret_cast<uint32_t *>(dev + desc_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 4 * (size_t)n_q, ctx->stream);
  int rc = e == cudaSuccess ? MPF_OK : MPF_ECUDA;
  const bool fork = groups.size() > 1;
  std::vector<cudaEvent_t> evs;
  if (fork && rc == MPF_OK) {
    while (ctx->n_fork < 8 && (size_t)ctx->n_fork < groups.size()) {
      if (cudaStreamCreateWithFlags(&ctx->fork[ctx->n_fork], cudaStreamNonBlocking) != cudaSuccess) break;
      ++ctx->n_fork;
    }
    for (size_t i = 0; i <= groups.size() && rc == MPF_OK; ++i) {
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = MPF_ECUDA;
      else evs.push_back(ev);
    }
    if (ctx->n_fork < 1) rc = MPF_ECUDA;
    if (rc == MPF_OK && cudaEventRecord(evs.back(), ctx->stream) != cudaSuccess) rc = MPF_ECUDA;
  }
  for (size_t gi = 0; gi < groups.size() && rc == MPF_OK; ++gi) {
    const int first = groups[gi].first, last = groups[gi].second;
    const int key = std::get<0>(order[(size_t)first]);
    int max_Mpad = 32;
    for (int i = first; i < last; ++i) max_Mpad = std::max(max_Mpad, std::get<1>(order[(size_t)i]));
    cudaStream_t st = ctx->stream;
    if (fork) {
      st = ctx->fork[gi % (size_t)ctx->n_fork];
      if (cudaStreamWaitEvent(st, evs.back(), 0) != cudaSuccess) {
        rc = MPF_ECUDA;
        break;
      }
    }
    VitParams p;
    p.residues = db->d_words;
    p.n_words = db->n_words;
    p.status = ctx->d_status;
    p.seq_word = db->d_seq_word;
    p.seq_len = db->d_seq_len;
    p.seq_orig = db->d_seq_orig;
    p.n_seqs = (uint32_t)n;
    p.n_queries = (uint32_t)(last - first);
    p.max_Mpad = max_Mpad;
    p.queries = reinterpret_cast<const VitQuery *>(dev) + first;
    p.counters = counters + first;
    p.state = state_len[gi] ? reinterpret_cast<uint2 *>(dev + state_off[gi]) : nullptr;
    p.state_bytes = state_len[gi];
    const int lr = launch_viterbi(p, key, db->n_codes, ctx->max_smem, ctx->num_sms, st);
    if (lr) rc = lr == 2 ? MPF_EUNSUPPORTED : MPF_ECUDA;
    if (fork && cudaEventRecord(evs[gi], st) != cudaSuccess) rc = MPF_ECUDA;
  }
  if (fork) {
    // Join every fork stream that may have work queued, then release the events.
    for (size_t gi = 0; gi < groups.size() && gi + 1 < evs.size(); ++gi)
      if (cudaStreamWaitEvent(ctx->stream, evs[gi], 0) != cudaSuccess) rc = MPF_ECUDA;
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  }
  cudaFreeAsync(dev, ctx->stream);
  (void)cudaGetLastError();
  return rc;
}

bool vit_args_ok(mpf_ctx *ctx, const mpf_vprofile *const *vps, int n_q, const mpf_db *db) {
  if (!ctx || !vps || n_q < 1 || !db || db->ctx->device != ctx->device) return false;
  for (int q = 0; q < n_q; ++q)
    if (!vps[q] || vps[q]->ctx->device != ctx->device) return false;
  return true;
}

}  // namespace

extern "C" {

int mpf_vit_profile_create(mpf_ctx *ctx, int M, int K, const int16_t *msc, const int16_t *trans,
                           const int16_t *special, int base, float scale, mpf_vprofile **out) {
  if (!out) return MPF_EINVAL;
  *out = nullptr;
  if (!ctx || !msc || !trans || !special || M < 1 || K < 1 || K > kVitRows) return MPF_EINVAL;
  if (base < -32768 || base > 32767 || !isfinite(scale) || !(scale > 0.f)) return MPF_EINVAL;
  if (M > kMaxLongM) return MPF_EUNSUPPORTED;
  const int Mpad = (M + 31) & ~31, Q = Mpad / 32;
  bool fast = true;
  for (size_t i = 0; i < (size_t)kVitTrans * M; ++i) fast = fast && trans[i] <= 0;
  for (int i = 0; i < kVitSpecial; ++i) fast = fast && special[i] <= 0;
  std::vector<int16_t> hm((size_t)kVitRows * Mpad, (int16_t)-32768);
  std::vector<int16_t> ht((size_t)kVitTrans * Mpad, (int16_t)-32768);
  // Striped: node k = l*Q + j in slot j*32 + l; transitions 8 per slot.
  for (int k = 0; k < M; ++k) {
    const size_t slot = (size_t)(k % Q) * 32 + (size_t)(k / Q);
    for (int x = 0; x < K; ++x) hm[(size_t)x * Mpad + slot] = msc[(size_t)x * M + k];
    for (int t = 0; t < kVitTrans; ++t) ht[slot * kVitTrans + t] = trans[(size_t)t * M + k];
  }
  mpf_vprofile *v = new (std::nothrow) mpf_vprofile;
  if (!v) return MPF_ENOMEM;
  v->fast = fast;
  v->ctx = ctx;
  v->M = M;
  v->K = K;
  v->Mpad = Mpad;
  for (int i = 0; i < kVitSpecial; ++i) v->sp[i] = special[i];
  v->base = base;
  v->scale = scale;
  DeviceGuard dg(ctx->device);
  cudaError_t e = cudaMalloc(&v->d_msc, hm.size() * sizeof(int16_t));
  if (e == cudaSuccess) e = cudaMalloc(&v->d_trans, ht.size() * sizeof(int16_t));
  if (e == cudaSuccess) e = cudaMemcpy(v->d_msc, hm.data(), hm.size() * sizeof(int16_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v->d_trans, ht.data(), ht.size() * sizeof(int16_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    mpf_vit_profile_destroy(v);
    return e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA;
  }
  *out = v;
  return MPF_OK;
}

void mpf_vit_profile_destroy(mpf_vprofile *v) {
  if (!v) return;
  DeviceGuard dg(v->ctx->device);
  cudaStreamSynchronize(v->ctx->stream);
  cudaFree(v->d_msc);
  cudaFree(v->d_trans);
  (void)cudaGetLastError();
  delete v;
}

int mpf_viterbi_scan(mpf_ctx *ctx, const mpf_vprofile *const *vps, int n_q, const mpf_db *db,
                     int16_t *score, uint8_t *overflow, float *nat) {
  if (!vit_args_ok(ctx, vps, n_q, db) || !score || !overflow) return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  const uint64_t n = (uint64_t)n_q * db->n_seqs;
  if (db->n_seqs == 0) return MPF_OK;
  const bool device_out = is_device_ptr(score) && is_device_ptr(overflow) && (!nat || is_device_ptr(nat));
  if (device_out) return viterbi_enqueue(ctx, vps, n_q, db, score, overflow, nat, nullptr, nullptr);
  int rc = ensure_out_scratch(ctx, (size_t)n * 7 + 64);
  if (rc) return rc;
  uint8_t *base = (uint8_t *)ctx->d_out;
  float *k_nat = nat ? (float *)base : nullptr;
  int16_t *k_score = reinterpret_cast<int16_t *>(base + (size_t)n * 4);
  uint8_t *k_flag = base + (size_t)n * 6;
  rc = viterbi_enqueue(ctx, vps, n_q, db, k_score, k_flag, k_nat, nullptr, nullptr);
  if (rc == MPF_OK) {
    cudaError_t e = cudaMemcpyAsync(score, k_score, n * 2, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(overflow, k_flag, n, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess && nat) e = cudaMemcpyAsync(nat, k_nat, n * 4, cudaMemcpyDefault, ctx->stream);
    if (e != cudaSuccess) rc = MPF_ECUDA;
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == MPF_OK) rc = MPF_ECUDA;
  (void)cudaGetLastError();
  return rc;
}

int mpf_viterbi_rescore(mpf_ctx *ctx, const mpf_vprofile *const *vps, int n_q, const mpf_db *db,
                        const uint8_t *msv_flag, const float *msv_nat, float msv_min_nat,
                        int16_t *score, uint8_t *overflow, float *nat, uint32_t *n_pass) {
  if (!vit_args_ok(ctx, vps, n_q, db) || !msv_flag || !msv_nat || !score || !overflow || !n_pass ||
      isnan(msv_min_nat))
    return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  for (const void *ptr : {(const void *)msv_flag, (const void *)msv_nat, (const void *)score,
                          (const void *)overflow, (const void *)n_pass})
    if (!is_device_ptr(ptr)) return MPF_EINVAL;
  if (nat && !is_device_ptr(nat)) return MPF_EINVAL;
  const uint64_t n = db->n_seqs;
  {  // The hand-off reads the MSV outputs while it writes the Viterbi ones: no two may share memory.
    const uint64_t nq = (uint64_t)n_q * n;
    const void *ptr[6] = {msv_flag, msv_nat, score, overflow, nat, n_pass};
    const uint64_t bytes[6] = {nq, 4 * nq, 2 * nq, nq, nat ? 4 * nq : 0, 4 * (uint64_t)n_q};
    if (ranges_overlap(ptr, bytes, 6)) return MPF_EINVAL;
  }
  const uint64_t n_chunks = (n + kSelectChunk - 1) / kSelectChunk;
  uint32_t *ranks = nullptr, *n_ranks = nullptr, *chunk = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&ranks, std::max<uint64_t>(1, (uint64_t)n_q * n) * 4, ctx->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&n_ranks, (size_t)n_q * 4, ctx->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&chunk, std::max<uint64_t>(1, 2 * (uint64_t)n_q * n_chunks) * 4, ctx->stream);
  int rc = e == cudaSuccess ? MPF_OK : (e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA);
  if (rc == MPF_OK && launch_select(db->d_seq_orig, n, n_q, msv_flag, msv_nat, msv_min_nat, score, 2,
                                    overflow, nat, chunk, chunk + (uint64_t)n_q * n_chunks, ranks,
                                    n_ranks, ctx->stream) != 0)
    rc = MPF_ECUDA;
  if (rc == MPF_OK && n > 0) rc = viterbi_enqueue(ctx, vps, n_q, db, score, overflow, nat, ranks, n_ranks);
  if (rc == MPF_OK && cudaMemcpyAsync(n_pass, n_ranks, (size_t)n_q * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
    rc = MPF_ECUDA;
  if (ranks) cudaFreeAsync(ranks, ctx->stream);
  if (n_ranks) cudaFreeAsync(n_ranks, ctx->stream);
  if (chunk) cudaFreeAsync(chunk, ctx->stream);
  (void)cudaGetLastError();
  return rc;
}

}  // extern "C"

