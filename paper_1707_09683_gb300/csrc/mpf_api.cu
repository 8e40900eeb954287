// mpf_api.cu -- host side of the C ABI declared in include/mpf.h: contexts,
// byte-filter profiles, the resident database, scans, plans, the SSV -> MSV
// pipeline and P-values (the allocation-free entry point is in
// mpf_noalloc.cu, the Viterbi calls in mpf_vit_api.cu).
//
// Owns device memory and streams, lays the database out in HBM, builds the
// striped cost tables, chooses kernel configurations and launches the scan
// kernels.  Every step of a scan itself runs in the kernels
// (mpf_scan_kernel.cuh, mpf_long_kernel.cu, mpf_pipeline.cu).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/mpf.h"
#include "mpf_handles.h"
#include "mpf_internal.h"

using namespace mpf;
using namespace mpf::host;

namespace mpf {
KernelFn kernel_for(int lanes, int words, int mode) {
  switch (lanes) {
    case 1: return kernel_lg1(words, mode);
    case 2: return kernel_lg2(words, mode);
    case 4: return kernel_lg4(words, mode);
    case 8: return kernel_lg8(words, mode);
    case 16: return kernel_lg16(words, mode);
    case 32: return kernel_lg32(words, mode);
    default: return nullptr;
  }
}
KernelFn kernel_qp_tm(int lanes, int words, int mode) {
  switch (lanes) {
    case 1: return kernel_qp_tm_lg1(words, mode);
    case 2: return kernel_qp_tm_lg2(words, mode);
    case 4: return kernel_qp_tm_lg4(words, mode);
    case 8: return kernel_qp_tm_lg8(words, mode);
    case 16: return kernel_qp_tm_lg16(words, mode);
    default: return nullptr;
  }
}
}  // namespace mpf

// ---------------------------------------------------------------- helpers --

namespace mpf {
namespace host {

const int kLanes[6] = {1, 2, 4, 8, 16, 32};

bool words_built(int w) { return w >= 4 && w <= kMaxWords && (w % 4 == 0 || w % 4 == 2); }

int smem_need(int lanes, int words) { return (int)table_geom(lanes, words).table_bytes; }

// Default (lanes, words) for a kernel mode: the fewest lanes per sequence
// whose rows need at most 40 words (48 for whole-warp groups), using the
// smallest built word count that covers M and whose table fits on chip.
void default_config(const mpf_ctx *ctx, int M, int mode, int *lanes, int *words) {
  for (int i = 0; i < 6; ++i) {
    const int lg = kLanes[i];
    int w = (M + 2 * lg - 1) / (2 * lg);
    w = std::max(4, (w + 1) / 2 * 2);
    if (!kernel_for(lg, w, mode)) w = (w + 3) / 4 * 4;
    const int wmax = lg == 32 ? kMaxWords : 40;
    if (w <= wmax && kernel_for(lg, w, mode) && smem_need(lg, w) <= ctx->max_smem) {
      *lanes = lg;
      *words = w;
      return;
    }
  }
  *lanes = 0;
  *words = 0;
}

// MSV_FAST needs the first begin score of every sequence below 255 - bias.
bool msv_fast_ok(const mpf_profile *p) {
  int xb = p->base - (p->tjb_min + p->tbm);
  xb = std::min(255, std::max(0, xb));
  return p->bias < 255 && xb < 255 - p->bias;
}

// IEEE half bits of an integer that half represents exactly (|v| <= 2048,
// or the padding score -16384).
uint16_t half_bits(int v) {
  if (v == 0) return 0;
  const uint16_t sign = v < 0 ? 0x8000 : 0;
  unsigned a = (unsigned)(v < 0 ? -v : v);
  int e = 31 - __builtin_clz(a);                        // a in [2^e, 2^(e+1))
  const unsigned m = e <= 10 ? (a << (10 - e)) - 1024u : (a >> (e - 10)) - 1024u;
  return (uint16_t)(sign | ((unsigned)(e + 15) << 10) | (m & 0x3ffu));
}

// Fill the striped shared-memory image of a profile for (lanes, words) in
// table format fmt: 16-bit scores s = bias - cost per (copy, residue row,
// word quad, lane, word, half), then 33 int16 per-code best scores.
void fill_table_image(const mpf_profile *p, const TableGeom &g, int fmt, uint8_t *img) {
  memset(img, 0, g.table_bytes);
  const int M = p->M, lanes = g.lanes, words = g.words;
  // Signed score of node k (0-based) for residue code x; padding nodes and
  // the padding code score kNegInf.
  auto score = [&](int x, int k) -> int {
    if (x >= 32 || k >= M) return kNegInf;
    const int c = x < p->K ? (int)p->cost[(size_t)x * M + k] : 255;
    return p->bias - c;
  };
  auto put = [&](size_t off, int x, int k) {
    const int sv = score(x, k);
    const uint16_t bits = fmt == TABLE_F16 ? half_bits(sv) : (uint16_t)(int16_t)sv;
    memcpy(&img[off], &bits, 2);
  };
  const int qw = 4 * g.quads;   // words held in the quad region
  for (int x = 0; x < kTableRows; ++x)
    for (int l = 0; l < lanes; ++l)
      for (int q = 0; q < words; ++q)
        for (int h = 0; h < 2; ++h) {
          const int k = (2 * l + h) * words + q;   // striped cell of (lane, half, word)
          if (q < qw) {
            for (int c = 0; c < g.copies; ++c)
              put((size_t)c * g.copy_bytes + (size_t)x * g.row_bytes +
                      ((size_t)(q / 4) * lanes + l) * 16 + (q % 4) * 4 + h * 2, x, k);
          } else {
            for (int c = 0; c < g.tail_copies; ++c)
              put(g.tail_off + (size_t)x * g.tail_row_bytes + ((size_t)c * lanes + l) * 8 +
                      (q - qw) * 4 + h * 2, x, k);
          }
        }
  for (int x = 0; x < kTableRows; ++x) {
    int m = kNegInf;
    if (x < 32)
      for (int k = 0; k < M; ++k) m = std::max(m, score(x, k));
    const int16_t sv = (int16_t)m;
    memcpy(&img[g.smax_off + 2 * x], &sv, 2);
  }
}

// Build (or fetch) the device copy of a profile's table image.
int get_table(const mpf_profile *p, int lanes, int words, int fmt, DevTable *out) {
  std::lock_guard<std::mutex> lk(p->mu);
  auto key = std::make_tuple(lanes, words, fmt);
  auto it = p->tables.find(key);
  if (it != p->tables.end()) {
    *out = it->second;
    return MPF_OK;
  }
  const TableGeom g = table_geom(lanes, words, fmt == TABLE_I16_PACKED);
  std::vector<uint8_t> img(g.table_bytes, 0);
  fill_table_image(p, g, fmt, img.data());
  mpf_ctx *ctx = p->ctx;
  DeviceGuard dg(ctx->device);
  uint4 *d = nullptr;
  MPF_CUDA(cudaMallocAsync((void **)&d, g.table_bytes, ctx->util));
  cudaError_t e = cudaMemcpyAsync(d, img.data(), g.table_bytes, cudaMemcpyHostToDevice, ctx->util);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->util);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFreeAsync(d, ctx->util);
    return MPF_ECUDA;
  }
  DevTable t;
  t.ptr = d;
  t.geom = g;
  p->tables[key] = t;
  *out = t;
  return MPF_OK;
}

// Device copy of a long profile's cost bytes in the long-model kernel's order:
// residue row x, word w of lane l at (x * seg_words + w) * 32 + l, four nodes
// (l * 4 * seg_words + 4w .. +3) per word; codes >= K and nodes past M cost 255.
int get_long_table(const mpf_profile *p, const uint8_t **out) {
  std::lock_guard<std::mutex> lk(p->mu);
  auto key = std::make_tuple(32, 0, 2);
  auto it = p->tables.find(key);
  if (it != p->tables.end()) {
    *out = reinterpret_cast<const uint8_t *>(it->second.ptr);
    return MPF_OK;
  }
  const int sw = p->seg_words, Q = 4 * sw, M = p->M;
  const size_t row = (size_t)sw * 32 * 4;
  std::vector<uint8_t> img(32 * row, 255);
  for (int x = 0; x < p->K; ++x)
    for (int k = 0; k < M; ++k) {
      const int l = k / Q, j = k % Q;
      img[(size_t)x * row + ((size_t)(j / 4) * 32 + l) * 4 + (j % 4)] = p->cost[(size_t)x * M + k];
    }
  mpf_ctx *ctx = p->ctx;
  DeviceGuard dg(ctx->device);
  uint4 *d = nullptr;
  MPF_CUDA(cudaMallocAsync((void **)&d, img.size(), ctx->util));
  cudaError_t e = cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, ctx->util);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->util);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFreeAsync(d, ctx->util);
    return MPF_ECUDA;
  }
  DevTable t;
  t.ptr = d;
  p->tables[key] = t;
  *out = reinterpret_cast<const uint8_t *>(d);
  return MPF_OK;
}

// Device copy of a long profile's scores for the tiled kernel: per tile of
// kTileNodes nodes, [code][chunk][lane] x 4 pairs of int16, lane l's pair
// p = (node l * kTileC + p, the same + kTileC / 2) of the tile, chunk p / 4;
// s = bias - cost (codes >= K cost 255), -32768 past M; then the 32 per-code
// maxima of s over the model.
int get_tile_table(const mpf_profile *p, const uint4 **out) {
  std::lock_guard<std::mutex> lk(p->mu);
  auto key = std::make_tuple(32, 0, 3);
  auto it = p->tables.find(key);
  if (it != p->tables.end()) {
    *out = it->second.ptr;
    return MPF_OK;
  }
  const int M = p->M, nt = (M + kTileNodes - 1) / kTileNodes;
  constexpr int kChunks = kTileC / 8;
  std::vector<int16_t> img((size_t)nt * kTileTableBytes / 2 + 32);
  for (int x = 0; x < 32; ++x) {
    int m = p->bias - 255;
    if (x < p->K)
      for (int k = 0; k < M; ++k) m = std::max(m, p->bias - (int)p->cost[(size_t)x * M + k]);
    img[(size_t)nt * kTileTableBytes / 2 + x] = (int16_t)m;
  }
  for (int t = 0; t < nt; ++t)
    for (int x = 0; x < 32; ++x)
      for (int l = 0; l < 32; ++l)
        for (int c = 0; c < kTileC; ++c) {
          const int k = t * kTileNodes + l * kTileC + c;
          int16_t s = -32768;
          if (k < M) s = (int16_t)(p->bias - (x < p->K ? (int)p->cost[(size_t)x * M + k] : 255));
          const int pr = c % (kTileC / 2), half = c / (kTileC / 2);
          const size_t chunk = (((size_t)t * 32 + x) * kChunks + pr / 4) * 32 + l;
          img[chunk * 8 + (pr % 4) * 2 + half] = s;
        }
  mpf_ctx *ctx = p->ctx;
  DeviceGuard dg(ctx->device);
  uint4 *d = nullptr;
  const size_t bytes = img.size() * sizeof(int16_t);
  MPF_CUDA(cudaMallocAsync((void **)&d, bytes, ctx->util));
  cudaError_t e = cudaMemcpyAsync(d, img.data(), bytes, cudaMemcpyHostToDevice, ctx->util);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->util);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFreeAsync(d, ctx->util);
    return MPF_ECUDA;
  }
  DevTable t;
  t.ptr = d;
  p->tables[key] = t;
  *out = d;
  return MPF_OK;
}

int ensure_out_scratch(mpf_ctx *ctx, size_t bytes) {
  if (ctx->d_out_bytes >= bytes) return MPF_OK;
  if (ctx->d_out) {
    MPF_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_out);
    ctx->d_out = nullptr;
    ctx->d_out_bytes = 0;
  }
  MPF_CUDA(cudaMalloc(&ctx->d_out, bytes));
  ctx->d_out_bytes = bytes;
  return MPF_OK;
}

// Kernel mode of a profile for a filter.  Automatic arithmetic: 16-bit
// integer cells (DPX on the integer pipe); fp16 cells only when asked for.
int kernel_mode(const mpf_profile *p, int filter) {
  if (p->seg_words) return filter == MPF_SSV ? MODE_TILE_SSV : msv_fast_ok(p) ? MODE_TILE_MSV : MODE_LONG_MSV;
  const bool f16 = p->arith[filter] == MPF_ARITH_F16;
  if (filter == MPF_SSV) return f16 ? MODE_SSV_F16 : MODE_SSV;
  if (!msv_fast_ok(p)) return MODE_MSV_DIRECT;
  return f16 ? MODE_MSV_HELD_F16 : MODE_MSV_HELD;
}

// The mode that scores a profile for both filters in one sweep, or -1:
// MSV runs a held pass (striped or tiled) and SSV the matching integer
// kernel; striped profiles also need the same configuration and table
// memory for both filters.
int fused_mode(const mpf_profile *p) {
  const int mm = kernel_mode(p, MPF_MSV), ms = kernel_mode(p, MPF_SSV);
  if (mm == MODE_TILE_MSV && ms == MODE_TILE_SSV) return MODE_TILE_MSV_SSV;
  const bool same = p->cfg_lanes[MPF_MSV] == p->cfg_lanes[MPF_SSV] && p->cfg_words[MPF_MSV] == p->cfg_words[MPF_SSV] &&
                    p->table_mem[MPF_MSV] == p->table_mem[MPF_SSV];
  return (mm == MODE_MSV_HELD && ms == MODE_SSV && same) ? MODE_MSV_SSV : -1;
}

// Whether a striped scan of this profile reads its table from tensor memory:
// one sequence per warp, enough words per lane, a mode with a TMEM kernel,
// and the profile's choice (automatic: yes).
bool use_tmem(const mpf_profile *p, int filter, int lanes, int words, int mode) {
  if (p->table_mem[filter] == MPF_TABLE_SHARED) return false;
  return lanes == 32 && words >= kTmMinWords && mode != MODE_MSV_DIRECT &&
         kernel_lg32_tm(words, mode) != nullptr;
}

// Packed sets of the candidates of one (lanes, mode), their word counts
// ascending: runs [a, b) of consecutive queries; a run of two or more is a
// set, padded to its largest word count, a run of one keeps its one-query
// kernel.  The runs minimise a cost in warp-words per sequence row (times 4
// below): a set costs (32 / lanes) x H, a query alone 5/4 of its own words
// (the one-query kernels read every word from shared memory and run at about
// 4/5 of the tensor-memory kernels' rate).  A set holds at most 32 / lanes
// queries and needs a built kernel for H and tables that fit max_smem.
std::vector<std::pair<size_t, size_t>> pack_runs(int lanes, int mode, const std::vector<int> &words,
                                                 int max_smem) {
  const size_t n = words.size();
  const int QP = 32 / lanes;
  auto packable = [&](int H) {
    return kernel_qp_tm(lanes, H, mode) != nullptr &&
           (uint64_t)QP * packed_table_stride(lanes, H) <= (uint64_t)max_smem;
  };
  // cost[b]: least cost of the first b queries; from[b]: start of the last run.
  std::vector<int64_t> cost(n + 1, 0);
  std::vector<size_t> from(n + 1, 0);
  for (size_t b = 1; b <= n; ++b) {
    cost[b] = cost[b - 1] + 5 * (int64_t)words[b - 1];
    from[b] = b - 1;
    const int H = words[b - 1];
    if (!packable(H)) continue;
    for (size_t a = b >= (size_t)QP ? b - (size_t)QP : 0; a + 2 <= b; ++a) {
      const int64_t c = cost[a] + 4 * (int64_t)QP * H;
      if (c < cost[b]) {
        cost[b] = c;
        from[b] = a;
      }
    }
  }
  std::vector<std::pair<size_t, size_t>> runs;
  for (size_t b = n; b > 0; b = from[b]) runs.emplace_back(from[b], b);
  std::reverse(runs.begin(), runs.end());
  return runs;
}

}  // namespace host
}  // namespace mpf

// One launch of the scan kernel over a set of queries sharing a kernel
// configuration.  Device arrays are owned by the group.
struct LaunchGroup {
  KernelFn fn = nullptr;
  int lanes = 0, words = 0, mode = 0;
  uint32_t smem = 0;
  int grid = 0;
  int threads = kBlockThreads;
  uint32_t long_words = 0;       // long-model kernel: largest seg_words of the group
  int n_codes = 32;              // distinct residue codes of the database
  uint32_t n_shards = 0;
  QueryDesc *d_queries = nullptr;
  uint32_t n_queries = 0;
  uint32_t *d_counter = nullptr;
  uint8_t *d_col = nullptr;      // tiled kernel: two columns of col_stride bytes per resident warp
  uint32_t col_stride = 0;
  uint64_t col_bytes = 0;
  uint32_t *d_fallback = nullptr;   // tiled MSV: per query a count, then n_seqs ranks per query
  bool tm = false;                  // striped kernel with the table in tensor memory
  int shard_factor = 1;             // striped kernels: shards = factor x resident blocks
  uint32_t n_real = 0;              // queries of the group (n_queries less empty slots of packed sets)
  int qp = 1;                       // tensor-memory kernels: queries scored per warp and sequence
  uint32_t qp_stride = 0;           //   and shared-memory bytes per staged table (qp > 1)
  std::shared_ptr<LaunchGroup> next;   // launched after this group on the same stream
};

struct mpf_plan {
  mpf_ctx *ctx = nullptr;
  const mpf_db *db = nullptr;
  std::vector<LaunchGroup> groups;
  std::vector<cudaEvent_t> events;   // fork/join events (more than one group)
  cudaGraphExec_t graph = nullptr;
};

namespace {

void plan_free(mpf_plan *pl) {
  if (!pl) return;
  DeviceGuard dg(pl->ctx->device);
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  // Ordered after the plan's last launch, which joins back into this stream.
  for (auto &g0 : pl->groups)
    for (LaunchGroup *g = &g0; g; g = g->next.get()) {
      if (g->d_queries) cudaFreeAsync(g->d_queries, pl->ctx->stream);
      if (g->d_counter) cudaFreeAsync(g->d_counter, pl->ctx->stream);
      if (g->d_col) cudaFreeAsync(g->d_col, pl->ctx->stream);
      if (g->d_fallback) cudaFreeAsync(g->d_fallback, pl->ctx->stream);
    }
  for (auto e : pl->events) cudaEventDestroy(e);
  (void)cudaGetLastError();
  delete pl;
}

int free_pending(mpf_ctx *ctx) {
  if (ctx->pending.empty()) return MPF_OK;
  MPF_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto *pl : ctx->pending) plan_free(pl);
  ctx->pending.clear();
  return MPF_OK;
}

int configure_kernel(mpf_ctx *ctx, LaunchGroup *g) {
  if (g->mode == MODE_TILE_SSV || g->mode == MODE_TILE_MSV || g->mode == MODE_TILE_MSV_SSV) {
    // Blocks of kTileWarps warps with one tile's scores in shared memory, or
    // (tm) one block of kTileWarpsTm warps per SM with the tile in TMEM: it
    // asks for more than half the shared memory so that no second block of
    // the kernel shares the SM.
    g->fn = tile_kernel_fn(g->mode, g->tm);
    g->threads = (g->tm ? kTileWarpsTm : kTileWarps) * 32;
    g->smem = g->tm ? (uint32_t)ctx->max_smem / 2 + 1024 : (uint32_t)kTileTableBytes;
    MPF_CUDA(cudaFuncSetAttribute((const void *)g->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)g->smem));
    MPF_CUDA(cudaFuncSetAttribute((const void *)g->fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    MPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)g->fn, g->threads,
                                                           g->smem));
    if (per_sm < 1 || (g->tm && per_sm != 1)) return MPF_EUNSUPPORTED;
    g->grid = ctx->num_sms * per_sm;
    g->n_shards = (uint32_t)g->grid;
    return MPF_OK;
  }
  if (g->mode == MODE_LONG_MSV) {
    // Each warp reads the cost rows of its residues from device memory, so
    // when the rows of the codes the database uses (n_codes x 128 x
    // seg_words bytes) fit in the L1 of the smallest carveout (156 KB, with
    // margin: 124 KB), take among the shared-memory carveouts that leave that
    // much L1 the one that keeps the most warps resident; when they cannot
    // fit, just keep the most warps resident (blocks of up to
    // kLongThreads / 32 warps).
    // The DP row is kept as 16-bit pairs unless that leaves fewer than four
    // warps per SM; then as bytes (half the shared memory per warp).
    const bool bytes = 4 * long_smem_per_warp((int)g->long_words, false) > 228 * 1024;
    g->fn = long_kernel_for(g->mode, bytes, (int)g->long_words);
    const size_t per_warp = long_smem_per_warp((int)g->long_words, bytes);
    constexpr size_t kKB = 1024;
    size_t ws = (size_t)std::max(g->n_codes, 1) * 128 * g->long_words;
    if (ws > 124 * kKB) ws = 0;
    static const int carves_kb[] = {228, 196, 164, 132, 100};
    int best_w = 0, best_b = 0, carve = 0;
    for (int c : carves_kb) {
      const size_t C = (size_t)c * kKB;
      if (256 * kKB - C < ws) continue;
      for (int w = kLongThreads / 32; w >= 1; --w) {
        const size_t sm = per_warp * (size_t)w;
        if (sm > (size_t)ctx->max_smem || sm + kKB > C) continue;
        const int b = std::min((int)(C / (sm + kKB)), 64 / w);
        if (w * b > best_w * best_b) {
          best_w = w;
          best_b = b;
        }
      }
      if (best_w) {
        carve = c;
        break;
      }
    }
    if (!best_w) return MPF_EUNSUPPORTED;
    g->threads = best_w * 32;
    g->smem = (uint32_t)(per_warp * (size_t)best_w);
    MPF_CUDA(cudaFuncSetAttribute((const void *)g->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)g->smem));
    // The driver takes the smallest supported carveout at or above the
    // preference: ask for just under the chosen one.
    MPF_CUDA(cudaFuncSetAttribute((const void *)g->fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)std::min<size_t>(100, (((size_t)carve - 1) * 100) / 228)));
    int per_sm = 0;
    MPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)g->fn, g->threads,
                                                           g->smem));
    if (per_sm < 1) return MPF_EUNSUPPORTED;
    g->grid = ctx->num_sms * std::min(per_sm, best_b);
    g->n_shards = (uint32_t)g->grid;
    return MPF_OK;
  }
  g->fn = g->qp > 1 ? kernel_qp_tm(g->lanes, g->words, g->mode)
         : g->tm    ? kernel_lg32_tm(g->words, g->mode)
                    : kernel_for(g->lanes, g->words, g->mode);
  if (!g->fn) return MPF_EINVAL;
  g->smem = g->qp > 1 ? (uint32_t)g->qp * g->qp_stride : (uint32_t)smem_need(g->lanes, g->words);
  if (g->smem > (uint32_t)ctx->max_smem) return MPF_EUNSUPPORTED;
  // A block with the table in tensor memory takes all of the SM's TMEM
  // columns: ask for more than half the shared memory, so no second block of
  // the kernel is placed on the SM.
  if (g->tm) g->smem = std::max<uint32_t>(g->smem, (uint32_t)ctx->max_smem / 2 + 1024);
  MPF_CUDA(cudaFuncSetAttribute((const void *)g->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)g->smem));
  int per_sm = 0;
  MPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)g->fn,
                                                         kBlockThreads, g->smem));
  if (per_sm < 1 || (g->tm && per_sm != 1)) return MPF_EUNSUPPORTED;
  g->grid = ctx->num_sms * per_sm;
  g->n_shards = (uint32_t)g->grid * (uint32_t)std::max(1, g->shard_factor);
  return MPF_OK;
}

// Build a plan: queries grouped by kernel configuration.
// ranks/n_ranks (nullable): query i scores only the n_ranks[i] length ranks
// listed at ranks + i * n_seqs (device memory).
int plan_create(mpf_ctx *ctx, int filter, const mpf_profile *const *profs, int n_q,
                const mpf_db *db, uint8_t *raw, uint8_t *flag, float *nat, mpf_plan **out,
                const uint32_t *ranks = nullptr, const uint32_t *n_ranks = nullptr) {
  if (!ctx || !profs || n_q < 1 || !db || !raw || !flag || !out) return MPF_EINVAL;
  if (filter != MPF_MSV && filter != MPF_SSV && filter != MPF_MSV_SSV) return MPF_EINVAL;
  if (filter == MPF_MSV_SSV && ranks) return MPF_EINVAL;
  if (db->ctx->device != ctx->device) return MPF_EINVAL;
  mpf_plan *pl = new (std::nothrow) mpf_plan;
  if (!pl) return MPF_ENOMEM;
  pl->ctx = ctx;
  pl->db = db;
  // Launch groups by (lanes, words, mode, table in tensor memory, queries
  // per warp).
  using GroupKey = std::tuple<int, int, int, int, int>;
  std::map<GroupKey, std::vector<QueryDesc>> byconf;
  std::map<GroupKey, std::vector<DevTable>> fb_table;   // tables of the exact rescoring launch
  std::map<GroupKey, std::vector<uint32_t>> fb_seg_words;
  std::map<GroupKey, int> group_shards;   // largest shard factor of a group's profiles
  // Queries that may share a warp's sequence with others (fewer than 32
  // lanes; integer SSV, held MSV or both), by (lanes, mode): placed after the loop.
  struct QpCand {
    int words, sf;
    const mpf_profile *p;
    QueryDesc q;
    DevTable fb;
  };
  std::map<std::pair<int, int>, std::vector<QpCand>> qp_cand;
  // One job per (query, kernel mode): MPF_MSV_SSV scores a query once for
  // both filters where it can (MODE_MSV_SSV, with the MSV settings), else
  // runs each filter's kernel into its output block (0: MSV, 1: SSV).
  struct Job {
    int i, filter, mode, block;
  };
  std::vector<Job> jobs;
  for (int i = 0; i < n_q; ++i) {
    const mpf_profile *p = profs[i];
    if (!p || p->ctx->device != ctx->device) {
      plan_free(pl);
      return MPF_EINVAL;
    }
    if (filter != MPF_MSV_SSV) {
      jobs.push_back(Job{i, filter, kernel_mode(p, filter), 0});
    } else if (fused_mode(p) >= 0) {
      jobs.push_back(Job{i, MPF_MSV, fused_mode(p), 0});
    } else {
      jobs.push_back(Job{i, MPF_MSV, kernel_mode(p, MPF_MSV), 0});
      jobs.push_back(Job{i, MPF_SSV, kernel_mode(p, MPF_SSV), 1});
    }
  }
  auto set_table = [](QueryDesc &q, const DevTable &t) {
    q.table = t.ptr;
    q.table_bytes = t.geom.table_bytes;
    q.row_bytes = t.geom.row_bytes;
    q.copy_bytes = t.geom.copy_bytes;
    q.smax_off = t.geom.smax_off;
    q.tail_off = t.geom.tail_off;
    q.tail_row_bytes = t.geom.tail_row_bytes;
  };
  for (const Job &jb : jobs) {
    const int i = jb.i, f = jb.filter, mode = jb.mode;
    const mpf_profile *p = profs[i];
    DevTable fb{};   // held MSV: the integer table of the rescoring launch
    QueryDesc q;
    memset(&q, 0, sizeof(q));
    int lanes = 32, words = 0;
    if (mode == MODE_TILE_SSV || mode == MODE_TILE_MSV || mode == MODE_TILE_MSV_SSV) {
      const uint4 *tt = nullptr;
      int rc = get_tile_table(p, &tt);
      if (rc) {
        plan_free(pl);
        return rc;
      }
      q.table = tt;
      q.M = (uint32_t)p->M;
      q.smax_off = (uint32_t)(((size_t)(p->M + kTileNodes - 1) / kTileNodes) * kTileTableBytes);
      const int ttm = p->table_mem[f] == MPF_TABLE_SHARED ? 0 : 1;   // tiles in TMEM
      if (mode != MODE_TILE_SSV) {   // the lane-segment kernel's table, for the fallback
        const uint8_t *lt = nullptr;
        rc = get_long_table(p, &lt);
        if (rc) {
          plan_free(pl);
          return rc;
        }
        DevTable lt_t{};
        lt_t.ptr = reinterpret_cast<uint4 *>(const_cast<uint8_t *>(lt));
        fb_table[GroupKey(lanes, words, mode, ttm, 1)].push_back(lt_t);
        fb_seg_words[GroupKey(lanes, words, mode, ttm, 1)].push_back((uint32_t)p->seg_words);
      }
    } else if (p->seg_words) {
      const uint8_t *lt = nullptr;
      int rc = get_long_table(p, &lt);
      if (rc) {
        plan_free(pl);
        return rc;
      }
      q.table = reinterpret_cast<const uint4 *>(lt);
      q.M = (uint32_t)p->M;
      q.seg_words = (uint32_t)p->seg_words;
    } else {
      lanes = p->cfg_lanes[f];
      words = p->cfg_words[f];
      if (!lanes) default_config(ctx, p->M, mode, &lanes, &words);
      if (!lanes || !kernel_for(lanes, words, mode)) {
        plan_free(pl);
        return MPF_EUNSUPPORTED;
      }
      DevTable t;
      int rc = get_table(p, lanes, words, table_format(mode), &t);
      if (rc) {
        plan_free(pl);
        return rc;
      }
      set_table(q, t);
      q.M = (uint32_t)p->M;
      if (mode == MODE_MSV_HELD || mode == MODE_MSV_HELD_F16 || mode == MODE_MSV_SSV) {
        // The integer table of the same layout, for the exact kernel that
        // rescores the sequences the held pass lists.
        DevTable ti = t;
        if (mode == MODE_MSV_HELD_F16) rc = get_table(p, lanes, words, TABLE_I16, &ti);
        if (rc) {
          plan_free(pl);
          return rc;
        }
        fb = ti;
      }
    }
    q.bias = p->bias;
    q.tbm = p->tbm;
    q.tec = p->tec;
    q.base = p->base;
    q.tjb_fixed = p->tjb_fixed;
    q.scale = p->scale;
    q.tjb = p->d_tjb;
    q.n_tjb = p->n_tjb;
    const size_t off = ((size_t)jb.block * (size_t)n_q + (size_t)i) * db->n_seqs;
    q.raw = raw + off;
    q.flag = flag + off;
    q.nat = nat ? nat + off : nullptr;
    if (mode == MODE_MSV_SSV || mode == MODE_TILE_MSV_SSV) {   // the SSV block
      const size_t off2 = ((size_t)n_q + (size_t)i) * db->n_seqs;
      q.raw2 = raw + off2;
      q.flag2 = flag + off2;
      q.nat2 = nat ? nat + off2 : nullptr;
    }
    q.ranks = ranks ? ranks + off : nullptr;
    q.n_ranks = ranks ? n_ranks + i : nullptr;
    const bool tiled = mode == MODE_TILE_SSV || mode == MODE_TILE_MSV || mode == MODE_TILE_MSV_SSV;
    const int tm = tiled ? (p->table_mem[f] == MPF_TABLE_SHARED ? 0 : 1)
                         : p->seg_words ? 0 : (use_tmem(p, f, lanes, words, mode) ? 1 : 0);
    const int sf = p->seg_words ? 1 : p->shard_factor[f];
    if (n_q >= 2 && !ranks && !p->seg_words && lanes < 32 &&
        (mode == MODE_SSV || mode == MODE_MSV_HELD || mode == MODE_MSV_SSV) && words >= kTmMinWords &&
        p->table_mem[f] != MPF_TABLE_SHARED) {
      qp_cand[std::make_pair(lanes, mode)].push_back(QpCand{words, sf, p, q, fb});
      continue;
    }
    const GroupKey key(lanes, words, mode, tm, 1);
    byconf[key].push_back(q);
    if (fb.ptr) fb_table[key].push_back(fb);
    group_shards[key] = std::max(group_shards[key], sf);
  }
  // Several queries per warp: 32 / lanes queries of one (lanes, mode) score
  // the same sequence in one warp, with the table rows in tensor memory.
  // Sorted by words per lane, runs of consecutive queries form a warp's set
  // (pack_runs), all padded to the run's largest word count H (padding nodes
  // score kNegInf, so the scores are those of the query's own layout), with
  // their tables in the packed geometry; empty slots of a set hold
  // descriptors without a table.  The held MSV pass's rescoring launch (one
  // query per warp) reads the integer table of the usual geometry at H words.
  for (auto &kv : qp_cand) {
    const int lanes = kv.first.first, mode = kv.first.second, QP = 32 / lanes;
    std::vector<QpCand> &v = kv.second;
    std::stable_sort(v.begin(), v.end(), [](const QpCand &a, const QpCand &b) { return a.words < b.words; });
    std::vector<int> words(v.size());
    for (size_t j = 0; j < v.size(); ++j) words[j] = v[j].words;
    const std::vector<std::pair<size_t, size_t>> runs = pack_runs(lanes, mode, words, ctx->max_smem);
    for (const auto &r : runs) {
      const size_t a = r.first, b = r.second;
      const bool pack = b - a >= 2;
      const int H = v[b - 1].words;
      const GroupKey key0(lanes, H, mode, 1, QP);
      for (size_t j = a; j < b; ++j) {
        QueryDesc q = v[j].q;
        DevTable fb = v[j].fb;
        if (pack) {
          DevTable t;
          int rc = get_table(v[j].p, lanes, H, TABLE_I16_PACKED, &t);
          if (rc == MPF_OK && mode != MODE_SSV) rc = get_table(v[j].p, lanes, H, TABLE_I16, &fb);
          if (rc) {
            plan_free(pl);
            return rc;
          }
          set_table(q, t);
        }
        const GroupKey key = pack ? key0 : GroupKey(lanes, v[j].words, mode, 0, 1);
        byconf[key].push_back(q);
        if (mode != MODE_SSV) fb_table[key].push_back(fb);
        group_shards[key] = std::max(group_shards[key], v[j].sf);
      }
      if (pack) {
        QueryDesc empty;
        memset(&empty, 0, sizeof(empty));
        for (size_t j = b - a; j < (size_t)QP; ++j) {
          byconf[key0].push_back(empty);
          if (mode != MODE_SSV) fb_table[key0].push_back(DevTable{});
        }
      }
    }
  }
  DeviceGuard dg(ctx->device);
  for (auto &kv : byconf) {
    LaunchGroup g;
    g.lanes = std::get<0>(kv.first);
    g.words = std::get<1>(kv.first);
    g.mode = std::get<2>(kv.first);
    g.tm = std::get<3>(kv.first) != 0;
    g.qp = std::get<4>(kv.first);
    if (g.qp > 1) g.qp_stride = packed_table_stride(g.lanes, g.words);
    g.shard_factor = group_shards[kv.first];
    for (const QueryDesc &qd : kv.second) g.long_words = std::max(g.long_words, qd.seg_words);
    g.n_codes = db->n_codes;
    int rc = configure_kernel(ctx, &g);
    if (rc) {
      plan_free(pl);
      return rc;
    }
    g.n_queries = (uint32_t)kv.second.size();
    for (const QueryDesc &qd : kv.second) g.n_real += qd.table ? 1u : 0u;
    cudaError_t e = cudaMallocAsync((void **)&g.d_queries, sizeof(QueryDesc) * kv.second.size(), ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&g.d_counter, sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess && (g.mode == MODE_TILE_SSV || g.mode == MODE_TILE_MSV || g.mode == MODE_TILE_MSV_SSV)) {
      // Per resident warp two columns (positions 0..max_len and the
      // prefetch's overrun), col_stride bytes each: int16, or for the TMEM
      // kernel the 32-bit pair holding the node.
      g.col_stride = (uint32_t)((((uint64_t)db->max_len + 12) * (g.tm ? 4 : 2) + 15) & ~(uint64_t)15);
      g.col_bytes = (uint64_t)g.grid * (uint64_t)(g.threads / 32) * 2 * g.col_stride;
      e = cudaMallocAsync((void **)&g.d_col, g.col_bytes, ctx->stream);
    }
    const bool held = g.mode == MODE_MSV_HELD || g.mode == MODE_MSV_HELD_F16 || g.mode == MODE_MSV_SSV;
    if (e == cudaSuccess && (g.mode == MODE_TILE_MSV || g.mode == MODE_TILE_MSV_SSV || held)) {
      // Fallback lists, and the launch that scores them exactly: the
      // lane-segment kernel after the tiled MSV pass, the striped kernel
      // with the J/B update every row after the held pass.
      const size_t nq = kv.second.size(), ns = std::max<uint64_t>(db->n_seqs, 1);
      e = cudaMallocAsync((void **)&g.d_fallback, (nq + nq * ns) * 4, ctx->stream);
      if (e == cudaSuccess) {
        auto nx = std::make_shared<LaunchGroup>();
        nx->mode = held ? MODE_MSV_DIRECT : MODE_LONG_MSV;
        nx->lanes = g.lanes;
        nx->words = g.words;
        nx->n_codes = db->n_codes;
        std::vector<QueryDesc> fq;   // the group's queries (not the empty slots of packed sets)
        for (size_t i = 0; i < nq; ++i) {
          kv.second[i].fallback_count = g.d_fallback + i;
          kv.second[i].fallback_ranks = g.d_fallback + nq + i * ns;
          if (!kv.second[i].table) continue;
          QueryDesc f = kv.second[i];
          if (held) {
            set_table(f, fb_table[kv.first][i]);
          } else {
            f.table = fb_table[kv.first][i].ptr;
            f.seg_words = fb_seg_words[kv.first][i];
          }
          f.ranks = kv.second[i].fallback_ranks;
          f.n_ranks = kv.second[i].fallback_count;
          nx->long_words = std::max(nx->long_words, f.seg_words);
          fq.push_back(f);
        }
        g.next = nx;
        int rc2 = configure_kernel(ctx, nx.get());
        if (rc2) {
          pl->groups.push_back(g);
          plan_free(pl);
          return rc2;
        }
        nx->n_queries = (uint32_t)fq.size();
        nx->n_real = nx->n_queries;
        e = cudaMallocAsync((void **)&nx->d_queries, sizeof(QueryDesc) * fq.size(), ctx->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&nx->d_counter, sizeof(uint32_t), ctx->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(nx->d_queries, fq.data(), sizeof(QueryDesc) * fq.size(),
                              cudaMemcpyHostToDevice, ctx->stream);
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.d_queries, kv.second.data(), sizeof(QueryDesc) * kv.second.size(),
                          cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      pl->groups.push_back(g);   // plan_free releases what the group holds
      plan_free(pl);
      return e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA;
    }
    pl->groups.push_back(g);
  }
  if (pl->groups.size() > 1) {
    while (ctx->n_fork < 8 && (size_t)ctx->n_fork < pl->groups.size()) {
      if (cudaStreamCreateWithFlags(&ctx->fork[ctx->n_fork], cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        plan_free(pl);
        return MPF_ECUDA;
      }
      ++ctx->n_fork;
    }
    for (size_t i = 0; i <= pl->groups.size(); ++i) {
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        plan_free(pl);
        return MPF_ECUDA;
      }
      pl->events.push_back(ev);
    }
  }
  *out = pl;
  return MPF_OK;
}

int enqueue_group(const mpf_db *db, mpf_ctx *ctx, LaunchGroup &g, cudaStream_t st) {
  MPF_CUDA(cudaMemsetAsync(g.d_counter, 0, sizeof(uint32_t), st));
  if (g.d_fallback) MPF_CUDA(cudaMemsetAsync(g.d_fallback, 0, sizeof(uint32_t) * g.n_queries, st));
  ScanParams sp{};
  sp.residues = db->d_words;
  sp.n_words = db->n_words;
  sp.seq_word = db->d_seq_word;
  sp.seq_len = db->d_seq_len;
  sp.seq_orig = db->d_seq_orig;
  sp.n_seqs = (uint32_t)db->n_seqs;
  sp.pad_word = db->pad_word;
  sp.queries = g.d_queries;
  sp.n_queries = g.n_queries;
  sp.n_shards = g.n_shards;
  sp.item_counter = g.d_counter;
  sp.status = ctx->d_status;
  sp.long_words = g.long_words;
  sp.tile_col = g.d_col;
  sp.tile_col_stride = g.col_stride;
  sp.tile_col_bytes = g.col_bytes;
  sp.qp_table_stride = g.qp_stride;
  const uint64_t n_items = ((uint64_t)g.n_queries + (uint64_t)g.qp - 1) / (uint64_t)g.qp * g.n_shards;
  const int grid = (int)std::min<uint64_t>((uint64_t)g.grid, n_items);
  g.fn<<<grid, g.threads, g.smem, st>>>(sp);
  MPF_CUDA(cudaGetLastError());
  if (g.next) return enqueue_group(db, ctx, *g.next, st);
  return MPF_OK;
}

// Enqueue every launch group on `st`; several groups fork onto the context's
// side streams and join back.
int plan_enqueue(mpf_plan *pl, cudaStream_t st) {
  mpf_ctx *ctx = pl->ctx;
  if (pl->groups.size() == 1) return enqueue_group(pl->db, ctx, pl->groups[0], st);
  const size_t ng = pl->groups.size();
  MPF_CUDA(cudaEventRecord(pl->events[ng], st));
  for (size_t i = 0; i < ng; ++i) {
    cudaStream_t fs = ctx->fork[i % (size_t)ctx->n_fork];
    MPF_CUDA(cudaStreamWaitEvent(fs, pl->events[ng], 0));
    int rc = enqueue_group(pl->db, ctx, pl->groups[i], fs);
    if (rc) return rc;
    MPF_CUDA(cudaEventRecord(pl->events[i], fs));
  }
  for (size_t i = 0; i < ng; ++i) MPF_CUDA(cudaStreamWaitEvent(st, pl->events[i], 0));
  return MPF_OK;
}

int plan_launch(mpf_plan *pl) {
  if (pl->graph) {
    MPF_CUDA(cudaGraphLaunch(pl->graph, pl->ctx->stream));
    return MPF_OK;
  }
  return plan_enqueue(pl, pl->ctx->stream);
}

// Run a plan into the caller's buffers; host buffers go through scratch.
int run_scan(mpf_ctx *ctx, int filter, const mpf_profile *const *profs, int n_q,
             const mpf_db *db, uint8_t *raw, uint8_t *flag, float *nat) {
  if (!ctx || !db || !raw || !flag || n_q < 1) return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  const bool dev_raw = is_device_ptr(raw), dev_flag = is_device_ptr(flag);
  const bool dev_nat = nat ? is_device_ptr(nat) : true;
  const uint64_t n = (uint64_t)n_q * db->n_seqs * (filter == MPF_MSV_SSV ? 2u : 1u);
  if (n == 0) return MPF_OK;
  uint8_t *k_raw = raw, *k_flag = flag;
  float *k_nat = nat;
  const bool staged = !(dev_raw && dev_flag && dev_nat);
  if (staged) {
    int rc = ensure_out_scratch(ctx, (size_t)n * 6 + 64);
    if (rc) return rc;
    uint8_t *base = (uint8_t *)ctx->d_out;
    k_nat = nat ? (float *)base : nullptr;
    k_raw = base + (size_t)n * 4;
    k_flag = k_raw + n;
  }
  mpf_plan *pl = nullptr;
  int rc = plan_create(ctx, filter, profs, n_q, db, k_raw, k_flag, k_nat, &pl);
  if (rc) return rc;
  rc = plan_enqueue(pl, ctx->stream);
  if (!staged) {
    // Device outputs: asynchronous; the plan is freed at the next sync.
    ctx->pending.push_back(pl);
    if (rc == MPF_OK && ctx->pending.size() > 64) rc = free_pending(ctx);
    return rc;
  }
  if (rc == MPF_OK) {
    cudaError_t e = cudaMemcpyAsync(raw, k_raw, n, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag, k_flag, n, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess && nat) e = cudaMemcpyAsync(nat, k_nat, n * 4, cudaMemcpyDefault, ctx->stream);
    if (e != cudaSuccess) rc = MPF_ECUDA;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (rc == MPF_OK && e != cudaSuccess) rc = MPF_ECUDA;
  plan_free(pl);
  if (rc == MPF_OK) {
    int st = 0;
    if (cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MPF_ECUDA;
    if (st) return status_code(st);
  }
  return rc;
}

}  // namespace

// ================================================================ C ABI ====

extern "C" {

int mpf_max_model_length(void) { return kMaxLongM; }

int mpf_max_striped_length(void) { return kStripedMaxM; }

const char *mpf_strerror(int status) {
  switch (status) {
    case MPF_OK: return "ok";
    case MPF_EINVAL: return "invalid argument";
    case MPF_ENOMEM: return "out of memory";
    case MPF_ECUDA: return "CUDA runtime error";
    case MPF_ETIMEOUT: return "bounded device wait timed out";
    case MPF_EUNSUPPORTED: return "unsupported request";
    case MPF_EDEVICE: return "a kernel's index check failed (debug build)";
    default: return "unknown status";
  }
}

int mpf_ctx_create(int device, void *cuda_stream, mpf_ctx **out) {
  if (!out) return MPF_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    (void)cudaGetLastError();
    return MPF_ECUDA;
  }
  if (device < 0 || device >= ndev) return MPF_EINVAL;
  DeviceGuard dg(device);
  mpf_ctx *ctx = new (std::nothrow) mpf_ctx;
  if (!ctx) return MPF_ENOMEM;
  ctx->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = (e == cudaSuccess);
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->util, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    mpf_ctx_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA;
  }
  ctx->max_smem -= 64;  // static shared memory of the kernel
  *out = ctx;
  return MPF_OK;
}

void mpf_ctx_destroy(mpf_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto *pl : ctx->pending) plan_free(pl);
  ctx->pending.clear();
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_out);
  for (int i = 0; i < ctx->n_fork; ++i) cudaStreamDestroy(ctx->fork[i]);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->util) {
    cudaStreamSynchronize(ctx->util);
    cudaStreamDestroy(ctx->util);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  (void)cudaGetLastError();
  delete ctx;
}

void *mpf_ctx_stream(mpf_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

int mpf_sync(mpf_ctx *ctx) {
  if (!ctx) return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  MPF_CUDA(cudaStreamSynchronize(ctx->stream));
  int rc = free_pending(ctx);
  if (rc) return rc;
  int st = 0;
  MPF_CUDA(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return status_code(st);
}

int mpf_profile_create(mpf_ctx *ctx, int M, int K, const uint8_t *cost, uint8_t bias_b,
                       uint8_t tbm_b, uint8_t tec_b, uint8_t tjb_b, const uint8_t *tjb_by_len,
                       uint32_t n_tjb, float scale_b, uint8_t base_b, mpf_profile **out) {
  if (!out) return MPF_EINVAL;
  *out = nullptr;
  if (!ctx || !cost || M < 1 || K < 1 || K > 32) return MPF_EINVAL;
  if (!(scale_b > 0.f) || !isfinite(scale_b)) return MPF_EINVAL;
  if (tjb_by_len && n_tjb == 0) return MPF_EINVAL;
  if (M > mpf_max_model_length()) return MPF_EUNSUPPORTED;
  mpf_profile *p = new (std::nothrow) mpf_profile;
  if (!p) return MPF_ENOMEM;
  p->ctx = ctx;
  p->M = M;
  p->K = K;
  p->cost.assign(cost, cost + (size_t)K * M);
  p->bias = bias_b;
  p->tbm = tbm_b;
  p->tec = tec_b;
  p->tjb_fixed = tjb_b;
  p->base = base_b;
  p->scale = scale_b;
  p->tjb_min = tjb_b;
  if (tjb_by_len) {
    p->tjb_min = *std::min_element(tjb_by_len, tjb_by_len + n_tjb);
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaMallocAsync((void **)&p->d_tjb, n_tjb, ctx->util);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_tjb, tjb_by_len, n_tjb, cudaMemcpyHostToDevice, ctx->util);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->util);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      if (p->d_tjb) cudaFreeAsync(p->d_tjb, ctx->util);
      delete p;
      return e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA;
    }
    p->n_tjb = n_tjb;
  }
  if (M > kStripedMaxM) {
    // Longer than the striped table holds: the long-model kernel, lane
    // segments of 4 * seg_words nodes, one warp's DP row in shared memory.
    p->seg_words = ((M + 31) / 32 + 3) / 4;
    if (long_smem_per_warp(p->seg_words, true) > (size_t)ctx->max_smem) {
      mpf_profile_destroy(p);
      return MPF_EUNSUPPORTED;
    }
    *out = p;
    return MPF_OK;
  }
  int lanes = 0, words = 0;
  default_config(ctx, M, kernel_mode(p, MPF_MSV), &lanes, &words);
  if (!lanes) {
    mpf_profile_destroy(p);
    return MPF_EUNSUPPORTED;
  }
  *out = p;
  return MPF_OK;
}

void mpf_profile_destroy(mpf_profile *p) {
  if (!p) return;
  DeviceGuard dg(p->ctx->device);
  // Ordered after the scans queued on the profile's context stream.
  for (auto &kv : p->tables) cudaFreeAsync(kv.second.ptr, p->ctx->stream);
  if (p->d_tjb) cudaFreeAsync(p->d_tjb, p->ctx->stream);
  (void)cudaGetLastError();
  delete p;
}

int mpf_profile_set_config(mpf_profile *p, int filter, int lanes, int words) {
  if (!p || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  if (lanes == 0 && words == 0) {  // back to the default
    p->cfg_lanes[filter] = p->cfg_words[filter] = 0;
    return MPF_OK;
  }
  if (p->seg_words) return MPF_EINVAL;   // long models have one configuration
  if (!words_built(words) || !kernel_for(lanes, words, kernel_mode(p, filter))) return MPF_EINVAL;
  if (2 * lanes * words < p->M) return MPF_EINVAL;
  if (smem_need(lanes, words) > p->ctx->max_smem) return MPF_EUNSUPPORTED;
  p->cfg_lanes[filter] = lanes;
  p->cfg_words[filter] = words;
  return MPF_OK;
}

int mpf_profile_set_arith(mpf_profile *p, int filter, int arith) {
  if (!p || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  if (arith != MPF_ARITH_AUTO && arith != MPF_ARITH_I16 && arith != MPF_ARITH_F16) return MPF_EINVAL;
  p->arith[filter] = arith;
  // A configured (lanes, words) pair without a kernel in the new arithmetic
  // falls back to the default configuration.
  if (p->cfg_lanes[filter] && !kernel_for(p->cfg_lanes[filter], p->cfg_words[filter], kernel_mode(p, filter)))
    p->cfg_lanes[filter] = p->cfg_words[filter] = 0;
  return MPF_OK;
}

int mpf_profile_set_shard_factor(mpf_profile *p, int filter, int factor) {
  if (!p || (filter != MPF_MSV && filter != MPF_SSV) || factor < 1 || factor > 16) return MPF_EINVAL;
  p->shard_factor[filter] = factor;
  return MPF_OK;
}

int mpf_profile_get_shard_factor(const mpf_profile *p, int filter, int *factor) {
  if (!p || !factor || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  *factor = p->seg_words ? 1 : p->shard_factor[filter];
  return MPF_OK;
}

int mpf_profile_set_table_memory(mpf_profile *p, int filter, int where) {
  if (!p || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  if (where != MPF_TABLE_AUTO && where != MPF_TABLE_SHARED) return MPF_EINVAL;
  p->table_mem[filter] = where;
  return MPF_OK;
}

int mpf_profile_get_table_memory(const mpf_profile *p, int filter, int *where) {
  if (!p || !where || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  const int mode = kernel_mode(p, filter);
  if (p->seg_words) {   // tiled kernels: the tile in TMEM unless set to shared; lane segments: shared
    *where = (mode != MODE_LONG_MSV && p->table_mem[filter] != MPF_TABLE_SHARED) ? MPF_TABLE_TENSOR
                                                                                 : MPF_TABLE_SHARED;
    return MPF_OK;
  }
  int lanes = p->cfg_lanes[filter], words = p->cfg_words[filter];
  if (!lanes) default_config(p->ctx, p->M, mode, &lanes, &words);
  *where = use_tmem(p, filter, lanes, words, mode) ? MPF_TABLE_TENSOR : MPF_TABLE_SHARED;
  return MPF_OK;
}

int mpf_profile_get_config(const mpf_profile *p, int filter, int *lanes, int *words) {
  if (!p || !lanes || !words || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  if (p->seg_words) {
    *lanes = 32;
    *words = 0;
  } else if (p->cfg_lanes[filter]) {
    *lanes = p->cfg_lanes[filter];
    *words = p->cfg_words[filter];
  } else {
    default_config(p->ctx, p->M, kernel_mode(p, filter), lanes, words);
  }
  return MPF_OK;
}

int mpf_profile_footprint(const mpf_profile *p, int filter, uint32_t *smem_bytes, uint64_t *table_bytes) {
  if (!p || !smem_bytes || !table_bytes || (filter != MPF_MSV && filter != MPF_SSV)) return MPF_EINVAL;
  const int mode = kernel_mode(p, filter);
  if (mode == MODE_TILE_SSV || mode == MODE_TILE_MSV || mode == MODE_LONG_MSV) {
    const uint64_t tiles = (uint64_t)(p->M + kTileNodes - 1) / kTileNodes;
    const uint64_t long_table = (uint64_t)32 * p->seg_words * 32 * 4;   // cost bytes, lane-segment order
    if (mode == MODE_LONG_MSV) {
      *smem_bytes = (uint32_t)long_smem_per_warp(p->seg_words, 4 * long_smem_per_warp(p->seg_words, false) > 228 * 1024);
      *table_bytes = long_table;
    } else {
      // The TMEM variant holds the tile in tensor memory and asks for more
      // than half the shared memory (one block per SM).
      *smem_bytes = p->table_mem[filter] == MPF_TABLE_SHARED ? (uint32_t)kTileTableBytes
                                                             : (uint32_t)p->ctx->max_smem / 2 + 1024;
      *table_bytes = tiles * kTileTableBytes + 64 + (mode == MODE_TILE_MSV ? long_table : 0);
    }
    return MPF_OK;
  }
  int lanes = p->cfg_lanes[filter], words = p->cfg_words[filter];
  if (!lanes) default_config(p->ctx, p->M, mode, &lanes, &words);
  if (!lanes) return MPF_EUNSUPPORTED;
  const TableGeom g = table_geom(lanes, words);
  *smem_bytes = g.table_bytes;
  *table_bytes = g.table_bytes;
  return MPF_OK;
}

int mpf_db_upload(mpf_ctx *ctx, const uint8_t *residues, uint64_t n_residues,
                  const uint64_t *offsets, const uint32_t *lengths, uint64_t n_seqs,
                  mpf_db **out) {
  if (!out) return MPF_EINVAL;
  *out = nullptr;
  if (!ctx || (n_seqs && (!offsets || !lengths)) || (n_residues && !residues)) return MPF_EINVAL;
  if (n_seqs >= (1ull << 31)) return MPF_EINVAL;
  // Validate ranges and codes; total padded size in 16-byte chunks.
  uint64_t chunks = 1;  // chunk 0 holds the padding word
  for (uint64_t s = 0; s < n_seqs; ++s) {
    if (offsets[s] > n_residues || lengths[s] > n_residues - offsets[s]) return MPF_EINVAL;
    chunks += (lengths[s] + 15u) / 16u;
  }
  uint32_t seen = 0;
  for (uint64_t i = 0; i < n_residues; ++i) {
    if (residues[i] >= 32) return MPF_EINVAL;
    seen |= 1u << residues[i];
  }
  chunks += 1;  // the kernel prefetches one word past a sequence
  if (chunks * 4 >= (1ull << 32)) return MPF_EUNSUPPORTED;
  // Length ranks: longest first, ties by sequence number.
  std::vector<uint32_t> order(n_seqs);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return lengths[a] > lengths[b]; });
  std::vector<uint32_t> seq_word(n_seqs), seq_len(n_seqs);
  uint8_t *host = nullptr;
  DeviceGuard dg(ctx->device);
  MPF_CUDA(cudaMallocHost(&host, chunks * 16));
  memset(host, kPadCode, 16);
  uint64_t c = 1;
  for (uint64_t rnk = 0; rnk < n_seqs; ++rnk) {
    const uint32_t s = order[rnk];
    const uint32_t L = lengths[s];
    seq_len[rnk] = L;
    if (L == 0) {
      seq_word[rnk] = 0;
      continue;
    }
    seq_word[rnk] = (uint32_t)(c * 4);
    const uint64_t nch = (L + 15u) / 16u;
    memcpy(host + c * 16, residues + offsets[s], L);
    memset(host + c * 16 + L, kPadCode, nch * 16 - L);
    c += nch;
  }
  memset(host + c * 16, kPadCode, (chunks - c) * 16);
  mpf_db *db = new (std::nothrow) mpf_db;
  if (!db) {
    cudaFreeHost(host);
    return MPF_ENOMEM;
  }
  db->ctx = ctx;
  db->n_seqs = n_seqs;
  db->n_residues = 0;
  for (uint64_t s = 0; s < n_seqs; ++s) db->n_residues += lengths[s];
  db->pad_word = 0;
  db->n_codes = __builtin_popcount(seen);
  db->max_len = n_seqs ? seq_len[0] : 0;
  const size_t ns = std::max<uint64_t>(n_seqs, 1);
  db->n_words = (uint32_t)(chunks * 4);
  cudaError_t e = cudaMalloc(&db->d_words, chunks * 16);
  if (e == cudaSuccess) e = cudaMalloc(&db->d_seq_word, ns * 4);
  if (e == cudaSuccess) e = cudaMalloc(&db->d_seq_len, ns * 4);
  if (e == cudaSuccess) e = cudaMalloc(&db->d_seq_orig, ns * 4);
  if (e == cudaSuccess) e = cudaMemcpy(db->d_words, host, chunks * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_seqs) {
    e = cudaMemcpy(db->d_seq_word, seq_word.data(), n_seqs * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db->d_seq_len, seq_len.data(), n_seqs * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db->d_seq_orig, order.data(), n_seqs * 4, cudaMemcpyHostToDevice);
  }
  cudaFreeHost(host);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    mpf_db_destroy(db);
    return e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA;
  }
  *out = db;
  return MPF_OK;
}

void mpf_db_destroy(mpf_db *db) {
  if (!db) return;
  DeviceGuard dg(db->ctx->device);
  cudaFree(db->d_words);
  cudaFree(db->d_seq_word);
  cudaFree(db->d_seq_len);
  cudaFree(db->d_seq_orig);
  (void)cudaGetLastError();
  delete db;
}

uint64_t mpf_db_n_seqs(const mpf_db *db) { return db ? db->n_seqs : 0; }
uint64_t mpf_db_n_residues(const mpf_db *db) { return db ? db->n_residues : 0; }

int mpf_msv_scan(mpf_ctx *ctx, const mpf_profile *prof, const mpf_db *db, uint8_t *raw,
                 uint8_t *overflow, float *nat) {
  return run_scan(ctx, MPF_MSV, &prof, 1, db, raw, overflow, nat);
}

int mpf_ssv_scan(mpf_ctx *ctx, const mpf_profile *prof, const mpf_db *db, uint8_t *raw,
                 uint8_t *overflow, float *nat) {
  return run_scan(ctx, MPF_SSV, &prof, 1, db, raw, overflow, nat);
}

int mpf_scan_batch(mpf_ctx *ctx, int filter, const mpf_profile *const *profs, int n_q,
                   const mpf_db *db, uint8_t *raw, uint8_t *overflow, float *nat) {
  return run_scan(ctx, filter, profs, n_q, db, raw, overflow, nat);
}

int mpf_plan_create(mpf_ctx *ctx, int filter, const mpf_profile *const *profs, int n_q,
                    const mpf_db *db, uint8_t *raw, uint8_t *overflow, float *nat,
                    mpf_plan **out) {
  if (!out) return MPF_EINVAL;
  *out = nullptr;
  if (!ctx || !raw || !overflow) return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  if (!is_device_ptr(raw) || !is_device_ptr(overflow) || (nat && !is_device_ptr(nat)))
    return MPF_EINVAL;
  return plan_create(ctx, filter, profs, n_q, db, raw, overflow, nat, out);
}

int mpf_plan_launch(mpf_plan *plan) {
  if (!plan) return MPF_EINVAL;
  DeviceGuard dg(plan->ctx->device);
  return plan_launch(plan);
}

int mpf_plan_capture_graph(mpf_plan *plan) {
  if (!plan) return MPF_EINVAL;
  mpf_ctx *ctx = plan->ctx;
  DeviceGuard dg(ctx->device);
  if (!ctx->capture) MPF_CUDA(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
  // The capture stream must see the plan's uploads queued on the context stream.
  MPF_CUDA(cudaStreamSynchronize(ctx->stream));
  MPF_CUDA(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
  int rc = plan_enqueue(plan, ctx->capture);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->capture, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    return rc;
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return MPF_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return MPF_ECUDA;
  }
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  plan->graph = exec;
  return MPF_OK;
}

int mpf_plan_kernel_launches(const mpf_plan *plan) {
  if (!plan) return 0;
  int n = 0;
  for (const LaunchGroup &g0 : plan->groups)
    for (const LaunchGroup *g = &g0; g; g = g->next.get()) ++n;   // with the rescoring launches
  return n;
}

int mpf_plan_pack_sets(int lanes, const int *words, int n, int max_smem, int *set_start) {
  if ((lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16) || n < 0 || (n && (!words || !set_start)))
    return MPF_EINVAL;
  std::vector<int> w(words, words + n);
  for (int i = 0; i < n; ++i)
    if (w[i] < 1 || (i && w[i] < w[i - 1])) return MPF_EINVAL;
  for (const auto &r : pack_runs(lanes, MODE_SSV, w, max_smem))
    for (size_t j = r.first; j < r.second; ++j) set_start[j] = r.second - r.first >= 2 ? (int)r.first : -1;
  return MPF_OK;
}

int mpf_plan_group_count(const mpf_plan *plan) { return plan ? (int)plan->groups.size() : 0; }

int mpf_plan_group_info(const mpf_plan *plan, int i, int *lanes, int *words, int *table_memory,
                        int *queries_per_warp, int *n_queries, int *filters) {
  if (!plan || i < 0 || (size_t)i >= plan->groups.size()) return MPF_EINVAL;
  const LaunchGroup &g = plan->groups[(size_t)i];
  if (lanes) *lanes = g.lanes;
  if (words) *words = g.words;
  if (table_memory) *table_memory = g.tm ? MPF_TABLE_TENSOR : MPF_TABLE_SHARED;
  if (queries_per_warp) *queries_per_warp = g.qp;
  if (n_queries) *n_queries = (int)g.n_real;
  if (filters) {
    switch (g.mode) {
      case MODE_MSV_SSV: case MODE_TILE_MSV_SSV: *filters = 3; break;
      case MODE_SSV: case MODE_SSV_F16: case MODE_TILE_SSV: *filters = 2; break;
      default: *filters = 1;
    }
  }
  return MPF_OK;
}

int mpf_pipeline_scan(mpf_ctx *ctx, const mpf_profile *const *profs, int n_q, const mpf_db *db,
                      float ssv_min_nat, uint8_t *ssv_raw, uint8_t *ssv_flag, float *ssv_nat,
                      uint8_t *msv_raw, uint8_t *msv_flag, float *msv_nat, uint32_t *n_pass) {
  if (!ctx || !profs || n_q < 1 || !db || !ssv_raw || !ssv_flag || !ssv_nat || !msv_raw ||
      !msv_flag || !n_pass || isnan(ssv_min_nat))
    return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  for (const void *ptr : {(const void *)ssv_raw, (const void *)ssv_flag, (const void *)ssv_nat,
                          (const void *)msv_raw, (const void *)msv_flag, (const void *)n_pass})
    if (!is_device_ptr(ptr)) return MPF_EINVAL;
  if (msv_nat && !is_device_ptr(msv_nat)) return MPF_EINVAL;
  const uint64_t n = db->n_seqs;
  {  // The hand-off reads the SSV outputs while it writes the MSV ones: no two may share memory.
    const uint64_t nq = (uint64_t)n_q * n;
    const void *ptr[7] = {ssv_raw, ssv_flag, ssv_nat, msv_raw, msv_flag, msv_nat, n_pass};
    const uint64_t bytes[7] = {nq, nq, 4 * nq, nq, nq, msv_nat ? 4 * nq : 0, 4 * (uint64_t)n_q};
    if (ranges_overlap(ptr, bytes, 7)) return MPF_EINVAL;
  }
  const uint64_t n_chunks = (n + kSelectChunk - 1) / kSelectChunk;
  uint32_t *ranks = nullptr, *n_ranks = nullptr, *chunk = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&ranks, std::max<uint64_t>(1, (uint64_t)n_q * n) * 4, ctx->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&n_ranks, (size_t)n_q * 4, ctx->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&chunk, std::max<uint64_t>(1, 2 * (uint64_t)n_q * n_chunks) * 4, ctx->stream);
  int rc = e == cudaSuccess ? MPF_OK : (e == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA);
  mpf_plan *ssv = nullptr, *msv = nullptr;
  if (rc == MPF_OK) rc = plan_create(ctx, MPF_SSV, profs, n_q, db, ssv_raw, ssv_flag, ssv_nat, &ssv);
  if (rc == MPF_OK) rc = plan_enqueue(ssv, ctx->stream);
  if (rc == MPF_OK && launch_select(db->d_seq_orig, n, n_q, ssv_flag, ssv_nat, ssv_min_nat, msv_raw, 1,
                                    msv_flag, msv_nat, chunk, chunk + (uint64_t)n_q * n_chunks,
                                    ranks, n_ranks, ctx->stream) != 0)
    rc = MPF_ECUDA;
  if (rc == MPF_OK) rc = plan_create(ctx, MPF_MSV, profs, n_q, db, msv_raw, msv_flag, msv_nat, &msv, ranks, n_ranks);
  if (rc == MPF_OK) rc = plan_enqueue(msv, ctx->stream);
  if (rc == MPF_OK && cudaMemcpyAsync(n_pass, n_ranks, (size_t)n_q * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
    rc = MPF_ECUDA;
  // Stream-ordered release after the MSV scan; plans are freed at the next sync.
  if (ranks) cudaFreeAsync(ranks, ctx->stream);
  if (n_ranks) cudaFreeAsync(n_ranks, ctx->stream);
  if (chunk) cudaFreeAsync(chunk, ctx->stream);
  if (ssv) ctx->pending.push_back(ssv);
  if (msv) ctx->pending.push_back(msv);
  (void)cudaGetLastError();
  return rc;
}

int mpf_pvalues(mpf_ctx *ctx, const float *nat, uint64_t n, float mu, float lambda, float *p) {
  if (!ctx || (n && (!nat || !p)) || !isfinite(mu) || !(lambda > 0.f) || !isfinite(lambda)) return MPF_EINVAL;
  DeviceGuard dg(ctx->device);
  if (n && (!is_device_ptr(nat) || !is_device_ptr(p))) return MPF_EINVAL;
  return launch_pvalues(nat, n, mu, lambda, p, ctx->num_sms, ctx->stream) ? MPF_ECUDA : MPF_OK;
}

void mpf_plan_destroy(mpf_plan *plan) {
  if (!plan) return;
  {
    DeviceGuard dg(plan->ctx->device);
    cudaStreamSynchronize(plan->ctx->stream);
  }
  plan_free(plan);
}

}  // extern "C"
