// mpf_noalloc.cu -- the allocation-free scan entry point (mpf_scan_noalloc).
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/mpf.h"
#include "mpf_handles.h"
#include "mpf_internal.h"

using namespace mpf;
using namespace mpf::host;

//
// mpf_scan_noalloc serves callers that must not allocate device memory at
// call time: services that account for every byte of device memory up front
// and run under a fixed budget, and plug-ins whose host application owns the
// device allocator (its pool holds the memory, and a cudaMalloc beside it can
// fail or stall the device).  Everything the scan kernel needs beyond its
// inputs and outputs -- the query descriptor, the work-item counter and the
// striped cost table -- lives in the file-scope device array below instead
// of memory from cudaMalloc; the kernel reports through the context's status
// word, like the regular scan.
namespace {

constexpr size_t kNoAllocHeader = 512;                 // descriptor, counter
constexpr size_t kNoAllocTableMax = 224u * 1024u;      // largest staged table image
constexpr size_t kNoAllocBytes = kNoAllocHeader + kNoAllocTableMax;

// Device scratch (one copy per GPU that loads the library, kept until exit).
// In host code this name is a host-side stand-in, never a device address:
// the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

// Host staging of the table image (pageable; a copy from it returns only
// after the driver has taken the bytes, so the next call may refill it).
static uint8_t g_noalloc_image[kNoAllocTableMax];
static std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
static uint8_t *g_noalloc_dev[kNoAllocMaxDevices];   // scratch address per device

}  // namespace

extern "C" int mpf_scan_noalloc(mpf_ctx *ctx, int filter, const mpf_profile *prof,
                                const mpf_db *db, uint8_t *raw, uint8_t *overflow, float *nat) {
  if (!ctx || !prof || !db || !raw || !overflow) return MPF_EINVAL;
  if (filter != MPF_MSV && filter != MPF_SSV) return MPF_EINVAL;
  if (prof->ctx->device != ctx->device || db->ctx->device != ctx->device) return MPF_EINVAL;
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices) return MPF_EUNSUPPORTED;
  DeviceGuard dg(ctx->device);
  if (!is_device_ptr(raw) || !is_device_ptr(overflow) || (nat && !is_device_ptr(nat)))
    return MPF_EINVAL;
  if (db->n_seqs == 0) return MPF_OK;

  if (prof->seg_words) return MPF_EUNSUPPORTED;   // long models need the table in device memory
  // The held-begin-score MSV lists sequences for a second kernel in device
  // memory; here the MSV kernel that tests the threshold row by row runs.
  int mode = kernel_mode(prof, filter);
  if (mode == MODE_MSV_HELD) mode = MODE_MSV_FAST;
  if (mode == MODE_MSV_HELD_F16) mode = MODE_MSV_FAST_F16;
  int lanes = prof->cfg_lanes[filter], words = prof->cfg_words[filter];
  if (!lanes) default_config(ctx, prof->M, mode, &lanes, &words);
  if (!lanes) return MPF_EUNSUPPORTED;
  const TableGeom g = table_geom(lanes, words);
  if (g.table_bytes > kNoAllocTableMax) return MPF_EUNSUPPORTED;   // beyond the scratch size
  KernelFn fn = kernel_for(lanes, words, mode);
  if (!fn) return MPF_EINVAL;

  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  // Set-up, once per device with that device current (the first call on a
  // device does it; make that first call outside any stream capture).
  if (!g_noalloc_dev[ctx->device]) {
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
      (void)cudaGetLastError();
      return MPF_ECUDA;
    }
    g_noalloc_dev[ctx->device] = (uint8_t *)addr;
  }
  uint8_t *scratch = g_noalloc_dev[ctx->device];

  // Striped table image (same layout the kernel stages into shared memory).
  fill_table_image(prof, g, table_format(mode), g_noalloc_image);

  QueryDesc q;
  memset(&q, 0, sizeof(q));
  q.table = reinterpret_cast<const uint4 *>(scratch + kNoAllocHeader);
  q.table_bytes = g.table_bytes;
  q.row_bytes = g.row_bytes;
  q.copy_bytes = g.copy_bytes;
  q.smax_off = g.smax_off;
  q.tail_off = g.tail_off;
  q.tail_row_bytes = g.tail_row_bytes;
  q.bias = prof->bias;
  q.tbm = prof->tbm;
  q.tec = prof->tec;
  q.base = prof->base;
  q.tjb_fixed = prof->tjb_fixed;
  q.scale = prof->scale;
  q.tjb = prof->d_tjb;
  q.n_tjb = prof->n_tjb;
  q.raw = raw;
  q.flag = overflow;
  q.nat = nat;
  static_assert(sizeof(QueryDesc) + 16 <= 256, "descriptor fits the scratch header");
  uint32_t *counter = reinterpret_cast<uint32_t *>(scratch + 256);

  const int smem = (int)g.table_bytes;
  MPF_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  MPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBlockThreads, smem));
  if (per_sm < 1) return MPF_EUNSUPPORTED;
  const uint32_t n_shards = (uint32_t)(ctx->num_sms * per_sm);

  // Every call reuses the same scratch: the table and descriptor are
  // rewritten and the counter cleared on the stream.
  MPF_CUDA(cudaMemcpyAsync(scratch + kNoAllocHeader, g_noalloc_image, g.table_bytes,
                           cudaMemcpyHostToDevice, ctx->stream));
  MPF_CUDA(cudaMemcpyAsync(scratch, &q, sizeof(q), cudaMemcpyHostToDevice, ctx->stream));
  MPF_CUDA(cudaMemsetAsync(scratch + 256, 0, 4, ctx->stream));

  ScanParams sp{};
  sp.residues = db->d_words;
  sp.n_words = db->n_words;
  sp.seq_word = db->d_seq_word;
  sp.seq_len = db->d_seq_len;
  sp.seq_orig = db->d_seq_orig;
  sp.n_seqs = (uint32_t)db->n_seqs;
  sp.pad_word = db->pad_word;
  sp.queries = reinterpret_cast<const QueryDesc *>(scratch);
  sp.n_queries = 1;
  sp.n_shards = n_shards;
  sp.item_counter = counter;
  sp.status = ctx->d_status;   // debug builds: failed index checks reach mpf_sync
  fn<<<(int)n_shards, kBlockThreads, smem, ctx->stream>>>(sp);
  MPF_CUDA(cudaGetLastError());
  return MPF_OK;
}

