// mpf_handles.h -- the library's handle structures and the host helpers
// shared by its translation units (mpf_api.cu, mpf_noalloc.cu,
// mpf_vit_api.cu).  Private: not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/mpf.h"
#include "mpf_internal.h"

using mpf::TableGeom;

struct mpf_plan;

struct mpf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int max_smem = 0;
  int *d_status = nullptr;
  // Scratch for host-pointer outputs (grown on demand).
  void *d_out = nullptr;
  size_t d_out_bytes = 0;
  // Streams for overlapping launch groups and for graph capture.
  cudaStream_t fork[8] = {};
  int n_fork = 0;
  cudaStream_t capture = nullptr;
  // Side stream for uploads that other streams must see complete (tables,
  // length tables): allocated and copied on it, then synchronised.
  cudaStream_t util = nullptr;
  // One-shot plans whose kernels may still be running.
  std::vector<mpf_plan *> pending;
};

struct DevTable {
  uint4 *ptr = nullptr;
  TableGeom geom{};
};

struct mpf_profile {
  mpf_ctx *ctx = nullptr;
  int M = 0, K = 0;
  std::vector<uint8_t> cost;  // K x M
  int bias = 0, tbm = 0, tec = 0, tjb_fixed = 0, base = 0;
  float scale = 1.f;
  uint8_t *d_tjb = nullptr;
  uint32_t n_tjb = 0;
  int tjb_min = 0;
  int cfg_lanes[2] = {0, 0}, cfg_words[2] = {0, 0};
  int shard_factor[2] = {1, 1};   // striped kernels: work items per query = factor x resident blocks
  int arith[2] = {MPF_ARITH_AUTO, MPF_ARITH_AUTO};
  int table_mem[2] = {MPF_TABLE_AUTO, MPF_TABLE_AUTO};
  int seg_words = 0;            // > 0: longer than the striped kernels hold (long-model kernel)
  mutable std::map<std::tuple<int, int, int>, DevTable> tables;
  mutable std::mutex mu;
};

struct mpf_db {
  mpf_ctx *ctx = nullptr;
  uint64_t n_seqs = 0, n_residues = 0;
  uint32_t *d_words = nullptr;      // residue words, sequences 16-byte aligned
  uint32_t n_words = 0;             // words in d_words
  uint32_t *d_seq_word = nullptr;   // per length rank
  uint32_t *d_seq_len = nullptr;
  uint32_t *d_seq_orig = nullptr;
  uint32_t pad_word = 0;
  int n_codes = 0;                  // distinct residue codes present
  uint32_t max_len = 0;             // longest sequence
};

// ---------------------------------------------------------------- helpers --

#define MPF_CUDA(call)                        \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) {                  \
      (void)cudaGetLastError();               \
      return e_ == cudaErrorMemoryAllocation ? MPF_ENOMEM : MPF_ECUDA; \
    }                                         \
  } while (0)

namespace mpf {
namespace host {


struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// True when any two of the n byte ranges [ptr, ptr + bytes) overlap (empty
// ranges overlap nothing).
inline bool ranges_overlap(const void *const *ptr, const uint64_t *bytes, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      if (!ptr[i] || !ptr[j] || !bytes[i] || !bytes[j]) continue;
      const uintptr_t a = (uintptr_t)ptr[i], b = (uintptr_t)ptr[j];
      if (a < b + bytes[j] && b < a + bytes[i]) return true;
    }
  return false;
}

// C status code of a nonzero device status word.
inline int status_code(int st) {
  if (st == 0) return MPF_OK;
  return st == kStatusBadIndex ? MPF_EDEVICE : MPF_ETIMEOUT;
}

// Default (lanes, words) of the striped kernels for a kernel mode.
void default_config(const mpf_ctx *ctx, int M, int mode, int *lanes, int *words);
// Kernel mode of a profile for a filter (arithmetic, MSV variant, long model).
int kernel_mode(const mpf_profile *p, int filter);
// Whether a striped scan in this configuration reads its table from TMEM.
bool use_tmem(const mpf_profile *p, int filter, int lanes, int words, int mode);
// Striped shared-memory image of a profile's score table.
void fill_table_image(const mpf_profile *p, const TableGeom &g, int fmt, uint8_t *img);
// Grow the context's device scratch for host-pointer outputs.
int ensure_out_scratch(mpf_ctx *ctx, size_t bytes);

}  // namespace host
}  // namespace mpf
