// mpf_pipeline.cu -- filter-to-filter hand-off and P-values (Sec. 2.1).
//
// In the HMMER3 pipeline SSV scores every sequence, only the sequences whose
// SSV score passes a threshold are re-scored by MSV, and only the MSV
// survivors by the Viterbi filter.  Between two stages these kernels compact,
// per query, the length ranks of the passing sequences into an ascending list
// (stable, so the next scan keeps its length-homogeneous batches) and mark
// every other sequence as filtered in the next stage's outputs.  A sequence
// passes when the earlier stage flagged it as overflowed (flag 1) or its nat
// score is >= the threshold; a sequence the earlier stage itself filtered
// (flag 2, nat NaN) never passes.  A separate element-wise kernel turns nat
// scores into Gumbel P-values.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "mpf_internal.h"

namespace mpf {

namespace {

constexpr int kSelThreads = 256;

struct SelectParams {
  const uint32_t *seq_orig;   // per length rank: original sequence number
  uint64_t n;                 // sequences
  uint32_t n_chunks;          // ceil(n / kSelectChunk)
  const uint8_t *in_flag;     // [q][n] by original number: earlier stage
  const float *in_nat;        // [q][n]
  float min_nat;              // a sequence passes if its nat >= min_nat or it overflowed
  void *out_raw;              // next stage's outputs: raw scores of raw_bytes each
  int raw_bytes;              // 1 (byte filters, filtered = 0) or 2 (Viterbi, filtered = -32768)
  uint8_t *out_flag;
  float *out_nat;             // nullable
  uint32_t *chunk_count;      // [q][n_chunks]
  uint32_t *chunk_offset;     // [q][n_chunks]
  uint32_t *ranks;            // [q][n] passing ranks, ascending
  uint32_t *n_ranks;          // [q]
};

__device__ __forceinline__ bool passes(const SelectParams &p, uint64_t idx) {
  return p.in_flag[idx] == 1 || p.in_nat[idx] >= p.min_nat;
}

// Pass 1: count the passing sequences of one chunk of ranks of one query and
// mark every sequence of the chunk as filtered (raw 0 or -32768, flag 2, nat
// NaN); the next scan overwrites the passing ones.
__global__ void __launch_bounds__(kSelThreads) select_count(SelectParams p) {
  const uint32_t q = blockIdx.y;
  const uint64_t lo = (uint64_t)blockIdx.x * kSelectChunk;
  const uint64_t hi = min(lo + (uint64_t)kSelectChunk, p.n);
  uint32_t c = 0;
  for (uint64_t r = lo + threadIdx.x; r < hi; r += blockDim.x) {
    const uint64_t idx = (uint64_t)q * p.n + p.seq_orig[r];
    c += passes(p, idx) ? 1u : 0u;
    if (p.raw_bytes == 2)
      static_cast<int16_t *>(p.out_raw)[idx] = (int16_t)-32768;
    else
      static_cast<uint8_t *>(p.out_raw)[idx] = 0;
    p.out_flag[idx] = 2;
    if (p.out_nat) p.out_nat[idx] = __int_as_float(0x7fc00000);
  }
  __shared__ uint32_t warp_sum[kSelThreads / 32];
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) t += warp_sum[w];
    p.chunk_count[(uint64_t)q * p.n_chunks + blockIdx.x] = t;
  }
}

// Pass 2: exclusive prefix sum of the chunk counts of one query (one block
// per query, tiles of blockDim chunks with a running carry); total -> n_ranks.
__global__ void __launch_bounds__(1024) select_scan(SelectParams p) {
  const uint32_t q = blockIdx.x;
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const uint32_t *cnt = p.chunk_count + (uint64_t)q * p.n_chunks;
  uint32_t *off = p.chunk_offset + (uint64_t)q * p.n_chunks;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (uint32_t base = 0; base < p.n_chunks; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < p.n_chunks ? cnt[i] : 0u;
    uint32_t x = v;   // inclusive warp scan
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < nwarps ? warp_sum[lane] : 0u;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += y;
      }
      if (lane < nwarps) warp_sum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const uint32_t before_warp = warp > 0 ? warp_sum[warp - 1] : 0u;
    if (i < p.n_chunks) off[i] = carry + before_warp + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nwarps - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) p.n_ranks[q] = carry;
}

// Pass 3: write the passing ranks of one chunk, in order, at the chunk's offset.
__global__ void __launch_bounds__(kSelThreads) select_write(SelectParams p) {
  const uint32_t q = blockIdx.y;
  const uint64_t lo = (uint64_t)blockIdx.x * kSelectChunk;
  const uint64_t hi = min(lo + (uint64_t)kSelectChunk, p.n);
  __shared__ uint32_t warp_sum[kSelThreads / 32];
  uint32_t pos = p.chunk_offset[(uint64_t)q * p.n_chunks + blockIdx.x];
  uint32_t *out = p.ranks + (uint64_t)q * p.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t t = lo; t < hi; t += blockDim.x) {
    const uint64_t r = t + threadIdx.x;
    const bool pass = r < hi && passes(p, (uint64_t)q * p.n + p.seq_orig[r]);
    const uint32_t bal = __ballot_sync(0xffffffffu, pass);
    if (lane == 0) warp_sum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
      const uint32_t s = warp_sum[w];
      before += w < warp ? s : 0u;
      total += s;
    }
    if (pass) out[pos + before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)r;
    pos += total;
    __syncthreads();
  }
}

// P-value of a nat score under a Gumbel distribution (location mu, slope
// lambda): P(S > x) = 1 - exp(-exp(-lambda (x - mu))); +inf scores (overflow)
// have P = 0, NaN (filtered) stays NaN.
__global__ void pvalue_kernel(const float *nat, uint64_t n, float mu, float lambda, float *p) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float x = nat[i];
    float r;
    if (isnan(x)) {
      r = x;
    } else if (isinf(x)) {
      r = x > 0.f ? 0.f : 1.f;
    } else {
      const float y = expf(-lambda * (x - mu));
      r = -expm1f(-y);
    }
    p[i] = r;
  }
}

}  // namespace

int launch_select(const uint32_t *seq_orig, uint64_t n, int n_q, const uint8_t *in_flag,
                  const float *in_nat, float min_nat, void *out_raw, int raw_bytes,
                  uint8_t *out_flag, float *out_nat, uint32_t *chunk_count,
                  uint32_t *chunk_offset, uint32_t *ranks, uint32_t *n_ranks, cudaStream_t st) {
  SelectParams p;
  p.seq_orig = seq_orig;
  p.n = n;
  p.n_chunks = (uint32_t)((n + kSelectChunk - 1) / kSelectChunk);
  p.in_flag = in_flag;
  p.in_nat = in_nat;
  p.min_nat = min_nat;
  p.out_raw = out_raw;
  p.raw_bytes = raw_bytes;
  p.out_flag = out_flag;
  p.out_nat = out_nat;
  p.chunk_count = chunk_count;
  p.chunk_offset = chunk_offset;
  p.ranks = ranks;
  p.n_ranks = n_ranks;
  if (n == 0) return cudaMemsetAsync(n_ranks, 0, sizeof(uint32_t) * (size_t)n_q, st) == cudaSuccess ? 0 : 1;
  const dim3 grid(p.n_chunks, (unsigned)n_q);
  select_count<<<grid, kSelThreads, 0, st>>>(p);
  select_scan<<<(unsigned)n_q, 1024, 0, st>>>(p);
  select_write<<<grid, kSelThreads, 0, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int launch_pvalues(const float *nat, uint64_t n, float mu, float lambda, float *p, int num_sms,
                   cudaStream_t st) {
  if (n == 0) return 0;
  const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms * 8);
  pvalue_kernel<<<(unsigned)blocks, 256, 0, st>>>(nat, n, mu, lambda, p);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace mpf
