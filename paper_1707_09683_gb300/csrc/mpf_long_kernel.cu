// mpf_long_kernel.cu -- MSV scans (Alg. 2) of models longer than the striped
// shared-memory table holds.  (SSV of such models runs tiled, with the DP row
// in registers: mpf_tile_kernel.cu.  MSV couples every row through xE, so it
// keeps the whole row, here in shared memory.)
//
// One warp scores one sequence.  Lane l owns the contiguous node segment
// [l*Q, l*Q + Q) (Q = 4 * seg_words); the byte costs are read from global
// memory in the same order (row x, word w of lane l at (x*seg_words + w)*32
// + l, four nodes per word), so every load of a warp is one 128-byte line,
// and the DP row lives in the warp's slice of shared memory, as 16-bit pairs
// (B8 = false) or, for the longest models, as bytes (B8 = true: half the
// shared memory per warp, so twice the warps, for two unpacking and one
// packing permute per four cells).
//
// Cells are held as u = 255 - v (v the byte score) in 16-bit halves, so that
// every byte saturation of the recurrence becomes one DPX add-then-min/max
// on a pair of cells with no wrap-around (all values stay in [0, 510]):
//   v = sat(sat(max(v'[k-1], xB) + bias) - c)
//   u = min(min(max(u'[k-1] - bias, 0), max(uB - bias, 0)) + c, 255)
// and the row maximum of v is 255 minus the row minimum of u.  Node k-1 of
// the previous row is the previous half of the same lane, or for a
// segment's first node the last node of the lane before (one shuffle per
// row).  Nodes past M cost 255 and are forced to u = 255.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mpf_internal.h"

namespace mpf {

namespace {

constexpr uint32_t kAll = 0xffffffffu;
constexpr uint32_t kU255 = 0x00ff00ffu;   // two cells at v = 0

__device__ __forceinline__ uint32_t lo_cost_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }
__device__ __forceinline__ uint32_t hi_cost_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }
// (u[k-1], u[k]) for the pair (k, k+1): high half of the previous pair, low half of this one.
__device__ __forceinline__ uint32_t diag_pair(uint32_t prev, uint32_t cur) { return __byte_perm(prev, cur, 0x5432); }

__device__ __forceinline__ uint32_t cell_pair(uint32_t d, uint32_t c, uint32_t negbias2, uint32_t uBb2) {
  const uint32_t t = __vimin_s16x2_relu(__viaddmax_s16x2(d, negbias2, 0u), uBb2);
  return __viaddmin_s16x2(t, c, kU255);
}

// Force the halves of pair `p` (nodes 2p, 2p+1 of the lane's last word) that
// lie at or past the lane's valid count `part` (1..3 nodes of this word) to
// u = 255.
__device__ __forceinline__ uint32_t pad_mask(int pair, int part) {
  const int first = 2 * pair;
  uint32_t m = 0;
  if (first >= part) m |= 0x000000ffu;
  if (first + 1 >= part) m |= 0x00ff0000u;
  return m;
}

// DP row slot of one lane word (four cells): two 16-bit pairs or four bytes.
template <bool B8>
struct RowSlot;
template <>
struct RowSlot<false> {
  typedef uint2 T;
  static __device__ __forceinline__ T fill() { return make_uint2(kU255, kU255); }
  static __device__ __forceinline__ void split(T s, uint32_t &x, uint32_t &y) {
    x = s.x;
    y = s.y;
  }
  static __device__ __forceinline__ T join(uint32_t u0, uint32_t u1) { return make_uint2(u0, u1); }
};
template <>
struct RowSlot<true> {
  typedef uint32_t T;
  static __device__ __forceinline__ T fill() { return 0xffffffffu; }
  static __device__ __forceinline__ void split(T s, uint32_t &x, uint32_t &y) {
    x = lo_cost_pair(s);
    y = hi_cost_pair(s);
  }
  static __device__ __forceinline__ T join(uint32_t u0, uint32_t u1) { return __byte_perm(u0, u1, 0x6420); }
};

template <bool B8, int U, bool PF>
__global__ void __launch_bounds__(kLongThreads) long_kernel(ScanParams sp) {
  typedef RowSlot<B8> Slot;
  extern __shared__ __align__(16) uint32_t lsm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  typename Slot::T *st = reinterpret_cast<typename Slot::T *>(lsm) + (size_t)warp * sp.long_words * 32 + lane;
  // Debug builds: the warps' DP rows must fit the block's shared memory.
  if (!MPF_DCHECK(sp.status, (size_t)(blockDim.x >> 5) * sp.long_words * 32 * sizeof(typename Slot::T) <=
                                 dynamic_smem_bytes()))
    return;

  for (;;) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(sp.item_counter, 1u);
    it = __shfl_sync(kAll, it, 0);
    // Item it: the (it - earlier queries' counts)-th selected rank of a query.
    uint32_t qi = 0;
    uint64_t rem = it;
    for (; qi < sp.n_queries; ++qi) {
      const QueryDesc &qd = sp.queries[qi];
      const uint64_t n_sel = qd.ranks ? (uint64_t)*qd.n_ranks : (uint64_t)sp.n_seqs;
      if (rem < n_sel) break;
      rem -= n_sel;
    }
    if (qi == sp.n_queries) break;
    const QueryDesc &qd = sp.queries[qi];
    if (!MPF_DCHECK(sp.status, rem < sp.n_seqs && qd.seg_words <= sp.long_words)) continue;
    const uint32_t r = qd.ranks ? __ldg(qd.ranks + rem) : (uint32_t)rem;
    if (!MPF_DCHECK(sp.status, r < sp.n_seqs)) continue;
    const uint32_t w0 = __ldg(sp.seq_word + r);
    const uint32_t len = __ldg(sp.seq_len + r);
    const uint32_t orig = __ldg(sp.seq_orig + r);
    if (!MPF_DCHECK(sp.status, (uint64_t)w0 + ((len + 3u) >> 2) <= sp.n_words && orig < sp.n_seqs)) continue;
    const int t = qd.tjb ? (int)__ldg(qd.tjb + min(len, qd.n_tjb - 1u)) : qd.tjb_fixed;
    const int bias = qd.bias;
    const int sw = (int)qd.seg_words;
    const int nv = min(max((int)qd.M - lane * 4 * sw, 0), 4 * sw);   // real nodes of this lane
    const int nfull = nv >> 2, part = nv & 3;
    const int nw = nfull + (part ? 1 : 0);
    const uint32_t *tab = reinterpret_cast<const uint32_t *>(qd.table) + lane;
    const uint32_t negbias2 = ((uint32_t)(-bias) & 0xffffu) * 0x00010001u;
    const uint32_t pm0 = part ? pad_mask(0, part) : 0u, pm1 = part ? pad_mask(1, part) : 0u;

    for (int w = 0; w < nw; ++w) st[(size_t)w * 32] = Slot::fill();
    int xJ = 0;
    int xB = min(255, max(0, qd.base - (t + qd.tbm)));
    uint32_t uBb2 = (uint32_t)max(255 - xB - bias, 0) * 0x00010001u;
    uint32_t carry = 255;                 // u of the node before the segment, previous row
    bool ovf = false;
    uint32_t word = 0;
    for (uint32_t i = 0; i < len; ++i) {
      if ((i & 3) == 0) word = __ldg(sp.residues + w0 + (i >> 2));
      uint32_t x = (word >> (8 * (i & 3))) & 0xffu;
      if (!MPF_DCHECK(sp.status, x < 32u)) x = 0;
      const uint32_t *row = tab + (size_t)x * sw * 32;
      uint32_t umin2 = kU255;             // row minimum
      uint32_t prev = carry << 16, last = kU255;
      // PF: a rolling window of the next four cost words, so four loads per
      // lane stay in flight whatever the unroll depth (the cost rows come
      // from L2 once they no longer fit in L1).
      uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      if (PF) {
        q0 = nfull > 0 ? __ldg(row) : 0u;
        q1 = nfull > 1 ? __ldg(row + 32) : 0u;
        q2 = nfull > 2 ? __ldg(row + 64) : 0u;
        q3 = nfull > 3 ? __ldg(row + 96) : 0u;
      }
#pragma unroll U
      for (int w = 0; w < nfull; ++w) {
        uint32_t cw;
        if (PF) {
          cw = q0;
          q0 = q1;
          q1 = q2;
          q2 = q3;
          q3 = w + 4 < nfull ? __ldg(row + (size_t)(w + 4) * 32) : 0u;
        } else {
          cw = __ldg(row + (size_t)w * 32);
        }
        uint32_t sx, sy;
        Slot::split(st[(size_t)w * 32], sx, sy);
        const uint32_t u0 = cell_pair(diag_pair(prev, sx), lo_cost_pair(cw), negbias2, uBb2);
        const uint32_t u1 = cell_pair(diag_pair(sx, sy), hi_cost_pair(cw), negbias2, uBb2);
        umin2 = __vimin3_u16x2(umin2, u0, u1);
        st[(size_t)w * 32] = Slot::join(u0, u1);
        prev = sy;
        last = u1;
      }
      if (part) {
        const uint32_t cw = __ldg(row + (size_t)nfull * 32);
        uint32_t sx, sy;
        Slot::split(st[(size_t)nfull * 32], sx, sy);
        uint32_t u0 = cell_pair(diag_pair(prev, sx), lo_cost_pair(cw), negbias2, uBb2);
        uint32_t u1 = cell_pair(diag_pair(sx, sy), hi_cost_pair(cw), negbias2, uBb2);
        u0 = __vimax_s16x2_relu(u0, pm0);
        u1 = __vimax_s16x2_relu(u1, pm1);
        umin2 = __vimin3_u16x2(umin2, u0, u1);
        st[(size_t)nfull * 32] = Slot::join(u0, u1);
        last = u1;
      }
      carry = __shfl_up_sync(kAll, last >> 16, 1);
      if (lane == 0) carry = 255;
      const int umin = (int)__reduce_min_sync(kAll, min(umin2 & 0xffffu, umin2 >> 16));
      const int xE = 255 - umin;
      if (xE >= 255 - bias) {
        ovf = true;
        break;
      }
      xJ = max(xJ, max(0, xE - qd.tec));
      xB = min(255, max(0, max(qd.base, xJ) - (t + qd.tbm)));
      uBb2 = (uint32_t)max(255 - xB - bias, 0) * 0x00010001u;
    }
    const int raw = ovf ? 255 : xJ;
    const int flag = ovf ? 1 : 0;
    const int num = xJ - t - qd.base;
    if (lane == 0) {
      qd.raw[orig] = (uint8_t)raw;
      qd.flag[orig] = (uint8_t)flag;
      if (qd.nat)
        qd.nat[orig] = flag ? __int_as_float(0x7f800000)
                            : __fsub_rn(__fdiv_rn(__int2float_rn(num), qd.scale), 3.0f);
    }
    __syncwarp();
  }
}

}  // namespace

// Unroll depth of the word loop and the rolling cost prefetch (measured on
// one query against 3,000-40,000 sequences): unroll 8 for segments of at most
// 48 words (M <= 6,144; 9-16% faster than 4), 16 with byte rows (M = 40,000:
// 35% faster), 4 in between; the prefetch in those two bands (M = 12,345:
// 1,597 against 1,138 GCUPS; M = 40,000: 934 against 877), not at unroll 8
// (mixed).
KernelFn long_kernel_for(int mode, bool bytes, int seg_words) {
  if (mode != MODE_LONG_MSV) return nullptr;
  if (bytes) return long_kernel<true, 16, true>;
  if (seg_words <= 48) return long_kernel<false, 8, false>;
  return long_kernel<false, 4, true>;
}

size_t long_smem_per_warp(int seg_words, bool bytes) {
  return (size_t)seg_words * 32 * (bytes ? sizeof(uint32_t) : sizeof(uint2));
}

}  // namespace mpf
