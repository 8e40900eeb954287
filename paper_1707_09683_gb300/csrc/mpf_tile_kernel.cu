// mpf_tile_kernel.cu -- SSV (Alg. 7) and MSV (Alg. 2) for models longer
// than the striped shared-memory table holds, tiled along the model.
//
// SSV has no coupling across a row except its running maximum, so the model
// can be cut into tiles of kTileNodes nodes swept one after the other over
// the whole sequence: the cell at the first node of a tile reads, on the
// previous row, the last node of the tile before (Alg. 7's diagonal), and
// nothing else crosses the cut.  A block of warps takes a batch of
// consecutive length ranks (one sequence per warp, similar lengths) through
// all tiles of its query together: per tile the block stages the tile's
// scores into shared memory, and each warp sweeps its sequence with the
// tile's DP row in registers.  Lane l holds the kTileC consecutive nodes
// l*kTileC + c as kTileC/2 16-bit pairs, pair p = (node p, node p + kTileC/2)
// of the lane, so the diagonal of pair p is the previous row's pair p - 1 as
// it stands and only pair 0 is assembled (from the lane before's last node
// and this lane's node kTileC/2 - 1).  The previous tile's last node reaches
// lane 0 through the warp's boundary column in device memory: one int16 per
// row, written by lane 31 one row later than read (position i + 1 holds row
// i), two buffers by tile parity.
//
// Cells are the unsaturated form r = max(0, r'[k-1] + s) with s = bias -
// cost, one DPX add-then-max per pair of cells; R >= 255 is the overflow
// (the Sec. 2.1 reading of Alg. 7 the other kernels use).  Values above
// 32767 wrap to negative and restart at 0, which only happens after some
// cell has passed 255, so after R >= 255.  Nodes past M score -32768, which
// keeps them at 0.
//
// MSV couples the rows through xE -> xJ -> xB, which a tile cannot see.  As
// in the striped kernels' lazy form, v = max(0, dp - b) follows the same
// recurrence as SSV while the begin score b stays constant, and b moves
// only once xJ passes base.  So the tiles are swept with b held at its
// initial value.  What decides the sequence is the first row whose maximum
// over the whole model passes T = min(base + tec - b, 255 - bias - b - 1),
// and that maximum: a row's maximum passes T exactly when some lane of some
// tile has a cell above T in it, so each lane keeps the first such row of
// its own cells (over the tiles) and its largest cell there, and one warp
// reduction per sequence gives the row and the row maximum.  Then: no such
// row (raw from the largest cell, or, if no cell rose above b, from the
// best single-cell score of the residues); an overflow there (raw 255,
// flag); the last row (raw as if none); or a row after which xB would move
// -- the sequence's rank goes to the query's fallback list, which the exact
// lane-segment kernel scores next (Alg. 2 row by row).
//
// With b held the swept cells are the SSV cells, so the MSV kernel's largest
// cell is also SSV's R: the both-filter variant (MODE_TILE_MSV_SSV) writes
// the SSV outputs from it in the same sweep.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mpf_internal.h"
#include "mpf_tmem.cuh"

namespace mpf {

namespace {

constexpr uint32_t kAll = 0xffffffffu;
constexpr uint32_t kNone = 0xffffffffu;
constexpr int kChunks = kTileC / 8;   // 16-byte chunks (4 pairs) per lane and residue row
constexpr int kPairs = kTileC / 2;

// The larger of the two 16-bit halves.
__device__ __forceinline__ int half_max(uint32_t w) { return max((int)(int16_t)(w & 0xffffu), (int)(int16_t)(w >> 16)); }

// One row of the lane's tile segment: v holds the previous row and receives
// this row; `in` is the previous row's score of the node before the lane's
// segment.  rmax collects the row's cells (pair-wise maxima).
__device__ __forceinline__ void tile_row(uint32_t (&v)[kPairs], uint32_t in, const uint4 *srow,
                                         uint32_t &rmax) {
  // Pair 0's diagonal: (node before the segment, node kPairs - 1), previous row.
  const uint32_t d0 = __byte_perm(in, v[kPairs - 1], 0x5410);
#pragma unroll
  for (int q = kChunks - 1; q >= 0; --q) {
    const uint4 s = srow[q * 32];
    const uint32_t sq[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
    for (int e = 3; e >= 0; --e) {
      const int p = q * 4 + e;
      v[p] = __viaddmax_s16x2(p > 0 ? v[p - 1] : d0, sq[e], 0u);
    }
    rmax = __vimax3_s16x2(rmax, v[q * 4], v[q * 4 + 1]);
    rmax = __vimax3_s16x2(rmax, v[q * 4 + 2], v[q * 4 + 3]);
  }
}

// tile_row with the row's scores in registers (word p = pair p).
__device__ __forceinline__ void tile_row_regs(uint32_t (&v)[kPairs], uint32_t in, const uint32_t (&sc)[kPairs],
                                              uint32_t &rmax) {
  const uint32_t d0 = __byte_perm(in, v[kPairs - 1], 0x5410);
#pragma unroll
  for (int q = kChunks - 1; q >= 0; --q) {
#pragma unroll
    for (int e = 3; e >= 0; --e) {
      const int p = q * 4 + e;
      v[p] = __viaddmax_s16x2(p > 0 ? v[p - 1] : d0, sc[p], 0u);
    }
    rmax = __vimax3_s16x2(rmax, v[q * 4], v[q * 4 + 1]);
    rmax = __vimax3_s16x2(rmax, v[q * 4 + 2], v[q * 4 + 3]);
  }
}

// The same with the node before the segment in the high half of `in_word`
// (the lane before's pair 15, or a boundary-column word): no extraction.
__device__ __forceinline__ void tile_row_regs_w(uint32_t (&v)[kPairs], uint32_t in_word,
                                                const uint32_t (&sc)[kPairs], uint32_t &rmax) {
  const uint32_t d0 = __byte_perm(in_word, v[kPairs - 1], 0x5432);
#pragma unroll
  for (int q = kChunks - 1; q >= 0; --q) {
#pragma unroll
    for (int e = 3; e >= 0; --e) {
      const int p = q * 4 + e;
      v[p] = __viaddmax_s16x2(p > 0 ? v[p - 1] : d0, sc[p], 0u);
    }
    rmax = __vimax3_s16x2(rmax, v[q * 4], v[q * 4 + 1]);
    rmax = __vimax3_s16x2(rmax, v[q * 4 + 2], v[q * 4 + 3]);
  }
}

// MSV result of one sequence, by the whole warp: frow / fval, this lane's
// first row with a cell above T and its largest cell there (kNone: none),
// V this lane's largest cell.
__device__ __noinline__ void msv_finish(const ScanParams &sp, const QueryDesc &qd, uint32_t r, uint32_t len,
                                        uint32_t orig, int lane, int b, int t, uint32_t frow, int fval, int V,
                                        bool both) {
  const int cap = 255 - qd.bias;
  const uint32_t first = __reduce_min_sync(kAll, frow);
  const int m = __reduce_max_sync(kAll, frow == first ? fval : -1);
  V = __reduce_max_sync(kAll, V);
  if (both && lane == 0) {   // SSV from the same largest cell
    const int raw = min(V, 255);
    const int flag = V >= 255 ? 1 : 0;
    qd.raw2[orig] = (uint8_t)raw;
    qd.flag2[orig] = (uint8_t)flag;
    if (qd.nat2)
      qd.nat2[orig] = flag ? __int_as_float(0x7f800000)
                           : __fsub_rn(__fdiv_rn(__int2float_rn(raw - qd.tbm - qd.tec - 2 * t), qd.scale), 3.0f);
  }
  // No cell rose above b: the best row maximum is the best single-cell
  // score of the residues (per-code maxima stored after the tiles).
  int g = -(1 << 20);
  if (V == 0 && len > 0 && first == kNone) {
    const int16_t *smax =
        reinterpret_cast<const int16_t *>(reinterpret_cast<const uint8_t *>(qd.table) + qd.smax_off);
    const int mine = (int)__ldg(smax + lane);
    const uint32_t w0 = __ldg(sp.seq_word + r);
    for (uint32_t j0 = 0; j0 < len; j0 += 32) {
      const uint32_t j = j0 + lane;
      uint32_t x = 0;
      if (j < len) x = (__ldg(sp.residues + w0 + (j >> 2)) >> (8 * (j & 3))) & 0xffu;
      if (!MPF_DCHECK(sp.status, x < 32u)) x = 0;
      const int sx = __shfl_sync(kAll, mine, (int)x);
      if (j < len) g = max(g, sx);
    }
    g = __reduce_max_sync(kAll, g);
  }
  if (lane != 0) return;
  int raw = 0, flag = 0;
  if (len > 0) {
    if (first != kNone) {
      if (b + m >= cap) {
        raw = 255;
        flag = 1;
      } else if (first + 1 < len) {
        // xB moves after this row: score the sequence exactly.
        const uint32_t k = atomicAdd(qd.fallback_count, 1u);
        if (MPF_DCHECK(sp.status, k < sp.n_seqs)) qd.fallback_ranks[k] = r;
        return;
      } else {
        raw = max(0, b + V - qd.tec);
      }
    } else {
      raw = V > 0 ? max(0, b + V - qd.tec) : max(0, b + g - qd.tec);
    }
  }
  qd.raw[orig] = (uint8_t)raw;
  qd.flag[orig] = (uint8_t)flag;
  if (qd.nat)
    qd.nat[orig] = flag ? __int_as_float(0x7f800000)
                        : __fsub_rn(__fdiv_rn(__int2float_rn(raw - t - qd.base), qd.scale), 3.0f);
}

template <bool MSV, bool BOTH = false>
__global__ void __launch_bounds__(kTileWarps * 32) tile_kernel(ScanParams sp) {
  static_assert(MSV || !BOTH, "the both-filter sweep is the MSV sweep");
  // Shared memory: the tile's scores, [code][chunk][lane] x 4 pairs.
  extern __shared__ __align__(16) uint4 tsm[];
  __shared__ uint32_t s_item;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  constexpr int kTileWords = 32 * kChunks * 32;   // uint4 per tile
  const uint64_t cw = (uint64_t)blockIdx.x * W + warp;
  // This warp's two boundary columns (int16 per row, position i + 1 = row i).
  int16_t *colbuf = reinterpret_cast<int16_t *>(sp.tile_col + cw * 2 * (uint64_t)sp.tile_col_stride);
  const uint32_t col_elems = sp.tile_col_stride / 2;
  // Debug builds: the table and this warp's columns within their buffers.
  if (!MPF_DCHECK(sp.status, (size_t)kTileWords * 16 <= dynamic_smem_bytes() &&
                                 (cw + 1) * 2 * sp.tile_col_stride <= sp.tile_col_bytes &&
                                 (sp.tile_col_stride & 15) == 0))
    return;

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(sp.item_counter, 1u);
    __syncthreads();
    uint64_t rem = s_item;
    __syncthreads();   // read by all before the next item's write
    // Item: the rem-th batch of W consecutive selected ranks of a query.
    uint32_t qi = 0;
    uint64_t n_sel = 0;
    for (; qi < sp.n_queries; ++qi) {
      const QueryDesc &qd = sp.queries[qi];
      n_sel = qd.ranks ? (uint64_t)*qd.n_ranks : (uint64_t)sp.n_seqs;
      const uint64_t nb = (n_sel + W - 1) / W;
      if (rem < nb) break;
      rem -= nb;
    }
    if (qi == sp.n_queries) break;
    const QueryDesc &qd = sp.queries[qi];
    const uint64_t ri = rem * W + warp;
    bool active = ri < n_sel && MPF_DCHECK(sp.status, n_sel <= sp.n_seqs);
    uint32_t r = 0, w0 = 0, len = 0, orig = 0;
    if (active) {
      r = qd.ranks ? __ldg(qd.ranks + ri) : (uint32_t)ri;
      active = MPF_DCHECK(sp.status, r < sp.n_seqs);
    }
    if (active) {
      w0 = __ldg(sp.seq_word + r);
      len = __ldg(sp.seq_len + r);
      orig = __ldg(sp.seq_orig + r);
      // The columns hold positions 0..len, and the prefetch reads up to
      // position len + 10.
      active = MPF_DCHECK(sp.status, (uint64_t)w0 + ((len + 3u) >> 2) <= sp.n_words && orig < sp.n_seqs &&
                                         (uint64_t)len + 11 <= col_elems);
    }
    const int tj = qd.tjb ? (int)__ldg(qd.tjb + min(len, qd.n_tjb - 1u)) : qd.tjb_fixed;
    // MSV: the begin score held over the tiles, and the threshold T.
    const int b = min(min(255, max(0, qd.base - (tj + qd.tbm))), 255 - qd.bias);
    const int T = min(qd.base + qd.tec - b, 255 - qd.bias - b - 1);
    uint32_t frow = kNone;   // MSV: this lane's first row with a cell above T
    int fval = -1;
    const int nt = (int)((qd.M + kTileNodes - 1) / kTileNodes);
    uint32_t rmax = 0;   // running maximum, two 16-bit halves
    for (int t = 0; t < nt; ++t) {
      __syncthreads();   // every warp is done with the previous tile
      const uint4 *g = qd.table + (size_t)t * kTileWords;
      for (int i = threadIdx.x; i < kTileWords; i += blockDim.x) tsm[i] = __ldg(g + i);
      __syncthreads();
      if (!active) continue;
      const int16_t *cin = colbuf + (size_t)((t + 1) & 1) * col_elems;   // previous tile's column
      int16_t *cout = colbuf + (size_t)(t & 1) * col_elems;              // this tile's column
      const bool first = t == 0, write = t + 1 < nt;
      if (write && lane == 31) cout[0] = 0;   // row -1
      uint32_t v[kPairs];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) v[p] = 0u;
      const uint4 *sbase = tsm + lane;
      // Rolling prefetch of the boundary column, four rows per 64-bit word.
      uint2 cur = make_uint2(0, 0), nxt = make_uint2(0, 0);
      if (lane == 0 && !first) {
        cur = __ldcg(reinterpret_cast<const uint2 *>(cin));
        nxt = __ldcg(reinterpret_cast<const uint2 *>(cin) + 1);
      }
      for (uint32_t i0 = 0; i0 < len; i0 += 4) {
        const uint32_t word = __ldg(sp.residues + w0 + (i0 >> 2));
        uint2 c = cur;
        if (lane == 0 && !first) {
          cur = nxt;
          nxt = __ldcg(reinterpret_cast<const uint2 *>(cin) + (i0 >> 2) + 2);
        }
        const uint32_t xs[4] = {__byte_perm(word, 0u, 0x4440), __byte_perm(word, 0u, 0x4441),
                                __byte_perm(word, 0u, 0x4442), __byte_perm(word, 0u, 0x4443)};
        const uint32_t cs[4] = {c.x & 0xffffu, c.x >> 16, c.y & 0xffffu, c.y >> 16};
        uint32_t rq[4] = {0u, 0u, 0u, 0u};   // MSV: this lane's maxima of the four rows
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (i0 + u < len) {
            uint32_t x = xs[u];
            if (!MPF_DCHECK(sp.status, x < 32u)) x = 0;
            // The node before the lane's segment, previous row: the lane
            // before's last node; for lane 0 the previous tile's last node.
            uint32_t in = __shfl_up_sync(kAll, v[kPairs - 1] >> 16, 1);
            if (lane == 0) in = cs[u];
            tile_row(v, in, sbase + x * (kChunks * 32), MSV ? rq[u] : rmax);
            if (write && lane == 31) cout[i0 + u + 1] = (int16_t)(v[kPairs - 1] >> 16);
          }
        }
        if (MSV) {
          // (Cells are >= 0 until an overflow, so the relu forms are exact.)
          const uint32_t r4 = __vimax3_s16x2(rq[0], rq[1], __vimax_s16x2_relu(rq[2], rq[3]));
          rmax = __vimax_s16x2_relu(rmax, r4);
          // The first of these rows with a cell above T, if not later than
          // this lane's first so far (rows after it cannot matter; the same
          // row in another tile keeps the larger cell).  Rows past the end
          // hold 0, which T = -1 would count: they are left out.
          if (i0 <= frow && half_max(r4) > T) {
#pragma unroll
            for (int u = 3; u >= 0; --u) {
              const int mu = half_max(rq[u]);
              const uint32_t row = i0 + u;
              if (mu > T && row < len) {
                if (row < frow) {
                  frow = row;
                  fval = mu;
                } else if (row == frow) {
                  fval = max(fval, mu);
                }
              }
            }
          }
        }
      }
    }
    if (MSV) {
      if (active) msv_finish(sp, qd, r, len, orig, lane, b, tj, frow, fval, half_max(rmax), BOTH);
      continue;
    }
    // R over the sequence: the largest half of any lane.
    int R = 0;
    if (active) R = half_max(rmax);
    R = __reduce_max_sync(kAll, R);
    if (active && lane == 0) {
      const int raw = min(R, 255);
      const int flag = R >= 255 ? 1 : 0;
      qd.raw[orig] = (uint8_t)raw;
      qd.flag[orig] = (uint8_t)flag;
      if (qd.nat)
        qd.nat[orig] = flag ? __int_as_float(0x7f800000)
                            : __fsub_rn(__fdiv_rn(__int2float_rn(raw - qd.tbm - qd.tec - 2 * tj), qd.scale), 3.0f);
    }
  }
}

// The tensor-memory variant: blocks of kTileWarpsTm warps, one block per SM
// (it allocates all of the SM's TMEM columns).  The tile's scores are not
// staged in shared memory: every lane quarter of TMEM holds the whole tile,
// code x's kPairs words of lane l at columns x * kPairs .. + kPairs - 1 of
// the quarter's lane l (32 codes x 16 words = the 512 columns), and warp w
// reads quarter w mod 4.  Warp w fills codes 8 (w / 4) .. + 7 of its quarter
// from the tile in device memory.  One sequence per warp makes the residue
// code of a row warp-uniform, so a row's 16 words are one tcgen05.ld, issued
// a row ahead into the other of two register buffers.
template <bool MSV, bool BOTH>
__global__ void __launch_bounds__(kTileWarpsTm * 32, 1) tile_kernel_tm(ScanParams sp) {
  static_assert(MSV || !BOTH, "the both-filter sweep is the MSV sweep");
  static_assert(32 * kPairs == (int)kTmemColumns && kTileWarpsTm % 4 == 0, "a tile fills a lane quarter");
  __shared__ uint32_t s_item, s_tmem;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  constexpr int kTileWords = 32 * kChunks * 32;   // uint4 per tile
  const uint64_t cw = (uint64_t)blockIdx.x * W + warp;
  // Boundary columns of 32-bit words: position i + 1 holds row i's pair 15
  // of lane 31 (node 31 in the high half), read by the next tile's lane 0.
  uint32_t *colbuf = reinterpret_cast<uint32_t *>(sp.tile_col + cw * 2 * (uint64_t)sp.tile_col_stride);
  const uint32_t col_elems = sp.tile_col_stride / 4;
  // Debug builds: the block shape and the block's columns within their
  // buffers (a block-uniform test, before the allocation).
  if (!MPF_DCHECK(sp.status, W == kTileWarpsTm &&
                                 ((uint64_t)blockIdx.x + 1) * W * 2 * sp.tile_col_stride <= sp.tile_col_bytes &&
                                 (sp.tile_col_stride & 15) == 0))
    return;
  if (warp == 0) tm_alloc(&s_tmem);
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  const uint32_t tm_lane = s_tmem + ((uint32_t)((warp & 3) * 32) << 16);

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(sp.item_counter, 1u);
    __syncthreads();
    uint64_t rem = s_item;
    __syncthreads();
    uint32_t qi = 0;
    uint64_t n_sel = 0;
    for (; qi < sp.n_queries; ++qi) {
      const QueryDesc &qd = sp.queries[qi];
      n_sel = qd.ranks ? (uint64_t)*qd.n_ranks : (uint64_t)sp.n_seqs;
      const uint64_t nb = (n_sel + W - 1) / W;
      if (rem < nb) break;
      rem -= nb;
    }
    if (qi == sp.n_queries) break;   // block-uniform
    const QueryDesc &qd = sp.queries[qi];
    const uint64_t ri = rem * W + warp;
    bool active = ri < n_sel && MPF_DCHECK(sp.status, n_sel <= sp.n_seqs);
    uint32_t r = 0, w0 = 0, len = 0, orig = 0;
    if (active) {
      r = qd.ranks ? __ldg(qd.ranks + ri) : (uint32_t)ri;
      active = MPF_DCHECK(sp.status, r < sp.n_seqs);
    }
    if (active) {
      w0 = __ldg(sp.seq_word + r);
      len = __ldg(sp.seq_len + r);
      orig = __ldg(sp.seq_orig + r);
      active = MPF_DCHECK(sp.status, (uint64_t)w0 + ((len + 3u) >> 2) <= sp.n_words && orig < sp.n_seqs &&
                                         (uint64_t)len + 11 <= col_elems);
    }
    const int tj = qd.tjb ? (int)__ldg(qd.tjb + min(len, qd.n_tjb - 1u)) : qd.tjb_fixed;
    const int b = min(min(255, max(0, qd.base - (tj + qd.tbm))), 255 - qd.bias);
    const int T = min(qd.base + qd.tec - b, 255 - qd.bias - b - 1);
    uint32_t frow = kNone;
    int fval = -1;
    const int nt = (int)((qd.M + kTileNodes - 1) / kTileNodes);
    uint32_t rmax = 0;
    for (int t = 0; t < nt; ++t) {
      // Every thread waited for its loads of the previous tile: order them
      // before this tile's TMEM writes.
      tm_fence_before();
      __syncthreads();
      tm_fence_after();
      {
        const uint4 *g = qd.table + (size_t)t * kTileWords + lane;
        const int x0 = 8 * (warp >> 2);
#pragma unroll 2
        for (int x = x0; x < x0 + 8; ++x) {
          const uint4 c0 = __ldg(g + x * 128), c1 = __ldg(g + x * 128 + 32), c2 = __ldg(g + x * 128 + 64),
                      c3 = __ldg(g + x * 128 + 96);
          const uint32_t col = tm_lane + (uint32_t)(x * kPairs);
          tm_st4(col, c0.x, c0.y, c0.z, c0.w);
          tm_st4(col + 4, c1.x, c1.y, c1.z, c1.w);
          tm_st4(col + 8, c2.x, c2.y, c2.z, c2.w);
          tm_st4(col + 12, c3.x, c3.y, c3.z, c3.w);
        }
        tm_wait_st();
      }
      tm_fence_before();
      __syncthreads();
      tm_fence_after();
      if (!active) continue;
      const uint32_t *cin = colbuf + (size_t)((t + 1) & 1) * col_elems;
      uint32_t *cout = colbuf + (size_t)(t & 1) * col_elems;
      const bool first = t == 0, write = t + 1 < nt;
      if (write && lane == 31) cout[0] = 0;
      uint32_t v[kPairs];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) v[p] = 0u;
      uint4 cur = make_uint4(0, 0, 0, 0), nxt = make_uint4(0, 0, 0, 0);
      if (lane == 0 && !first) {
        cur = __ldcg(reinterpret_cast<const uint4 *>(cin));
        nxt = __ldcg(reinterpret_cast<const uint4 *>(cin) + 1);
      }
      // Score rows of the current and the next row.  Codes are < 32 in a
      // sequence; the load issued for the row after the last one takes any
      // code (only waited for).
      uint32_t TA[kPairs], TB[kPairs];
      uint32_t word = len ? __ldg(sp.residues + w0) : 0u;
      tm_ld<kPairs>(TA, tm_lane + (word & 31u) * (uint32_t)kPairs);
      for (uint32_t i0 = 0; i0 < len; i0 += 4) {
        const uint32_t nword = i0 + 4 < len ? __ldg(sp.residues + w0 + (i0 >> 2) + 1) : 0u;
        const uint4 c = cur;
        if (lane == 0 && !first) {
          cur = nxt;
          nxt = __ldcg(reinterpret_cast<const uint4 *>(cin) + (i0 >> 2) + 2);
        }
        const uint32_t cs[4] = {c.x, c.y, c.z, c.w};
        uint32_t rq[4] = {0u, 0u, 0u, 0u};
        // One row: wait for its scores, issue the next row's load, update.
        // The next row's code is masked to 0..31 (a column of the tile): in
        // the sequence's last group of rows it may be a padding byte, whose
        // load is only waited for.
        auto one_row = [&](const int u, uint32_t (&Tc)[kPairs], uint32_t (&Tn)[kPairs]) {
          tm_wait_ld<kPairs>(Tc);
          MPF_DCHECK(sp.status, __byte_perm(word, 0u, 0x4440 + u) < 32u);
          const uint32_t xn = (u < 3 ? __byte_perm(word, 0u, 0x4441 + u) : nword) & 31u;
          tm_ld<kPairs>(Tn, tm_lane + xn * (uint32_t)kPairs);
          uint32_t in = __shfl_up_sync(kAll, v[kPairs - 1], 1);   // node 31 (high half), previous row
          if (lane == 0) in = cs[u];
          tile_row_regs_w(v, in, Tc, MSV ? rq[u] : rmax);
          if (write && lane == 31) cout[i0 + u + 1] = v[kPairs - 1];
        };
        if (i0 + 4 <= len) {   // warp-uniform: four rows, no row test
          one_row(0, TA, TB);
          one_row(1, TB, TA);
          one_row(2, TA, TB);
          one_row(3, TB, TA);
        } else {
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            if (i0 + u < len) {
              if (u & 1)
                one_row(u, TB, TA);
              else
                one_row(u, TA, TB);
            }
          }
        }
        word = nword;
        if (MSV) {
          const uint32_t r4 = __vimax3_s16x2(rq[0], rq[1], __vimax_s16x2_relu(rq[2], rq[3]));
          rmax = __vimax_s16x2_relu(rmax, r4);
          if (i0 <= frow && half_max(r4) > T) {
#pragma unroll
            for (int u = 3; u >= 0; --u) {
              const int mu = half_max(rq[u]);
              const uint32_t row = i0 + u;
              if (mu > T && row < len) {
                if (row < frow) {
                  frow = row;
                  fval = mu;
                } else if (row == frow) {
                  fval = max(fval, mu);
                }
              }
            }
          }
        }
      }
      tm_wait_ld<kPairs>(TA);   // the load issued after the last row
    }
    if (MSV) {
      if (active) msv_finish(sp, qd, r, len, orig, lane, b, tj, frow, fval, half_max(rmax), BOTH);
      continue;
    }
    int R = 0;
    if (active) R = half_max(rmax);
    R = __reduce_max_sync(kAll, R);
    if (active && lane == 0) {
      const int raw = min(R, 255);
      const int flag = R >= 255 ? 1 : 0;
      qd.raw[orig] = (uint8_t)raw;
      qd.flag[orig] = (uint8_t)flag;
      if (qd.nat)
        qd.nat[orig] = flag ? __int_as_float(0x7f800000)
                            : __fsub_rn(__fdiv_rn(__int2float_rn(raw - qd.tbm - qd.tec - 2 * tj), qd.scale), 3.0f);
    }
  }
  tm_fence_before();
  __syncthreads();
  if (warp == 0) {
    tm_fence_after();
    tm_dealloc(s_tmem);
  }
}

}  // namespace

KernelFn tile_kernel_fn(int mode, bool tm) {
  if (tm)
    return mode == MODE_TILE_MSV_SSV ? tile_kernel_tm<true, true>
           : mode == MODE_TILE_MSV   ? tile_kernel_tm<true, false>
                                     : tile_kernel_tm<false, false>;
  return mode == MODE_TILE_MSV_SSV ? tile_kernel<true, true> : mode == MODE_TILE_MSV ? tile_kernel<true> : tile_kernel<false>;
}

}  // namespace mpf
