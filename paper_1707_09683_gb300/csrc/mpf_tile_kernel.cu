// mpf_tile_kernel.cu -- SSV (Alg. 7) for models longer than the striped
// shared-memory table holds, tiled along the model.
//
// SSV has no coupling across a row except its running maximum, so the model
// can be cut into tiles of kTileNodes nodes swept one after the other over
// the whole sequence: the cell at the first node of a tile reads, on the
// previous row, the last node of the tile before (Alg. 7's diagonal), and
// nothing else crosses the cut.  A block of warps takes a batch of
// consecutive length ranks (one sequence per warp, similar lengths) through
// all tiles of its query together: per tile the block stages the tile's
// scores into shared memory, and each warp sweeps its sequence with the
// tile's DP row in registers -- lane l holds kTileC consecutive nodes as
// 16-bit pairs -- reading the previous tile's boundary value for each row
// from, and writing its own to, the warp's column in device memory (one
// byte per row).
//
// Cells are the unsaturated form r = max(0, r'[k-1] + s) with s = bias -
// cost, one DPX add-then-max per pair of cells; R >= 255 is the overflow
// (Sec. 2.1 reading of Alg. 7, as in the other kernels).  A boundary value is
// stored as min(r, 255): a value of 255 there means R >= 255 already, so
// the result no longer depends on what follows.  Values above 32767 wrap to
// negative and restart at 0, which likewise only happens after R >= 255.
// Nodes past M score -32768, which keeps them at 0.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mpf_internal.h"

namespace mpf {

namespace {

constexpr uint32_t kAll = 0xffffffffu;
constexpr int kChunks = kTileC / 8;   // 16-byte chunks (8 cells) per lane and residue row

// (r[k-1], r[k]) for the pair (k, k+1): high half of the previous pair, low
// half of this one.
__device__ __forceinline__ uint32_t diag(uint32_t prev, uint32_t cur) { return __byte_perm(prev, cur, 0x5432); }

__global__ void __launch_bounds__(kTileWarps * 32) tile_ssv_kernel(ScanParams sp) {
  // Shared memory: the tile's scores, [code][chunk][lane] x 8 int16.
  extern __shared__ __align__(16) uint4 tsm[];
  __shared__ uint32_t s_item;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  constexpr int kTileWords = 32 * kChunks * 32;   // uint4 per tile
  const uint64_t cw = (uint64_t)blockIdx.x * W + warp;
  uint8_t *col = sp.tile_col + cw * sp.tile_col_stride;
  // Debug builds: the table and this warp's column within their buffers.
  if (!MPF_DCHECK(sp.status, (size_t)kTileWords * 16 <= dynamic_smem_bytes() &&
                                 (cw + 1) * sp.tile_col_stride <= sp.tile_col_bytes))
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
      active = MPF_DCHECK(sp.status, (uint64_t)w0 + ((len + 3u) >> 2) <= sp.n_words && orig < sp.n_seqs &&
                                         len <= sp.tile_col_stride);
    }
    const int nt = (int)((qd.M + kTileNodes - 1) / kTileNodes);
    uint32_t rmax = 0;   // running maximum, two 16-bit halves
    for (int t = 0; t < nt; ++t) {
      __syncthreads();   // every warp is done with the previous tile
      const uint4 *g = qd.table + (size_t)t * kTileWords;
      for (int i = threadIdx.x; i < kTileWords; i += blockDim.x) tsm[i] = __ldg(g + i);
      __syncthreads();
      if (!active) continue;
      const bool first = t == 0, last_tile = t == nt - 1;
      uint32_t v[kTileC / 2];
#pragma unroll
      for (int p = 0; p < kTileC / 2; ++p) v[p] = 0u;
      uint32_t word = 0, cin = 0, cout = 0, cprev = 0;
      for (uint32_t i = 0; i < len; ++i) {
        if ((i & 3) == 0) {
          word = __ldg(sp.residues + w0 + (i >> 2));
          if (lane == 0 && !first) cin = __ldcg(reinterpret_cast<const uint32_t *>(col) + (i >> 2));
        }
        uint32_t x = (word >> (8 * (i & 3))) & 0xffu;
        if (!MPF_DCHECK(sp.status, x < 32u)) x = 0;
        // Diagonal into the lane's first node: the lane before's last node
        // of the previous row; for lane 0 the previous tile's boundary
        // value of the previous row (0 before the first tile and row).
        uint32_t in = __shfl_up_sync(kAll, v[kTileC / 2 - 1] >> 16, 1);
        if (lane == 0) in = cprev;
        const uint4 *srow = tsm + (size_t)x * kChunks * 32 + lane;
#pragma unroll
        for (int q = kChunks - 1; q >= 0; --q) {
          const uint4 s = srow[q * 32];
          const uint32_t sq[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
          for (int e = 3; e >= 0; --e) {
            const int p = q * 4 + e;
            const uint32_t prev = p > 0 ? v[p - 1] : (in << 16);
            v[p] = __viaddmax_s16x2(diag(prev, v[p]), sq[e], 0u);
          }
          rmax = __vimax3_s16x2(rmax, v[q * 4], v[q * 4 + 1]);
          rmax = __vimax3_s16x2(rmax, v[q * 4 + 2], v[q * 4 + 3]);
        }
        if (lane == 0 && !first) cprev = (cin >> (8 * (i & 3))) & 0xffu;
        if (!last_tile) {
          const uint32_t b = min(v[kTileC / 2 - 1] >> 16, 255u);   // this row's last node (>= 0 here)
          cout |= b << (8 * (i & 3));
          if (lane == 31 && ((i & 3) == 3 || i + 1 == len)) {
            __stcg(reinterpret_cast<uint32_t *>(col) + (i >> 2), cout);
          }
          if ((i & 3) == 3) cout = 0;
        }
      }
    }
    // R over the sequence: the largest half of any lane.
    int R = 0;
    if (active) {
      const int m = max((int)(int16_t)(rmax & 0xffffu), (int)(int16_t)(rmax >> 16));
      R = m;
    }
    R = __reduce_max_sync(kAll, R);
    if (active && lane == 0) {
      const int t = qd.tjb ? (int)__ldg(qd.tjb + min(len, qd.n_tjb - 1u)) : qd.tjb_fixed;
      const int raw = min(R, 255);
      const int flag = R >= 255 ? 1 : 0;
      qd.raw[orig] = (uint8_t)raw;
      qd.flag[orig] = (uint8_t)flag;
      if (qd.nat)
        qd.nat[orig] = flag ? __int_as_float(0x7f800000)
                            : __fsub_rn(__fdiv_rn(__int2float_rn(raw - qd.tbm - qd.tec - 2 * t), qd.scale), 3.0f);
    }
  }
}

}  // namespace

KernelFn tile_ssv_kernel_fn() { return tile_ssv_kernel; }

}  // namespace mpf
