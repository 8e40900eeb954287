// mpf_scan_kernel.cuh -- the MSV / SSV scan kernel for sm_103a.
//
// One kernel serves the single-query scan and the batched scan: resident
// thread blocks pull work items (query, database shard) from a counter,
// stage the query's striped cost table in shared memory, and stream the
// shard's sequences through their warps.
//
// Parallel decomposition (the five tiers of Sec. 3.1, re-mapped to GB300):
//   tier 1  thread blocks on the 152 SMs pull work items;
//   tier 2  warps pull batches of 32 / LG consecutive length ranks of their
//           item's shard from a shared-memory counter and run them in lock
//           step (sequences are length-sorted and shards interleave the
//           ranks, so the lengths of a batch nearly agree and a block's
//           batches shrink as it drains -- this replaces the pre-built warp
//           data blocks of Sec. 3.2 and Alg. 1);
//   tier 3  a group of LG lanes holds one sequence's DP row, striped over the
//           group (Farrar layout: cell k = (2*lane + half) * H + word);
//   tier 4  32 / LG groups per warp score different sequences at once;
//   tier 5  every 32-bit register holds two 16-bit cells updated by one
//           DPX instruction (byte SIMD -- vaddus4 etc. of Alg. 2 -- is not a
//           native instruction on sm_103, the 16x2 DPX forms are).
//
// Cell arithmetic.  With s = bias - cost (a signed score) and b = min(xB,
// 255 - bias), the byte update of Alg. 2 is exactly
//     dp = max(0, max(dp'[k-1], b) + s)
// because every dp' of a row that did not overflow is below 255 - bias, so
// clamping xB reproduces the saturating bias addition.  The SSV update of
// Alg. 7 is r = max(0, r'[k-1] + s) kept unsaturated in 16 bits; R >= 255 is
// the overflow and R is capped at the end.  MSV_FAST keeps v = max(0, dp - b),
// which follows the SSV recurrence while b is constant; b only changes when
// xJ passes base, so each lane keeps a running maximum and the group reduces
// it (Alg. 6) only on rows where some lane crosses the threshold at which xJ
// would pass base or the score would overflow.  After the first such row
// the group reduces every row (exact mode) until the sequence ends.  A row
// can raise the running maximum by at most `bias`, so a warp runs four rows
// without any per-row test whenever no lane is within 4 * bias of T.
//
// The F16 modes hold the same integers as IEEE half values and update a cell
// pair with one fused add-and-clamp-at-zero (HFMA2.RELU, v * 1 + s), which
// issues on the FMA pipe instead of the integer ALU pipe that the DPX
// instructions use.  Every value a scored cell takes before its sequence
// has reached the overflow threshold is an integer of magnitude below 2048,
// which half precision represents exactly; later values only need to stay
// above the threshold, and rounding is monotone.  Running maxima compare the
// half bit patterns of non-negative values as unsigned integers.
//
// Tensor-memory variant (TM, one sequence per warp, LG = 32).  The table is
// staged in shared memory as usual; then the first HT words of each lane's
// row (all H up to 14 words, else 12) of all 33 residue rows are copied into
// the block's tensor memory (thread t of warp w owns TMEM lane 32 (w mod 4) +
// t: its row of code x is columns x * HT .. x * HT + HT - 1).  The TMEM loads
// of a row are issued while the previous row is computed; the row then
// updates its words past HT from shared memory and its first HT words from
// the loaded registers.  Every row takes the same path, so the kernel has no
// per-row branch on the table source.  The cell arithmetic is unchanged.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include <type_traits>

#include "mpf_internal.h"
#include "mpf_tmem.cuh"

namespace mpf {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ int half_max(uint32_t w) {  // both halves are >= 0
  return max((int)(w & 0xffffu), (int)(w >> 16));
}

__device__ __forceinline__ uint32_t pack2(int v) {
  const uint32_t h = (uint32_t)(uint16_t)(int16_t)v;
  return (h << 16) | h;
}

__device__ __forceinline__ int sat8(int v) { return min(255, max(0, v)); }

// PTX prmt in its default mode: each selector nibble picks one of the eight
// bytes of (a, b) with its low three bits, and with its high bit set copies
// that byte's sign bit into all eight bits (the CUDA __byte_perm intrinsic
// uses only the low three bits).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}

template <int LG>
__device__ __forceinline__ int group_max(int v) {
#pragma unroll
  for (int off = LG / 2; off >= 1; off >>= 1) v = max(v, __shfl_xor_sync(kFull, v, off, LG));
  return v;
}

__device__ __forceinline__ float nat_score(int num, float scale) {
  return __fsub_rn(__fdiv_rn(__int2float_rn(num), scale), 3.0f);
}

// Order-preserving key of a cell value: the integer itself, or the bit
// pattern of a non-negative half.
template <bool F16>
__device__ __forceinline__ int value_key(int v) {
  if (!F16) return v;
  return (int)__half_as_ushort(__int2half_rn(v));
}

template <bool F16>
__device__ __forceinline__ int key_value(int k) {
  if (!F16) return k;
  if (k >= 0x7c00) return 1 << 20;   // +inf: far above every threshold
  return __half2int_rn(__ushort_as_half((unsigned short)k));
}

__device__ __forceinline__ uint32_t hfma2_relu_u32(uint32_t a, uint32_t b, uint32_t c) {
  const __half2 r = __hfma2_relu(*reinterpret_cast<const __half2 *>(&a),
                                 *reinterpret_cast<const __half2 *>(&b),
                                 *reinterpret_cast<const __half2 *>(&c));
  return *reinterpret_cast<const uint32_t *>(&r);
}

__device__ __forceinline__ uint32_t pack2_half(int v) {
  const uint32_t h = (uint32_t)__half_as_ushort(__int2half_rn(v));
  return (h << 16) | h;
}

template <int LG, int H, int MODE, bool TM = false, int QP = 1>
__global__ void __launch_bounds__(kBlockThreads, 1) scan_kernel(ScanParams p) {
  static_assert((H % 4 == 0 || H % 4 == 2) && H >= 4 && H <= kMaxWords, "words per lane");
  static_assert(!TM || ((LG == 32 || QP * LG == 32) && H >= kTmMinWords && MODE != MODE_MSV_DIRECT),
                "tensor-memory variant");
  static_assert(QP == 1 || (TM && QP * LG == 32), "queries per warp");
  constexpr int HT = TM ? tm_words(H) : 0;   // words per lane from TMEM
  static_assert(HT == H || HT % 4 == 0, "shared-memory words start on a chunk");
  constexpr int Q = H / 4;               // full 4-word chunks per lane and row
  constexpr bool kTail = (H % 4) == 2;   // two more words from the tail region
  constexpr int NT = LG >= 16 ? 1 : 16 / LG;
  static_assert(LG == 1 || LG == 2 || LG == 4 || LG == 8 || LG == 16 || LG == 32, "lanes");
  constexpr int NC = LG >= 8 ? 1 : 8 / LG;
  constexpr int G = 32 / LG;
  constexpr bool kF16 = (MODE == MODE_SSV_F16 || MODE == MODE_MSV_FAST_F16 || MODE == MODE_MSV_HELD_F16);
  static_assert(QP == 1 || !kF16, "packed sets use integer cells");
  constexpr bool kSSV = (MODE == MODE_SSV || MODE == MODE_SSV_F16);
  constexpr bool kFast = (MODE == MODE_MSV_FAST || MODE == MODE_MSV_FAST_F16);
  constexpr bool kBoth = (MODE == MODE_MSV_SSV);   // held MSV and SSV outputs from one sweep
  constexpr bool kHeld = (MODE == MODE_MSV_HELD || MODE == MODE_MSV_HELD_F16 || kBoth);
  constexpr bool kDirect = (MODE == MODE_MSV_DIRECT);
  const uint32_t one2 = 0x3c003c00u;   // (1.0, 1.0) as half2
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_item, s_next;
  __shared__ uint32_t s_tmem;

  const int lane = threadIdx.x & 31;
  const int gl = lane & (LG - 1);
  const int grp = lane / LG;
  // Byte selector of the diagonal shift: bytes 2, 3 of the lane before's last
  // word, then bytes 0, 1 of this lane's.  With integer cells (0 .. 32767)
  // the group's first lane takes the sign copies of its own byte 1, which
  // are zero; fp16 cells zero it with a select instead.
  const uint32_t shift_sel = (LG > 1 && gl != 0) ? 0x5432u : 0x54ddu;
  // QP > 1: the 32 / LG groups of a warp score one sequence against QP
  // queries (the QP consecutive queries of a work item), so every lane of
  // the warp reads the same residue and the TMEM column of a row is uniform.
  const uint32_t n_items = (p.n_queries + QP - 1) / QP * p.n_shards;
  const int warp = (int)(threadIdx.x >> 5);
  uint32_t tm_lane = 0;   // TMEM address of this warp's lane quarter, column 0
  if constexpr (TM) {
    if (warp == 0) tm_alloc(&s_tmem);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    tm_lane = s_tmem + ((uint32_t)((warp & 3) * 32) << 16);
  }

  for (;;) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(p.item_counter, 1u);
      s_next = 0u;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= n_items) break;
    const uint32_t shard = item % p.n_shards;
    const uint32_t qbase = item / p.n_shards * QP;
    const uint32_t qi = qbase + (QP > 1 ? (uint32_t)grp : 0u);
    // QP > 1: a set may have empty slots (descriptors without a table, after
    // its queries), and the last item fewer queries.
    const bool qvalid = qi < p.n_queries && (QP == 1 || p.queries[qi].table != nullptr);
    const QueryDesc *qd = p.queries + (qvalid ? qi : qbase);
    const uint32_t tstride = QP > 1 ? p.qp_table_stride : 0u;   // shared-memory bytes per query's table
    // Debug builds: the table must fit the block's shared memory and the
    // selected ranks the database (the item is skipped otherwise).
    if (!MPF_DCHECK(p.status, (QP > 1 ? qd->table_bytes <= tstride && tstride % 16 == 0 &&
                                            QP * tstride <= dynamic_smem_bytes() && !qd->ranks
                                      : qd->table_bytes <= dynamic_smem_bytes()) &&
                                  p.pad_word < p.n_words && (!qd->ranks || *qd->n_ranks <= p.n_seqs))) {
      __syncthreads();
      continue;
    }
    // A shard without sequences (a short rank list, such as the few
    // sequences a held MSV pass leaves for rescoring) stages nothing.
    if ((uint64_t)shard >= (qd->ranks ? (uint64_t)*qd->n_ranks : (uint64_t)p.n_seqs)) {
      __syncthreads();
      continue;
    }

    // Stage the striped table(s) (16-byte vector copies, coalesced); with
    // QP > 1 query g's table at g * tstride.
#pragma unroll 1
    for (int g = 0; g < QP; ++g) {
      if (qbase + (uint32_t)g >= p.n_queries) break;
      const QueryDesc *qg = p.queries + qbase + g;
      if (!qg->table) continue;
      const uint32_t nvec = qg->table_bytes >> 4;
      const uint4 *src = qg->table;
      uint4 *dst = reinterpret_cast<uint4 *>(smem + (uint32_t)g * tstride);
      for (uint32_t i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    // A group past the last query computes on the first query's table and
    // writes nothing (its lanes must still follow the warp's sequence).
    const uint8_t *tbl_base = smem + (QP > 1 && qvalid ? (uint32_t)grp * tstride : 0u);
    const uint8_t *tbl_lane = tbl_base + (QP > 1 ? 0u : (grp % NC) * qd->copy_bytes) + gl * 16;
    // QP > 1: packed tables (one copy of each region; the table stride
    // spreads the groups of a phase over the banks).
    const uint8_t *tail_lane = tbl_base + qd->tail_off + ((QP > 1 ? 0 : grp % NT) * LG + gl) * 8;
    if constexpr (TM) {
      // Copy the first HT words of every lane's row of every code from the
      // staged table into tensor memory: warp q < 4 writes lane quarter q.
      tm_fence_after();
      if (warp < 4) {
        for (uint32_t x = 0; x < (uint32_t)kTableRows; ++x) {
          const uint32_t col = tm_lane + x * (uint32_t)HT;
#pragma unroll
          for (int j = 0; j < HT / 4; ++j) {
            const uint4 s4 = *reinterpret_cast<const uint4 *>(tbl_lane + x * qd->row_bytes + j * LG * 16);
            tm_st4(col + 4 * j, s4.x, s4.y, s4.z, s4.w);
          }
          if constexpr (HT % 4 == 2) {   // HT == H: the two tail words
            const uint2 t2 = *reinterpret_cast<const uint2 *>(tail_lane + x * qd->tail_row_bytes);
            tm_st2(col + 4 * (HT / 4), t2.x, t2.y);
          }
        }
        tm_wait_st();
      }
      tm_fence_before();
      __syncthreads();
      tm_fence_after();
    }

    const int bias = qd->bias, tbm = qd->tbm, tec = qd->tec, base = qd->base;
    const int cap = 255 - bias;
    const float scale = qd->scale;
    const uint8_t *tjb = qd->tjb;
    const uint32_t n_tjb = qd->n_tjb;
    const int tjb_fixed = qd->tjb_fixed;
    uint8_t *out_raw = qd->raw;
    uint8_t *out_flag = qd->flag;
    float *out_nat = qd->nat;
    const uint32_t row_bytes = qd->row_bytes;
    const uint32_t tail_row_bytes = qd->tail_row_bytes;
    const int16_t *smax = reinterpret_cast<const int16_t *>(tbl_base + qd->smax_off);
    const uint32_t *ranks = qd->ranks;
    const uint64_t n_sel = ranks ? (uint64_t)*qd->n_ranks : (uint64_t)p.n_seqs;

    for (;;) {
      // ---- take G consecutive length ranks of this shard (one per group;
      // QP > 1: one rank, the same sequence for every group) ----
      uint32_t k0 = 0;
      if (lane == 0) k0 = atomicAdd(&s_next, QP > 1 ? 1u : (uint32_t)G);
      k0 = __shfl_sync(kFull, k0, 0);
      const uint64_t kr = (uint64_t)shard + (uint64_t)(k0 + (QP > 1 ? 0 : grp)) * p.n_shards;
      bool active = kr < n_sel;
      if (!__any_sync(kFull, active)) break;
      const uint64_t r = (ranks && active) ? (uint64_t)__ldg(ranks + kr) : kr;
      if (active && !MPF_DCHECK(p.status, r < p.n_seqs)) active = false;

      // Group state (identical in every lane of a group).
      uint32_t wptr = p.pad_word, orig = 0;
      int len = 0, t = 0;
      if (active) {
        wptr = __ldg(p.seq_word + r);
        len = (int)__ldg(p.seq_len + r);
        orig = __ldg(p.seq_orig + r);
        t = tjb ? (int)__ldg(tjb + min((uint32_t)len, n_tjb - 1u)) : tjb_fixed;
        if (!MPF_DCHECK(p.status, (uint64_t)wptr + (uint64_t)((len + 3) >> 2) <= p.n_words &&
                                      orig < p.n_seqs)) {
          active = false;
          wptr = p.pad_word;
          len = 0;
        }
      }
      const uint32_t wstart = wptr;
      const int nsteps = (len + 3) >> 2;           // residue words of this sequence
      const int wsteps = (int)__reduce_max_sync(kFull, (uint32_t)nsteps);
      int xJ = 0;
      int b = min(sat8(base - (t + tbm)), cap);
      uint32_t b2 = pack2(b);
      const int T = min(base + tec - b, cap - b - 1);
      const int Tk = value_key<kF16>(max(T, 0));          // threshold as a key
      const int Tnear = T - 4 * max(bias, 0);              // no trigger possible in 4 rows below it
      const int Tnear_k = value_key<kF16>(max(Tnear, 0));
      // "Some half of the running maximum is above the key K" as one add and
      // one mask: the halves (keys <= 0x7fff) plus 0x7fff - K reach bit 15
      // exactly when they exceed K, and no sum carries into the other half.
      const uint32_t Tk2 = pack2(0x7fff - Tk), Tnear2 = pack2(0x7fff - Tnear_k);
      bool done = false, exact = false;

      // Lane state: H words of two 16-bit cells and a running maximum (key).
      uint32_t v[H];
#pragma unroll
      for (int q = 0; q < H; ++q) v[q] = 0u;
      uint32_t vacc = 0u;
      uint32_t cur = __ldg(p.residues + (nsteps > 0 ? wptr : p.pad_word));

      // Tensor-memory words of the current and the next row: the loads of
      // row i + 1 are issued while row i is computed.  Every residue code,
      // the padding code included, has a TMEM row (code x: columns x * HT ..).
      // Whole-warp kernels of up to 16 words per lane: one 16-column load per
      // row (tcgen05.ld .x16, one uniform address) in place of two or three
      // narrower ones; the columns past a code's HT words belong to the next
      // code (or lie past the 33 codes, inside the allocation) and are not
      // used.  Measured per row of M = 600-1000: 3.5-8.5% faster; from 22
      // words on, where a row has more work to hide the loads behind, the
      // exact-width loads were up to 2% faster.  Packed kernels load HT
      // columns (their group state leaves no registers for wider buffers).
      constexpr int HL = TM ? ((QP == 1 && H <= 16) ? 16 : HT) : 1;
      static_assert(!TM || (HT <= 16 && (kTableRows - 1) * HT + 16 <= (int)kTmemColumns), "load width");
      uint32_t TA[HL], TB[HL];
      auto tm_col = [&](uint32_t xc) -> uint32_t {
        if (!MPF_DCHECK(p.status, xc < (uint32_t)kTableRows)) xc = kPadCode;
        return tm_lane + xc * (uint32_t)HT;
      };
      if constexpr (TM) tm_ld<HL>(TA, tm_col(cur & 0xffu));   // first row of the sequence

      // Four rows of one residue word (nxt: the next word).  CHECK: test every
      // row for the MSV threshold (only needed when some lane is near it, or
      // in exact mode).
      auto four_rows = [&](const int step, auto check_tag, const uint32_t nxt) {
        constexpr bool CHECK = decltype(check_tag)::value;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
         auto one_row = [&](auto &Tc, auto &Tn) {
          // Rows past the end of a sequence read padding codes: their cells
          // score kNegInf, and the special states must not see them.
          const bool real = active && (4 * step + rr) < len;
          uint32_t x = __byte_perm(cur, 0u, 0x4440u + rr);   // residue code of row rr
          if (!MPF_DCHECK(p.status, x < (uint32_t)kTableRows)) x = kPadCode;
          if constexpr (TM) {
            // This row's TMEM words (issued one row earlier), then the next
            // row's loads: a wait covers every earlier load of the thread.
            tm_wait_ld<HL>(Tc);
            tm_ld<HL>(Tn, tm_col(rr < 3 ? __byte_perm(cur, 0u, 0x4440u + rr + 1) : nxt & 0xffu));
          }
          const uint8_t *rowp = tbl_lane + x * row_bytes;
          // Diagonal shift (Alg. 5): cell k-1 of the previous row feeds cell k.
          const uint32_t wl = v[H - 1];
          uint32_t up = 0u;
          if (LG > 1) {
            up = __shfl_up_sync(kFull, wl, 1, LG);
            if (kF16 && gl == 0) up = 0u;
          }
          // Cell k - 1 of the previous row: the lane before's last cell and
          // this lane's high-half cell of the last word.  The group's first
          // lane takes zero instead, as sign copies of a non-negative cell.
          const uint32_t mpv = prmt(up, wl, kF16 ? 0x5432u : shift_sel);
          uint32_t rmax = 0u;
          // Update word q from the previous row's word q - 1 and score word sc.
          auto cell = [&](const int q, const uint32_t sc) {
            const uint32_t prev = (q == 0) ? mpv : v[q - 1];
            if (kF16)
              v[q] = hfma2_relu_u32(prev, one2, sc);
            else if (kDirect)
              v[q] = __viaddmax_s16x2(__vimax_s16x2_relu(prev, b2), sc, 0u);
            else
              v[q] = __viaddmax_s16x2(prev, sc, 0u);
          };
          // Fold words q + 1 and q into the row / running maximum.
          auto fold = [&](const int q) {
            if (kDirect)
              rmax = __vimax3_u16x2(rmax, v[q + 1], v[q]);
            else
              vacc = __vimax3_u16x2(vacc, v[q + 1], v[q]);
          };
          // Words from shared memory, highest first (in-place update): the
          // two-word tail, then the 4-word chunks down to chunk j_lo.
          auto smem_words = [&](const int j_lo) {
            if (kTail) {   // words 4Q+1 and 4Q
              const uint2 t2 = *reinterpret_cast<const uint2 *>(tail_lane + x * tail_row_bytes);
              cell(4 * Q + 1, t2.y);
              cell(4 * Q, t2.x);
              fold(4 * Q);
            }
#pragma unroll
            for (int j = Q - 1; j >= j_lo; --j) {
              const uint4 s4 = *reinterpret_cast<const uint4 *>(rowp + j * LG * 16);
              cell(4 * j + 3, s4.w);
              cell(4 * j + 2, s4.z);
              cell(4 * j + 1, s4.y);
              cell(4 * j, s4.x);
              fold(4 * j + 2);
              fold(4 * j);
            }
          };
          if constexpr (TM) {
            if constexpr (HT < H) smem_words(HT / 4);
#pragma unroll
            for (int q = HT - 1; q >= 1; q -= 2) {
              cell(q, Tc[q]);
              cell(q - 1, Tc[q - 1]);
              fold(q - 1);
            }
          } else {
            smem_words(0);
          }
          if (kDirect) {
            // xE of this row (Alg. 6), then the J and B special states.
            const int xE = group_max<LG>(half_max(rmax));
            if (real && !done) {
              if (xE >= cap) {
                done = true;
              } else {
                xJ = max(xJ, xE - tec);
                b = min(sat8(max(base, xJ) - (t + tbm)), cap);
                b2 = pack2(b);
              }
            }
          } else if (kFast && CHECK) {
            const bool trig = real && !done && (exact || ((vacc + Tk2) & 0x80008000u) != 0u);
            if (__any_sync(kFull, trig)) {
              const int mm = key_value<kF16>(group_max<LG>(half_max(vacc)));
              if (real && !done && (exact || mm > T)) {
                const int xE = b + mm;
                if (xE >= cap) {
                  done = true;
                } else {
                  xJ = exact ? max(xJ, xE - tec) : max(0, xE - tec);
                  const int bn = min(sat8(max(base, xJ) - (t + tbm)), cap);
                  if (bn > b) {
#pragma unroll
                    for (int q = 0; q < H; ++q)
                      v[q] = kF16 ? hfma2_relu_u32(v[q], one2, pack2_half(b - bn))
                                  : __viaddmax_s16x2(v[q], pack2(b - bn), 0u);
                  }
                  b = bn;
                  exact = true;
                }
              }
              if (exact) vacc = 0u;
            }
          }
         };
          if (rr & 1)
            one_row(TB, TA);
          else
            one_row(TA, TB);
        }
      };

      for (int step = 0; step < wsteps; ++step) {
        // Prefetch the next residue word; past the end a group reads padding.
        const uint32_t nxt = __ldg(p.residues + (step + 1 < nsteps ? wptr + (uint32_t)step + 1u : p.pad_word));
        if (kFast) {
          const bool near = active && !done && (exact || Tnear < 0 || ((vacc + Tnear2) & 0x80008000u) != 0u);
          if (__any_sync(kFull, near))
            four_rows(step, std::true_type{}, nxt);
          else
            four_rows(step, std::false_type{}, nxt);
        } else {
          four_rows(step, std::false_type{}, nxt);
        }
        cur = nxt;
      }

      if constexpr (TM) tm_wait_ld<HL>(TA);   // the load issued after the last row

      // ---- finalise the G sequences -------------------------------------
      const bool own = active && qvalid;   // this group writes its sequence's outputs
      const int V = key_value<kF16>(group_max<LG>(half_max(vacc)));
      if (kFast || kHeld) {
        // A sequence whose cells never rose above the begin score: its best
        // row maximum is the best single-cell score of its residues.
        const bool rescue = active && !done && !exact && V == 0 && len > 0;
        int g = INT_MIN / 2;
        if (rescue) {
          for (int w = gl; w < nsteps; w += LG) {
            const uint32_t word = __ldg(p.residues + wstart + (uint32_t)w);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (4 * w + i < len && MPF_DCHECK(p.status, ((word >> (8 * i)) & 0xffu) < (uint32_t)kTableRows))
                g = max(g, (int)smax[(word >> (8 * i)) & 0xffu]);
          }
        }
        g = group_max<LG>(g);
        if (kBoth && own && gl == 0) {
          // SSV (Alg. 7) from the same largest cell: with b held the MSV
          // cells minus b are exactly the SSV cells.
          const bool ovf = V >= 255;
          const int raw = ovf ? 255 : V;
          qd->raw2[orig] = (uint8_t)raw;
          qd->flag2[orig] = ovf ? 1 : 0;
          if (qd->nat2) qd->nat2[orig] = ovf ? __int_as_float(0x7f800000) : nat_score(raw - tbm - tec - 2 * t, scale);
        }
        if (kHeld && own && gl == 0) {
          // The begin score b was held for every row.  V, the largest cell
          // of any row, decides: at or above 255 - bias - b some row
          // overflowed (with b held or after it rose, cells only grow);
          // at most T no row could move xJ past base, so the held rows are
          // exact; in between xB would have moved: an exact kernel rescores
          // the sequence.
          if (V >= cap - b) {
            out_raw[orig] = 255;
            out_flag[orig] = 1;
            if (out_nat) out_nat[orig] = __int_as_float(0x7f800000);
          } else if (V > T) {
            const uint32_t slot = atomicAdd(qd->fallback_count, 1u);
            if (MPF_DCHECK(p.status, slot < p.n_seqs)) qd->fallback_ranks[slot] = (uint32_t)r;
          } else {
            const int G2 = V > 0 ? V : g;
            const int raw = len > 0 ? max(0, b + G2 - tec) : 0;
            out_raw[orig] = (uint8_t)raw;
            out_flag[orig] = 0;
            if (out_nat) out_nat[orig] = nat_score(raw - t - base, scale);
          }
        }
        if (kFast && own && gl == 0) {
          int raw;
          uint8_t flag = 0;
          if (done) {
            raw = 255;
            flag = 1;
          } else if (exact) {
            raw = xJ;
          } else {
            const int G2 = V > 0 ? V : g;
            raw = len > 0 ? max(0, b + G2 - tec) : 0;
          }
          out_raw[orig] = (uint8_t)raw;
          out_flag[orig] = flag;
          if (out_nat) out_nat[orig] = flag ? __int_as_float(0x7f800000) : nat_score(raw - t - base, scale);
        }
      } else if (kDirect) {
        if (own && gl == 0) {
          const int raw = done ? 255 : xJ;
          out_raw[orig] = (uint8_t)raw;
          out_flag[orig] = done ? 1 : 0;
          if (out_nat) out_nat[orig] = done ? __int_as_float(0x7f800000) : nat_score(raw - t - base, scale);
        }
      } else {  // SSV
        if (own && gl == 0) {
          const bool ovf = V >= 255;
          const int raw = ovf ? 255 : V;
          out_raw[orig] = (uint8_t)raw;
          out_flag[orig] = ovf ? 1 : 0;
          if (out_nat) out_nat[orig] = ovf ? __int_as_float(0x7f800000) : nat_score(raw - tbm - tec - 2 * t, scale);
        }
      }
    }
    if constexpr (TM) tm_fence_before();   // this item's TMEM reads before the next item's writes
    __syncthreads();
  }
  if constexpr (TM) {
    if (warp == 0) {
      tm_fence_after();
      tm_dealloc(s_tmem);
    }
  }
}

}  // namespace mpf
