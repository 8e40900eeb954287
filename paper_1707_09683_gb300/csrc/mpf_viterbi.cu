// mpf_viterbi.cu -- the P7Viterbi filter (Eq. 1 of Sec. 2.1) for sm_103a.
//
// One warp scores one sequence against one query, in the 16-bit saturating
// word arithmetic of the Viterbi filter carried in 32-bit registers.  Lane l
// owns a contiguous segment of Q = ceil(M/32) nodes (Farrar's striped order:
// node l*Q + j sits in slot j*32 + l, so every shared access of a warp is one
// contiguous line).  Per DP row each lane sweeps its segment once:
//   * the diagonal terms of Eq. 1 (node k-1 of the previous row) come from
//     the lane's previous node, or for a segment's first node from the last
//     node of the lane before (one shuffle per row);
//   * the insert term uses the same node of the previous row;
//   * the delete chain D[k] = max(M[k-1] + tMD, D[k-1] + tDD) runs along the
//     row.  Each lane computes a segment-local chain that assumes minus
//     infinity enters the segment; each segment is a map d -> max(A,
//     min(d + B, C)) of the delete score entering it, these maps compose, and
//     a 5-step warp scan gives the true delete score entering every segment.
//     The next row completes the previous row's chain on the fly (D' =
//     max(local D', carried chain)), so no second pass is needed;
//   * E is a warp maximum, then the N, C, J, B special states are scalar.
//
// viterbi_fast_kernel takes profiles whose transition and special scores are
// all <= 0 (any profile of log-probabilities).  Then no sum can pass the
// upper bound except M[k] itself, whose saturation at 32767 is the overflow,
// so every sat() reduces to max(., -32768), a chain of them to one DPX
// add-then-max per term, the maps lose their cap (C), and D[k] <= max of the
// M of earlier nodes, so E is the maximum of M alone.
//
// viterbi_general_kernel takes any int16 scores: every sum is clamped on
// both sides, the maps keep their cap, -32768 is a number that positive moves
// can raise (so the carried chain of the row before the first starts at true
// minus infinity, not at -32768, and D_1 = -32768 re-enters every row), and
// E also takes the true delete scores: the local chain's maximum and the
// carried chain's, whose maximum over a segment is its entry value plus the
// largest prefix sum of tDD there (once a cap binds the row has overflowed).
//
// The transition table is staged once per query into shared memory and read
// by all warps of a block; match scores are read from global memory in the
// same striped order.  Models longer than 3,072 nodes take the same kernels
// with their DP rows in device memory (GM, below).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <array>

#include "mpf_internal.h"

namespace mpf {

namespace {

constexpr uint32_t kAll = 0xffffffffu;

// ------------------------------------------------------------ fast kernel

constexpr int kNeg = -32768;

__device__ __forceinline__ int lo16(uint32_t w) { return (int)(int16_t)(w & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t w) { return ((int)w) >> 16; }
// max(a + b, c), one DPX instruction.
__device__ __forceinline__ int addmax(int a, int b, int c) { return __viaddmax_s32(a, b, c); }

// Where a kernel keeps its tables and DP rows.  Models that fit (GM =
// false): the query's transitions staged into shared memory, read by every
// warp of the block, and each warp's M, I, D rows in shared memory.  Longer
// models (GM = true): transitions read through the L1 from device memory,
// and each warp's rows in its slice of a device scratch buffer as one 8-byte
// record per node (M | I, D), at slot j*32 + lane like the shared rows, so a
// warp's access is 256 contiguous bytes (4-byte records M | I in the fast
// kernel's variant without the stored D row); the rows are read and written
// at the L2 (ld/st.global.cg), which keeps the L1 for the tables.
template <bool GM>
__device__ __forceinline__ void stage_transitions(uint4 *tr, const uint4 *gtr, int nq) {
  if (GM) return;
  __syncthreads();   // every warp is done with the previous query's table
  for (int i = threadIdx.x; i < nq * 32; i += blockDim.x) tr[i] = __ldg(gtr + i);
  __syncthreads();
}

template <bool GM>
struct TransSrc {
  const uint4 *s, *g;
  __device__ __forceinline__ uint4 operator[](int i) const { return GM ? __ldg(g + i) : s[i]; }
};

// This warp's records in the device scratch (GM), or nullptr (also when the
// scratch is too small: debug builds report it).
template <bool GM>
__device__ __forceinline__ uint2 *warp_rows(const VitParams &p, int Qmax, int warp) {
  if (!GM) return nullptr;
  const uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (uint64_t)warp;
  const uint64_t per = (uint64_t)Qmax * 32;
  if (!MPF_DCHECK(p.status, p.state && (w + 1) * per * sizeof(uint2) <= p.state_bytes)) return nullptr;
  return p.state + w * per;
}

__device__ __forceinline__ void load_rows(const uint2 *g, int sl, int &Mo, int &Io, int &Dl) {
  const uint2 r = __ldcg(g + sl);
  Mo = (int)(int16_t)(r.x & 0xffffu);
  Io = ((int)r.x) >> 16;
  Dl = (int)r.y;
}

__device__ __forceinline__ void store_rows(uint2 *g, int sl, int Mn, int In, int d) {
  __stcg(g + sl, make_uint2(__byte_perm((uint32_t)Mn, (uint32_t)In, 0x5410), (uint32_t)d));
}

// Whether a launch scores query Q: the team kernel takes it when it selects
// at most Q.team_max sequences (a count the host may not know: rank lists
// are counted on the device), the one-warp kernels otherwise.
__device__ __forceinline__ bool takes_query(const VitQuery &Q, uint32_t n_seqs, bool team) {
  const int64_t n = Q.ranks ? (int64_t)*Q.n_ranks : (int64_t)n_seqs;
  return team ? n <= Q.team_max : n > Q.team_max;
}

// One node of a lane's sweep (fast kernel): the previous row's M, I and
// segment-local D of this node arrive in Mo, Io, Dl; the node's new M, I and
// local D leave in Mn, In, d.  dM, dI, dD hold the previous row's values of
// the node before (true D), X the carried delete chain, mprev this row's M of
// the node before.
struct FastCell {
  int dM, dI, dD, X, mprev, d, mx, Mn, In;
  int mop, Dlp;   // recomputed previous-row chain: M' of the node before (in the segment), local D'
  __device__ __forceinline__ void step(const uint4 t, int e, int Mo, int Io, int Dl, int xB) {
    const int tDD = hi16(t.w);
    X += tDD;
    const int Do = max(Dl, X);
    cell(t, tDD, e, Mo, Io, Do, xB);
  }
  // The same node when the previous row's local delete chain is not stored:
  // it is recomputed here from the previous row's M (2 DPX operations).
  __device__ __forceinline__ void step_nd(const uint4 t, int e, int Mo, int Io, int xB) {
    const int tDD = hi16(t.w);
    X += tDD;
    Dlp = addmax(Dlp, tDD, addmax(mop, lo16(t.w), kNeg));
    mop = Mo;
    const int Do = max(Dlp, X);
    cell(t, tDD, e, Mo, Io, Do, xB);
  }
  __device__ __forceinline__ void cell(const uint4 t, int tDD, int e, int Mo, int Io, int Do, int xB) {
    int best = addmax(dM, hi16(t.x), kNeg);      // M' + tMM
    best = addmax(dI, lo16(t.y), best);           // I' + tIM
    best = addmax(dD, hi16(t.y), best);           // D' + tDM
    best = addmax(xB, lo16(t.x), best);           // xB + tBM
    Mn = addmax(best, e, kNeg);
    In = addmax(Io, hi16(t.z), addmax(Mo, lo16(t.z), kNeg));
    d = addmax(d, tDD, addmax(mprev, lo16(t.w), kNeg));
    mx = max(mx, Mn);
    dM = Mo;
    dI = Io;
    dD = Do;
    mprev = Mn;
  }
};

// Shared memory: the query's transitions, Qmax*32 uint4 (8 int16 per node:
// BM|MM, IM|DM, MI|II, MD|DD), then per warp three arrays of Qmax*32 int16
// (M, I, D), slot j*32 + lane (sign-extending 16-bit loads, no unpacking).
// With ND the D array is not kept: the next row recomputes the local delete
// chain from the stored M row (4 bytes of state per node instead of 6, two
// more DPX operations per node), so more warps fit on long models.  U is the
// unroll depth of the node loop.
template <int U, bool ND, bool GM>
__global__ void __launch_bounds__(kVitFastMaxThreads, 1) viterbi_fast_kernel(VitParams p) {
  extern __shared__ __align__(16) uint4 fsm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int Qmax = p.max_Mpad >> 5;
  uint4 *tr = fsm;
  int16_t *sM = reinterpret_cast<int16_t *>(fsm + (size_t)Qmax * 32) + (size_t)warp * Qmax * 32 * (ND ? 2 : 3);
  int16_t *sI = sM + (size_t)Qmax * 32;
  int16_t *sD = sI + (size_t)Qmax * 32;   // unused with ND
  uint2 *gst = warp_rows<GM>(p, Qmax, warp);
  uint32_t *gst32 = reinterpret_cast<uint32_t *>(gst);   // GM with ND: 4-byte records (M | I)
  // Debug builds: the transitions and the warps' DP rows must fit the block's
  // shared memory (or the rows the device scratch).
  if (!GM && !MPF_DCHECK(p.status, (size_t)Qmax * 32 * (16 + (blockDim.x >> 5) * (ND ? 4 : 6)) <= dynamic_smem_bytes()))
    return;
  if (GM && !gst) return;

  for (uint32_t qi = 0; qi < p.n_queries; ++qi) {
    const VitQuery Q = p.queries[qi];
    const int nq = Q.Mpad >> 5;
    if (!MPF_DCHECK(p.status, Q.Mpad <= p.max_Mpad && (!Q.ranks || *Q.n_ranks <= p.n_seqs))) continue;
    if (!takes_query(Q, p.n_seqs, false)) continue;
    const uint4 *gtr = reinterpret_cast<const uint4 *>(Q.trans);
    stage_transitions<GM>(tr, gtr, nq);
    const TransSrc<GM> T{tr, gtr};

    // Per-lane constants of the query.
    const int nv = min(max(Q.M - lane * nq, 0), nq);   // real nodes in this lane's segment
    int tMD0 = kNeg, tDD0 = 0, Bl = 0;
    if (nv > 0) {
      tMD0 = lo16(T[lane].w);
      tDD0 = hi16(T[lane].w);
    }
    for (int j = 0; j < nv; ++j) Bl += hi16(T[j * 32 + lane].w);
    const int Bsuf = Bl - tDD0;
    // Inclusive prefix over lanes, modulo 2^32: the whole model's sum of tDD
    // can pass the int32 range at 100,000 nodes, a window of 16 lanes cannot,
    // so the differences below are exact.
    uint32_t P = (uint32_t)Bl;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(kAll, P, off);
      if (lane >= off) P += y;
    }
    int Wn[5];    // sum of B over lanes (lane - 2^r, lane], or a sentinel
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const uint32_t y = __shfl_up_sync(kAll, P, 1 << r);
      Wn[r] = lane >= (1 << r) ? (int)(P - y) : -(1 << 29);
    }
    const int tNN = Q.sp[0], tNB = Q.sp[1], tEC = Q.sp[2], tCC = Q.sp[3];
    const int tCT = Q.sp[4], tEJ = Q.sp[5], tJJ = Q.sp[6], tJB = Q.sp[7];
    const uint64_t n_sel = Q.ranks ? (uint64_t)*Q.n_ranks : (uint64_t)p.n_seqs;

    for (;;) {
      uint32_t q = 0;
      if (lane == 0) q = atomicAdd(p.counters + qi, 1u);
      q = __shfl_sync(kAll, q, 0);
      if ((uint64_t)q >= n_sel) break;
      const uint32_t r = Q.ranks ? __ldg(Q.ranks + q) : q;
      if (!MPF_DCHECK(p.status, r < p.n_seqs)) continue;
      const uint32_t w0 = __ldg(p.seq_word + r);
      const int len = (int)__ldg(p.seq_len + r);
      const uint32_t orig = __ldg(p.seq_orig + r);
      if (!MPF_DCHECK(p.status, (uint64_t)w0 + (uint64_t)((len + 3) >> 2) <= p.n_words && orig < p.n_seqs))
        continue;

      for (int j = 0; j < nq; ++j) {
        if (GM && ND) {
          __stcg(gst32 + j * 32 + lane, __byte_perm((uint32_t)kNeg, (uint32_t)kNeg, 0x5410));
        } else if (GM) {
          store_rows(gst, j * 32 + lane, kNeg, kNeg, kNeg);
        } else {
          sM[j * 32 + lane] = sI[j * 32 + lane] = (int16_t)kNeg;
          if (!ND) sD[j * 32 + lane] = (int16_t)kNeg;
        }
      }
      int xN = Q.base, xJ = kNeg, xC = kNeg;
      int xB = addmax(xN, tNB, kNeg);
      // Previous row: M, I and true D of the node before the segment, and the
      // delete score carried into the segment (X0m + tDD of node 0 is its
      // value at node 0; row 0 carries minus infinity).
      int pM0 = kNeg, pI0 = kNeg, pD0 = kNeg, X0m = kNeg - tDD0;
      bool ovf = false;
      uint32_t word = 0;
      for (int i = 0; i < len; ++i) {
        if ((i & 3) == 0) word = __ldg(p.residues + w0 + (uint32_t)(i >> 2));
        int x = (int)((word >> (8 * (i & 3))) & 0xffu);
        if (!MPF_DCHECK(p.status, x < kVitRows)) x = 0;
        const int16_t *erow = Q.msc + (size_t)x * nq * 32 + lane;

        // Sweep the segment: the previous row's delete chain is completed on
        // the fly (D' = max(local D', carried chain)), then M, I and this
        // row's segment-local delete chain.
        FastCell c{pM0, pI0, pD0, X0m, kNeg, kNeg, kNeg, kNeg, kNeg, kNeg, kNeg};
#pragma unroll U
        for (int j = 0; j < nv; ++j) {
          const int sl = j * 32 + lane;
          if (GM && ND) {
            const uint32_t rr = __ldcg(gst32 + sl);
            c.step_nd(T[sl], __ldg(erow + j * 32), lo16(rr), hi16(rr), xB);
            __stcg(gst32 + sl, __byte_perm((uint32_t)c.Mn, (uint32_t)c.In, 0x5410));
          } else if (GM) {
            int Mo, Io, Dl;
            load_rows(gst, sl, Mo, Io, Dl);
            c.step(T[sl], __ldg(erow + j * 32), Mo, Io, Dl, xB);
            store_rows(gst, sl, c.Mn, c.In, c.d);
          } else if (ND) {
            c.step_nd(tr[sl], __ldg(erow + j * 32), sM[sl], sI[sl], xB);
            sM[sl] = (int16_t)c.Mn;
            sI[sl] = (int16_t)c.In;
          } else {
            c.step(tr[sl], __ldg(erow + j * 32), sM[sl], sI[sl], sD[sl], xB);
            sD[sl] = (int16_t)c.d;
            sM[sl] = (int16_t)c.Mn;
            sI[sl] = (int16_t)c.In;
          }
        }
        const int xE = __reduce_max_sync(kAll, c.mx);
        if (xE >= 32767) {
          ovf = true;
          break;
        }

        // True delete score at the end of every segment: inclusive scan of
        // the segments' maps d -> max(A, d + B).
        int Mlp = __shfl_up_sync(kAll, c.Mn, 1);
        int Ilp = __shfl_up_sync(kAll, c.In, 1);
        if (lane == 0) Mlp = Ilp = kNeg;
        int A = addmax(Mlp, tMD0 + Bsuf, c.d);
#pragma unroll
        for (int r = 0; r < 5; ++r) A = addmax(__shfl_up_sync(kAll, A, 1 << r), Wn[r], A);
        int carry = __shfl_up_sync(kAll, A, 1);
        if (lane == 0) carry = kNeg;
        pM0 = Mlp;
        pI0 = Ilp;
        pD0 = carry;
        X0m = max(carry + tDD0, Mlp + tMD0) - tDD0;

        xN = addmax(xN, tNN, kNeg);
        xC = addmax(xC, tCC, addmax(xE, tEC, kNeg));
        xJ = addmax(xJ, tJJ, addmax(xE, tEJ, kNeg));
        xB = addmax(xN, tNB, addmax(xJ, tJB, kNeg));
      }
      if (lane == 0) {
        if (ovf) {
          Q.score[orig] = 32767;
          Q.flag[orig] = 1;
          if (Q.nat) Q.nat[orig] = __int_as_float(0x7f800000);
        } else {
          const int sc = addmax(xC, tCT, kNeg);
          Q.score[orig] = (int16_t)sc;
          Q.flag[orig] = 0;
          if (Q.nat) Q.nat[orig] = __fsub_rn(__fdiv_rn(__int2float_rn(sc - Q.base), Q.scale), 3.0f);
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------- general kernel

constexpr int kPos = 32767;
constexpr int kMinusInf = -(1 << 29);   // true minus infinity in 32-bit registers

// sat(a + b), the 16-bit saturating add of the Viterbi filter.
__device__ __forceinline__ int satadd(int a, int b) { return max(__viaddmin_s32(a, b, kPos), kNeg); }

// Any int16 scores (see the file comment).  Shared memory as for the plain
// fast kernel: transitions, then per warp the M, I and segment-local D rows.
template <int U, bool GM>
__global__ void __launch_bounds__(kVitFastMaxThreads, 1) viterbi_general_kernel(VitParams p) {
  extern __shared__ __align__(16) uint4 fsm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int Qmax = p.max_Mpad >> 5;
  uint4 *tr = fsm;
  int16_t *sM = reinterpret_cast<int16_t *>(fsm + (size_t)Qmax * 32) + (size_t)warp * Qmax * 32 * 3;
  int16_t *sI = sM + (size_t)Qmax * 32;
  int16_t *sD = sI + (size_t)Qmax * 32;
  uint2 *gst = warp_rows<GM>(p, Qmax, warp);
  if (!GM && !MPF_DCHECK(p.status, (size_t)Qmax * 32 * (16 + (blockDim.x >> 5) * 6) <= dynamic_smem_bytes()))
    return;
  if (GM && !gst) return;

  for (uint32_t qi = 0; qi < p.n_queries; ++qi) {
    const VitQuery Q = p.queries[qi];
    const int nq = Q.Mpad >> 5;
    if (!MPF_DCHECK(p.status, Q.Mpad <= p.max_Mpad && (!Q.ranks || *Q.n_ranks <= p.n_seqs))) continue;
    if (!takes_query(Q, p.n_seqs, false)) continue;
    const uint4 *gtr = reinterpret_cast<const uint4 *>(Q.trans);
    stage_transitions<GM>(tr, gtr, nq);
    const TransSrc<GM> T{tr, gtr};

    // Per-lane constants: the segment's map of the delete score entering it
    // is d -> max(A, min(d + Bl, Cl)), built from tDD of the first node (t0)
    // and the composite (Bsuf, Csuf) of x -> min(x + tDD, 32767) over the
    // others; maxP is the largest prefix sum of those tDD (0 included).
    const int nv = min(max(Q.M - lane * nq, 0), nq);
    int t0 = 0, tMD0 = kNeg, Bsuf = 0, Csuf = 1 << 29, maxP = 0;
    if (nv > 0) {
      t0 = hi16(T[lane].w);
      tMD0 = lo16(T[lane].w);
    }
    for (int j = 1; j < nv; ++j) {
      const int t = hi16(T[j * 32 + lane].w);
      Bsuf += t;
      Csuf = min(Csuf + t, kPos);
      maxP = max(maxP, Bsuf);
    }
    // Lane 0's segment starts at node 1, whose delete state is fixed: a
    // constant map.  Lanes without nodes pass the entering score through.
    int Bl = lane == 0 ? kMinusInf : t0 + Bsuf;
    int Cl = nv > 0 ? min(kPos + Bsuf, Csuf) : kPos;
    if (nv == 0 && lane > 0) Bl = 0;
    // Composites of the maps over the windows (lane - 2^r, lane] of the
    // Hillis-Steele scan, or a sentinel below the window.
    int Wb[5], Wc[5];
    {
      int B = Bl, C = Cl;
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        Wb[r] = lane >= (1 << r) ? B : kMinusInf;
        Wc[r] = C;
        if (r == 4) break;        // the 32-lane composite is never used
        const int Bp = __shfl_up_sync(kAll, B, 1 << r);
        const int Cp = __shfl_up_sync(kAll, C, 1 << r);
        if (lane >= (1 << r)) {   // this lane's window after the earlier one
          C = min(Cp + B, C);
          B = Bp + B;
        }
      }
    }
    const int tNN = Q.sp[0], tNB = Q.sp[1], tEC = Q.sp[2], tCC = Q.sp[3];
    const int tCT = Q.sp[4], tEJ = Q.sp[5], tJJ = Q.sp[6], tJB = Q.sp[7];
    const uint64_t n_sel = Q.ranks ? (uint64_t)*Q.n_ranks : (uint64_t)p.n_seqs;

    for (;;) {
      uint32_t q = 0;
      if (lane == 0) q = atomicAdd(p.counters + qi, 1u);
      q = __shfl_sync(kAll, q, 0);
      if ((uint64_t)q >= n_sel) break;
      const uint32_t r = Q.ranks ? __ldg(Q.ranks + q) : q;
      if (!MPF_DCHECK(p.status, r < p.n_seqs)) continue;
      const uint32_t w0 = __ldg(p.seq_word + r);
      const int len = (int)__ldg(p.seq_len + r);
      const uint32_t orig = __ldg(p.seq_orig + r);
      if (!MPF_DCHECK(p.status, (uint64_t)w0 + (uint64_t)((len + 3) >> 2) <= p.n_words && orig < p.n_seqs))
        continue;

      for (int j = 0; j < nq; ++j) {
        if (GM) store_rows(gst, j * 32 + lane, kNeg, kNeg, kNeg);
        else sM[j * 32 + lane] = sI[j * 32 + lane] = sD[j * 32 + lane] = (int16_t)kNeg;
      }
      int xN = Q.base, xJ = kNeg, xC = kNeg;
      int xB = satadd(xN, tNB);
      // Previous row: M, I and true D of the node before the segment, and the
      // carried delete chain at the segment's first node (row 0 carries none).
      int pM0 = kNeg, pI0 = kNeg, pD0 = kNeg, X0 = kMinusInf;
      bool ovf = false;
      uint32_t word = 0;
      for (int i = 0; i < len; ++i) {
        if ((i & 3) == 0) word = __ldg(p.residues + w0 + (uint32_t)(i >> 2));
        int x = (int)((word >> (8 * (i & 3))) & 0xffu);
        if (!MPF_DCHECK(p.status, x < kVitRows)) x = 0;
        const int16_t *erow = Q.msc + (size_t)x * nq * 32 + lane;

        int dM = pM0, dI = pI0, dD = pD0, X = X0, mprev = kNeg, d = kMinusInf;
        int mxM = kNeg, mxD = kNeg, Mn = kNeg, In = kNeg;
#pragma unroll U
        for (int j = 0; j < nv; ++j) {
          const int sl = j * 32 + lane;
          int Mo, Io, Dl;
          if (GM) {
            load_rows(gst, sl, Mo, Io, Dl);
          } else {
            Mo = sM[sl];
            Io = sI[sl];
            Dl = sD[sl];
          }
          const uint4 t = T[sl];
          const int e = __ldg(erow + j * 32);
          const int tDD = hi16(t.w);
          if (j > 0) X = __viaddmin_s32(X, tDD, kPos);   // previous row's carried chain
          const int Do = max(Dl, X);
          const int best = max(max(__viaddmin_s32(dM, hi16(t.x), kPos), __viaddmin_s32(dI, lo16(t.y), kPos)),
                               max(__viaddmin_s32(dD, hi16(t.y), kPos), __viaddmin_s32(xB, lo16(t.x), kPos)));
          Mn = satadd(max(best, kNeg), e);
          In = max(max(__viaddmin_s32(Mo, lo16(t.z), kPos), __viaddmin_s32(Io, hi16(t.z), kPos)), kNeg);
          // Segment-local chain: minus infinity enters the segment's first node.
          d = j > 0 ? max(satadd(mprev, lo16(t.w)), __viaddmin_s32(d, tDD, kPos)) : kMinusInf;
          mxM = max(mxM, Mn);
          mxD = max(mxD, d);
          if (GM) {
            store_rows(gst, sl, Mn, In, j > 0 ? d : kNeg);
          } else {
            sM[sl] = (int16_t)Mn;
            sI[sl] = (int16_t)In;
            sD[sl] = (int16_t)(j > 0 ? d : kNeg);
          }
          dM = Mo;
          dI = Io;
          dD = Do;
          mprev = Mn;
        }

        // True delete score at the end of every segment (inclusive scan of
        // the segments' maps), the chain carried into the next row, and E.
        int Mlp = __shfl_up_sync(kAll, Mn, 1);
        int Ilp = __shfl_up_sync(kAll, In, 1);
        if (lane == 0) Mlp = Ilp = kNeg;
        const int a0 = satadd(Mlp, tMD0);
        int A = nv > 0 ? max(d, min((lane == 0 ? kNeg : a0) + Bsuf, Csuf)) : kMinusInf;
#pragma unroll
        for (int rr = 0; rr < 5; ++rr) {
          const int Ap = __shfl_up_sync(kAll, A, 1 << rr);
          A = max(A, min(Ap + Wb[rr], Wc[rr]));
        }
        int carry = __shfl_up_sync(kAll, A, 1);
        if (lane == 0) carry = kNeg;
        const int newX0 = lane == 0 ? kNeg : max(__viaddmin_s32(carry, t0, kPos), a0);
        const int xd = nv > 0 ? max(mxD, newX0 + maxP) : kNeg;
        const int xE = __reduce_max_sync(kAll, max(mxM, min(xd, kPos)));
        if (xE >= kPos) {
          ovf = true;
          break;
        }
        pM0 = Mlp;
        pI0 = Ilp;
        pD0 = carry;
        X0 = newX0;
        xN = satadd(xN, tNN);
        xC = max(satadd(xC, tCC), satadd(xE, tEC));
        xJ = max(satadd(xJ, tJJ), satadd(xE, tEJ));
        xB = max(satadd(xN, tNB), satadd(xJ, tJB));
      }
      if (lane == 0) {
        if (ovf) {
          Q.score[orig] = 32767;
          Q.flag[orig] = 1;
          if (Q.nat) Q.nat[orig] = __int_as_float(0x7f800000);
        } else {
          const int sc = satadd(xC, tCT);
          Q.score[orig] = (int16_t)sc;
          Q.flag[orig] = 0;
          if (Q.nat) Q.nat[orig] = __fsub_rn(__fdiv_rn(__int2float_rn(sc - Q.base), Q.scale), 3.0f);
        }
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------ team kernel
//
// One team of kTeamW warps scores one sequence (fast-kernel scores).  Lane
// l's segment of Q nodes is cut into kTeamW sub-segments of ceil(Q/kTeamW)
// nodes, sub-segment w swept by warp w of the team, so a row takes about
// Q/kTeamW node steps instead of Q.  In node order the sub-segments form
// one chain, lane-major: (0,0) .. (0,W-1), (1,0) ...  After its sweep each
// warp publishes, per lane, the M and I of its sub-segment's last node, its
// local delete-chain end and its row maximum; one named barrier per row
// makes them visible to the team (two buffers, by row parity).  Every warp
// then composes, per lane, the maps d -> max(A, d + B) of the lane's
// sub-segments in order, runs the warp scan over lanes as the one-warp
// kernel does, and applies the first w maps of its lane to the delete score
// entering the lane: the true delete score entering its own sub-segment.
// All warps of a team keep identical special states and leave a sequence
// together.  For launches with few sequences per warp, whose time is set by
// the longest sequences' rows.

constexpr int kTeamW = 4;

struct TeamExchange {
  int Mlast[kTeamW][32];
  int Ilast[kTeamW][32];
  int dlast[kTeamW][32];
  int xe[kTeamW];
};

__host__ __device__ constexpr size_t team_bytes(int Qmax) {
  return (((size_t)Qmax * 32 * 6 + 2 * sizeof(TeamExchange) + 16) + 15) & ~(size_t)15;
}

__device__ __forceinline__ void team_barrier(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kTeamW * 32) : "memory");
}

template <int U>
__global__ void __launch_bounds__(kVitFastMaxThreads, 1) viterbi_team_kernel(VitParams p) {
  extern __shared__ __align__(16) uint4 fsm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int team = warp / kTeamW, w = warp % kTeamW;
  const int Qmax = p.max_Mpad >> 5;
  uint4 *tr = fsm;
  uint8_t *tb = reinterpret_cast<uint8_t *>(fsm + (size_t)Qmax * 32) + (size_t)team * team_bytes(Qmax);
  int16_t *sM = reinterpret_cast<int16_t *>(tb);
  int16_t *sI = sM + (size_t)Qmax * 32;
  int16_t *sD = sI + (size_t)Qmax * 32;
  TeamExchange *ex = reinterpret_cast<TeamExchange *>(tb + (size_t)Qmax * 32 * 6);
  volatile uint32_t *bcast = reinterpret_cast<volatile uint32_t *>(ex + 2);
  const int bar = 1 + team;   // named barrier of this team (0 is __syncthreads)
  // Debug builds: whole teams, at most 15 per block, and their rows and
  // exchange buffers within the block's shared memory.
  if (!MPF_DCHECK(p.status, (blockDim.x & (kTeamW * 32 - 1)) == 0 && (blockDim.x >> 5) / kTeamW <= 15 &&
                                (size_t)Qmax * 32 * 16 + ((blockDim.x >> 5) / kTeamW) * team_bytes(Qmax) <=
                                    dynamic_smem_bytes()))
    return;

  for (uint32_t qi = 0; qi < p.n_queries; ++qi) {
    const VitQuery Q = p.queries[qi];
    const int nq = Q.Mpad >> 5;
    if (!MPF_DCHECK(p.status, Q.Mpad <= p.max_Mpad && (!Q.ranks || *Q.n_ranks <= p.n_seqs))) continue;
    if (!takes_query(Q, p.n_seqs, true)) continue;
    const uint4 *gtr = reinterpret_cast<const uint4 *>(Q.trans);
    stage_transitions<false>(tr, gtr, nq);

    // Per-lane constants.  Whole segment: nv nodes, Bl = sum of tDD, the
    // window sums Wn of the lane scan (as in the one-warp kernel).  Per
    // sub-segment v of this lane: Bw[v] = sum of its tDD, and cMB[v] = tMD +
    // (Bw - tDD) of its first node, so that its map's A is max(M of the node
    // before + cMB, local chain end); an empty sub-segment is the identity.
    const int nv = min(max(Q.M - lane * nq, 0), nq);
    const int qw = (nq + kTeamW - 1) / kTeamW;
    int Bw[kTeamW], cMB[kTeamW];
    int Bl = 0, tDDf = 0, tMDf = kNeg;
#pragma unroll
    for (int v = 0; v < kTeamW; ++v) {
      const int jb = v * qw, je = min(nv, jb + qw);
      int B = 0;
      for (int j = jb; j < je; ++j) B += hi16(tr[j * 32 + lane].w);
      Bw[v] = B;
      Bl += B;
      cMB[v] = -(1 << 29);
      if (je > jb) {
        const uint32_t t = tr[jb * 32 + lane].w;
        cMB[v] = lo16(t) + (B - hi16(t));
        if (v == w) {
          tMDf = lo16(t);
          tDDf = hi16(t);
        }
      }
    }
    const int jb = w * qw, je = min(nv, jb + qw);   // this warp's nodes of the lane
    const int vlast = (nq - 1) / qw;                  // last non-empty sub-segment of a full lane
    uint32_t P = (uint32_t)Bl;   // prefix over lanes modulo 2^32 (see the one-warp kernel)
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(kAll, P, off);
      if (lane >= off) P += y;
    }
    int Wn[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const uint32_t y = __shfl_up_sync(kAll, P, 1 << r);
      Wn[r] = lane >= (1 << r) ? (int)(P - y) : -(1 << 29);
    }
    const int tNN = Q.sp[0], tNB = Q.sp[1], tEC = Q.sp[2], tCC = Q.sp[3];
    const int tCT = Q.sp[4], tEJ = Q.sp[5], tJJ = Q.sp[6], tJB = Q.sp[7];
    const uint64_t n_sel = Q.ranks ? (uint64_t)*Q.n_ranks : (uint64_t)p.n_seqs;

    for (;;) {
      if (w == 0 && lane == 0) bcast[0] = atomicAdd(p.counters + qi, 1u);
      team_barrier(bar);
      const uint32_t q = bcast[0];
      team_barrier(bar);   // read by all before the next sequence's write
      if ((uint64_t)q >= n_sel) break;
      const uint32_t r = Q.ranks ? __ldg(Q.ranks + q) : q;
      if (!MPF_DCHECK(p.status, r < p.n_seqs)) continue;
      const uint32_t w0 = __ldg(p.seq_word + r);
      const int len = (int)__ldg(p.seq_len + r);
      const uint32_t orig = __ldg(p.seq_orig + r);
      if (!MPF_DCHECK(p.status, (uint64_t)w0 + (uint64_t)((len + 3) >> 2) <= p.n_words && orig < p.n_seqs))
        continue;

      for (int j = jb; j < min(nq, jb + qw); ++j)
        sM[j * 32 + lane] = sI[j * 32 + lane] = sD[j * 32 + lane] = (int16_t)kNeg;
      int xN = Q.base, xJ = kNeg, xC = kNeg;
      int xB = addmax(xN, tNB, kNeg);
      // Previous row: M, I and true D of the node before this sub-segment,
      // and the carried delete chain (X0m + tDD of the first node is its
      // value there).
      int pM0 = kNeg, pI0 = kNeg, pD0 = kNeg, X0m = kNeg - tDDf;
      bool ovf = false;
      int par = 0;
      uint32_t word = 0;
      for (int i = 0; i < len; ++i) {
        if ((i & 3) == 0) word = __ldg(p.residues + w0 + (uint32_t)(i >> 2));
        int x = (int)((word >> (8 * (i & 3))) & 0xffu);
        if (!MPF_DCHECK(p.status, x < kVitRows)) x = 0;
        const int16_t *erow = Q.msc + (size_t)x * nq * 32 + lane;

        FastCell c{pM0, pI0, pD0, X0m, kNeg, kNeg, kNeg, kNeg, kNeg, kNeg, kNeg};
#pragma unroll U
        for (int j = jb; j < je; ++j) {
          const int sl = j * 32 + lane;
          c.step(tr[sl], __ldg(erow + j * 32), sM[sl], sI[sl], sD[sl], xB);
          sD[sl] = (int16_t)c.d;
          sM[sl] = (int16_t)c.Mn;
          sI[sl] = (int16_t)c.In;
        }
        TeamExchange &E = ex[par];
        E.Mlast[w][lane] = c.Mn;
        E.Ilast[w][lane] = c.In;
        E.dlast[w][lane] = c.d;
        const int mx = __reduce_max_sync(kAll, c.mx);
        if (lane == 0) E.xe[w] = mx;
        team_barrier(bar);
        int xE = E.xe[0];
#pragma unroll
        for (int v = 1; v < kTeamW; ++v) xE = max(xE, E.xe[v]);
        if (xE >= 32767) {
          ovf = true;
          break;
        }

        // The lane's map, composed over its sub-segments in node order; the
        // node before sub-segment 0 is the last node of the lane before (a
        // full lane: its last non-empty sub-segment is vlast).
        const int Mbefore = lane > 0 ? E.Mlast[vlast][lane - 1] : kNeg;
        const int Ibefore = lane > 0 ? E.Ilast[vlast][lane - 1] : kNeg;
        int Av[kTeamW];
        int AF = -(1 << 29);
#pragma unroll
        for (int v = 0; v < kTeamW; ++v) {
          const int Mp = v == 0 ? Mbefore : E.Mlast[v - 1][lane];
          Av[v] = addmax(Mp, cMB[v], E.dlast[v][lane]);
          AF = addmax(AF, Bw[v], Av[v]);
        }
        int A = AF;
#pragma unroll
        for (int rr = 0; rr < 5; ++rr) A = addmax(__shfl_up_sync(kAll, A, 1 << rr), Wn[rr], A);
        int din = __shfl_up_sync(kAll, A, 1);
        if (lane == 0) din = kNeg;
#pragma unroll
        for (int v = 0; v < kTeamW; ++v)
          if (v < w) din = addmax(din, Bw[v], Av[v]);
        const int Mp = w == 0 ? Mbefore : E.Mlast[w - 1][lane];
        const int Ip = w == 0 ? Ibefore : E.Ilast[w - 1][lane];
        pM0 = Mp;
        pI0 = Ip;
        pD0 = din;
        X0m = max(din + tDDf, Mp + tMDf) - tDDf;
        par ^= 1;

        xN = addmax(xN, tNN, kNeg);
        xC = addmax(xC, tCC, addmax(xE, tEC, kNeg));
        xJ = addmax(xJ, tJJ, addmax(xE, tEJ, kNeg));
        xB = addmax(xN, tNB, addmax(xJ, tJB, kNeg));
      }
      if (w == 0 && lane == 0) {
        if (ovf) {
          Q.score[orig] = 32767;
          Q.flag[orig] = 1;
          if (Q.nat) Q.nat[orig] = __int_as_float(0x7f800000);
        } else {
          const int sc = addmax(xC, tCT, kNeg);
          Q.score[orig] = (int16_t)sc;
          Q.flag[orig] = 0;
          if (Q.nat) Q.nat[orig] = __fsub_rn(__fdiv_rn(__int2float_rn(sc - Q.base), Q.scale), 3.0f);
        }
      }
    }
  }
}

}  // namespace

size_t viterbi_fast_smem_bytes(int Mpad, int warps) {
  return (size_t)(Mpad >> 5) * 32 * (16 + 6 * (size_t)warps);
}

namespace {

// Shared memory of a block: transitions + per warp the DP rows (M, I and D,
// or M and I with ND; the general kernel always keeps D).
size_t fast_smem(int Mpad, int warps, bool nd) {
  const size_t q = (size_t)(Mpad >> 5);
  return q * 32 * 16 + (size_t)warps * q * 32 * (nd ? 4 : 6);
}

typedef void (*VitKernelFn)(VitParams);

// Variants: the unroll depth of the node loop (8 for segments of 32 nodes or
// more, which measured 5-10% faster there; 4 below, where the deeper unroll
// measured slower) and whether the D row is stored.  The general kernel
// takes the same unroll rule and always stores D.
VitKernelFn vit_kernel_for(bool general, int Q, bool nd) {
  if (general) return Q >= 32 ? viterbi_general_kernel<8, false> : viterbi_general_kernel<4, false>;
  if (nd) return viterbi_fast_kernel<8, true, false>;
  return Q >= 32 ? viterbi_fast_kernel<8, false, false> : viterbi_fast_kernel<4, false, false>;
}

// Device rows of the fast kernel without the stored D row (4-byte records
// M | I; the next row recomputes the local delete chain, two more DPX
// operations per cell) where the tables overflow the L1: then every cell
// also fetches its transitions and match score from L2, and halving the
// row traffic pays (one query, 14,000-40,000 sequences, GCUPS with / without
// D: M = 5,000 604 / 644, 7,000 354 / 606, 10,000 298 / 454; at M = 2,405
// and 3,500, tables in L1, 655 / 626 and 663 / 645).
VitKernelFn gm_kernel_for(bool general, bool nd = false) {
  if (general) return viterbi_general_kernel<8, true>;
  return nd ? viterbi_fast_kernel<8, true, true> : viterbi_fast_kernel<8, false, true>;
}

constexpr size_t kGmL1TableBytes = 224 * 1024;
bool gm_no_d(int Mpad, int n_codes) {
  return (16 + 2 * (size_t)std::max(n_codes, 1)) * (size_t)Mpad > kGmL1TableBytes;
}

// Launch shape of the device-row variants: blocks of kGmWarps warps, as
// many blocks per SM as registers allow, at most kGmWarpsPerSm warps (each
// warp's rows are 8 bytes per node, so this bounds the scratch: 16 warps x
// 152 SMs x 8 B x 100,000 nodes = 1.9 GB at the longest model).  No shared
// memory, so the carveout leaves the whole L1 to the tables.
constexpr int kGmWarps = 8, kGmWarpsPerSm = 16;

int gm_blocks_per_sm(bool general) {
  // The smallest occupancy of the kernel's variants (the scratch is sized for it).
  static const std::array<int, 2> occ = [] {
    std::array<int, 2> t{};
    for (int g = 0; g < 2; ++g) {
      int best = kGmWarpsPerSm / kGmWarps;
      for (int nd = 0; nd < 2; ++nd) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void *)gm_kernel_for(g == 1, nd == 1),
                                                          kGmWarps * 32, 0) != cudaSuccess)
          b = 0;
        best = std::min(best, b);
      }
      t[g] = best;
    }
    return t;
  }();
  return occ[general ? 1 : 0];
}

// Launch shape of a kernel: variant, warps per block, resident blocks
// per SM and the shared-memory carveout.  Each warp reads the match-score
// rows of its residues from global memory, so the L1 left beside shared
// memory should hold the rows of the codes the database uses (n_codes x Mpad
// x 2 bytes, at most 124 KB); among the carveouts that leave that much L1,
// take the shape that keeps the most warps resident (registers permitting).
// The variant without a stored D row trades two DPX operations per cell for
// a third less shared memory per warp; it is taken where the plain kernel
// keeps five warps or fewer per SM (measured, one query against 10,000
// sequences: M = 2800 510 against 435 GCUPS, M = 3072 513 against 377; at
// M = 2000-2405, with 6-11 plain warps, it measured 6-13% slower).  The
// general kernel has no such variant.
struct FastShape {
  bool nd = false;
  int warps = 0, blocks = 1;
  size_t smem = 0;
  int carve_pct = 100;
};

FastShape fast_shape(bool general, int Mpad, int n_codes, int max_smem_block) {
  constexpr size_t kKB = 1024, kUnified = 256 * kKB, kCarveMax = 228 * kKB;
  const int Q = Mpad >> 5;
  // Registers per thread of every instantiation, looked up once (thread-safe
  // static initialisation).
  static const std::array<int, 5> regs_tab = [] {
    std::array<int, 5> t{};
    const VitKernelFn fns[5] = {viterbi_fast_kernel<4, false, false>, viterbi_fast_kernel<8, false, false>,
                                viterbi_fast_kernel<8, true, false>, viterbi_general_kernel<4, false>,
                                viterbi_general_kernel<8, false>};
    for (int i = 0; i < 5; ++i) {
      cudaFuncAttributes a;
      t[i] = cudaFuncGetAttributes(&a, (const void *)fns[i]) == cudaSuccess ? a.numRegs : 255;
    }
    return t;
  }();
  const int regs[2] = {regs_tab[(general ? 3 : 0) + (Q >= 32 ? 1 : 0)], regs_tab[2]};
  const size_t ws = std::min((size_t)std::max(n_codes, 1) * 2 * (size_t)Mpad, 124 * kKB);
  static const int carves_kb[] = {228, 196, 164, 132, 100};   // supported carveouts
  for (int c : carves_kb) {
    const size_t C = (size_t)c * kKB;
    if (kUnified - C < ws && c != 100) continue;
    FastShape best;
    for (int v = 0; v < 2; ++v) {
      const bool nd = v == 1;
      if (nd && (general || best.warps * best.blocks > 5)) continue;
      const int warp_regs = ((regs[v] + 7) / 8) * 8 * 32;
      FastShape cand;
      for (int w = kVitFastMaxThreads / 32; w >= 1; --w) {
        const size_t sm = fast_smem(Mpad, w, nd);
        if (sm > (size_t)max_smem_block || sm + kKB > C) continue;
        int b = (int)(C / (sm + kKB));
        b = std::min(b, 65536 / (warp_regs * w));
        b = std::min(b, 64 / w);
        if (b < 1) continue;
        if (w * b > cand.warps * cand.blocks || (w * b == cand.warps * cand.blocks && b > cand.blocks)) {
          cand.nd = nd;
          cand.warps = w;
          cand.blocks = b;
          cand.smem = sm;
        }
      }
      if (cand.warps * cand.blocks > best.warps * best.blocks) best = cand;
    }
    if (best.warps == 0) continue;
    // The driver takes the smallest supported carveout at or above the
    // preference: ask for just under C.
    best.carve_pct = (int)std::min<size_t>(100, ((C - kKB) * 100) / kCarveMax);
    return best;
  }
  return FastShape();
}

// Launch shape of the team kernel: teams of kTeamW warps per block (at most
// 512 threads), each team with its own DP rows and exchange buffers, the
// same L1-aware carveout choice as fast_shape.
FastShape team_shape(int Mpad, int n_codes, int max_smem_block) {
  constexpr size_t kKB = 1024, kUnified = 256 * kKB, kCarveMax = 228 * kKB;
  const int Q = Mpad >> 5;
  static const int regs = [] {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, (const void *)viterbi_team_kernel<4>) == cudaSuccess ? a.numRegs : 255;
  }();
  const int warp_regs = ((regs + 7) / 8) * 8 * 32;
  const size_t ws = std::min((size_t)std::max(n_codes, 1) * 2 * (size_t)Mpad, 124 * kKB);
  static const int carves_kb[] = {228, 196, 164, 132, 100};
  for (int c : carves_kb) {
    const size_t C = (size_t)c * kKB;
    if (kUnified - C < ws && c != 100) continue;
    FastShape best;
    for (int t = kVitFastMaxThreads / (32 * kTeamW); t >= 1; --t) {
      const int w = t * kTeamW;
      const size_t sm = (size_t)Q * 32 * 16 + (size_t)t * team_bytes(Q);
      if (sm > (size_t)max_smem_block || sm + kKB > C) continue;
      int b = (int)(C / (sm + kKB));
      b = std::min(b, 65536 / (warp_regs * w));
      b = std::min(b, 64 / w);
      if (b < 1) continue;
      if (w * b > best.warps * best.blocks) {
        best.warps = w;
        best.blocks = b;
        best.smem = sm;
      }
    }
    if (best.warps == 0) continue;
    best.carve_pct = (int)std::min<size_t>(100, ((C - kKB) * 100) / kCarveMax);
    return best;
  }
  return FastShape();
}

}  // namespace

size_t viterbi_state_bytes(bool fast, int Mpad, int num_sms) {
  return (size_t)num_sms * gm_blocks_per_sm(!fast) * kGmWarps * (size_t)Mpad * sizeof(uint2);
}

// Rows in shared memory pay off while they leave enough warps resident to
// hide the latency of the match-score loads; with six or fewer per SM the
// device-memory rows (16 warps per SM, the whole L1 for the tables) were
// faster when every warp had several sequences to score (one query against
// 20,000-40,000 sequences, 8-16 per warp; GCUPS shared / device rows: fast
// kernel, 6 warps, M = 2350: 488 / 678, 2405: 488 / 612, 2500: 491 / 523;
// general kernel, 4-6 warps, M = 2405: 417 / 529, 2800: 381 / 530, 3072:
// 340 / 505; with 7-12 warps the shared rows were within 12% either way,
// and ahead below M = 2200).  With few sequences per warp the launch ends
// with the longest sequences, which a warp scores more slowly among 16 than
// among 6 (M = 3500, device rows: 40,000 sequences 665 GCUPS, 16,326 470;
// the MSV -> Viterbi stage over 2% of 500,000 sequences, M = 48-2405: 486
// GCUPS with shared rows, 351 with device rows for M = 2405).  So device
// rows are taken there only with at least 8 sequences per warp.
constexpr int kVitSmemMinWarps = 7;
constexpr uint64_t kGmMinSeqsPerWarp = 8;
// Teams where the host cannot count the sequences (rank lists of the MSV ->
// Viterbi stage, whose survivors are few per warp), for segments of at
// least 8 nodes per lane (M > 224): with fewer, the per-row exchange costs
// more than the shorter sweep saves.
constexpr int kTeamMinQ = 8;

int shape_bits(const FastShape &s) { return s.warps * 10000 + s.blocks * 100 + s.carve_pct; }

// Sequences up to which the team kernel is ahead of the one-warp kernel of
// shape s.  Measured (one query, the first N sequences of the sweep
// database, GCUPS one-warp / team): N = 1,000 and 3,000, M = 256-2405: the
// team ahead everywhere (1.3-2.2x); N = 15,000: M = 400 397 / 245, 800 514 /
// 444, 1600 539 / 562, 2405 (six one-warp warps per SM) 486 / 614.  So the
// team takes every count where the one-warp shape keeps six or fewer warps
// per SM, and otherwise up to about Q/8 sequences per resident one-warp
// worker (the break-even grows with the segment length Q).
int64_t team_max_for(const FastShape &s, int Mpad, int num_sms) {
  if (s.warps * s.blocks < kVitSmemMinWarps) return INT64_MAX;
  return (int64_t)(Mpad >> 5) * num_sms * s.warps * s.blocks / 8;
}

int viterbi_shape_key(bool fast, int Mpad, int n_codes, int max_smem, int num_sms, uint64_t n_seqs) {
  const int gb = gm_blocks_per_sm(!fast);
  const int gm_key =
      gb > 0 ? (fast ? kVitFastDevice : kVitGeneralDevice) * kVitKeyKind + (fast && gm_no_d(Mpad, n_codes) ? 1 : 0)
             : -1;
  if (Mpad > kStripedMaxM) return gm_key;
  const FastShape s = fast_shape(!fast, Mpad, n_codes, max_smem);
  const uint64_t gm_warps = (uint64_t)num_sms * gb * kGmWarps;
  const bool few_warps = s.warps * s.blocks < kVitSmemMinWarps;
  if (gm_key >= 0 && (s.warps == 0 || (few_warps && n_seqs >= kGmMinSeqsPerWarp * gm_warps))) return gm_key;
  if (s.warps == 0) return -1;
  const int one_kind = !fast ? kVitGeneralShared : s.nd ? kVitFastSharedNoD : kVitFastShared;
  const int one_key = one_kind * kVitKeyKind + shape_bits(s);
  if (!fast || (Mpad >> 5) < kTeamMinQ) return one_key;
  const FastShape t = team_shape(Mpad, n_codes, max_smem);
  if (t.warps == 0) return one_key;
  const int team_key = kVitFastTeam * kVitKeyKind + shape_bits(t);
  if (n_seqs > 0) return (int64_t)n_seqs <= team_max_for(s, Mpad, num_sms) ? team_key : one_key;
  return few_warps ? team_key : kVitFastDual * kVitKeyKind + shape_bits(s);
}

int64_t viterbi_team_max(int key, int Mpad, int n_codes, int max_smem, int num_sms) {
  switch (vit_key_kind(key)) {
    case kVitFastTeam:
      return INT64_MAX;
    case kVitFastDual:
      return team_max_for(fast_shape(false, Mpad, n_codes, max_smem), Mpad, num_sms);
    default:
      return -1;
  }
}

int launch_viterbi(const VitParams &p, int key, int n_codes, int max_smem, int num_sms, cudaStream_t st) {
  if (p.n_queries == 0) return 0;
  const int kind = vit_key_kind(key);
  if (kind == kVitFastDevice || kind == kVitGeneralDevice) {
    const bool general = kind == kVitGeneralDevice;
    const int b = gm_blocks_per_sm(general);
    if (b < 1) return 2;
    if (!p.state || p.state_bytes < viterbi_state_bytes(!general, p.max_Mpad, num_sms)) return 1;
    const bool nd = key % kVitKeyKind == 1;   // fast kernel without the stored D row
    const VitKernelFn k = gm_kernel_for(general, nd);
    if (cudaFuncSetAttribute((const void *)k, cudaFuncAttributePreferredSharedMemoryCarveout, 0) != cudaSuccess)
      return 1;
    k<<<num_sms * b, kGmWarps * 32, 0, st>>>(p);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
  }
  // Shared-memory kernels; a dual launch runs the one-warp kernel, then the
  // team kernel, each scoring the queries on its side of team_max (the
  // other exits at once).
  int rc = 0;
  const int passes = kind == kVitFastDual ? 2 : 1;
  for (int pass = 0; pass < passes && rc == 0; ++pass) {
    const bool team = kind == kVitFastTeam || (kind == kVitFastDual && pass == 1);
    FastShape s;
    VitKernelFn k;
    if (team) {
      s = team_shape(p.max_Mpad, n_codes, max_smem);
      k = viterbi_team_kernel<4>;
    } else {
      const bool general = kind == kVitGeneralShared;
      s = fast_shape(general, p.max_Mpad, n_codes, max_smem);
      k = vit_kernel_for(general, p.max_Mpad >> 5, s.nd);
    }
    if (s.warps == 0) return 2;
    const void *fn = (const void *)k;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, s.carve_pct) != cudaSuccess)
      return 1;
    k<<<num_sms * s.blocks, s.warps * 32, s.smem, st>>>(p);
    rc = cudaGetLastError() == cudaSuccess ? 0 : 1;
  }
  return rc;
}

}  // namespace mpf
