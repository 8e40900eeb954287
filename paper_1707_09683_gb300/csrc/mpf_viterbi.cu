// mpf_viterbi.cu -- the P7Viterbi filter (Eq. 1 of Sec. 2.1) for sm_103a.
//
// One warp scores one sequence.  The DP row (M, I, D scores of every node)
// lives in the warp's slice of shared memory as 16-bit words and is swept in
// chunks of 32 consecutive nodes, node k handled by lane k mod 32:
//   * the diagonal terms of Eq. 1 (node k-1 of the previous row) come from the
//     neighbouring lane by one shuffle, and from the previous chunk's last
//     lane across a chunk boundary;
//   * the insert term uses the same node of the previous row (lane-local);
//   * the delete chain D[k] = max(M[k-1] + tMD, D[k-1] + tDD) runs along the
//     row: each node is the map d -> max(A, min(d + B, C)) of its
//     predecessor, these maps compose, and a 5-step warp scan gives every lane
//     its node's value from the chunk's carry-in;
//   * E is a warp max, then the N, C, J, B special states are scalar.
// All arithmetic is the 16-bit saturating word arithmetic of the Viterbi
// filter, computed in 32-bit registers with explicit clamps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mpf_internal.h"

namespace mpf {

namespace {

constexpr uint32_t kAll = 0xffffffffu;

__device__ __forceinline__ int sat16(int v) { return min(32767, max(-32768, v)); }

// Score one sequence (length-rank r) against query Q; the warp's three DP
// rows are sM, sI, sD (Mpad int16 each).
__device__ __forceinline__ void viterbi_one(const VitParams &p, const VitQuery &Q, uint32_t r,
                                            int16_t *sM, int16_t *sI, int16_t *sD, int lane) {
  const int Mpad = Q.Mpad, M = Q.M;
  const int nch = Mpad >> 5;
  const int tNN = Q.sp[0], tNB = Q.sp[1], tEC = Q.sp[2], tCC = Q.sp[3];
  const int tCT = Q.sp[4], tEJ = Q.sp[5], tJJ = Q.sp[6], tJB = Q.sp[7];
  const uint32_t w0 = __ldg(p.seq_word + r);
  const int len = (int)__ldg(p.seq_len + r);
  const uint32_t orig = __ldg(p.seq_orig + r);

  for (int k = lane; k < Mpad; k += 32) sM[k] = sI[k] = sD[k] = (int16_t)-32768;
  __syncwarp();
  int xN = Q.base, xJ = -32768, xC = -32768;
  int xB = sat16(xN + tNB);
  bool ovf = false;
  uint32_t word = 0;
  for (int i = 0; i < len; ++i) {
    if ((i & 3) == 0) word = __ldg(p.residues + w0 + (uint32_t)(i >> 2));
    const int x = (int)((word >> (8 * (i & 3))) & 0xffu);
    const int16_t *msc_row = Q.msc + (size_t)x * Mpad;
    int coM = -32768, coI = -32768, coD = -32768;   // previous row, node before the chunk
    int cnM = -32768, cnD = -32768;                  // this row, node before the chunk
    int xE = -32768;
    for (int c = 0; c < nch; ++c) {
      const int k = (c << 5) + lane;                 // 0-based node index
      const int Mo = sM[k], Io = sI[k], Do = sD[k];
      int pM = __shfl_up_sync(kAll, Mo, 1);
      int pI = __shfl_up_sync(kAll, Io, 1);
      int pD = __shfl_up_sync(kAll, Do, 1);
      if (lane == 0) {
        pM = coM;
        pI = coI;
        pD = coD;
      }
      coM = __shfl_sync(kAll, Mo, 31);
      coI = __shfl_sync(kAll, Io, 31);
      coD = __shfl_sync(kAll, Do, 31);
      const int e = __ldg(msc_row + k);
      const int16_t *t = Q.trans + k;
      const int tBM = __ldg(t), tMM = __ldg(t + Mpad), tIM = __ldg(t + 2 * Mpad);
      const int tDM = __ldg(t + 3 * Mpad), tMI = __ldg(t + 4 * Mpad), tII = __ldg(t + 5 * Mpad);
      const int tMD = __ldg(t + 6 * Mpad), tDD = __ldg(t + 7 * Mpad);
      const int best = max(max(sat16(pM + tMM), sat16(pI + tIM)), max(sat16(pD + tDM), sat16(xB + tBM)));
      const int Mn = sat16(best + e);
      const int In = (k < M - 1) ? max(sat16(Mo + tMI), sat16(Io + tII)) : -32768;
      // Delete chain along the row: node k maps the delete score of node k-1
      // to max(A, min(d + B, C)); an inclusive warp scan composes the maps.
      int pMn = __shfl_up_sync(kAll, Mn, 1);
      if (lane == 0) pMn = cnM;
      int A = sat16(pMn + tMD), B = tDD, C = 32767;
      if (k == 0) {               // node 1 has no delete state
        A = -32768;
        B = -(1 << 20);
      }
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int Ap = __shfl_up_sync(kAll, A, off);
        const int Bp = __shfl_up_sync(kAll, B, off);
        const int Cp = __shfl_up_sync(kAll, C, off);
        if (lane >= off) {        // this lane's map after the earlier lanes' maps
          A = max(A, min(Ap + B, C));
          C = min(Cp + B, C);
          B = Bp + B;
        }
      }
      const int Dn = max(A, min(cnD + B, C));
      cnM = __shfl_sync(kAll, Mn, 31);
      cnD = __shfl_sync(kAll, Dn, 31);
      if (k < M) {
        xE = max(xE, max(Mn, Dn));
        sM[k] = (int16_t)Mn;
        sI[k] = (int16_t)In;
        sD[k] = (int16_t)Dn;
      }
    }
    xE = __reduce_max_sync(kAll, xE);
    if (xE >= 32767) {
      ovf = true;
      break;
    }
    xN = sat16(xN + tNN);
    xC = max(sat16(xC + tCC), sat16(xE + tEC));
    xJ = max(sat16(xJ + tJJ), sat16(xE + tEJ));
    xB = max(sat16(xN + tNB), sat16(xJ + tJB));
  }
  if (lane == 0) {
    if (ovf) {
      Q.score[orig] = 32767;
      Q.flag[orig] = 1;
      if (Q.nat) Q.nat[orig] = __int_as_float(0x7f800000);
    } else {
      const int sc = sat16(xC + tCT);
      Q.score[orig] = (int16_t)sc;
      Q.flag[orig] = 0;
      if (Q.nat) Q.nat[orig] = __fsub_rn(__fdiv_rn(__int2float_rn(sc - Q.base), Q.scale), 3.0f);
    }
  }
  __syncwarp();
}

// Persistent kernel: every warp walks the queries in order and, within a
// query, pulls the next length rank from that query's counter.
__global__ void __launch_bounds__(kVitThreads) viterbi_kernel(VitParams p) {
  extern __shared__ __align__(16) int16_t vsm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int16_t *sM = vsm + (size_t)warp * 3 * p.max_Mpad;
  int16_t *sI = sM + p.max_Mpad;
  int16_t *sD = sI + p.max_Mpad;
  for (uint32_t qi = 0; qi < p.n_queries; ++qi) {
    const VitQuery Q = p.queries[qi];
    const uint64_t n_sel = Q.ranks ? (uint64_t)*Q.n_ranks : (uint64_t)p.n_seqs;
    for (;;) {
      uint32_t q = 0;
      if (lane == 0) q = atomicAdd(p.counters + qi, 1u);
      q = __shfl_sync(kAll, q, 0);
      if ((uint64_t)q >= n_sel) break;
      const uint32_t r = Q.ranks ? __ldg(Q.ranks + q) : q;
      viterbi_one(p, Q, r, sM, sI, sD, lane);
    }
  }
}

}  // namespace

size_t viterbi_smem_bytes(int Mpad) { return (size_t)(kVitThreads / 32) * 3 * (size_t)Mpad * sizeof(int16_t); }

int launch_viterbi(const VitParams &p, int num_sms, cudaStream_t st) {
  if (p.n_queries == 0) return 0;
  const size_t smem = viterbi_smem_bytes(p.max_Mpad);
  if (cudaFuncSetAttribute((const void *)viterbi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)viterbi_kernel, kVitThreads,
                                                    smem) != cudaSuccess || per_sm < 1)
    return 1;
  viterbi_kernel<<<num_sms * per_sm, kVitThreads, smem, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace mpf
