// mpf_tmem.cuh -- tensor-memory (TMEM) helpers for the scan kernels (sm_103a).
//
// The striped scan kernels read one row of their score table per DP row.
// Shared memory delivers 128 B per SM clock, which caps a kernel that reads
// 2 B of table per cell at 64 cells per clock.  The 256 KB of tensor memory
// next to each SM's tensor cores is read into registers by tcgen05.ld at
// about three times that rate (measured: 386 B/clk/SM with 32x32b.x16 loads),
// so the one-sequence-per-warp kernels keep the score rows of the residue
// codes a database uses in TMEM and read the rest from shared memory.
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM.  Warp w of a block
// may read only lanes 32 (w mod 4) .. 32 (w mod 4) + 31, thread t of the warp
// lane 32 (w mod 4) + t; the column is a warp-uniform operand.  A block
// allocates columns with tcgen05.alloc (one warp, power of two >= 32) and
// must free them with tcgen05.dealloc before it exits.
#pragma once
#include <stdint.h>

namespace mpf {

constexpr uint32_t kTmemCols = kTmemColumns;   // the whole tensor memory of an SM, one block per SM

__device__ __forceinline__ uint32_t smem_addr_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Warp-collective: allocate kTmemCols columns; the TMEM address is written
// to *dst (shared memory).  Then give up the right to allocate again (a
// block allocates once, at its start).
__device__ __forceinline__ void tm_alloc(uint32_t *dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr_u32(dst)),
               "r"(kTmemCols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

// Warp-collective: free the columns (every tcgen05.ld / st of the block must
// have completed: waited for, then ordered by a fenced barrier).
__device__ __forceinline__ void tm_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols));
}

// Order tcgen05 operations across a thread barrier (before / after it).
__device__ __forceinline__ void tm_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Loads of 16, 8, 4, 2 or 1 consecutive columns of the thread's lane into
// registers (32x32b shape).  The registers are valid only after tm_wait_ld.
template <int N>
__device__ __forceinline__ void tm_ld_pow2(uint32_t *r, uint32_t a);

template <>
__device__ __forceinline__ void tm_ld_pow2<16>(uint32_t *r, uint32_t a) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(a));
}
template <>
__device__ __forceinline__ void tm_ld_pow2<8>(uint32_t *r, uint32_t a) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(a));
}
template <>
__device__ __forceinline__ void tm_ld_pow2<4>(uint32_t *r, uint32_t a) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
template <>
__device__ __forceinline__ void tm_ld_pow2<2>(uint32_t *r, uint32_t a) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
template <>
__device__ __forceinline__ void tm_ld_pow2<1>(uint32_t *r, uint32_t a) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[0]) : "r"(a));
}

// N (< 32) consecutive columns starting at column address a.
template <int N>
__device__ __forceinline__ void tm_ld(uint32_t *r, uint32_t a) {
  static_assert(N > 0 && N < 32, "columns per load");
  constexpr int A = N & 16, B = N & 8, C = N & 4, D = N & 2, E = N & 1;
  if constexpr (A) tm_ld_pow2<16>(r, a);
  if constexpr (B) tm_ld_pow2<8>(r + A, a + A);
  if constexpr (C) tm_ld_pow2<4>(r + A + B, a + A + B);
  if constexpr (D) tm_ld_pow2<2>(r + A + B + C, a + A + B + C);
  if constexpr (E) tm_ld_pow2<1>(r + A + B + C + D, a + A + B + C + D);
}

// Wait for this thread's outstanding tcgen05.ld; the empty asm statements
// after it make every register of r depend on the wait, so no use of them is
// scheduled before it.
template <int N>
__device__ __forceinline__ void tm_wait_ld(uint32_t *r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}

// Stores of 4 or 2 consecutive columns of the thread's lane.
__device__ __forceinline__ void tm_st4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y),
               "r"(z), "r"(w)
               : "memory");
}
__device__ __forceinline__ void tm_st2(uint32_t a, uint32_t x, uint32_t y) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(a), "r"(x), "r"(y) : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace mpf
