// mpf_inst.cu -- scan-kernel instantiations for one lane-group size.
//
// Compiled once per size (-DMPF_LG=1, 2, 4, 8, 16, 32; see build.py) into
// kernel_lg<MPF_LG>(): every mode of the striped scan kernel (eight) for each
// built word count -- multiples of four, and the counts with a two-word tail.
// With -DMPF_LG=32 -DMPF_TM=1 it builds kernel_lg32_tm() instead: the
// tensor-memory variants (every mode but MSV_DIRECT, at least kTmMinWords
// words).  With -DMPF_QP=1 (lanes 1 to 16) it builds kernel_qp_tm_lg<lanes>():
// the tensor-memory variants that score one sequence against 32 / lanes
// queries per warp (integer SSV, the held MSV pass and the two together).
#include "mpf_scan_kernel.cuh"

#ifndef MPF_LG
#error "compile with -DMPF_LG=<lanes per sequence>"
#endif
#define MPF_CAT2(a, b) a##b
#define MPF_CAT(a, b) MPF_CAT2(a, b)

namespace mpf {

#if defined(MPF_QP)

#define MPF_WORDS_CASE(W)                                                                             \
  case W:                                                                                             \
    if (mode == MODE_SSV) return scan_kernel<MPF_LG, W, MODE_SSV, true, 32 / MPF_LG>;                 \
    if (mode == MODE_MSV_HELD) return scan_kernel<MPF_LG, W, MODE_MSV_HELD, true, 32 / MPF_LG>;       \
    if (mode == MODE_MSV_SSV) return scan_kernel<MPF_LG, W, MODE_MSV_SSV, true, 32 / MPF_LG>;         \
    return nullptr;

KernelFn MPF_CAT(kernel_qp_tm_lg, MPF_LG)(int words, int mode) {
  switch (words) {
    MPF_WORDS_CASE(8)
    MPF_WORDS_CASE(10)
    MPF_WORDS_CASE(12)
    MPF_WORDS_CASE(14)
    MPF_WORDS_CASE(16)
    MPF_WORDS_CASE(18)
    MPF_WORDS_CASE(20)
    MPF_WORDS_CASE(22)
    MPF_WORDS_CASE(24)
    MPF_WORDS_CASE(26)
    MPF_WORDS_CASE(28)
    MPF_WORDS_CASE(30)
    MPF_WORDS_CASE(32)
    MPF_WORDS_CASE(34)
    MPF_WORDS_CASE(36)
    MPF_WORDS_CASE(38)
    MPF_WORDS_CASE(40)
    MPF_WORDS_CASE(42)
    MPF_WORDS_CASE(44)
    MPF_WORDS_CASE(46)
    MPF_WORDS_CASE(48)
    default:
      return nullptr;
  }
}

#elif defined(MPF_TM) && MPF_LG == 32

#define MPF_WORDS_CASE(W)                                                                  \
  case W:                                                                                  \
    if (mode == MODE_SSV) return scan_kernel<32, W, MODE_SSV, true>;                       \
    if (mode == MODE_MSV_FAST) return scan_kernel<32, W, MODE_MSV_FAST, true>;             \
    if (mode == MODE_SSV_F16) return scan_kernel<32, W, MODE_SSV_F16, true>;               \
    if (mode == MODE_MSV_FAST_F16) return scan_kernel<32, W, MODE_MSV_FAST_F16, true>;     \
    if (mode == MODE_MSV_HELD) return scan_kernel<32, W, MODE_MSV_HELD, true>;             \
    if (mode == MODE_MSV_HELD_F16) return scan_kernel<32, W, MODE_MSV_HELD_F16, true>;     \
    if (mode == MODE_MSV_SSV) return scan_kernel<32, W, MODE_MSV_SSV, true>;               \
    return nullptr;

KernelFn kernel_lg32_tm(int words, int mode) {
  switch (words) {
    MPF_WORDS_CASE(8)
    MPF_WORDS_CASE(10)
    MPF_WORDS_CASE(12)
    MPF_WORDS_CASE(14)
    MPF_WORDS_CASE(16)
    MPF_WORDS_CASE(18)
    MPF_WORDS_CASE(20)
    MPF_WORDS_CASE(22)
    MPF_WORDS_CASE(24)
    MPF_WORDS_CASE(26)
    MPF_WORDS_CASE(28)
    MPF_WORDS_CASE(30)
    MPF_WORDS_CASE(32)
    MPF_WORDS_CASE(34)
    MPF_WORDS_CASE(36)
    MPF_WORDS_CASE(38)
    MPF_WORDS_CASE(40)
    MPF_WORDS_CASE(42)
    MPF_WORDS_CASE(44)
    MPF_WORDS_CASE(46)
    MPF_WORDS_CASE(48)
    default:
      return nullptr;
  }
}

#else

#define MPF_WORDS_CASE(W)                                                            \
  case W:                                                                            \
    if (mode == MODE_SSV) return scan_kernel<MPF_LG, W, MODE_SSV>;                   \
    if (mode == MODE_MSV_FAST) return scan_kernel<MPF_LG, W, MODE_MSV_FAST>;         \
    if (mode == MODE_MSV_DIRECT) return scan_kernel<MPF_LG, W, MODE_MSV_DIRECT>;     \
    if (mode == MODE_SSV_F16) return scan_kernel<MPF_LG, W, MODE_SSV_F16>;           \
    if (mode == MODE_MSV_FAST_F16) return scan_kernel<MPF_LG, W, MODE_MSV_FAST_F16>; \
    if (mode == MODE_MSV_HELD) return scan_kernel<MPF_LG, W, MODE_MSV_HELD>;         \
    if (mode == MODE_MSV_HELD_F16) return scan_kernel<MPF_LG, W, MODE_MSV_HELD_F16>; \
    if (mode == MODE_MSV_SSV) return scan_kernel<MPF_LG, W, MODE_MSV_SSV>;           \
    return nullptr;

KernelFn MPF_CAT(kernel_lg, MPF_LG)(int words, int mode) {
  switch (words) {
    MPF_WORDS_CASE(4)
    MPF_WORDS_CASE(6)
    MPF_WORDS_CASE(8)
    MPF_WORDS_CASE(10)
    MPF_WORDS_CASE(12)
    MPF_WORDS_CASE(14)
    MPF_WORDS_CASE(16)
    MPF_WORDS_CASE(18)
    MPF_WORDS_CASE(20)
    MPF_WORDS_CASE(22)
    MPF_WORDS_CASE(24)
    MPF_WORDS_CASE(26)
    MPF_WORDS_CASE(28)
    MPF_WORDS_CASE(30)
    MPF_WORDS_CASE(32)
    MPF_WORDS_CASE(34)
    MPF_WORDS_CASE(36)
    MPF_WORDS_CASE(38)
    MPF_WORDS_CASE(40)
    MPF_WORDS_CASE(42)
    MPF_WORDS_CASE(44)
    MPF_WORDS_CASE(46)
    MPF_WORDS_CASE(48)
    default:
      return nullptr;
  }
}

#endif

}  // namespace mpf
