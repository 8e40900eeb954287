// Kernel instantiations for groups of 8 lane(s) per sequence.
#include "mpf_scan_kernel.cuh"

namespace mpf {

#define MPF_WORDS_CASE(W)                                   \
  case W:                                                   \
    if (mode == MODE_SSV) return scan_kernel<8, W, MODE_SSV>;             \
    if (mode == MODE_MSV_FAST) return scan_kernel<8, W, MODE_MSV_FAST>;   \
    if (mode == MODE_MSV_DIRECT) return scan_kernel<8, W, MODE_MSV_DIRECT>; \
    if (mode == MODE_SSV_F16) return scan_kernel<8, W, MODE_SSV_F16>; \
    if (mode == MODE_MSV_FAST_F16) return scan_kernel<8, W, MODE_MSV_FAST_F16>; \
    return nullptr;

// Word counts with a two-word tail: the half-precision modes and the
// per-row MSV fallback.
#define MPF_WORDS_CASE_TAIL(W)                                          \
  case W:                                                               \
    if (mode == MODE_MSV_DIRECT) return scan_kernel<8, W, MODE_MSV_DIRECT>;     \
    if (mode == MODE_SSV_F16) return scan_kernel<8, W, MODE_SSV_F16>;           \
    if (mode == MODE_MSV_FAST_F16) return scan_kernel<8, W, MODE_MSV_FAST_F16>; \
    return nullptr;

KernelFn kernel_lg8(int words, int mode) {
  switch (words) {
    MPF_WORDS_CASE(4)
    MPF_WORDS_CASE(8)
    MPF_WORDS_CASE(12)
    MPF_WORDS_CASE(16)
    MPF_WORDS_CASE(20)
    MPF_WORDS_CASE(24)
    MPF_WORDS_CASE(28)
    MPF_WORDS_CASE(32)
    MPF_WORDS_CASE(36)
    MPF_WORDS_CASE(40)
    MPF_WORDS_CASE(44)
    MPF_WORDS_CASE(48)
    MPF_WORDS_CASE_TAIL(6)
    MPF_WORDS_CASE_TAIL(10)
    MPF_WORDS_CASE_TAIL(14)
    MPF_WORDS_CASE_TAIL(18)
    MPF_WORDS_CASE_TAIL(22)
    MPF_WORDS_CASE_TAIL(26)
    MPF_WORDS_CASE_TAIL(30)
    MPF_WORDS_CASE_TAIL(34)
    MPF_WORDS_CASE_TAIL(38)
    MPF_WORDS_CASE_TAIL(42)
    MPF_WORDS_CASE_TAIL(46)
    default:
      return nullptr;
  }
}

}  // namespace mpf
