// mpf_ubench.cu -- issue-rate and on-chip bandwidth microbenchmarks behind
// the roofline of the byte-filter kernels (libmpf_ubench.so; not part of the
// scan library).
//
// Every test runs one block per SM (grid = SM count, more dynamic shared
// memory than two blocks could share) of 1,024 threads (ALU tests) or 512
// (memory tests, which need more registers per thread)
// and times its loop with clock64() between two block barriers, so results
// are in SM clock cycles whatever the clock frequency: per SM and cycle,
//   ALU tests:    lane-operations (threads x operations / cycles)
//   memory tests: bytes delivered to registers (threads x bytes / cycles).
// Each thread runs 8 independent dependency chains so that issue, not
// latency, is the limit (32 warps per SM, 64 chains per scheduler).
//
// The operations are the candidates for one packed cell update of the MSV /
// SSV recurrences (Alg. 2, Alg. 7): 32-bit integer add, three-input logic
// (LOP3), byte permute (PRMT), integer multiply-add (IMAD), the 16x2 DPX
// forms (add-then-max, three-input max; and the 32-bit forms of the Viterbi
// filter), fp16x2 fused multiply-add with
// ReLU, and the 4x8-bit SIMD intrinsics of the paper's Kepler kernels
// (__vaddus4, __vsubus4, __vmaxu4).  The memory tests read 128-bit words
// from shared memory, and 32-bit columns from tensor memory (TMEM, tcgen05.ld
// of the 32x32b shape), alone and together.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace {

constexpr int kThreads = 1024;      // ALU tests: 32 warps per SM
constexpr int kMemThreads = 512;    // memory tests: 16 warps per SM (128 registers each)
constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr uint32_t kTmemCols = 256;      // columns allocated per block (power of two >= 32)
constexpr int kSmemBytes = 128 * 1024;   // forces one block per SM; the LDS tests read it

enum Op : int {
  OP_IADD = 0,
  OP_LOP3 = 1,
  OP_PRMT = 2,
  OP_IMAD = 3,
  OP_DPX_ADDMAX = 4,
  OP_DPX_MAX3 = 5,
  OP_HFMA2_RELU = 6,
  OP_VADDUS4 = 7,
  OP_VSUBUS4 = 8,
  OP_VMAXU4 = 9,
  OP_DPX_ADDMAX_HFMA2 = 10,   // one DPX and one HFMA2 per step: do the pipes co-issue?
  OP_DPX_ADDMAX_PRMT = 11,    // one DPX and one PRMT per step
  OP_DPX_ADDMAX_S32 = 12,     // 32-bit DPX forms (the Viterbi filter's cells)
  OP_DPX_MAX3_S32 = 13,
  OP_LDS128 = 20,
  OP_TMEM_LD = 21,
  OP_LDS128_TMEM_LD = 22,
  OP_SHFL = 23,
};

template <int OP>
__device__ __forceinline__ uint32_t alu_step(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  if constexpr (OP == OP_IADD) {
    asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  } else if constexpr (OP == OP_LOP3) {
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  } else if constexpr (OP == OP_PRMT) {
    asm volatile("prmt.b32 %0, %1, %2, 0x5432;" : "=r"(r) : "r"(a), "r"(b));
  } else if constexpr (OP == OP_IMAD) {
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  } else if constexpr (OP == OP_DPX_ADDMAX) {
    r = __viaddmax_s16x2(a, b, c);
  } else if constexpr (OP == OP_DPX_MAX3) {
    r = __vimax3_s16x2(a, b, c);
  } else if constexpr (OP == OP_DPX_ADDMAX_S32) {
    r = (uint32_t)__viaddmax_s32((int)a, (int)b, (int)c);
  } else if constexpr (OP == OP_DPX_MAX3_S32) {
    r = (uint32_t)__vimax3_s32((int)a, (int)b, (int)c);
  } else if constexpr (OP == OP_HFMA2_RELU) {
    const __half2 x = __hfma2_relu(*reinterpret_cast<const __half2 *>(&a),
                                   *reinterpret_cast<const __half2 *>(&b),
                                   *reinterpret_cast<const __half2 *>(&c));
    r = *reinterpret_cast<const uint32_t *>(&x);
  } else if constexpr (OP == OP_VADDUS4) {
    r = __vaddus4(a, b);
  } else if constexpr (OP == OP_VSUBUS4) {
    r = __vsubus4(a, b);
  } else {
    r = __vmaxu4(a, b);
  }
  return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ALU issue rate: kChains independent chains of one operation per thread
// (two operations per step for the pairs).
template <int OP>
__global__ void __launch_bounds__(kThreads, 1)
    ubench_alu(uint32_t seed, int iters, uint32_t *sink, long long *cycles) {
  uint32_t a[kChains], d[kChains];
  const uint32_t b = seed * 2654435761u + 0x00010001u, c = seed ^ 0x3c003c00u;
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = d[j] = seed + threadIdx.x * 977u + (uint32_t)j * 131u;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        if constexpr (OP == OP_DPX_ADDMAX_HFMA2) {
          a[j] = alu_step<OP_DPX_ADDMAX>(a[j], b, c);
          d[j] = alu_step<OP_HFMA2_RELU>(d[j], b, c);
        } else if constexpr (OP == OP_DPX_ADDMAX_PRMT) {
          a[j] = alu_step<OP_DPX_ADDMAX>(a[j], b, c);
          d[j] = alu_step<OP_PRMT>(d[j], b, c);
        } else {
          a[j] = alu_step<OP>(a[j], b, c);
        }
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) x ^= a[j] ^ d[j];
  if (x == 0x9e3779b9u) sink[blockIdx.x] = x;   // keeps the chains live
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Shared-memory bandwidth: conflict-free 128-bit loads (lane i of a warp reads
// the i-th 16-byte word of a 512-byte line), XOR-folded into registers.
__device__ __forceinline__ void lds_step(const uint4 *s, uint32_t idx, uint32_t &acc) {
  const uint4 v = s[idx];
  acc ^= v.x ^ v.y ^ v.z ^ v.w;
}

// TMEM: the block allocates kTmemCols columns; warp w reads the 32 lanes of
// its quarter (w mod 4) of the tensor memory.  Two tcgen05.ld of 16 columns
// (64 bytes per thread each), then one wait.
__device__ __forceinline__ uint32_t tmem_ld2x16(uint32_t taddr) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr + 16u));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) x ^= r[i];
  return x;
}

template <int OP>
__global__ void __launch_bounds__(kMemThreads, 1)
    ubench_mem(uint32_t seed, int iters, uint32_t *sink, long long *cycles) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_taddr;
  const uint4 *s = reinterpret_cast<const uint4 *>(smem);
  const int warp = threadIdx.x >> 5;
  constexpr bool kTmem = (OP == OP_TMEM_LD || OP == OP_LDS128_TMEM_LD);
  // Fill the shared memory (every word written before the timed loop).
  for (uint32_t i = threadIdx.x; i < kSmemBytes / 4; i += kMemThreads)
    reinterpret_cast<uint32_t *>(smem)[i] = seed + i;
  uint32_t taddr = 0;
  if constexpr (kTmem) {
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&s_taddr)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if constexpr (kTmem) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    taddr = s_taddr + ((uint32_t)((warp & 3) * 32) << 16);
    // Write every column this warp will read (16 columns per store).
    for (uint32_t col = 0; col < kTmemCols; col += 16) {
      const uint32_t v = seed ^ (threadIdx.x * 7u + col);
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16};" ::"r"(taddr + col),
          "r"(v), "r"(v + 1), "r"(v + 2), "r"(v + 3), "r"(v + 4), "r"(v + 5), "r"(v + 6), "r"(v + 7),
          "r"(v + 8), "r"(v + 9), "r"(v + 10), "r"(v + 11), "r"(v + 12), "r"(v + 13), "r"(v + 14),
          "r"(v + 15));
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  // Per iteration and thread: 16 128-bit shared loads (256 B); 4 x two
  // 16-column TMEM loads (512 B); 16 x 8 independent shuffles.
  uint32_t acc = 0, sh[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) sh[j] = seed + threadIdx.x + (uint32_t)j;
  const uint32_t lane_word = threadIdx.x & 31u;
  const uint32_t nlines = kSmemBytes / 512;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if constexpr (OP == OP_LDS128 || OP == OP_LDS128_TMEM_LD) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const uint32_t line = ((uint32_t)it * kUnroll + (uint32_t)u + (uint32_t)warp * 3u) & (nlines - 1);
        lds_step(s, line * 32u + lane_word, acc);
      }
    }
    if constexpr (kTmem) {
#pragma unroll
      for (int g = 0; g < 4; ++g)
        acc ^= tmem_ld2x16(taddr + (((uint32_t)it * 128u + (uint32_t)g * 32u) & (kTmemCols - 1)));
    }
    if constexpr (OP == OP_SHFL) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int j = 0; j < kChains; ++j) sh[j] = __shfl_xor_sync(0xffffffffu, sh[j] + (uint32_t)u, 1);
    }
  }
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc ^= sh[j];
  __syncthreads();
  const long long t1 = clock64();
  if constexpr (kTmem) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_taddr), "r"(kTmemCols));
    }
  }
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

typedef void (*UbenchFn)(uint32_t, int, uint32_t *, long long *);

UbenchFn ubench_fn(int op) {
  switch (op) {
    case OP_IADD: return ubench_alu<OP_IADD>;
    case OP_LOP3: return ubench_alu<OP_LOP3>;
    case OP_PRMT: return ubench_alu<OP_PRMT>;
    case OP_IMAD: return ubench_alu<OP_IMAD>;
    case OP_DPX_ADDMAX: return ubench_alu<OP_DPX_ADDMAX>;
    case OP_DPX_MAX3: return ubench_alu<OP_DPX_MAX3>;
    case OP_HFMA2_RELU: return ubench_alu<OP_HFMA2_RELU>;
    case OP_VADDUS4: return ubench_alu<OP_VADDUS4>;
    case OP_VSUBUS4: return ubench_alu<OP_VSUBUS4>;
    case OP_VMAXU4: return ubench_alu<OP_VMAXU4>;
    case OP_DPX_ADDMAX_HFMA2: return ubench_alu<OP_DPX_ADDMAX_HFMA2>;
    case OP_DPX_ADDMAX_PRMT: return ubench_alu<OP_DPX_ADDMAX_PRMT>;
    case OP_DPX_ADDMAX_S32: return ubench_alu<OP_DPX_ADDMAX_S32>;
    case OP_DPX_MAX3_S32: return ubench_alu<OP_DPX_MAX3_S32>;
    case OP_LDS128: return ubench_mem<OP_LDS128>;
    case OP_TMEM_LD: return ubench_mem<OP_TMEM_LD>;
    case OP_LDS128_TMEM_LD: return ubench_mem<OP_LDS128_TMEM_LD>;
    case OP_SHFL: return ubench_mem<OP_SHFL>;
    default: return nullptr;
  }
}

}  // namespace

extern "C" {

// Run test `op` with `iters` loop iterations on every SM of `device`.
// Writes the per-SM rate (lane-operations or bytes per SM clock cycle,
// averaged over the blocks) to *rate and the mean cycle count to *cycles_out.
// Returns 0, 1 for an unknown op, 2 for a CUDA error.
int mpf_ubench_run(int device, int op, int iters, double *rate, double *cycles_out) {
  UbenchFn fn = ubench_fn(op);
  if (!fn || iters < 1 || !rate || !cycles_out) return 1;
  if (cudaSetDevice(device) != cudaSuccess) return 2;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 2;
  uint32_t *sink = nullptr;
  long long *cyc = nullptr;
  if (cudaMalloc(&sink, sizeof(uint32_t) * nsm) != cudaSuccess) return 2;
  if (cudaMalloc(&cyc, sizeof(long long) * nsm) != cudaSuccess) {
    cudaFree(sink);
    return 2;
  }
  const int smem = kSmemBytes;   // one block per SM in every test
  const int threads = op >= OP_LDS128 ? kMemThreads : kThreads;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    fn<<<nsm, threads, smem>>>(0x1234567u, iters, sink, cyc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<long long> h(nsm);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(long long) * nsm, cudaMemcpyDeviceToHost);
  cudaFree(sink);
  cudaFree(cyc);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return 2;
  }
  double mean = 0;
  for (long long c : h) mean += (double)c;
  mean /= nsm;
  const double per_thread_steps = (double)iters * kUnroll;
  double work;   // per block
  switch (op) {
    case OP_DPX_ADDMAX_HFMA2:
    case OP_DPX_ADDMAX_PRMT: work = kThreads * per_thread_steps * kChains * 2; break;
    case OP_LDS128: work = (double)kMemThreads * iters * 256; break;
    case OP_TMEM_LD: work = (double)kMemThreads * iters * 512; break;
    case OP_LDS128_TMEM_LD: work = (double)kMemThreads * iters * (256 + 512); break;
    case OP_SHFL: work = kMemThreads * per_thread_steps * kChains; break;
    default: work = kThreads * per_thread_steps * kChains; break;
  }
  *rate = work / mean;
  *cycles_out = mean;
  return 0;
}

}  // extern "C"
