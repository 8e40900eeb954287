// mpf_debug.cu -- self-test of the kernels' debug index checks.
//
// In the debug build (-DMPF_DEBUG_CHECKS) one block evaluates an index
// check that fails -- an index one past the end of a length it was given --
// with no memory access behind it, so the context's status word must read
// "bad index" afterwards.  It shows that a failed check reaches mpf_sync as
// MPF_EDEVICE without ever making the access the check guards.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpf.h"
#include "mpf_handles.h"
#include "mpf_internal.h"

#ifdef MPF_DEBUG_CHECKS
namespace {

__global__ void index_check_selftest(int *status, uint32_t n, uint32_t *sink) {
  const uint32_t idx = n + threadIdx.x;   // one past the end and beyond
  if (MPF_DCHECK(status, idx < n)) sink[0] = idx;   // never taken: idx >= n
}

}  // namespace
#endif

extern "C" int mpf_debug_check_selftest(mpf_ctx *ctx) {
  if (!ctx) return MPF_EINVAL;
#ifdef MPF_DEBUG_CHECKS
  mpf::host::DeviceGuard dg(ctx->device);
  index_check_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_status, 16u, nullptr);
  return cudaGetLastError() == cudaSuccess ? MPF_OK : MPF_ECUDA;
#else
  return MPF_EUNSUPPORTED;
#endif
}
