// Failure-detection check: a bounded wait that nothing completes.
//
// The library's kernels never spin without a limit: every mbarrier wait
// (mbar_wait_bounded, common.cuh) polls against the GPU clock, and when the
// limit passes it records DEV_ERR_TIMEOUT in the context's device error word,
// raises its CTA's abort flag and returns false; the kernel's roles then stop
// at their next check, drain what they issued and return.  This kernel
// drives the same helper into its timeout on purpose (one thread waits on a
// freshly initialised barrier that no thread or copy ever arrives on), so a
// test can check the whole path (device word, host status, a GPU that stays
// usable) without a fault or a hang.
#include "ctx.h"
#include "common.cuh"

namespace osar {
namespace {

__global__ void k_wait_probe(DevScalars* sc, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    mbar_wait_bounded(&bar, 0, &abort_flag, &sc->error, limit_ns);
  __syncthreads();
}

}  // namespace
}  // namespace osar

extern "C" osar_status osar_probe_bounded_wait(osar_ctx* ctx, int64_t limit_ns) {
  if (!ctx) return OSAR_E_INVALID;
  if (ctx->sticky != OSAR_OK) return ctx->sticky;
  if (limit_ns < 1000000 || limit_ns > 10000000000ll) {
    ctx->last_error = "osar_probe_bounded_wait: limit_ns must be in [1e6, 1e10]";
    return OSAR_E_INVALID;
  }
  osar::k_wait_probe<<<1, 32, 0, ctx->stream>>>(ctx->scal, (uint64_t)limit_ns);
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  int32_t err = 0;
  if (e == cudaSuccess)
    e = cudaMemcpy(&err, reinterpret_cast<const char*>(ctx->scal) +
                             offsetof(osar::DevScalars, error),
                   sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    ctx->last_error = std::string("osar_probe_bounded_wait: ") + cudaGetErrorName(e);
    ctx->sticky = OSAR_E_CUDA;
    return OSAR_E_CUDA;
  }
  if (err == osar::DEV_ERR_TIMEOUT) {
    ctx->last_error = "osar_probe_bounded_wait: the bounded wait gave up (as designed)";
    return OSAR_E_TIMEOUT;
  }
  ctx->last_error = "osar_probe_bounded_wait: the wait ended without a timeout";
  return OSAR_E_STATE;
}
