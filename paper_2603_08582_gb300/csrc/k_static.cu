// Allocation-free variant of the Gram apply (y = A_n x).
//
// Some callers cannot let a library allocate device memory while they run:
// flight or embedded pipelines that reserve all GPU memory once at start-up
// and forbid allocation afterwards (an allocation can fail under memory
// pressure, and cudaMalloc / cudaFree may synchronise the whole device and
// break a latency budget), and hosts that route every buffer through their
// own memory pool.  osar_gram_apply_static serves them: the caller supplies
// x and y in device memory, and the scratch the matvec needs (the working
// copy of x and the segment / block partials) comes from one file-scope
// device array instead of cudaMalloc.
//
// The array is GRAM_APPLY_STATIC_BYTES (4 MiB) on every GPU where a context
// is created, held until the process exits.  It fits the scratch of any Gram
// with M <= 4096 rows in every precision (atoms; pixels N in the pixel-space
// Gram form, whose apply works on P_n); larger contexts are rejected with
// OSAR_E_INVALID.  All calls on a device share the array and it keeps the
// last call's contents; every byte a call reads is written earlier in that
// call, so nothing needs clearing.  Calls whose work overlaps on the GPU
// (two streams, or two contexts on one device) race on the array and must be
// ordered by the caller.
//
// Set-up: the array's device address is looked up once per device, with that
// device current (cudaGetSymbolAddress).  osar_create does it for its device,
// so that the lookup, and the module load that places the array in device
// memory under CUDA's lazy loading, happen while the caller is still setting
// up.  Should that lookup fail, the first osar_gram_apply_static call on the
// device repeats it (then make that call before any stream capture).
//
// The caller's x and y are checked before any launch: both must be device
// (or managed) memory that the current device can address and 16-byte
// aligned.  A host pointer or a pointer into another GPU would otherwise make
// the first kernel fault and leave the CUDA context unusable.
#include <cstdint>
#include <mutex>
#include <string>

#include "ctx.h"

namespace {

constexpr size_t GRAM_APPLY_STATIC_BYTES = size_t(4) << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_apply_scratch[GRAM_APPLY_STATIC_BYTES];

std::mutex g_scratch_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_apply_scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Device or managed memory usable by the current device, 16-byte aligned.
bool device_vector_ok(const void* p, std::string* why) {
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) {
    *why = "not 16-byte aligned";
    return false;
  }
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the non-sticky error
    *why = "not a CUDA pointer";
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) {
    *why = a.type == cudaMemoryTypeHost ? "page-locked host memory, not device memory"
                                        : "host memory, not device memory";
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || a.device != dev) {
    *why = "memory of another device";
    return false;
  }
  return true;
}

}  // namespace

namespace osar {
// Called by osar_create with the context's device current: look the static
// array up once per device now rather than inside the first apply.
void prepare_static_scratch() {
  void* p = nullptr;
  if (scratch_address(&p) != cudaSuccess) cudaGetLastError();
}
}  // namespace osar

extern "C" osar_status osar_gram_apply_static(osar_ctx* ctx,
                                              const void* x_dev_c128,
                                              void* y_dev_c128) {
  if (!ctx) return OSAR_E_INVALID;
  if (ctx->sticky != OSAR_OK) return ctx->sticky;
  if (!x_dev_c128 || !y_dev_c128) {
    ctx->last_error = "osar_gram_apply_static: NULL vector";
    return OSAR_E_INVALID;
  }
  std::string why;
  if (!device_vector_ok(x_dev_c128, &why)) {
    ctx->last_error = "osar_gram_apply_static: x is " + why;
    return OSAR_E_INVALID;
  }
  if (!device_vector_ok(y_dev_c128, &why)) {
    ctx->last_error = "osar_gram_apply_static: y is " + why;
    return OSAR_E_INVALID;
  }
  const size_t need = osar::gram_apply_scratch_bytes(ctx);
  if (need > GRAM_APPLY_STATIC_BYTES) {
    ctx->last_error = "osar_gram_apply_static: this Gram needs " +
                      std::to_string(need) + " bytes of scratch, more than the " +
                      std::to_string(GRAM_APPLY_STATIC_BYTES) +
                      "-byte static array (M <= 4096 always fits)";
    return OSAR_E_INVALID;
  }
  void* scratch = nullptr;
  cudaError_t e = osar::settle_gram(ctx);  // a deferred update: its result
  if (e == cudaSuccess) e = scratch_address(&scratch);
  if (e == cudaSuccess)
    e = osar::launch_gram_apply_scratch(
        ctx, static_cast<const double2*>(x_dev_c128),
        static_cast<double2*>(y_dev_c128), scratch);
  if (e != cudaSuccess) {
    ctx->last_error = std::string("osar_gram_apply_static: ") +
                      cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    ctx->sticky = OSAR_E_CUDA;
    return OSAR_E_CUDA;
  }
  return OSAR_OK;
}
