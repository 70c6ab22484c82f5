// Guard regions behind device allocations; see guard.h.
#include "guard.h"

namespace osar {

cudaError_t guarded_malloc(Guards& g, void** p, size_t bytes, const char* name,
                           cudaStream_t st, size_t* total) {
  const size_t n = (bytes ? bytes : 16) + g.bytes;
  cudaError_t e = cudaMalloc(p, n);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  if (total) *total = n;
  e = cudaMemsetAsync(*p, 0, bytes ? bytes : 16, st);
  if (e == cudaSuccess && g.bytes) {
    unsigned char* guard = static_cast<unsigned char*>(*p) + (bytes ? bytes : 16);
    e = cudaMemsetAsync(guard, GUARD_BYTE, g.bytes, st);
    g.regions.push_back(GuardRegion{name, guard});
  }
  return e;
}

cudaError_t check_guards(const Guards& g, cudaStream_t st, int* bad,
                         std::string* first) {
  *bad = 0;
  if (!g.bytes) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(st);
  std::vector<unsigned char> h(g.bytes);
  for (const GuardRegion& r : g.regions) {
    if (e != cudaSuccess) break;
    e = cudaMemcpy(h.data(), r.addr, g.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    for (unsigned char b : h)
      if (b != GUARD_BYTE) {
        if (*bad == 0 && first) *first = r.name;
        ++*bad;
        break;
      }
  }
  return e;
}

}  // namespace osar
