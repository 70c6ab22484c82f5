// Guard regions behind device allocations (a sanitizer substitute).
//
// With guards on (osar_config.guard_bytes > 0) every buffer a context or a
// batch allocates gets guard_bytes more, filled with GUARD_BYTE right after
// the buffer's own bytes; check_guards copies each guard back and counts the
// ones whose bytes changed, i.e. buffers that a kernel wrote past their end.
// The buffer itself keeps its alignment (the guard follows it).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace osar {

constexpr unsigned char GUARD_BYTE = 0xA5;

struct GuardRegion {
  std::string name;     // the buffer (its allocation expression)
  unsigned char* addr;  // first guard byte (just past the buffer)
};

struct Guards {
  size_t bytes = 0;  // guard bytes per allocation, 0: off
  std::vector<GuardRegion> regions;
};

// cudaMalloc of `bytes` (+ the guard), the buffer zeroed and the guard
// filled on `st`; *total gets the bytes allocated.
cudaError_t guarded_malloc(Guards& g, void** p, size_t bytes, const char* name,
                           cudaStream_t st, size_t* total);

// Synchronises `st`, then counts the guards that changed; *first gets the
// first such buffer's name.
cudaError_t check_guards(const Guards& g, cudaStream_t st, int* bad,
                         std::string* first);

}  // namespace osar
