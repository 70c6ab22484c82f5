// NVTX ranges over the library's calls, so that a timeline profiler shows
// which call queued which kernels (header-only NVTX 3; with no tool
// attached a range costs a few nanoseconds).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace osar {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace osar
