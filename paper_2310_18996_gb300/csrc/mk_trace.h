// NVTX ranges around the C-ABI calls: a timeline profiler (Nsight Systems,
// or ncu --nvtx filters) shows each library call and the GPU work it
// enqueued.  NVTX3 is header-only; without a tool attached a range costs a
// function-pointer test.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mk {
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace mk

#define MK_TRACE(name) ::mk::TraceRange mk_trace_range_(name)
