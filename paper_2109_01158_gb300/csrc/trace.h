// trace.h -- NVTX ranges around the library's public calls, so that a timeline profiler
// (Nsight Systems, or any NVTX consumer) shows which call enqueued which kernels.  NVTX is
// header-only: without a profiler attached a range costs a branch on a null pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace fe {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace fe

#define FE_TRACE(name) ::fe::TraceRange fe_trace_range_(name)
