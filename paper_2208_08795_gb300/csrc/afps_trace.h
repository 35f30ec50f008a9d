// afps_trace.h -- NVTX ranges around the library's host entry points, so that
// a profiler's timeline (nsys, ncu's NVTX filters) shows which call issued
// which kernels.  NVTX3 is header-only: without an attached tool a range is
// a couple of function calls into a no-op stub.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace afps {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace afps

#define AFPS_TRACE(name) ::afps::TraceRange afps_trace_range_(name)
