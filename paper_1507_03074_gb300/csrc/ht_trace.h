// NVTX ranges around the library's host-side calls, so that a timeline
// (Nsight Systems, or ncu --nvtx filters) shows which ABI call enqueued
// which kernels.  Header-only NVTX v3: without a tool attached each range
// costs one test of an unset function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace hte {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

} // namespace hte
