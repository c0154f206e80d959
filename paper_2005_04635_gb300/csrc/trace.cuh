// trace.cuh -- NVTX ranges around the C ABI's compute calls, so a profiler's
// timeline shows init / iterate / measure / phase sweeps by name.  Without an
// attached tool the NVTX calls return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace grv {
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace grv

#define GROVER_TRACE(name) ::grv::TraceRange grover_trace_range_(name)
