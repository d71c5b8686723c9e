// NVTX ranges around the library's host-side work (header-only NVTX 3: a range costs nothing
// unless a profiler is attached). Ranges show up in nsys/ncu timelines.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace vpm {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace vpm
