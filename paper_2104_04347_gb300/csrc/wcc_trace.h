// NVTX ranges around the public calls that launch work or move data, so that
// a profiler (ncu --nvtx, Nsight Systems) can attribute kernels and copies to
// the API call that issued them.  NVTX3 is header-only; without a tool
// attached each range costs one predictable branch.
#pragma once
#include <nvtx3/nvToolsExt.h>

struct WccTraceRange {
    explicit WccTraceRange(const char* name) { nvtxRangePushA(name); }
    ~WccTraceRange() { nvtxRangePop(); }
    WccTraceRange(const WccTraceRange&) = delete;
    WccTraceRange& operator=(const WccTraceRange&) = delete;
};
