// NVTX ranges around the library's entry points, so that a profiler's
// timeline (Nsight Systems, or ncu --nvtx) shows which call launched which
// kernels.  NVTX v3 is header-only: without a tool attached each range costs
// a check of a function pointer and nothing is recorded.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace glbm_trace {

struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace glbm_trace
