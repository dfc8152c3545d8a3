// trace.h -- NVTX ranges around the host phases of the path (hoisting, launches, waiting for
// results, assembly, minimiser steps, the batch and server phases), for profilers that record
// NVTX (ncu --nvtx, Nsight Systems).  NVTX v3 is header-only: without an attached tool a range
// costs one call through a null-checked function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace gbnll {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace gbnll

#define GBNLL_TRACE_CAT2(a, b) a##b
#define GBNLL_TRACE_CAT(a, b) GBNLL_TRACE_CAT2(a, b)
// a range from here to the end of the enclosing scope
#define GBNLL_TRACE(name) ::gbnll::TraceRange GBNLL_TRACE_CAT(gbnll_trace_, __LINE__)(name)
