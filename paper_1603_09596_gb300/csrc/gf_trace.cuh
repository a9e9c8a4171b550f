// gf_trace.cuh -- NVTX ranges around the library's entry points and the build's levels, so that a
// profiler's timeline (ncu --nvtx, nsys) shows which call and which level a kernel belongs to.
// Host side only; without a profiler attached the NVTX calls return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

struct GfRange {
    explicit GfRange(const char *name) { nvtxRangePushA(name); }
    ~GfRange() { nvtxRangePop(); }
    GfRange(const GfRange &) = delete;
    GfRange &operator=(const GfRange &) = delete;
};
