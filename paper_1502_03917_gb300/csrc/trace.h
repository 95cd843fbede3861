// trace.h -- NVTX ranges of the library (internal).
//
// Host-side ranges in the "aaomg" NVTX domain around set-up, solves, refinement
// iterations, batch solves and every level's smoothing, transfer and coarse
// work, so that a timeline tool (nsys) attributes device time to the method's
// steps.  Inside a CUDA graph the ranges mark the recording of each step; the
// replays show up under the solve and iteration ranges.  Without a tool
// attached an NVTX call returns at once.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdio>

namespace aaomg {

inline nvtxDomainHandle_t trace_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("aaomg");
    return d;
}

class TraceRange {
  public:
    explicit TraceRange(const char* fmt, ...) {
        char buf[96];
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = buf;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace aaomg
