// Named ranges for timeline profilers: every public entry point (and each batch the
// serving runtime launches) opens a range in the "pm" domain.  NVTX v3 is header-only
// and costs a few instructions when no profiler is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace pm_trace {

inline nvtxDomainHandle_t domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("pm");
  return d;
}

struct Range {
  explicit Range(const char *name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(domain(), &a);
  }
  ~Range() { nvtxDomainRangePop(domain()); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

}  // namespace pm_trace

#define PM_TRACE(name) pm_trace::Range pm_trace_range_(name)
