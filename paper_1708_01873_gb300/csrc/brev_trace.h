// NVTX ranges around the library's entry points.  A profiler that reads
// NVTX (Nsight Systems, ncu's --nvtx filters) shows every call that enqueues
// work as a range named after the entry point, in the "brev" domain, on the
// calling thread.  NVTX v3 is header-only: with no tool attached, a push or
// pop is one call through a pointer to an empty function.  Compile with
// -DBREV_NO_NVTX to leave the ranges out.
#pragma once

#ifndef BREV_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace brev {

class TraceRange {
 public:
  explicit TraceRange(const char* name) {
#ifndef BREV_NO_NVTX
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(domain(), &a);
#else
    (void)name;
#endif
  }
  ~TraceRange() {
#ifndef BREV_NO_NVTX
    nvtxDomainRangePop(domain());
#endif
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;

 private:
#ifndef BREV_NO_NVTX
  static nvtxDomainHandle_t domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("brev");
    return d;
  }
#endif
};

}  // namespace brev

#define BREV_TRACE(name) ::brev::TraceRange brev_trace_range_(name)
