// smc_trace.h -- NVTX ranges (domain "libsmc") around the library's entry
// points and, in the profiling step, around each stage.  They mark host-side
// enqueue intervals; a profiler that attaches to the process (Nsight Systems,
// Nsight Compute's range mode) shows them beside the kernels.  NVTX v3 is
// header-only: with no tool attached a range costs a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace smc {

inline nvtxDomainHandle_t nvtx_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("libsmc");
  return d;
}

inline void range_push(const char* name) {
  nvtxEventAttributes_t a{};
  a.version = NVTX_VERSION;
  a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  a.messageType = NVTX_MESSAGE_TYPE_ASCII;
  a.message.ascii = name;
  nvtxDomainRangePushEx(nvtx_domain(), &a);
}

inline void range_pop() { nvtxDomainRangePop(nvtx_domain()); }

struct Range {
  explicit Range(const char* name) { range_push(name); }
  ~Range() { range_pop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

}  // namespace smc

// one range per scope, closed when the scope ends (every return path)
#define SMC_RANGE(name) ::smc::Range smc_scope_range_(name)
