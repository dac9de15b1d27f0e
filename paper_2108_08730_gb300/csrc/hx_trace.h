// NVTX ranges around the phases of a solve and of a served request, for
// timeline tools (Nsight Systems).  NVTX v3 is header-only; without a tool
// attached a range costs a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace hx {

// A range pushed on construction and popped at end() or destruction.
class TraceRange {
 public:
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
  void end() {
    if (open_) nvtxRangePop();
    open_ = false;
  }
  ~TraceRange() { end(); }

 private:
  bool open_ = true;
};

}  // namespace hx
