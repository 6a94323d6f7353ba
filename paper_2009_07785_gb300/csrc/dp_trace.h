// Names the library's calls on a profiler's timeline: an NVTX range per
// C-ABI call (and per launch group of a node batch).  NVTX v3 is header-only;
// without an attached tool a range costs a call through a null hook.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace dp {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace dp
