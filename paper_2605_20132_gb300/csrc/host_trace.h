// NVTX ranges around the C-ABI calls that enqueue GPU work, so that a
// timeline profiler shows each push by name.  NVTX v3 is header-only: with no
// tool attached a range costs a few nanoseconds and no library is linked.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace filark {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace filark
