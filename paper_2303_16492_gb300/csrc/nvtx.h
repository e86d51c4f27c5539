// NVTX ranges on the host side of every launch sequence (the header-only
// NVTX v3 API: no library to link; the calls cost a pointer test unless a
// profiler is attached), so that a timeline shows each iteration, each
// kernel launch of the whole-GPU path and each evaluation by name.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace trsgd {

struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace trsgd
