// NVTX ranges around the library's phases -- setup, factorization, right-hand side, solve,
// each GMRES cycle and each true-residual evaluation -- the counterparts of the paper's
// T_s / T_a / T_p columns in a Nsight timeline.  Without a tool attached a range costs a
// check of an unset function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace ls {

struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

}  // namespace ls
