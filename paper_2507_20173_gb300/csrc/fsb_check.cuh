// fsb_check.cuh -- run-time invariant checks of the debug build.
//
// Built with -DFSB_DEBUG_BOUNDS (build.py's debug library), a failed check
// latches FSB_ERR_STATE in the launch's status word, records the check's
// site, and returns false so the caller clamps the offending extent and
// every access stays in bounds (control flow stays uniform, so no barrier
// is skipped).  The release build compiles the checks away.
#pragma once

#include <cuda_runtime.h>

#include "fsb_internal.h"

namespace fsb {

__device__ __forceinline__ bool fsb_check(bool ok, int* status, unsigned* site, unsigned id) {
#ifdef FSB_DEBUG_BOUNDS
  if (!ok && atomicCAS(status, 0, static_cast<int>(FSB_ERR_STATE)) == 0) atomicExch(site, id);
  return ok;
#else
  (void)status;
  (void)site;
  (void)id;
  return true;
#endif
}

}  // namespace fsb
