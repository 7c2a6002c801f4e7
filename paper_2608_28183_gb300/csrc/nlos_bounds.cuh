// Index checks of the bounds-checked debug build (build flag
// NLOS_BOUNDS_CHECK; a stand-in for a device memory checker): an access whose
// element index falls outside [0, n) of its buffer records kDevErrBounds in
// the workspace's error word (read by nlos_workspace_check) and is skipped -
// no trap, the context stays usable. Extents of 0 mean "not known here" and
// pass. In normal builds every check is a constant true and compiles away.
#pragma once
#include "nlos_internal.h"

namespace nlos {

__device__ __forceinline__ bool bchk(long long i, long long n, int* err) {
#ifdef NLOS_BOUNDS_CHECK
  if (n > 0 && (i < 0 || i >= n)) {
    if (err) atomicExch(err, kDevErrBounds);
    return false;
  }
#else
  (void)i;
  (void)n;
  (void)err;
#endif
  return true;
}

}  // namespace nlos
