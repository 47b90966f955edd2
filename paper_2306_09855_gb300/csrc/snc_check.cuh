// snc_check.cuh -- optional device-side bounds checks (build with
// SNC_BOUNDS_CHECK defined).  A failed check skips the access and records
// the first offender (site id, index, limit) in the context's error block:
// err[0] |= kErrBounds; err[2] = site; err[4..5] = index; err[6..7] = limit.
#pragma once

#include <cstdint>

#ifdef SNC_BOUNDS_CHECK
__device__ __forceinline__ bool snc_in_bounds(uint32_t* err, uint32_t site, uint64_t idx, uint64_t limit) {
  if (idx < limit) return true;
  if (err) {
    atomicOr(err, 4u);
    if (atomicCAS(err + 2, 0u, site) == 0u) {
      err[4] = static_cast<uint32_t>(idx);
      err[5] = static_cast<uint32_t>(idx >> 32);
      err[6] = static_cast<uint32_t>(limit);
      err[7] = static_cast<uint32_t>(limit >> 32);
    }
  }
  return false;
}
#define SNC_IN_BOUNDS(err, site, idx, limit) snc_in_bounds((err), (site), (idx), (limit))
#else
#define SNC_IN_BOUNDS(err, site, idx, limit) true
#endif
