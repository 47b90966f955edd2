// deliver.cu -- spike delivery through the connection index (Sec. 2.3).
#include "deliver.h"

#include "snc_check.cuh"
#include "snc_internal.h"

namespace snc {

namespace {

// First connection and size of group k of source s, or false if the entry
// is outside the index.
__device__ __forceinline__ bool group_range(const DeliverArgs& a, uint32_t s, uint32_t k, uint64_t& start,
                                            uint64_t& size) {
  if (s >= a.n_nodes) return false;
  const uint64_t g0 = a.group_ptr[s], g1 = a.group_ptr[s + 1];
  if (static_cast<uint64_t>(k) >= g1 - g0) return false;
  const uint64_t g = g0 + k;
  start = a.group_first[g];
  const uint64_t end = g + 1 < g1 ? a.group_first[g + 1] : a.row_ptr[s + 1];
  if (end < start || end > a.n_syn) return false;
  size = end - start;
  return true;
}

}  // namespace

__global__ void deliver_size_kernel(DeliverArgs a) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t e = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < a.n_spikes; e += stride) {
    uint64_t start = 0, size = 0;
    if (!group_range(a, a.src[e], a.grp[e], start, size) || size > 0xFFFFFFFFull) {
      atomicOr(a.err, kErrBounds);
      size = 0;
    }
    a.sizes[e] = static_cast<uint32_t>(size);
    a.first[e] = start;
  }
}

__global__ void __launch_bounds__(kDeliverThreads) deliver_kernel(DeliverArgs a) {
  constexpr uint64_t kRange = static_cast<uint64_t>(kDeliverThreads) * kDeliverItems;
  __shared__ uint64_t e_lo, e_hi;  // entries holding the range's first and last connection
  const uint64_t total = a.offsets[a.n_spikes];
  // Largest e in [lo, hi] with offsets[e] <= q.
  const auto entry_of = [&](uint64_t q, uint64_t lo, uint64_t hi) {
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) >> 1;
      if (a.offsets[mid] <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  for (uint64_t q0 = static_cast<uint64_t>(blockIdx.x) * kRange; q0 < total; q0 += gridDim.x * kRange) {
    const uint64_t q_last = q0 + kRange - 1 < total ? q0 + kRange - 1 : total - 1;
    if (threadIdx.x == 0) {
      e_lo = entry_of(q0, 0, a.n_spikes - 1);
      e_hi = entry_of(q_last, e_lo, a.n_spikes - 1);
    }
    __syncthreads();
    const uint64_t lo = e_lo, hi = e_hi;
#pragma unroll
    for (int j = 0; j < kDeliverItems; ++j) {
      const uint64_t q = q0 + static_cast<uint64_t>(j) * kDeliverThreads + threadIdx.x;
      if (q >= total) break;
      const uint64_t e = entry_of(q, lo, hi);
      const uint64_t c = a.first[e] + (q - a.offsets[e]);  // invalid entries own no q
      if (!SNC_IN_BOUNDS(a.err, 40u, c, a.n_syn)) continue;
      const uint32_t t = a.target[c];
      if (!SNC_IN_BOUNDS(a.err, 41u, t, a.n_nodes)) continue;
      atomicAdd(a.input + t, a.weight[c] * a.mult[e]);
    }
    __syncthreads();  // e_lo / e_hi are rewritten
  }
}

}  // namespace snc
