// index_kernels.cu -- unpacking of the sorted keys and the group index of
// Sec. 2.2.
//
// A connection starts a group when its source or its delay differs from the
// previous connection's.  group_first[g] is the position of the g-th group
// start (a stream compaction whose tile offsets come from a decoupled
// look-back scan), row_ptr[i] the first connection of source i and
// group_ptr[i] = p_i = sum_{j<i} G_j the first group of source i (both found
// by binary search, one thread per node).
#include <cuda_runtime.h>

#include <cstdint>

#include "index_kernels.h"
#include "snc_check.cuh"
#include "snc_internal.h"

namespace snc {

namespace {
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;
}  // namespace

__global__ void __launch_bounds__(kIndexThreads) index_kernel(IndexArgs a) {
  constexpr int NW = kIndexThreads / 32;
  __shared__ uint32_t tile_sh;
  __shared__ uint32_t cnt[kIndexItems][NW];
  __shared__ uint64_t group_base_sh;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) tile_sh = atomicAdd(a.tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = tile_sh;
  const uint64_t base = static_cast<uint64_t>(tile) * kIndexTile;
  const int sd_shift = a.node_bits;
  const uint64_t node_mask = (1ull << a.node_bits) - 1;
  const uint32_t delay_mask = (1u << a.delay_bits) - 1u;
  uint32_t flags = 0;  // bit k: element k starts a group
#pragma unroll
  for (int k = 0; k < kIndexItems; ++k) {
    const uint64_t q = base + static_cast<uint64_t>(k) * kIndexThreads + tid;
    bool start = false;
    if (q < a.n) {
      const uint64_t key = a.keys[q];
      a.target[q] = static_cast<uint32_t>(key & node_mask);
      a.delay[q] = static_cast<uint16_t>((key >> sd_shift) & delay_mask);
      start = q == 0 || (key >> sd_shift) != (a.keys[q - 1] >> sd_shift);
    }
    const uint32_t b = __ballot_sync(0xffffffffu, start);
    if (lane == 0) cnt[k][warp] = __popc(b);
    if (start) flags |= 1u << k;
  }
  __syncthreads();
  // Exclusive offsets in tile order (k-major, then warp, then lane).
  if (tid == 0) {
    uint32_t run = 0;
    for (int k = 0; k < kIndexItems; ++k)
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = cnt[k][w];
        cnt[k][w] = run;
        run += c;
      }
    // Look-back over tiles for the number of groups before this tile.
    uint64_t* st = a.status + tile;
    const uint64_t total = run;
    *reinterpret_cast<volatile unsigned long long*>(st) = (tile == 0 ? kFlagInc : kFlagAgg) | total;
    uint64_t prefix = 0;
    if (tile > 0) {
      int64_t look = static_cast<int64_t>(tile) - 1;
      uint32_t spins = 0;
      while (look >= 0) {
        const uint64_t v = *reinterpret_cast<const volatile unsigned long long*>(a.status + look);
        const uint64_t f = v & (3ull << 62);
        if (f == 0) {
          if (++spins > kSpinLimit) {
            atomicOr(a.err, kErrLookbackTimeout);
            break;
          }
          continue;
        }
        prefix += v & kValMask;
        if (f == kFlagInc) break;
        --look;
      }
      *reinterpret_cast<volatile unsigned long long*>(st) = kFlagInc | (prefix + total);
    }
    group_base_sh = prefix;
    if (base + kIndexTile >= a.n) *a.n_groups = prefix + total;  // last tile
  }
  __syncthreads();
  const uint64_t g0 = group_base_sh;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kIndexItems; ++k) {
    const bool start = (flags >> k) & 1u;
    const uint32_t b = __ballot_sync(0xffffffffu, start);
    if (start) {
      const uint64_t g = g0 + cnt[k][warp] + __popc(b & lt);
      const uint64_t q = base + static_cast<uint64_t>(k) * kIndexThreads + tid;
      if (g < a.group_cap) a.group_first[g] = q;
      else atomicOr(a.err, kErrBounds);
    }
  }
}

// row_ptr[i] = first position whose source is >= i; group_ptr[i] = number of
// group starts before row_ptr[i].  i = 0 .. n_nodes.
__global__ void node_index_kernel(NodeIndexArgs a) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > a.n_nodes) return;
  const int src_shift = a.node_bits + a.delay_bits;
  uint64_t lo = 0, hi = a.n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if ((a.keys[mid] >> src_shift) < i) lo = mid + 1; else hi = mid;
  }
  if (!SNC_IN_BOUNDS(nullptr, 21u, lo, a.n + 1)) return;
  a.row_ptr[i] = lo;
  const uint64_t ng = *a.n_groups;
  uint64_t glo = 0, ghi = ng < a.group_cap ? ng : a.group_cap;
  while (glo < ghi) {
    const uint64_t mid = (glo + ghi) >> 1;
    if (a.group_first[mid] < lo) glo = mid + 1; else ghi = mid;
  }
  a.group_ptr[i] = glo;
}

// Source of every connection from row_ptr (for host copies).
__global__ void expand_sources_kernel(const uint64_t* row_ptr, uint64_t n_nodes, uint32_t* src) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  for (uint64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) src[q] = static_cast<uint32_t>(i);
}

}  // namespace snc
