// digit_hist.cuh -- per-pass digit histograms of packed sort keys, counted
// in shared memory and merged into global 64-bit counters.  Used by the
// generation kernels (the keys are at hand when they are produced) and by the
// standalone sort's histogram kernel.
#pragma once

#include <cstdint>

#include "sort_kernels.h"

namespace snc {

// Digit plan of the passes as the counting code needs it.
struct HistPlan {
  unsigned long long* global;  // [n_passes * stride] counters; null = no counting
  int n_passes;
  int stride;                  // bins per pass (1 << kernel digit width)
  int shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
};

// Shifts and masks held in registers (the loops below are unrolled over the
// maximum pass count, so nothing is indexed dynamically).
struct HistRegs {
  int n;
  int stride;
  int shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
};

__device__ __forceinline__ HistRegs hist_regs(const HistPlan& p) {
  HistRegs r;
  r.n = p.global ? p.n_passes : 0;
  r.stride = p.stride;
#pragma unroll
  for (int i = 0; i < kMaxPasses; ++i) {
    r.shift[i] = p.shift[i];
    r.mask[i] = p.mask[i];
  }
  return r;
}

__device__ __forceinline__ void hist_clear(uint32_t* sh, const HistRegs& r) {
  for (int i = threadIdx.x; i < r.n * r.stride; i += blockDim.x) sh[i] = 0u;
}

__device__ __forceinline__ void hist_add(uint32_t* sh, const HistRegs& r, uint64_t key) {
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p)
    if (p < r.n) atomicAdd(&sh[p * r.stride + (static_cast<uint32_t>(key >> r.shift[p]) & r.mask[p])], 1u);
}

__device__ __forceinline__ void hist_flush(const uint32_t* sh, const HistRegs& r, unsigned long long* global) {
  for (int i = threadIdx.x; i < r.n * r.stride; i += blockDim.x) {
    const uint32_t v = sh[i];
    if (v) atomicAdd(&global[(i / r.stride) * kMaxRadix + (i % r.stride)], static_cast<unsigned long long>(v));
  }
}

HistPlan hist_plan(const SortPasses& sp, unsigned long long* global);

inline size_t hist_smem_bytes(const HistPlan& p) {
  return p.global ? static_cast<size_t>(p.n_passes) * p.stride * sizeof(uint32_t) : 0;
}

}  // namespace snc
