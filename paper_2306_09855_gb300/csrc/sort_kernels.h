// sort_kernels.h -- interface of the onesweep radix sort.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace snc {

constexpr int kMaxPasses = 8;
constexpr int kMaxRadix = 2048;  // widest digit: 11 bits
constexpr int kDigitScanThreads = 256;

// Digit plan of one sort: pass p sorts on (key >> shift[p]) & mask[p].
struct SortPasses {
  int n_passes;
  int kernel_bits;  // digit width the pass kernel is instantiated for
  int shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
};

struct OnesweepArgs {
  const uint64_t* keys_in;
  const uint32_t* vals_in;
  uint64_t* keys_out;
  uint32_t* vals_out;
  uint64_t n;
  int shift;
  uint32_t mask;
  const uint64_t* digit_start;  // global exclusive digit offsets of this pass
  uint64_t* status;             // look-back words [tile][digit]
  uint32_t* tile_counter;       // dynamic tile ids, zero before the pass
  uint32_t epoch;               // 1..16383, distinct for every pass sharing `status`
  uint32_t* err;
};

SortPasses plan_passes(int key_bits);
int onesweep_tile(int bits);
size_t sort_scratch_bytes(uint64_t n, const SortPasses& sp);
cudaError_t radix_sort_run(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                           uint64_t* keys_tmp, uint32_t* vals_tmp, uint64_t n, const SortPasses& sp, void* scratch,
                           uint32_t* err, cudaStream_t st, cudaEvent_t* pass_events);

}  // namespace snc
