// copass.h -- COPASS block sort (Appendix A of the paper): a stable sort of
// (key, value) pairs that keeps the array's division in blocks and needs,
// besides the array itself, two blocks of working memory instead of a
// second copy of the whole array.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sort_kernels.h"

namespace snc {

constexpr int kCopassMaxRuns = 256;  // blocks (runs) of one sort
constexpr uint64_t kCopassAlign = 1024;  // block sizes are multiples of this (16-byte aligned bulk copies)

// Working memory of copass_sort_run: two blocks of (key, value) pairs, the
// radix sort scratch of one block, and the run tables.
size_t copass_scratch_bytes(uint64_t block, int key_bytes, int val_bytes, const SortPasses& sp);

// Sorts keys[0..n) with vals stably by the planned digits, in place, in
// blocks of `block` pairs (a multiple of kCopassAlign; at most
// kCopassMaxRuns blocks):
//   1. every block is sorted on its own (the onesweep radix sort);
//   2. for output block o: the COPASS partition of the remaining runs
//      (copass_partition_kernel) gives each run's share of the block's
//      pairs; the shares are gathered into the auxiliary block, the rest of
//      every run is shifted to the end of the array (windows of one block,
//      from the end), and the auxiliary block is sorted into block o's place.
// Runs keep their original order, so equal keys keep theirs (stable).
// scratch: copass_scratch_bytes(block, ...) bytes of device memory.
template <typename K, typename V>
cudaError_t copass_sort_run(K* keys, V* vals, uint64_t n, uint64_t block, const SortPasses& sp, void* scratch,
                            uint32_t* err, cudaStream_t st);

}  // namespace snc
