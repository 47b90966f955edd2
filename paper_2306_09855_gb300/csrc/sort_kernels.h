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
  int group_tiles;  // tiles per look-back unit (1, 4 or 8); 0 = bulk-copy kernel
  int items;        // bulk-copy kernel: keys per thread (8, 12 or 16)
  int shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
};

// Arguments of one pass over (key K, value V) pairs.  K is uint32_t or
// uint64_t, V uint32_t or uint64_t.
template <typename K, typename V>
struct OnesweepArgs {
  const K* keys_in;
  const V* vals_in;
  K* keys_out;
  V* vals_out;
  uint64_t n;
  int shift;
  uint32_t mask;
  const uint64_t* digit_start;  // global exclusive digit offsets of this pass
  uint64_t* status;             // look-back words [group][digit]
  uint32_t* tile_counter;       // dynamic group tickets, zero before the pass
  uint32_t epoch;               // 1..16383, distinct for every pass sharing `status`
  uint32_t* err;
  // Bound of every look-back wait (iterations) and a tile that publishes no
  // look-back word (0xFFFFFFFF = none): the second makes the waits of the
  // tiles after it expire, which tests use to reach the TIMEOUT path.
  uint32_t lookback_spin_limit;
  uint32_t withhold_unit;
  uint32_t* status32;           // bulk-copy kernel: 32-bit words [tile][digit], cleared per pass
  // Last pass of a build's sort: write the sorted values as separate target,
  // weight and delay arrays instead of vals_out (null otherwise).
  uint32_t* unpack_target;
  uint32_t* unpack_weight;
  uint16_t* unpack_delay;
  uint32_t unpack_delay_mask;
  // Segmented sort (bulk-copy kernel only): n_seg independent ranges
  // [seg_begin[s], seg_end[s]) with their tiles numbered from
  // seg_tile_begin[s]; digit_start then holds seg_digit_stride entries per
  // segment.  n_seg = 0: one range [0, n).
  int n_seg;
  const uint64_t* seg_begin;
  const uint64_t* seg_end;
  const uint32_t* seg_tile_begin;
  uint64_t seg_digit_stride;
};

// Separate output arrays of the last pass for (source, delay) keys with
// (target << 32 | weight bits) values.
struct SortUnpack {
  uint32_t* target;
  uint32_t* weight;
  uint16_t* delay;
  uint32_t delay_mask;
};

// Sort parameters chosen by the tuner: widest digit (8..11 bits) and tiles
// per look-back unit (1, 4, 8).
struct SortTuning {
  int max_digit_bits;
  int group_tiles;
  int items;      // keys per thread of the bulk-copy kernel
};
extern SortTuning g_sort_tuning;

// Look-back bound and withheld tile of later sorts (snc_set_wait_test).
struct WaitTest {
  uint32_t lookback_spin_limit;
  uint32_t withhold_unit;
};
extern WaitTest g_wait_test;
constexpr uint32_t kDefaultSpinLimit = 1u << 22;

SortPasses plan_passes(int key_bits);  // with g_sort_tuning
SortPasses plan_passes(int key_bits, const SortTuning& tune);
int onesweep_group(const SortPasses& sp);  // keys per look-back unit
// n_tiles / n_seg: the tiles and segments of a segmented sort (0 otherwise).
size_t sort_scratch_bytes(uint64_t n, const SortPasses& sp, uint64_t n_tiles = 0, int n_seg = 0);
// Where the parts of the sort's scratch live (sort_scratch_bytes in total).
struct SortScratch {
  uint64_t* status;
  size_t status_bytes;
  size_t hist_bytes;
  unsigned long long* hist;  // [kMaxPasses][kMaxRadix] digit counts
  uint64_t* start;           // [kMaxPasses][kMaxRadix] exclusive digit offsets
  uint32_t* counters;        // tile tickets, one per pass
};
SortScratch sort_scratch_layout(void* scratch, uint64_t n, const SortPasses& sp, uint64_t n_tiles = 0, int n_seg = 0);

// Independent ranges sorted by one launch per pass (a batched build's
// networks).  Device arrays: begin/end [n_seg], tile_begin [n_seg + 1] with
// tiles of onesweep_group(sp) keys; n_tiles = tile_begin[n_seg] (host copy).
// Every begin must be a multiple of 4.
struct SortSegments {
  int n_seg;
  const uint64_t* begin;
  const uint64_t* end;
  const uint32_t* tile_begin;
  uint64_t n_tiles;
  uint64_t max_len;  // longest segment (host copy)
};

// Stable LSD sort of n (key, value) pairs on the planned digits.
// hist_ready: the digit counts are already in the scratch's hist area (for
// example accumulated by the kernels that produced the keys).  Instantiated
// for (uint64_t, uint32_t), (uint32_t, uint64_t) and (uint64_t, uint64_t).
// unpack (64-bit values only): the last pass writes unpack's arrays instead
// of vals_out (which it then leaves untouched); *fused reports whether it did.
template <typename K, typename V>
cudaError_t radix_sort_run(const K* keys_in, const V* vals_in, K* keys_out, V* vals_out, K* keys_tmp, V* vals_tmp,
                           uint64_t n, const SortPasses& sp, void* scratch, uint32_t* err, cudaStream_t st,
                           cudaEvent_t* pass_events, bool hist_ready = false, const SortUnpack* unpack = nullptr,
                           bool* fused = nullptr, const SortSegments* segs = nullptr);

}  // namespace snc
