// source_major.h -- the sort of builds generated source by source.
//
// one_to_one, all_to_all and fixed_outdegree (with or without multapses)
// generate each projection's connections source after source (Sec. 2.1
// numbering: i = source * K + slot, or source row by row), so a build made
// only of such projections holds, for every source, one run per projection
// in generation order.  Its stable (source, delay) sort (Sec. 2.2) is then a
// stable counting sort of each source's runs by delay step: one read of the
// keys, one of the values, and the sorted keys, targets, weights and delays
// written at the source's CSR offset.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "snc_internal.h"

namespace snc {

constexpr int kSrcMajorMaxProj = 16;   // projections of a build on this path
constexpr int kSrcMajorMaxDelayBits = 9;
constexpr int kSrcMajorThreads = 256;
constexpr int kSrcMajorItems = 8;      // keys per thread and chunk
constexpr int kSrcMajorChunk = kSrcMajorThreads * kSrcMajorItems;
constexpr uint64_t kSrcMajorSmall = 256;  // sources up to this many connections: one warp each

struct SrcMajorArgs {
  const DevProj* projs;
  int n_proj;
  uint32_t n_nodes;          // sources [0, n_nodes) (a single network: ids are local)
  uint32_t* counts;          // connections per source
  const uint64_t* row_base;  // exclusive scan of counts (n_nodes + 1)
  const void* keys_in;       // generation order
  const uint64_t* vals_in;
  int key32;
  int delay_bits;
  void* keys_out;            // sorted keys
  uint32_t* target;          // sorted targets (network-local)
  uint32_t* weight;          // sorted fp32 weight bits
  uint16_t* delay;           // sorted delay steps
  uint64_t n;                // connections
  uint32_t* err;
  uint32_t* long_list;       // sources above kSrcMajorSmall connections (any order)
  uint32_t* n_long;          // their number
};

// True if every projection's rule generates source by source.
bool source_major_rule(uint32_t rule);

// counts[s] = connections of source s over all projections.
__global__ void src_major_count_kernel(SrcMajorArgs a);
// Stable counting sort of each source's runs by delay step: sources above
// kSrcMajorSmall connections (a block each), and the others (a warp each).
__global__ void src_major_sort_kernel(SrcMajorArgs a);
__global__ void src_major_small_kernel(SrcMajorArgs a);

}  // namespace snc
