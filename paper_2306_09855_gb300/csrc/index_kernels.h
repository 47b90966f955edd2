// index_kernels.h -- interface of the unpack / group-index kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace snc {

constexpr int kIndexThreads = 256;
constexpr int kIndexItems = 8;
constexpr int kIndexTile = kIndexThreads * kIndexItems;

struct IndexArgs {
  const uint64_t* keys;  // sorted packed keys
  uint64_t n;
  int node_bits, delay_bits;
  uint32_t* target;
  uint16_t* delay;
  uint32_t* starts;          // group-start bitmap, kIndexTile / 32 words per block
  uint32_t* block_counts;    // group starts per block
  const uint64_t* block_offsets;  // exclusive scan of block_counts (n_blocks + 1)
  uint64_t* group_first;
  uint64_t group_cap;
  uint64_t* n_groups;
  uint32_t* err;
};

struct NodeIndexArgs {
  const uint64_t* keys;
  uint64_t n;
  uint64_t n_nodes;
  int node_bits, delay_bits;
  const uint64_t* group_first;
  uint64_t group_cap;
  const uint64_t* n_groups;
  uint64_t* row_ptr;
  uint64_t* group_ptr;
};

__global__ void index_unpack_kernel(IndexArgs a);
__global__ void index_groups_kernel(IndexArgs a);
__global__ void node_index_kernel(NodeIndexArgs a);
__global__ void expand_sources_kernel(const uint64_t* row_ptr, uint64_t n_nodes, uint32_t* src);

}  // namespace snc
