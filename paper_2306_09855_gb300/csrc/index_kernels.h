// index_kernels.h -- interface of the unpack / group-index kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace snc {

constexpr int kIndexThreads = 256;
constexpr int kIndexItems = 8;
constexpr int kIndexTile = kIndexThreads * kIndexItems;

struct IndexArgs {
  const void* keys;          // sorted (source, delay) keys: uint32_t when key32, else uint64_t
  const uint64_t* vals;      // sorted (target, weight) values
  int key32;
  int unpacked;              // the sort already wrote target / delay / weight: starts only
  uint64_t n;
  int delay_bits;
  uint32_t* target;
  uint16_t* delay;
  uint32_t* weight;          // fp32 bits
  uint32_t* starts;          // group-start bitmap, kIndexTile / 32 words per block
  uint32_t* block_counts;    // group starts per block
  const uint64_t* block_offsets;  // exclusive scan of block_counts (n_blocks + 1)
  uint64_t* group_first;
  uint64_t group_cap;
  uint64_t* n_groups;
  uint32_t* err;
};

struct NodeIndexArgs {
  const void* keys;
  int key32;
  uint64_t n;
  uint64_t n_nodes;
  int delay_bits;
  const uint64_t* group_first;
  uint64_t group_cap;
  const uint64_t* n_groups;
  uint64_t* row_ptr;
  uint64_t* group_ptr;
};

// Launch the unpack / node-index kernel for the key width of the build.
cudaError_t launch_index_unpack(const IndexArgs& a, unsigned grid, cudaStream_t st);
__global__ void index_groups_kernel(IndexArgs a);
cudaError_t launch_node_index(const NodeIndexArgs& a, cudaStream_t st);
__global__ void expand_sources_kernel(const uint64_t* row_ptr, uint64_t n_nodes, uint32_t* src);

// Batches: per-network CSR offsets relative to the network's first
// connection / group, and group starts relative to its first connection.
struct RebaseArgs {
  const uint64_t* row_ptr;     // global node CSR of the build [total_nodes + 1]
  const uint64_t* group_ptr;   // [total_nodes + 1]
  const uint64_t* node_base;   // first global node of each network [n_nets + 1]
  const uint64_t* local_base;  // first entry of each network's local arrays [n_nets]
  int n_nets;
  uint64_t total_nodes;
  uint64_t* row_local;         // concatenated per-network arrays of (n + 1) entries
  uint64_t* group_local;
  uint64_t* group_first;       // rebased in place
  uint64_t n_groups_cap;
  const uint64_t* n_groups;
};
__global__ void rebase_nodes_kernel(RebaseArgs a);
__global__ void rebase_groups_kernel(RebaseArgs a);

}  // namespace snc
