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
  // Networks of the build: positions [seg_begin[m], seg_end[m]) hold network
  // m's connections; positions between them belong to none.
  int n_seg;
  const uint64_t* seg_begin;
  const uint64_t* seg_end;
};

// Per-network CSR and group offsets.  Network m owns entries
// [local_base[m], local_base[m] + n_nodes_m + 1) of row_local / group_local:
// row_local = first position (relative to seg_begin[m]) whose source is >= i,
// group_local = groups of the network before it.  gfirst[m] = first group of
// network m, gfirst[n_members] = all groups.
struct MemberIndexArgs {
  const void* keys;
  int key32;
  int delay_bits;
  int n_members;
  const uint64_t* seg_begin;
  const uint64_t* seg_end;
  const uint64_t* local_base;
  uint64_t n_entries;  // nodes of all networks + n_members
  const uint64_t* group_first;
  uint64_t group_cap;
  const uint64_t* n_groups;
  uint64_t* row_local;
  uint64_t* group_local;
  uint64_t* gfirst;
};

// Launch the unpack / node-index kernel for the key width of the build.
cudaError_t launch_index_unpack(const IndexArgs& a, unsigned grid, cudaStream_t st);
__global__ void index_groups_kernel(IndexArgs a);
cudaError_t launch_member_index(const MemberIndexArgs& a, cudaStream_t st);
// group_first[g] -= seg_begin of the network that owns group g.
__global__ void rebase_group_first_kernel(uint64_t* group_first, const uint64_t* n_groups, uint64_t group_cap,
                                          const uint64_t* gfirst, const uint64_t* seg_begin, int n_members);
__global__ void expand_sources_kernel(const uint64_t* row_ptr, uint64_t n_nodes, uint32_t* src);
// Target shards: flag the connections whose target is in [first, first +
// count), then keep them in generation order.
__global__ void shard_flag_kernel(const uint64_t* vals, uint64_t n, uint32_t first, uint32_t count, uint32_t* flags);
__global__ void shard_compact_kernel(const void* keys_in, const uint64_t* vals_in, int key32, uint64_t n,
                                     const uint64_t* offsets, uint32_t first, uint32_t count, void* keys_out,
                                     uint64_t* vals_out);

// In-place unpack after a block sort: targets over vals (as uint32), weight
// bits over keys (as uint32), delays into `delay`; tk / tv: a temporary
// block of `window` keys and values.
cudaError_t unpack_in_place(void* keys, int key32, uint64_t* vals, uint64_t n, uint64_t window, void* tk,
                            uint64_t* tv, uint32_t delay_mask, uint16_t* delay, int sms, cudaStream_t st);

}  // namespace snc
