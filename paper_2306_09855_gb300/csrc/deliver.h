// deliver.h -- spike delivery through the connection index (Sec. 2.3).
//
// A spike array entry names a source node, one of its connection groups
// (groups are the source's runs of equal delay, in increasing delay order)
// and a multiplicity.  Delivery adds weight * multiplicity to the input of
// the target of every connection of that group, one thread per connection.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace snc {

constexpr int kDeliverThreads = 256;
constexpr int kDeliverItems = 4;  // connections per thread and block range

struct DeliverArgs {
  const uint32_t* src;          // [n_spikes] source node (network-local id)
  const uint32_t* grp;          // [n_spikes] group index within the source (0 = smallest delay)
  const float* mult;            // [n_spikes] multiplicity
  uint64_t n_spikes;
  const uint64_t* row_ptr;      // [n_nodes + 1]
  const uint64_t* group_ptr;    // [n_nodes + 1]: p_i
  const uint64_t* group_first;  // [n_groups]
  const uint32_t* target;       // [n_syn]
  const float* weight;          // [n_syn]
  uint64_t n_nodes;
  uint64_t n_syn;
  uint32_t* sizes;              // [n_spikes]: connections of each entry's group (0 if invalid)
  uint64_t* first;              // [n_spikes]: first connection of each entry's group
  const uint64_t* offsets;      // [n_spikes + 1]: exclusive scan of sizes
  float* input;                 // [n_nodes], accumulated into
  uint32_t* err;
};

// sizes[e] = connections in entry e's group and first[e] its first
// connection; an entry outside the index sets the bounds bit of the error
// word and delivers nothing.
__global__ void deliver_size_kernel(DeliverArgs a);
// One thread per delivered connection (block ranges of
// kDeliverThreads * kDeliverItems connections).
__global__ void deliver_kernel(DeliverArgs a);

}  // namespace snc
