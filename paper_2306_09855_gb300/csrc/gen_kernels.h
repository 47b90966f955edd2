// gen_kernels.h -- launch interface of the generation kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "digit_hist.cuh"
#include "snc_internal.h"

namespace snc {

constexpr int kGenThreads = 256;
constexpr int kChunk = 4096;  // connections per generation chunk
// Sampler: one bitmap of the candidate range per warp in shared memory.
constexpr size_t kSamplerSmem = 200 * 1024;
constexpr uint64_t kSamplerMaxNodes = 1u << 20;

struct GenArgs {
  const DevProj* projs;
  int n_proj;
  uint64_t total_chunks;
  const uint32_t* thr_blob;
  const uint16_t* guide_blob;
  uint32_t max_delay_len;  // largest delay table among the launched projections
  KeyLayout layout;
  uint64_t* keys;
  uint32_t* vals;
  uint64_t cap;    // entries of keys / vals
  uint32_t* err;   // device error block (bounds checks)
  HistPlan hist;   // digit counts of the sort's passes, accumulated as keys are written
};

struct SamplerArgs {
  GenArgs gen;               // output arrays and layout
  const DevProj* proj;       // the one projection handled by the launch
  const uint32_t* thr_blob;
  const uint16_t* guide_blob;
  uint32_t max_delay_len;
  uint32_t bitmap_words;     // per warp
  const uint64_t* prim_offsets;  // Bernoulli: per-target offsets (n_primary + 1)
  uint32_t* err;
};

__global__ void gen_direct_kernel(GenArgs a);
__global__ void bernoulli_count_kernel(const DevProj* proj, const uint32_t* thr_blob,
                                       const uint16_t* guide_blob, uint32_t* counts);
__global__ void sampler_kernel(SamplerArgs a);

// fixed_total_number with autapses or multapses forbidden.
struct TotalArgs {
  const DevProj* proj;
  uint64_t* pairs;        // per slot: (source << 32) | target, global ids
  uint64_t* table_keys;   // open-addressing hash table of pairs (~0 = empty)
  uint64_t* table_vals;   // accepted: slot; claimed this round: 2^63 | slot
  uint64_t table_mask;
  // Packed table (one word per entry, used when it fits):
  // (pair_local << (slot_bits + 1)) | (claimed_this_round << slot_bits) | slot
  int packed;
  int slot_bits;
  int t_bits;           // bits of the target's local index in pair_local
  uint8_t* lost;        // round-0 marks (packed table or no table); null: resolve pass
  uint64_t* pending;      // slots still to redraw
  uint64_t* next_pending;
  unsigned long long* n_next;  // device counter of next_pending
  uint32_t* err;
};
__global__ void total_round0_kernel(TotalArgs a);
__global__ void total_collect_kernel(TotalArgs a);
__global__ void total_claim_kernel(TotalArgs a, const uint64_t* pending, uint64_t n_pending, uint32_t round);
__global__ void total_resolve_kernel(TotalArgs a, const uint64_t* pending, uint64_t n_pending, int all_slots);
__global__ void total_emit_kernel(GenArgs g, const DevProj* proj, const uint64_t* pairs);

cudaError_t exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* block_tmp,
                               cudaStream_t st);
uint64_t scan_tmp_entries(uint64_t n);

}  // namespace snc
