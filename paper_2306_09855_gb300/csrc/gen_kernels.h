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
  void* keys;      // uint32_t[cap] when key32, else uint64_t[cap]: (source, delay)
  uint64_t* vals;  // (target, weight bits)
  int key32;
  uint64_t cap;    // entries of keys / vals
  uint32_t* err;   // device error block (bounds checks)
  HistPlan hist;   // digit counts of the sort's passes, accumulated as keys are written
  ArrayBlobs arr;  // explicit arrays of the Connect calls (DevProj list offsets)
};

// One launch serves every listed sampler projection: warps take primary
// nodes of the concatenated list (prim_prefix), each warp keeping a bitmap
// and the delay table of its current projection in shared memory.
struct SamplerArgs {
  GenArgs gen;                   // output arrays and layout
  const DevProj* projs;          // projection table of the build
  const uint32_t* list;          // projections handled by the launch
  const uint64_t* prim_prefix;   // [n_list + 1] primaries before each listed projection
  int n_list;
  const uint32_t* thr_blob;
  const uint16_t* guide_blob;
  uint32_t max_delay_len;        // largest delay table among the listed projections
  uint32_t table_words;          // per-warp table area (thresholds + guide), uint32 units
  uint32_t bitmap_words;         // per-warp bitmap (largest candidate range)
  const uint64_t* prim_offsets;  // Bernoulli: exclusive scan of all per-target counts
  uint32_t* err;
};

__global__ void gen_direct_kernel(GenArgs a);
// Per-target Binomial counts of every listed pairwise_bernoulli projection
// (targets concatenated in list order, prefix[n_list] in total).
__global__ void bernoulli_count_kernel(const DevProj* projs, const uint32_t* list, const uint64_t* prefix, int n_list,
                                       const uint32_t* thr_blob, const uint16_t* guide_blob, ArrayBlobs arr,
                                       uint32_t* counts);
// out[j] = offsets[prefix[j + 1]] - offsets[prefix[j]]: connections per listed projection.
__global__ void segment_totals_kernel(const uint64_t* offsets, const uint64_t* prefix, int n_list, uint64_t* out);
__global__ void sampler_kernel(SamplerArgs a);
// Graph builds with pairwise_bernoulli projections.  Such a projection owns
// `count` positions, a capacity fixed when the graph is recorded; positions
// past the drawn total (totals[k] for list[k]) get the padding key, which
// sorts after every connection, and a zero value, and are added to the
// fused digit counts when the build counts digits in generation.
// kErrGraphCapacity when a total exceeds its capacity.  grid.y strides over
// the list.
__global__ void bern_pad_kernel(GenArgs g, const DevProj* projs, const uint32_t* list, int n_list,
                                const uint64_t* totals, uint64_t pad_key);
// Connections each network of the build really holds: fixed[m] plus the
// drawn totals of its pairwise_bernoulli projections (member[k] owns
// totals[k]), at most its segment [seg_begin[m], seg_end[m]) (a replay past
// a capacity is reported, never read past); real_end[m] = seg_begin[m] +
// that count.
__global__ void member_real_kernel(const uint64_t* totals, const uint32_t* member, int n_list, const uint64_t* fixed,
                                   const uint64_t* seg_begin, const uint64_t* seg_end, int n_members,
                                   uint64_t* real_end, uint64_t* real_count);

// fixed_total_number with autapses or multapses forbidden: the redraw
// projections of a build, their slots concatenated.
struct RedrawProj {
  uint32_t proj;        // index in the projection table
  int packed;           // one-word table entries
  int slot_bits;        // bits of a local slot
  int t_bits;           // bits of the target's local index (packed pair)
  uint64_t slot_base;   // first slot of this projection in the concatenation
  uint64_t chunk_base;  // first emit chunk (kChunk slots) of this projection
  uint64_t table_off;   // first entry of its hash table region
  uint64_t table_mask;  // entries - 1 (power of two)
  // Bucketed claims (RedrawArgs::bucketed): the projection's buckets are
  // [bucket_base, bucket_base + n_buckets), n_buckets = 1 << bucket_bits (0
  // when multapses are allowed: no pair table at all).
  uint64_t bucket_base;
  uint64_t n_buckets;
  int bucket_bits;
  // Round-0 entries first go to 2^super_bits super-buckets (the top bits of
  // the bucket index; at most 2^kSplitBits buckets each).  Super-bucket s
  // has kSuperLanes regions, one per residue of the emit chunk index:
  // region (s, l) holds sup[super_off + (s * kSuperLanes + l) * super_cap,
  // ...), its fill counter sfill[((super_base + s) * kSuperLanes + l) *
  // kFillStride].
  int super_bits;
  uint64_t super_base;
  uint64_t super_cap;
  uint64_t super_off;
  // Split units (kSplitUnit entries of one region): split_per_super per
  // region, the projection's first unit split_base.
  uint64_t split_base;
  uint64_t split_per_super;
};

struct RedrawArgs {
  const DevProj* projs;
  ArrayBlobs arr;              // explicit arrays (node lists compared for autapses)
  const RedrawProj* rp;
  int n;                       // redraw projections
  uint64_t n_slots;            // all slots
  uint64_t* pairs;             // per slot: (source << 32) | target, global ids
  uint8_t* lost;               // round-0 marks
  uint64_t* table_keys;        // hash tables (~0 = empty)
  uint64_t* table_vals;        // values of the two-array tables
  uint64_t* next_pending;
  unsigned long long* n_next;  // device counter of next_pending
  uint32_t* err;
  // Bucketed claims: every pair is owned by one bucket (the top bits of its
  // hash).  Round 0 fills ent[b * cap, b * cap + fill[b]) with the bucket's
  // entries; the round-0 kernel turns the region into an open-addressing
  // table of `cap` words (low bits of the hash, linear probing) holding the
  // accepted pairs, and the claims of later rounds go into that table.
  int bucketed;
  uint64_t* ent;
  uint32_t* fill;
  uint32_t cap;
  uint64_t n_buckets;
  // Bucketed claims: pairs[g] holds a slot's pair only if bit g is set here
  // (the slot redrew); every other slot keeps its round-0 draw, which the
  // emit kernel draws again.
  uint32_t* moved;
  uint64_t* sup;
  uint32_t* sfill;
  uint64_t n_super;
  uint32_t max_super;  // largest 2^super_bits of the build
  uint64_t n_split_units;
};
constexpr uint32_t kBucketCap = 2048;    // words of a bucket's table (mean 1024 entries, 32 sd)
constexpr uint32_t kBucketMean = 1024;   // target mean of round-0 entries per bucket
constexpr int kSplitBits = 9;            // buckets per super-bucket: 2^kSplitBits at most
constexpr int kMaxSuperBits = 12;        // super-buckets per projection: 2^12 at most
constexpr int kSuperLanes = 8;           // regions per super-bucket
constexpr int kFillStride = 8;           // region fill counters 32 bytes apart
constexpr int kSplitThreads = 512;       // split kernel block
constexpr uint32_t kSplitUnit = 8192;    // entries per split block and unit
__global__ void redraw_round0_kernel(RedrawArgs a);
__global__ void redraw_collect_kernel(RedrawArgs a);
// n_pending entries of `pending`, or *d_count of them when d_count is not
// null (graph builds: the count stays on the device).
__global__ void redraw_claim_kernel(RedrawArgs a, const uint64_t* pending, uint64_t n_pending, uint32_t round,
                                    const unsigned long long* d_count);
__global__ void redraw_resolve_kernel(RedrawArgs a, const uint64_t* pending, uint64_t n_pending,
                                      const unsigned long long* d_count);
// Graph builds: sets kErrGraphRounds when *d_count slots are still pending
// after the last recorded round.
__global__ void redraw_rounds_check_kernel(const unsigned long long* d_count, uint32_t* err);
// Bucketed claims: round 0 keeps the lowest slot of every pair in each
// bucket and leaves the bucket's table of accepted pairs; later rounds claim
// and resolve in those tables (redraw_claim_kernel, redraw_resolve_kernel).
// Round 0 with buckets: writes every slot's round-0 connection and sends
// its pair to its super-bucket.  Dynamic shared memory: histogram, delay
// table, guide, then 2 * max_super counters.
__global__ void redraw_draw_kernel(GenArgs g, RedrawArgs a, uint64_t total_chunks);
size_t redraw_draw_smem(const GenArgs& g, const RedrawArgs& a);
// Rewrites the connections of the slots that redrew (RedrawArgs::moved).
__global__ void redraw_patch_kernel(GenArgs g, RedrawArgs a);
__global__ void redraw_bucket_split_kernel(RedrawArgs a);  // dynamic shared memory: redraw_split_smem()
size_t redraw_split_smem();
__global__ void redraw_bucket0_kernel(RedrawArgs a);
__global__ void total_emit_kernel(GenArgs g, RedrawArgs a, uint64_t total_chunks);

cudaError_t exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* block_tmp,
                               cudaStream_t st);
uint64_t scan_tmp_entries(uint64_t n);

}  // namespace snc
