// snc_internal.h -- host-side context and the descriptors the kernels read.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <exception>
#include <string>
#include <vector>

#include "../../include/snc.h"

namespace snc {

// Device-side error bits, OR-ed into the context's error word by kernels
// instead of trapping; read back by snc_synchronize.
enum : uint32_t {
  kErrLookbackTimeout = 1u,  // a decoupled look-back wait hit its iteration bound
  kErrSamplerBound = 2u,     // a sampler exceeded its attempt bound
  kErrBounds = 4u,           // an internal index check failed
  // Graph replays (snc_batch_rebuild) run with bounds fixed when the graph
  // was recorded:
  kErrGraphCapacity = 8u,    // a pairwise_bernoulli projection drew past its capacity
  kErrGraphRounds = 16u,     // total-number redraws still pending after the recorded rounds
};

constexpr int kDelayGuide = 257;  // guide-table entries per threshold table

// One Connect call as the kernels see it (plain data, copied to the device).
struct DevProj {
  uint32_t s0, ns, t0, nt;  // global node ranges of the build
  uint32_t t_base;          // first node of the projection's network (targets are packed relative to it)
  uint32_t rule;
  uint32_t autapses, multapses;
  uint32_t w_normal;
  uint32_t k0, k1;        // Philox key of this projection
  uint64_t k;             // K or N
  uint64_t count;         // connections of this projection
  uint64_t out_off;       // position of its first connection in the generated arrays
  float w_mean, w_std;
  uint32_t d_const;       // delay step when the delay is constant (d_len == 0 && !d_table)
  uint32_t d_table;       // 1 if the delay is drawn from a threshold table
  uint32_t d_base, d_len; // value = d_base + #{thr <= u}
  uint32_t d_off;         // offset of the thresholds in the table blob (uint32 units)
  uint32_t d_goff;        // offset of the guide (uint16 units) in the guide blob
  // Bernoulli count tables, [0] all sources candidates, [1] one left out.
  uint32_t b_base[2], b_len[2], b_off[2], b_goff[2];
  uint64_t prim_off;      // offset of this projection's per-primary offsets (variable counts)
  uint64_t chunk_begin;   // first generation chunk of this projection
  uint64_t n_chunks;
  uint32_t chunks_per_row;  // all_to_all: chunks per source row
  uint32_t row_len;         // all_to_all: connections per source row (full row)
  // Primary node index of the projection's first primary in the Connect
  // call's own numbering: 0, except for a target shard, whose target-primary
  // projections (one_to_one, all_to_all, fixed_indegree,
  // pairwise_bernoulli) keep only the targets in the shard and key every
  // draw by primary + prim_shift, the index the whole network uses.
  uint32_t prim_shift;
  // floor(i / k) for 32-bit i as ((t + ((i - t) >> k_sh1)) >> k_sh2) with
  // t = umulhi(i, k_mul) (Granlund & Montgomery 1994, Fig. 4.1); set for
  // 1 <= k < 2^32 (division_magic).
  uint32_t k_mul;
  uint32_t k_sh1, k_sh2;
  // Explicit arrays of the Connect call (Sec. 2.1), as offsets into the
  // build's array blobs (kNoList: not given).  src_list / tgt_list: node ids
  // (network-local) in place of the ranges; w_list: per-connection weight
  // bits; d_list: per-connection delay steps (step blob); self_list: per
  // primary node, the position of its node in the list drawn from
  // (kNoPosition: absent), for per-primary rules without autapses;
  // row_list: one_to_one without autapses, the kept positions (id blob);
  // all_to_all without autapses, the dropped pairs before each source row
  // (offset blob, ns + 1 entries); drop_list: all_to_all, the dropped target
  // positions of every row, ascending per row (id blob).
  uint64_t src_list, tgt_list, w_list, d_list, self_list, row_list, drop_list;
};
// Multiplier and shifts of DevProj::k_mul for a divisor 1 <= d < 2^32:
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, shifts min(l, 1) and
// max(l - 1, 0) (Granlund & Montgomery 1994, Fig. 4.1).
inline void division_magic(uint64_t d, uint32_t* mul, uint32_t* sh1, uint32_t* sh2) {
  if (d == 0 || d > 0xFFFFFFFFull) {
    *mul = 0;
    *sh1 = *sh2 = 0;
    return;
  }
  int l = 0;
  while ((1ull << l) < d) ++l;
  *mul = static_cast<uint32_t>(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  *sh1 = l < 1 ? static_cast<uint32_t>(l) : 1u;
  *sh2 = l > 1 ? static_cast<uint32_t>(l - 1) : 0u;
}

constexpr uint64_t kNoList = ~0ull;
constexpr uint32_t kNoPosition = 0xFFFFFFFFu;

// The build's array blobs (device): node ids, weight bits and positions
// (uint32), delay steps (uint16), row offsets (uint64).
struct ArrayBlobs {
  const uint32_t* ids;
  const uint16_t* steps;
  const uint64_t* offs;
};

// Sort key and value of a connection.  The key packs source | delay step
// (Sec. 2.2 sorts by these two keys); it is 32 bits wide when the two fit,
// else 64.  The value packs the target above the fp32 weight's bits.  Source
// and target are local to the connection's network (equal to the node ids
// when a single network is built); a batch sorts each network's connections
// as a segment of its own.
struct KeyLayout {
  int src_bits;
  int delay_bits;
  int tgt_bits;  // bits of the largest network-local target (value field: 32)
  int total_bits() const { return src_bits + delay_bits; }
  bool key32() const { return total_bits() <= 32; }
};

__host__ __device__ inline uint64_t pack_key(uint32_t s, uint32_t d, int db) {
  return (static_cast<uint64_t>(s) << db) | d;
}

__host__ __device__ inline uint64_t pack_value(uint32_t t_local, uint32_t wbits) {
  return (static_cast<uint64_t>(t_local) << 32) | wbits;
}

// Host-side projection record.
struct Projection {
  snc_range src, tgt;
  snc_conn_rule rule;
  snc_syn_spec syn;
  bool exact_count;     // count known on the host
  uint64_t count;       // connections (after the count phase for Bernoulli)
  uint32_t d_const = 1;
  bool d_table = false;
  uint32_t d_base = 1;
  std::vector<uint32_t> d_thr;
  uint64_t b_base[2] = {0, 0};
  std::vector<uint32_t> b_thr[2];
  uint32_t max_step = 1;
  // Explicit arrays (snc_connect_arrays): node ids in place of the ranges
  // (src_list / tgt_list set), per-connection weight bits and delay steps
  // (empty: drawn).
  bool src_list = false, tgt_list = false;
  std::vector<uint32_t> src_ids, tgt_ids;
  std::vector<uint32_t> w_bits;
  std::vector<uint16_t> d_steps;
  bool has_lists() const { return src_list || tgt_list; }
  bool has_arrays() const { return has_lists() || !w_bits.empty() || !d_steps.empty(); }
};

// Device-memory estimate of finalizing one context (snc_runtime.cu).
struct BuildEstimate {
  uint64_t n_syn;           // connections (an upper bound for Bernoulli projections)
  uint64_t peak_bytes;      // device memory at the build's peak
  uint64_t resident_bytes;  // device memory the finished network keeps
  uint64_t n_nodes;
  uint32_t max_step;        // largest delay step
};
snc_status estimate_build(const snc_ctx* c, BuildEstimate* e);

// Runtime hooks of the server (snc_runtime.cu).  rebind_build replaces the
// stream (and, when alloc != nullptr, the allocator) a context builds with;
// allowed before finalize, and after a finished build to pick the stream its
// memory is released on.
void rebind_build(snc_ctx* c, cudaStream_t stream, const snc_allocator* alloc);
uint64_t storage_live_bytes(const snc_ctx* c);  // device bytes the context's storage holds
int ctx_device(const snc_ctx* c);
bool ctx_finalized(const snc_ctx* c);
bool ctx_sharded(const snc_ctx* c);  // a target shard (built alone, never in a batch)

// Admission of the served form (snc_server.cpp): one queued request as the
// admission sees it, and the limits it admits under.
struct AdmitRequest {
  uint64_t peak_bytes;  // estimated device memory at the build's peak
  uint64_t n_syn;       // connections
  uint64_t n_nodes;     // nodes of its network
  uint32_t max_step;    // largest delay step
  bool alone;           // built alone (a target shard)
};
struct AdmitLimits {
  uint64_t budget_bytes;    // the server's device-memory budget
  uint64_t reserved_bytes;  // reserved by running builds and resident results
  uint64_t batch_max_syn;   // connections of one batched build at most
  int batch_max_nets;       // networks of one batched build at most
};
// How many requests from the front of q[0..n) start as the next build, and
// the memory they reserve (*reserve): none while the front one does not fit
// the budget; else the front one, followed, when it is small (at most half
// of batch_max_syn connections) and not built alone, by the longest run of
// following small requests, none built alone, that keeps the batch within
// batch_max_nets networks, batch_max_syn connections, the budget and a
// batched key (global source | delay step | member-local target) of at most
// 64 bits over fewer than 2^32 nodes.
size_t admit_from_front(const AdmitRequest* q, size_t n, const AdmitLimits& lim, uint64_t* reserve);

// Entry points run their body through abi_guard: a C++ exception (host
// memory or threads exhausted inside the standard library) becomes
// SNC_ERR_OOM with a last-error message instead of crossing the C ABI.
snc_status abi_exception(const char* what) noexcept;  // snc_runtime.cu

template <class Body>
snc_status abi_guard(Body&& body) noexcept {
  try {
    return body();
  } catch (const std::exception& e) {
    return abi_exception(e.what());
  } catch (...) {
    return abi_exception("unknown exception");
  }
}

// Host threshold tables (tables.cpp).
int delay_thresholds(double mu, double sigma, double dt, std::vector<uint32_t>& thr, uint32_t& base);
int binomial_thresholds(uint64_t n, double p, std::vector<uint32_t>& thr, uint64_t& base);
void guide_table(const std::vector<uint32_t>& thr, uint16_t* guide);

}  // namespace snc
