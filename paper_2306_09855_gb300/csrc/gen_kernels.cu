// gen_kernels.cu -- connection generation directly in GPU memory (Sec. 2.1).
//
// Every kernel writes, for connection number `pos` of the concatenated
// generation order, the packed sort key (source | delay step) and the value
// (target | weight bits).  The paper's index formulas decide (source,
// target); the counter-based stream decides every random quantity, so the
// output does not depend on grid or block sizes.
//
//   gen_direct_kernel   one_to_one, all_to_all, in/out-degree with multapses,
//                       fixed_total_number with multapses and autapses
//   bernoulli_count     per-target Binomial counts of pairwise_bernoulli
//   sampler_kernel      in/out-degree without multapses and the Bernoulli
//                       subsets: one warp per primary node, distinct draws
//                       tracked in a shared-memory bitmap
//   redraw_*            fixed_total_number with autapses or multapses
//                       forbidden: round-based redraws; duplicates found per
//                       hash bucket in shared memory (global pair tables when
//                       a (pair, slot) entry does not fit 63 bits)
#include <cuda_runtime.h>

#include <cstdint>

#include "gen_kernels.h"
#include "snc_check.cuh"
#include "snc_device.cuh"

namespace snc {

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Projection owning chunk c (binary search over chunk_begin).
__device__ __forceinline__ int find_proj(const DevProj* projs, int n_proj, uint64_t c) {
  int lo = 0, hi = n_proj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (projs[mid].chunk_begin <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct SmemTables {
  uint32_t* thr;
  uint16_t* guide;
};

__device__ __forceinline__ uint32_t delay_step(const DevProj& P, const SmemTables& t, uint32_t u) {
  if (!P.d_table) return P.d_const;
  return P.d_base + table_lookup(t.thr, t.guide, P.d_len, u);
}

__device__ __forceinline__ uint32_t weight_bits(const DevProj& P, uint32_t w2, uint32_t w3) {
  const float w = P.w_normal ? normal_weight(P.w_mean, P.w_std, w2, w3) : P.w_mean;
  return __float_as_uint(w);
}

// Whether a projection record carries explicit arrays (Sec. 2.1); the
// kernels run their array-free instance for the others (ARR = false), which
// reads none of the list fields.
__device__ __forceinline__ bool has_arrays(const DevProj& P) {
  return P.src_list != kNoList || P.tgt_list != kNoList || P.w_list != kNoList || P.d_list != kNoList;
}

// Node (build id) at position pos of the projection's source / target list:
// the range, or the explicit ids of the Connect call (Sec. 2.1).
template <bool ARR>
__device__ __forceinline__ uint32_t src_node(const DevProj& P, const ArrayBlobs& A, uint32_t pos) {
  if constexpr (ARR) return P.src_list == kNoList ? P.s0 + pos : P.t_base + A.ids[P.src_list + pos];
  return P.s0 + pos;
}
template <bool ARR>
__device__ __forceinline__ uint32_t tgt_node(const DevProj& P, const ArrayBlobs& A, uint32_t pos) {
  if constexpr (ARR) return P.tgt_list == kNoList ? P.t0 + pos : P.t_base + A.ids[P.tgt_list + pos];
  return P.t0 + pos;
}

// Delay step and weight bits of connection number inew of the rule's own
// numbering: given per connection (Sec. 2.1), or drawn from the slot's WD
// words (which are drawn either way).
template <bool ARR>
__device__ __forceinline__ uint32_t conn_delay(const DevProj& P, const ArrayBlobs& A, const SmemTables& t,
                                               uint64_t inew, uint32_t u) {
  if constexpr (ARR) return P.d_list == kNoList ? delay_step(P, t, u) : A.steps[P.d_list + inew];
  return delay_step(P, t, u);
}
template <bool ARR>
__device__ __forceinline__ uint32_t conn_weight(const DevProj& P, const ArrayBlobs& A, uint64_t inew, uint32_t w2,
                                                uint32_t w3) {
  if constexpr (ARR) return P.w_list == kNoList ? weight_bits(P, w2, w3) : A.ids[P.w_list + inew];
  return weight_bits(P, w2, w3);
}

// Per-primary rules without autapses: whether primary b (build id `node`)
// appears in the list drawn from, and at which position *q.
template <bool ARR>
__device__ __forceinline__ bool self_in_other(const DevProj& P, const ArrayBlobs& A, uint32_t b, uint32_t node,
                                              uint32_t first_other, uint32_t n_other, uint32_t* q) {
  if (P.autapses) return false;
  if (ARR && P.self_list != kNoList) {
    const uint32_t v = A.ids[P.self_list + b];
    *q = v;
    return v != kNoPosition;
  }
  if (node >= first_other && node - first_other < n_other) {
    *q = node - first_other;
    return true;
  }
  return false;
}

// Stage the projection's delay table into shared memory.
__device__ void load_delay_table(const DevProj& P, const uint32_t* thr_blob, const uint16_t* guide_blob,
                                 SmemTables t) {
  if (!P.d_table) return;
  for (uint32_t i = threadIdx.x; i < P.d_len; i += blockDim.x) t.thr[i] = thr_blob[P.d_off + i];
  for (uint32_t i = threadIdx.x; i < kDelayGuide; i += blockDim.x) t.guide[i] = guide_blob[P.d_goff + i];
}

// Per-block digit counters in shared memory (at the start of the dynamic
// shared memory of every generation kernel).
struct BlockHist {
  uint32_t* sh;
  HistRegs r;
};

__device__ __forceinline__ BlockHist block_hist_begin(const GenArgs& a, uint32_t* smem) {
  BlockHist h{smem, hist_regs(a.hist)};
  hist_clear(h.sh, h.r);
  return h;  // the caller synchronises before the first store
}

__device__ __forceinline__ void block_hist_end(const GenArgs& a, const BlockHist& h) {
  __syncthreads();
  if (h.r.n) hist_flush(h.sh, h.r, a.hist.global);
}

__device__ __forceinline__ uint32_t hist_words(const GenArgs& a) {
  return a.hist.global ? static_cast<uint32_t>(a.hist.n_passes * a.hist.stride) : 0u;
}

// s and t are local to the connection's network (the build's node id minus
// the network's first node).
__device__ __forceinline__ void store(const GenArgs& a, const BlockHist& h, uint64_t pos, uint32_t s, uint32_t d,
                                      uint32_t t, uint32_t wbits) {
  if (!SNC_IN_BOUNDS(a.err, 1u, pos, a.cap)) return;
  const uint64_t key = pack_key(s, d, a.layout.delay_bits);
  if (a.key32)
    static_cast<uint32_t*>(a.keys)[pos] = static_cast<uint32_t>(key);
  else
    static_cast<uint64_t*>(a.keys)[pos] = key;
  a.vals[pos] = pack_value(t, wbits);
  hist_add(h.sh, h.r, key);
}

}  // namespace

namespace {
// One chunk of a direct rule (ARR: the projection carries explicit arrays).
template <bool ARR>
__device__ __forceinline__ void direct_chunk(const GenArgs& a, const BlockHist& bh, const SmemTables& tabs,
                                             const DevProj& P, uint64_t lc, uint32_t warp, uint32_t lane) {
  if (P.rule == SNC_ALL_TO_ALL) {
    // Row a (source s0 + a); targets b' in [part * kChunk, ...).  With
    // autapses off the diagonal target is skipped and later rows shift.
    // With explicit lists the dropped target positions of the row come
    // from the host (ascending).
    const uint32_t row = static_cast<uint32_t>(lc / P.chunks_per_row);
    const uint32_t part = static_cast<uint32_t>(lc % P.chunks_per_row);
    const uint32_t s = src_node<ARR>(P, a.arr, row);
    uint32_t n_drop = 0, diag_b = 0;
    uint64_t before = 0;  // dropped pairs in rows < row
    const uint32_t* drops = nullptr;
    if (P.row_list != kNoList) {
      before = a.arr.offs[P.row_list + row];
      n_drop = static_cast<uint32_t>(a.arr.offs[P.row_list + row + 1] - before);
      drops = a.arr.ids + P.drop_list + before;
    } else if (!P.autapses) {
      if (s >= P.t0 && s - P.t0 < P.nt) {
        n_drop = 1;
        diag_b = s - P.t0;
      }
      const uint32_t lo = max(P.s0, P.t0), hi = min(P.s0 + P.ns, P.t0 + P.nt);
      if (hi > lo && s > lo) before = min(s, hi) - lo;
    }
    const uint32_t row_len = P.nt - n_drop;
    const uint64_t row_out = P.out_off + static_cast<uint64_t>(row) * P.nt - before;
    for (uint32_t e = threadIdx.x; e < kChunk; e += blockDim.x) {
      const uint32_t bp = part * kChunk + e;
      if (bp >= row_len) break;
      uint32_t b = bp;
      if (drops) {
        for (uint32_t k = 0; k < n_drop; ++k) {
          if (drops[k] > b) break;
          ++b;
        }
      } else if (n_drop && bp >= diag_b) {
        b = bp + 1;
      }
      const Words W = draw(P.k0, P.k1, kTagWD, 0, b + P.prim_shift, row);
      const uint64_t inew = static_cast<uint64_t>(row) * P.nt + b;
      store(a, bh, row_out + bp, s - P.t_base, conn_delay<ARR>(P, a.arr, tabs, inew, W.x),
            tgt_node<ARR>(P, a.arr, b) - P.t_base, conn_weight<ARR>(P, a.arr, inew, W.z, W.w));
    }
    return;
  }
  const uint64_t start = lc * kChunk;
  const uint64_t end = min(start + kChunk, P.count);
  // Four windows of 128 per warp.
  for (int win = 0; win < kChunk / (128 * (kGenThreads / 32)); ++win) {
    const uint64_t wbase = start + (static_cast<uint64_t>(warp) * (kChunk / (kGenThreads / 32))) +
                           static_cast<uint64_t>(win) * 128;
    if (wbase >= end) break;
    Words X{0, 0, 0, 0};
    if (P.rule == SNC_FIXED_TOTAL_NUMBER) X = draw(P.k0, P.k1, kTagIdx, 0, kPrimaryNone, (wbase >> 2) + lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t i = wbase + static_cast<uint64_t>(q) * 32 + lane;
      uint32_t tw = 0;
      if (P.rule == SNC_FIXED_TOTAL_NUMBER) {
        const int src_lane = 8 * q + static_cast<int>(lane >> 2);
        const uint32_t vx = __shfl_sync(0xffffffffu, X.x, src_lane);
        const uint32_t vy = __shfl_sync(0xffffffffu, X.y, src_lane);
        const uint32_t vz = __shfl_sync(0xffffffffu, X.z, src_lane);
        const uint32_t vw = __shfl_sync(0xffffffffu, X.w, src_lane);
        const uint32_t sel = lane & 3u;
        tw = sel == 0 ? vx : sel == 1 ? vy : sel == 2 ? vz : vw;
      }
      if (i >= end) continue;
      uint32_t s, t, primary;
      uint64_t slot, inew = i;
      switch (P.rule) {
        case SNC_ONE_TO_ONE: {
          // pair i of the kept pairs (explicit lists without autapses)
          const uint32_t pos = P.row_list != kNoList ? a.arr.ids[P.row_list + i] : static_cast<uint32_t>(i);
          s = src_node<ARR>(P, a.arr, pos);
          t = tgt_node<ARR>(P, a.arr, pos);
          primary = pos;
          slot = 0;
          inew = pos;
          break;
        }
        case SNC_FIXED_INDEGREE:
        case SNC_FIXED_OUTDEGREE: {
          uint64_t b, j;
          if (P.count <= 0xFFFFFFFFull) {
            const uint32_t ii = static_cast<uint32_t>(i), kk = static_cast<uint32_t>(P.k);
            const uint32_t t = __umulhi(ii, P.k_mul);
            const uint32_t bq = (t + ((ii - t) >> P.k_sh1)) >> P.k_sh2;  // ii / kk
            b = bq;
            j = ii - bq * kk;
          } else {
            b = i / P.k;
            j = i - b * P.k;
          }
          primary = static_cast<uint32_t>(b);
          slot = j;
          s = t = 0;
          break;
        }
        default:  // fixed_total_number
          primary = kPrimaryNone;
          slot = i;
          s = t = 0;
          break;
      }
      const Words W = draw(P.k0, P.k1, kTagWD, 0, primary == kPrimaryNone ? primary : primary + P.prim_shift, slot);
      if (P.rule == SNC_FIXED_INDEGREE) {
        t = tgt_node<ARR>(P, a.arr, primary);
        uint32_t q = 0;
        const bool skip = self_in_other<ARR>(P, a.arr, primary, t, P.s0, P.ns, &q);
        s = src_node<ARR>(P, a.arr, endpoint(W.y, P.ns, skip, q));
      } else if (P.rule == SNC_FIXED_OUTDEGREE) {
        s = src_node<ARR>(P, a.arr, primary);
        uint32_t q = 0;
        const bool skip = self_in_other<ARR>(P, a.arr, primary, s, P.t0, P.nt, &q);
        t = tgt_node<ARR>(P, a.arr, endpoint(W.y, P.nt, skip, q));
      } else if (P.rule == SNC_FIXED_TOTAL_NUMBER) {
        s = src_node<ARR>(P, a.arr, rand_below(W.y, P.ns));
        t = tgt_node<ARR>(P, a.arr, rand_below(tw, P.nt));
      }
      store(a, bh, P.out_off + i, s - P.t_base, conn_delay<ARR>(P, a.arr, tabs, inew, W.x), t - P.t_base,
            conn_weight<ARR>(P, a.arr, inew, W.z, W.w));
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Direct rules.  A chunk is kChunk consecutive connections of one projection
// (for all_to_all: kChunk consecutive targets of one source row).  A warp
// works on windows of 128 consecutive connections; for fixed_total_number
// each lane computes one IDX draw (four target words) for the window and the
// words are passed around with shuffles.  At least four blocks per SM (64
// registers): with the projection record in registers the kernel would
// otherwise take 88 and run two blocks per SM, measured slower.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGenThreads, 4) gen_direct_kernel(GenArgs a) {
  extern __shared__ uint32_t smem_raw[];
  const uint32_t hw = hist_words(a);
  SmemTables tabs{smem_raw + hw, reinterpret_cast<uint16_t*>(smem_raw + hw + a.max_delay_len)};
  const BlockHist bh = block_hist_begin(a, smem_raw);
  __syncthreads();
  int cur = -1;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  for (uint64_t c = blockIdx.x; c < a.total_chunks; c += gridDim.x) {
    const int p = find_proj(a.projs, a.n_proj, c);
    if (p != cur) {
      __syncthreads();
      load_delay_table(a.projs[p], a.thr_blob, a.guide_blob, tabs);
      __syncthreads();
      cur = p;
    }
    // A copy in registers: the output stores below cannot alias it, so its
    // fields are not read again after every store.
    const DevProj P = a.projs[p];
    const uint64_t lc = c - P.chunk_begin;
    if (has_arrays(P))
      direct_chunk<true>(a, bh, tabs, P, lc, warp, lane);
    else
      direct_chunk<false>(a, bh, tabs, P, lc, warp, lane);
  }
  block_hist_end(a, bh);
}

// ---------------------------------------------------------------------------
// pairwise_bernoulli counts: target b draws n_b ~ Binomial(candidates, p)
// from word 0 of its COUNT draw (Sec. 4 names the rule; reading in the
// design notes).
// ---------------------------------------------------------------------------
// Index j of the segment holding element g: prefix[j] <= g < prefix[j + 1].
__device__ __forceinline__ int find_segment(const uint64_t* prefix, int n, uint64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void bernoulli_count_kernel(const DevProj* projs, const uint32_t* list, const uint64_t* prefix, int n_list,
                                       const uint32_t* thr_blob, const uint16_t* guide_blob, ArrayBlobs arr,
                                       uint32_t* counts) {
  const uint64_t total = prefix[n_list];
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int j = find_segment(prefix, n_list, g);
    const DevProj& P = projs[list[j]];
    const uint32_t b = static_cast<uint32_t>(g - prefix[j]);
    const uint32_t node = tgt_node<true>(P, arr, b);
    uint32_t q = 0;
    const int skip = self_in_other<true>(P, arr, b, node, P.s0, P.ns, &q) ? 1 : 0;
    const Words W = draw(P.k0, P.k1, kTagCount, 0, b + P.prim_shift, 0);
    const uint32_t i = table_lookup(thr_blob + P.b_off[skip], guide_blob + P.b_goff[skip], P.b_len[skip], W.x);
    counts[g] = P.b_base[skip] + i;
  }
}

__global__ void segment_totals_kernel(const uint64_t* offsets, const uint64_t* prefix, int n_list, uint64_t* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n_list) out[j] = offsets[prefix[j + 1]] - offsets[prefix[j]];
}

namespace {
// The connections of primary node b of a sampler projection (one warp).
template <bool ARR>
__device__ __forceinline__ void sample_primary(const SamplerArgs& a, const BlockHist& bh, uint32_t* bitmap,
                                               const SmemTables& tabs, const DevProj& P, uint32_t b,
                                               uint32_t lane) {
  const bool indeg = P.rule != SNC_FIXED_OUTDEGREE;  // indegree and Bernoulli pick sources
  const uint32_t n_other = indeg ? P.ns : P.nt;
  const uint32_t first_other = indeg ? P.s0 : P.t0;
  const uint32_t words = (n_other + 31u) >> 5;
  const ArrayBlobs& A = a.gen.arr;
  const uint32_t node = indeg ? tgt_node<ARR>(P, A, b) : src_node<ARR>(P, A, b);
  uint32_t skip_local = 0;
  const bool skip = self_in_other<ARR>(P, A, b, node, first_other, n_other, &skip_local);
  const uint32_t cand = n_other - (skip ? 1u : 0u);
  uint64_t want, out;
  if (P.rule == SNC_PAIRWISE_BERNOULLI) {
    const uint64_t rel = a.prim_offsets[P.prim_off + b] - a.prim_offsets[P.prim_off];
    want = a.prim_offsets[P.prim_off + b + 1] - a.prim_offsets[P.prim_off + b];
    out = P.out_off + rel;
    if (rel + want > P.count) {  // only a graph replay can draw past the projection's capacity
      if (lane == 0) atomicOr(a.err, kErrGraphCapacity);
      return;
    }
  } else {
    want = P.k;
    out = P.out_off + static_cast<uint64_t>(b) * P.k;
  }
  if (want == 0) return;
  const bool complement = 2 * want > cand;
  const uint32_t need = static_cast<uint32_t>(complement ? cand - want : want);
  // The bitmap area holds whole 16-byte units (bitmap_words is a multiple
  // of four), so clear it with 16-byte stores.
  for (uint32_t w = lane; w < (words + 3u) / 4u; w += 32) reinterpret_cast<uint4*>(bitmap)[w] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  uint32_t got = 0;
  uint64_t call = 0;
  const uint64_t max_calls = 16ull * cand + 64;  // far above any plausible need
  while (got < need) {
    if (call > max_calls) {
      if (lane == 0) atomicOr(a.err, kErrSamplerBound);
      break;
    }
    // One IDX draw per lane: attempts 4*(call + lane) .. +3.  The four
    // groups of 32 attempts are selected first; the WD draws of the kept
    // values then run together (four independent chains per lane).
    const Words X = draw(P.k0, P.k1, kTagIdx, 0, b + P.prim_shift, call + lane);
    call += 32;
    uint32_t kept_j[4], kept_r[4];
    bool kept[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      kept[q] = false;
      kept_j[q] = 0;
      kept_r[q] = 0;
      if (got >= need) continue;  // uniform over the warp
      const int src_lane = 8 * q + static_cast<int>(lane >> 2);
      const uint32_t vx = __shfl_sync(0xffffffffu, X.x, src_lane);
      const uint32_t vy = __shfl_sync(0xffffffffu, X.y, src_lane);
      const uint32_t vz = __shfl_sync(0xffffffffu, X.z, src_lane);
      const uint32_t vw = __shfl_sync(0xffffffffu, X.w, src_lane);
      const uint32_t sel = lane & 3u;
      const uint32_t u = sel == 0 ? vx : sel == 1 ? vy : sel == 2 ? vz : vw;
      const uint32_t r = endpoint(u, n_other, skip, skip_local);
      const uint32_t word = r >> 5, bit = 1u << (r & 31u);
      const bool seen = (bitmap[word] & bit) != 0u;
      __syncwarp();  // every lane has read its word before any lane sets a bit
      // Unseen values are set at once; a lane that finds its bit already set
      // by the group shares its value with another lane.  Only then (rarely:
      // about 32^2 / (2 n_other) of the groups) does the match instruction,
      // whose cost grows with the number of distinct values, pick the lowest
      // lane of each value; otherwise every unseen lane holds a value no other
      // lane holds and is the first of it.
      const uint32_t prev = seen ? bit : atomicOr(&bitmap[word], bit);
      bool fresh = !seen;
      if (__any_sync(0xffffffffu, !seen && (prev & bit) != 0u)) {
        const uint32_t peers = __match_any_sync(0xffffffffu, r);
        fresh = fresh && (__ffs(peers) - 1) == static_cast<int>(lane);
      }
      const uint32_t fresh_mask = __ballot_sync(0xffffffffu, fresh);
      const uint32_t rank = __popc(fresh_mask & ((1u << lane) - 1u));
      const uint32_t room = need - got;
      const bool take = fresh && rank < room;
      // New values beyond the room (last group only) leave the bitmap again:
      // no other lane's kept value shares their bit.
      if (fresh && !take) atomicAnd(&bitmap[word], ~bit);
      kept[q] = take;
      kept_j[q] = got + rank;
      kept_r[q] = r;
      got += min(static_cast<uint32_t>(__popc(fresh_mask)), room);
      __syncwarp();
    }
    if (!complement) {
      // Drawn for every lane (the chains interleave), stored for kept ones.
      Words W[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) W[q] = draw(P.k0, P.k1, kTagWD, 0, b + P.prim_shift, kept_j[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!kept[q]) continue;
        const uint32_t j = kept_j[q], r = kept_r[q];
        const uint32_t other = indeg ? src_node<ARR>(P, A, r) : tgt_node<ARR>(P, A, r);
        const uint32_t s = indeg ? other : node, t = indeg ? node : other;
        const uint64_t inew = static_cast<uint64_t>(b + P.prim_shift) * P.k + j;
        store(a.gen, bh, out + j, s - P.t_base, conn_delay<ARR>(P, A, tabs, inew, W[q].x), t - P.t_base,
              conn_weight<ARR>(P, A, inew, W[q].z, W[q].w));
      }
    }
  }
  if (complement) {
    // Kept values in ascending order: free bits of the bitmap, minus the
    // left-out node itself.
    uint32_t base = 0;
    for (uint32_t w0 = 0; w0 < words; w0 += 32) {
      const uint32_t w = w0 + lane;
      uint32_t free_bits = 0;
      if (w < words) {
        free_bits = ~bitmap[w];
        if (w == words - 1 && (n_other & 31u)) free_bits &= (1u << (n_other & 31u)) - 1u;
        if (skip && (skip_local >> 5) == w) free_bits &= ~(1u << (skip_local & 31u));
      }
      const uint32_t cnt = __popc(free_bits);
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (static_cast<int>(lane) >= o) incl += v;
      }
      uint32_t j = base + incl - cnt;
      while (free_bits) {
        const uint32_t bitpos = __ffs(free_bits) - 1;
        free_bits &= free_bits - 1;
        const uint32_t r = w * 32 + bitpos;
        if (j < want) {
          const Words W = draw(P.k0, P.k1, kTagWD, 0, b + P.prim_shift, j);
          const uint32_t other = indeg ? src_node<ARR>(P, A, r) : tgt_node<ARR>(P, A, r);
          const uint32_t s = indeg ? other : node, t = indeg ? node : other;
          const uint64_t inew = static_cast<uint64_t>(b + P.prim_shift) * P.k + j;
          store(a.gen, bh, out + j, s - P.t_base, conn_delay<ARR>(P, A, tabs, inew, W.x), t - P.t_base,
                conn_weight<ARR>(P, A, inew, W.z, W.w));
        } else {
          atomicOr(a.err, kErrBounds);
        }
        ++j;
      }
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncwarp();
}

}  // namespace

// ---------------------------------------------------------------------------
// Sampling without replacement, one warp per primary node.  Attempt a uses
// word (a mod 4) of IDX draw floor(a / 4); the first `need` distinct values
// are kept.  A warp examines 32 attempts at a time: a value is new if its
// bit is clear in the warp's bitmap and no lower lane drew it in the same
// group of 32; the first (need - got) new values in lane order are taken,
// which is exactly the sequential rule.  When more than half of the
// candidates are wanted the excluded values are drawn instead and the kept
// ones are listed in ascending order.
// ---------------------------------------------------------------------------
__global__ void sampler_kernel(SamplerArgs a) {
  extern __shared__ uint32_t smem_all[];
  const uint32_t lane = lane_id();
  const uint32_t warp_in_block = threadIdx.x >> 5;
  const uint32_t warps_per_block = blockDim.x >> 5;
  const BlockHist bh = block_hist_begin(a.gen, smem_all);
  __syncthreads();
  uint32_t* warp_area =
      smem_all + hist_words(a.gen) + static_cast<size_t>(warp_in_block) * (a.bitmap_words + a.table_words);
  uint32_t* bitmap = warp_area;
  SmemTables tabs{warp_area + a.bitmap_words, reinterpret_cast<uint16_t*>(warp_area + a.bitmap_words + a.max_delay_len)};
  const uint64_t total = a.prim_prefix[a.n_list];
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * warps_per_block + warp_in_block;
  const uint64_t n_warps = static_cast<uint64_t>(gridDim.x) * warps_per_block;
  int cur = -1;

  for (uint64_t gp = gw; gp < total; gp += n_warps) {
    const int j = find_segment(a.prim_prefix, a.n_list, gp);
    const DevProj P = a.projs[a.list[j]];
    if (j != cur) {
      // This warp's copy of the projection's delay table.
      if (P.d_table) {
        for (uint32_t i = lane; i < P.d_len; i += 32) tabs.thr[i] = a.thr_blob[P.d_off + i];
        for (uint32_t i = lane; i < kDelayGuide; i += 32) tabs.guide[i] = a.guide_blob[P.d_goff + i];
      }
      __syncwarp();
      cur = j;
    }
    const uint32_t b = static_cast<uint32_t>(gp - a.prim_prefix[j]);
    if (has_arrays(P))
      sample_primary<true>(a, bh, bitmap, tabs, P, b, lane);
    else
      sample_primary<false>(a, bh, bitmap, tabs, P, b, lane);
  }
  block_hist_end(a.gen, bh);
}

__global__ void bern_pad_kernel(GenArgs g, const DevProj* projs, const uint32_t* list, int n_list,
                                const uint64_t* totals, uint64_t pad_key) {
  const HistRegs hr = hist_regs(g.hist);
  for (int k = blockIdx.y; k < n_list; k += gridDim.y) {
    const DevProj& P = projs[list[k]];
    const uint64_t tot = totals[k];
    if (tot > P.count) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(g.err, kErrGraphCapacity);
      continue;
    }
    const uint64_t n_pad = P.count - tot;
    const uint64_t begin = P.out_off + tot;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
      const uint64_t pos = begin + i;
      if (!SNC_IN_BOUNDS(g.err, 3u, pos, g.cap)) break;
      if (g.key32)
        static_cast<uint32_t*>(g.keys)[pos] = static_cast<uint32_t>(pad_key);
      else
        static_cast<uint64_t*>(g.keys)[pos] = pad_key;
      g.vals[pos] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && n_pad > 0) {
#pragma unroll
      for (int p = 0; p < kMaxPasses; ++p)
        if (p < hr.n)
          atomicAdd(g.hist.global + p * kMaxRadix + (static_cast<uint32_t>(pad_key >> hr.shift[p]) & hr.mask[p]),
                    static_cast<unsigned long long>(n_pad));
    }
  }
}

__global__ void member_real_kernel(const uint64_t* totals, const uint32_t* member, int n_list, const uint64_t* fixed,
                                   const uint64_t* seg_begin, const uint64_t* seg_end, int n_members,
                                   uint64_t* real_end, uint64_t* real_count) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_members; m += gridDim.x * blockDim.x) {
    uint64_t cnt = fixed[m];
    for (int k = 0; k < n_list; ++k)
      if (member[k] == static_cast<uint32_t>(m)) cnt += totals[k];
    const uint64_t cap = seg_end[m] - seg_begin[m];
    if (cnt > cap) cnt = cap;
    real_count[m] = cnt;
    real_end[m] = seg_begin[m] + cnt;
  }
}

// ---------------------------------------------------------------------------
// fixed_total_number with autapses or multapses forbidden (not in the paper,
// Sec. 4).  Round 0 draws every slot as in the multapse case; a slot whose
// pair is not allowed redraws in round r >= 1 from its DEDUP draw.  With
// multapses forbidden a pair may be held by one slot only: pairs accepted in
// earlier rounds block it, and among the slots drawing it in the same round
// the lowest wins.  All redraw projections of a build are handled together
// (slots concatenated, one hash table region per projection), so every round
// costs one launch pair and one read-back however many projections redraw.
//
// Table entries.  Packed (when it fits in 63 bits): one word
//   (pair_local << (slot_bits + 1)) | (claimed_this_round << slot_bits) | slot.
// Otherwise keys (global pair) and values (claim bit 63 | slot) in two
// arrays.  Either way an accepted entry is smaller than any claim on the same
// pair, so atomicMin never replaces it, and among claims it keeps the lowest
// slot.  In round 0 a claimant that meets its pair marks the higher of the
// two slots lost; every claimant but the lowest is marked by someone, so no
// second pass over the table is needed and round-0 entries are written in
// the accepted form.
// ---------------------------------------------------------------------------
namespace {
constexpr uint64_t kEmpty = ~0ull;
constexpr uint64_t kClaim = 1ull << 63;

__device__ __forceinline__ uint64_t pair_hash(uint64_t key) {
  key ^= key >> 33;
  key *= 0xff51afd7ed558ccdull;
  key ^= key >> 33;
  key *= 0xc4ceb9fe1a85ec53ull;
  key ^= key >> 33;
  return key;
}

// (s, t): source and target positions offset by s0 / t0 (equal to the
// nodes for ranges); with explicit lists the nodes at those positions are
// compared.
__device__ __forceinline__ bool allowed_pair(const DevProj& P, const ArrayBlobs& A, uint32_t s, uint32_t t) {
  if (P.autapses) return true;
  if (P.src_list == kNoList && P.tgt_list == kNoList) return s != t;
  return src_node<true>(P, A, s - P.s0) != tgt_node<true>(P, A, t - P.t0);
}

// The slot g of the concatenated list: its projection and local slot.
struct SlotRef {
  const RedrawProj* r;
  const DevProj* P;
  uint64_t i;
};

__device__ __forceinline__ SlotRef slot_ref(const RedrawArgs& a, uint64_t g) {
  int lo = 0, hi = a.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.rp[mid].slot_base <= g) lo = mid; else hi = mid - 1;
  }
  const RedrawProj* r = &a.rp[lo];
  return SlotRef{r, &a.projs[r->proj], g - r->slot_base};
}

// Claim of `slot` on the pair (s, t) (global ids) in projection r's table.
// round0: accepted form plus lost marks; otherwise a claim for resolve().
__device__ void claim(const RedrawArgs& a, const RedrawProj& r, const DevProj& P, uint32_t s, uint32_t t,
                      uint64_t slot, uint64_t gslot, bool round0) {
  const uint64_t slot_mask = (1ull << r.slot_bits) - 1;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(a.table_keys + r.table_off);
  if (r.packed) {
    const int sh = r.slot_bits + 1;
    const uint64_t pair = (static_cast<uint64_t>(s - P.s0) << r.t_bits) | (t - P.t0);
    const uint64_t e = (pair << sh) | (round0 ? 0ull : (1ull << r.slot_bits)) | slot;
    uint64_t h = pair_hash(pair) & r.table_mask;
    for (uint64_t probe = 0; probe <= r.table_mask; ++probe) {
      const uint64_t old = atomicCAS(keys + h, kEmpty, e);
      if (old == kEmpty) return;
      if ((old >> sh) == pair) {
        const uint64_t prev = atomicMin(keys + h, e);
        if (round0) {
          if (prev < e) a.lost[gslot] = 1;
          else a.lost[gslot - slot + (prev & slot_mask)] = 1;
        }
        return;
      }
      h = (h + 1) & r.table_mask;
    }
  } else {
    unsigned long long* vals = reinterpret_cast<unsigned long long*>(a.table_vals + r.table_off);
    const uint64_t pair = (static_cast<uint64_t>(s) << 32) | t;
    const uint64_t v = (round0 ? 0ull : kClaim) | slot;
    uint64_t h = pair_hash(pair) & r.table_mask;
    for (uint64_t probe = 0; probe <= r.table_mask; ++probe) {
      uint64_t k = keys[h];
      if (k == kEmpty) k = atomicCAS(keys + h, kEmpty, pair);
      if (k == kEmpty || k == pair) {
        const uint64_t prev = atomicMin(vals + h, v);
        if (round0 && prev != kEmpty) {
          if (prev < v) a.lost[gslot] = 1;
          else a.lost[gslot - slot + (prev & ~kClaim)] = 1;
        }
        return;
      }
      h = (h + 1) & r.table_mask;
    }
  }
  atomicOr(a.err, kErrBounds);
}

// Round r >= 1: true if `slot` holds the lowest claim on its pair (and marks
// the entry accepted).
__device__ bool resolve(const RedrawArgs& a, const RedrawProj& r, const DevProj& P, uint32_t s, uint32_t t,
                        uint64_t slot) {
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(a.table_keys + r.table_off);
  if (r.packed) {
    const int sh = r.slot_bits + 1;
    const uint64_t pair = (static_cast<uint64_t>(s - P.s0) << r.t_bits) | (t - P.t0);
    const uint64_t e = (pair << sh) | (1ull << r.slot_bits) | slot;
    uint64_t h = pair_hash(pair) & r.table_mask;
    for (uint64_t probe = 0; probe <= r.table_mask; ++probe) {
      const uint64_t v = keys[h];
      if (v == kEmpty) return false;
      if ((v >> sh) == pair) {
        if (v != e) return false;
        keys[h] = e & ~(1ull << r.slot_bits);
        return true;
      }
      h = (h + 1) & r.table_mask;
    }
    return false;
  }
  unsigned long long* vals = reinterpret_cast<unsigned long long*>(a.table_vals + r.table_off);
  const uint64_t pair = (static_cast<uint64_t>(s) << 32) | t;
  uint64_t h = pair_hash(pair) & r.table_mask;
  for (uint64_t probe = 0; probe <= r.table_mask; ++probe) {
    const uint64_t k = keys[h];
    if (k == kEmpty) return false;
    if (k == pair) {
      if (vals[h] != (kClaim | slot)) return false;
      vals[h] = slot;
      return true;
    }
    h = (h + 1) & r.table_mask;
  }
  return false;
}

// Bucketed claims.  Entries are (pair << (slot_bits + 1)) | claim << slot_bits
// | slot with the pair and slot local to the projection, as in the packed
// table above.
__device__ __forceinline__ uint64_t local_pair(const RedrawProj& r, const DevProj& P, uint32_t s, uint32_t t) {
  return (static_cast<uint64_t>(s - P.s0) << r.t_bits) | (t - P.t0);
}

// Round r >= 1 with buckets: the claim of local slot i on (s, t) goes into
// the table of the pair's bucket (accepted entries have the claim bit clear
// and are smaller than any claim on their pair, so atomicMin keeps them;
// among claims it keeps the lowest slot).
__device__ void bucket_claim(const RedrawArgs& a, const RedrawProj& r, const DevProj& P, uint32_t s, uint32_t t,
                             uint64_t i) {
  const uint64_t pair = local_pair(r, P, s, t);
  const uint64_t hash = pair_hash(pair);
  const uint64_t b = r.bucket_base + (r.bucket_bits ? hash >> (64 - r.bucket_bits) : 0ull);
  unsigned long long* tab = reinterpret_cast<unsigned long long*>(a.ent + b * a.cap);
  const int sh = r.slot_bits + 1;
  const uint64_t e = (pair << sh) | (1ull << r.slot_bits) | i;
  const uint32_t mask = a.cap - 1;
  uint32_t h = static_cast<uint32_t>(hash) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint64_t old = atomicCAS(tab + h, kEmpty, e);
    if (old == kEmpty) return;
    if ((old >> sh) == pair) {
      atomicMin(tab + h, e);
      return;
    }
    h = (h + 1) & mask;
  }
  atomicOr(a.err, kErrBounds);  // full table: cannot happen below cap entries
}

// True if local slot i holds the lowest claim on (s, t) and no accepted pair
// blocks it; the entry then becomes accepted.
__device__ bool bucket_resolve(const RedrawArgs& a, const RedrawProj& r, const DevProj& P, uint32_t s, uint32_t t,
                               uint64_t i) {
  const uint64_t pair = local_pair(r, P, s, t);
  const uint64_t hash = pair_hash(pair);
  const uint64_t b = r.bucket_base + (r.bucket_bits ? hash >> (64 - r.bucket_bits) : 0ull);
  uint64_t* tab = a.ent + b * a.cap;
  const int sh = r.slot_bits + 1;
  const uint64_t e = (pair << sh) | (1ull << r.slot_bits) | i;
  const uint32_t mask = a.cap - 1;
  uint32_t h = static_cast<uint32_t>(hash) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint64_t v = tab[h];
    if (v == kEmpty) return false;
    if ((v >> sh) == pair) {
      if (v != e) return false;
      tab[h] = e & ~(1ull << r.slot_bits);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

// The redraw projection that owns bucket b.
__device__ __forceinline__ int bucket_owner(const RedrawArgs& a, uint64_t b) {
  int lo = 0, hi = a.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.rp[mid].bucket_base <= b) lo = mid; else hi = mid - 1;
  }
  while (lo > 0 && (a.rp[lo].n_buckets == 0 || b >= a.rp[lo].bucket_base + a.rp[lo].n_buckets)) --lo;
  return lo;
}

__device__ __forceinline__ void push_pending(const RedrawArgs& a, uint64_t g) {
  const unsigned long long at = atomicAdd(a.n_next, 1ull);
  if (at < a.n_slots) a.next_pending[at] = g;
  else atomicOr(a.err, kErrBounds);
}
}  // namespace

// Round 0 with global pair tables: every slot draws and stores its pair;
// claims go to the projection's table.
__global__ void redraw_round0_kernel(RedrawArgs a) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < a.n_slots; g += stride) {
    const SlotRef x = slot_ref(a, g);
    const DevProj& P = *x.P;
    const Words W = draw(P.k0, P.k1, kTagWD, 0, kPrimaryNone, x.i);
    const Words X = draw(P.k0, P.k1, kTagIdx, 0, kPrimaryNone, x.i >> 2);
    const uint32_t sel = static_cast<uint32_t>(x.i & 3u);
    const uint32_t tw = sel == 0 ? X.x : sel == 1 ? X.y : sel == 2 ? X.z : X.w;
    const uint32_t s = P.s0 + rand_below(W.y, P.ns);
    const uint32_t t = P.t0 + rand_below(tw, P.nt);
    a.pairs[g] = (static_cast<uint64_t>(s) << 32) | t;
    if (!allowed_pair(P, a.arr, s, t)) a.lost[g] = 1;
    else if (!P.multapses) claim(a, *x.r, P, s, t, x.i, g, true);
  }
}

// Round-0 slots marked lost become the first pending list.
__global__ void redraw_collect_kernel(RedrawArgs a) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < a.n_slots; g += stride)
    if (a.lost[g]) push_pending(a, g);
}

__global__ void redraw_claim_kernel(RedrawArgs a, const uint64_t* pending, uint64_t n_pending, uint32_t round,
                                    const unsigned long long* d_count) {
  if (d_count) n_pending = *d_count;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n_pending; q += stride) {
    const uint64_t g = pending[q];
    const SlotRef x = slot_ref(a, g);
    const DevProj& P = *x.P;
    const Words D = draw(P.k0, P.k1, kTagDedup, round, kPrimaryNone, x.i);
    const uint32_t s = P.s0 + rand_below(D.x, P.ns);
    const uint32_t t = P.t0 + rand_below(D.y, P.nt);
    a.pairs[g] = (static_cast<uint64_t>(s) << 32) | t;
    if (a.moved) atomicOr(a.moved + (g >> 5), 1u << (g & 31u));
    // The resolve kernel decides every slot (not allowed -> next round).
    if (!P.multapses && allowed_pair(P, a.arr, s, t)) {
      if (a.bucketed) bucket_claim(a, *x.r, P, s, t, x.i);
      else claim(a, *x.r, P, s, t, x.i, g, false);
    }
  }
}

// Target word of slot wbase + 32 q + lane from the IDX draws of a window of
// 128 slots (lane l holds IDX(wbase / 4 + l), four target words).
__device__ __forceinline__ uint32_t window_target_word(const Words& X, int q, uint32_t lane) {
  const int src_lane = 8 * q + static_cast<int>(lane >> 2);
  const uint32_t vx = __shfl_sync(0xffffffffu, X.x, src_lane);
  const uint32_t vy = __shfl_sync(0xffffffffu, X.y, src_lane);
  const uint32_t vz = __shfl_sync(0xffffffffu, X.z, src_lane);
  const uint32_t vw = __shfl_sync(0xffffffffu, X.w, src_lane);
  const uint32_t sel = lane & 3u;
  return sel == 0 ? vx : sel == 1 ? vy : sel == 2 ? vz : vw;
}

// The redraw projection that owns emit chunk c.
__device__ __forceinline__ int chunk_owner(const RedrawArgs& a, uint64_t c) {
  int lo = 0, hi = a.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.rp[mid].chunk_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Round 0 with buckets, fused with the emit: every slot draws its round-0
// connection (WD for source, delay and weight; the IDX draws of a 128-slot
// window give the targets, one draw per four slots) and writes it; slots
// that redraw later are rewritten by the patch kernel.  A pair that is not
// allowed joins the pending list.  Without multapses the pairs of half a
// chunk (2048 slots) are counted per super-bucket in shared memory, each
// super-bucket's run reserved with one global atomic (in the region of the
// chunk's lane) and every entry written into its run.
namespace {
constexpr int kDrawStage = kChunk / 2;  // entries of one partition round
}

size_t redraw_draw_smem(const GenArgs& g, const RedrawArgs& a) {
  const size_t words = (g.hist.global ? static_cast<size_t>(g.hist.n_passes) * g.hist.stride : 0u) +
                       g.max_delay_len + (kDelayGuide + 1) / 2 + 3u * a.max_super + 8u;
  return (words + 1) / 2 * sizeof(uint64_t) + kDrawStage * (sizeof(uint64_t) + sizeof(uint16_t));
}

// Four blocks per SM at least (64 registers), with the projection records in
// registers (measured faster than reading them through global memory).
__global__ void __launch_bounds__(kGenThreads, 4) redraw_draw_kernel(GenArgs g, RedrawArgs a, uint64_t total_chunks) {
  extern __shared__ uint32_t smem_raw[];
  const uint32_t hw = hist_words(g);
  SmemTables tabs{smem_raw + hw, reinterpret_cast<uint16_t*>(smem_raw + hw + g.max_delay_len)};
  uint32_t* cnt = smem_raw + hw + g.max_delay_len + (kDelayGuide + 1) / 2;  // entries per super-bucket
  uint32_t* base = cnt + a.max_super;                                        // reserved start of each run
  uint32_t* lstart = base + a.max_super;                                     // start of each run in the stage
  uint32_t* wsum = lstart + a.max_super;                                     // warp totals of the scan
  const size_t words = hw + g.max_delay_len + (kDelayGuide + 1) / 2 + 3u * a.max_super + 8u;
  uint64_t* stage = reinterpret_cast<uint64_t*>(smem_raw) + (words + 1) / 2;  // entries in super-bucket order
  uint16_t* stage_s = reinterpret_cast<uint16_t*>(stage + kDrawStage);     // their super-buckets
  const BlockHist bh = block_hist_begin(g, smem_raw);
  __syncthreads();
  constexpr int kWin = kChunk / (128 * (kGenThreads / 32));  // windows per warp and chunk
  constexpr int kHalf = kWin / 2;                             // windows per partition round
  constexpr int kPer = 4 * kHalf;                             // slots per thread and round
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  int cur = -1;
  for (uint64_t c = blockIdx.x; c < total_chunks; c += gridDim.x) {
    const int lo = chunk_owner(a, c);
    const RedrawProj r = a.rp[lo];
    const DevProj P = a.projs[r.proj];
    if (lo != cur) {
      __syncthreads();
      load_delay_table(P, g.thr_blob, g.guide_blob, tabs);
      __syncthreads();
      cur = lo;
    }
    const bool part = !P.multapses;  // uniform over the block
    const bool arr = has_arrays(P);   // uniform over the block
    const uint32_t n_sup = part ? (1u << r.super_bits) : 0u;
    const int fine_shift = r.bucket_bits - r.super_bits;
    const uint64_t lc = c - r.chunk_base;
    const uint32_t cl = static_cast<uint32_t>(lc % kSuperLanes);  // the chunk's lane
    const uint64_t start = lc * kChunk;
    const uint64_t end = min(start + kChunk, P.count);
    for (int h = 0; h < kWin / kHalf; ++h) {
      for (uint32_t s = threadIdx.x; s < n_sup; s += blockDim.x) cnt[s] = 0;
      __syncthreads();
      uint64_t ent[kPer];
      uint32_t rs[kPer];  // (super-bucket << 16) | rank in the run, ~0 = none
#pragma unroll
      for (int w2 = 0; w2 < kHalf; ++w2) {
        const uint64_t wbase = start + (static_cast<uint64_t>(warp) * (kChunk / (kGenThreads / 32))) +
                               static_cast<uint64_t>(h * kHalf + w2) * 128;
        Words X{0, 0, 0, 0};
        if (wbase < end) X = draw(P.k0, P.k1, kTagIdx, 0, kPrimaryNone, (wbase >> 2) + lane);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = w2 * 4 + q;
          const uint32_t tw = window_target_word(X, q, lane);
          const uint64_t i = wbase + static_cast<uint64_t>(q) * 32 + lane;
          rs[k] = ~0u;
          ent[k] = 0;
          if (i >= end) continue;
          const Words W = draw(P.k0, P.k1, kTagWD, 0, kPrimaryNone, i);
          const uint32_t ps = rand_below(W.y, P.ns), pt = rand_below(tw, P.nt);
          const uint32_t s = P.s0 + ps, t = P.t0 + pt;
          if (arr)
            store(g, bh, P.out_off + i, src_node<true>(P, g.arr, ps) - P.t_base,
                  conn_delay<true>(P, g.arr, tabs, i, W.x), tgt_node<true>(P, g.arr, pt) - P.t_base,
                  conn_weight<true>(P, g.arr, i, W.z, W.w));
          else
            store(g, bh, P.out_off + i, s - P.t_base, delay_step(P, tabs, W.x), t - P.t_base,
                  weight_bits(P, W.z, W.w));
          if (!allowed_pair(P, a.arr, s, t)) {
            push_pending(a, r.slot_base + i);
          } else if (part) {
            const uint64_t pair = local_pair(r, P, s, t);
            const uint64_t fine = r.bucket_bits ? pair_hash(pair) >> (64 - r.bucket_bits) : 0ull;
            const uint32_t sb = static_cast<uint32_t>(fine >> fine_shift);
            ent[k] = (pair << (r.slot_bits + 1)) | i;
            rs[k] = (sb << 16) | atomicAdd(cnt + sb, 1u);
          }
        }
      }
      __syncthreads();
      if (!part) continue;  // uniform over the block; nothing counted
      // Reserve each run; scan the counts (contiguous groups of super-buckets
      // per thread) for the stage.
      for (uint32_t s = threadIdx.x; s < n_sup; s += blockDim.x) {
        const uint32_t n = cnt[s];
        const uint64_t fi = ((r.super_base + s) * kSuperLanes + cl) * kFillStride;
        base[s] = n ? atomicAdd(a.sfill + fi, n) : 0u;
      }
      const uint32_t per = (n_sup + kGenThreads - 1) / kGenThreads;
      const uint32_t s0 = threadIdx.x * per;
      uint32_t sum = 0;
      for (uint32_t j = 0; j < per; ++j)
        if (s0 + j < n_sup) sum += cnt[s0 + j];
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncthreads();
      if (warp == 0) {
        uint32_t w = lane < kGenThreads / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
          if (lane >= static_cast<uint32_t>(o)) w += y;
        }
        if (lane < kGenThreads / 32) wsum[lane] = w;
      }
      __syncthreads();
      uint32_t run = x - sum + (warp ? wsum[warp - 1] : 0u);
      for (uint32_t j = 0; j < per; ++j)
        if (s0 + j < n_sup) {
          lstart[s0 + j] = run;
          run += cnt[s0 + j];
        }
      const uint32_t total = wsum[kGenThreads / 32 - 1];
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        if (rs[k] == ~0u) continue;
        const uint32_t sb = rs[k] >> 16;
        const uint32_t at = lstart[sb] + (rs[k] & 0xFFFFu);
        if (at < kDrawStage) {
          stage[at] = ent[k];
          stage_s[at] = static_cast<uint16_t>(sb);
        }
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < total && i < kDrawStage; i += blockDim.x) {
        const uint32_t sb = stage_s[i];
        const uint64_t pos = static_cast<uint64_t>(base[sb]) + (i - lstart[sb]);
        if (pos < r.super_cap)
          a.sup[r.super_off + (static_cast<uint64_t>(sb) * kSuperLanes + cl) * r.super_cap + pos] = stage[i];
        else
          atomicOr(a.err, kErrBounds);
      }
      __syncthreads();  // the counters and the stage are reused
    }
  }
  block_hist_end(g, bh);
}

// Rewrites the connection of every slot that redrew: its final pair (source
// in the key, target in the value) with the delay and weight it already has;
// the digit counts of the sort follow the key.
__global__ void redraw_patch_kernel(GenArgs g, RedrawArgs a) {
  extern __shared__ uint32_t delta[];  // per pass and digit: changes of the block, mod 2^32
  const HistRegs hr = hist_regs(g.hist);
  for (int i = threadIdx.x; i < hr.n * hr.stride; i += blockDim.x) delta[i] = 0u;
  __syncthreads();
  const uint64_t words = (a.n_slots + 31) / 32;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t dmask = (1ull << g.layout.delay_bits) - 1;
  for (uint64_t w = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < words; w += stride) {
    uint32_t m = a.moved[w];
    while (m) {
      const uint64_t gs = w * 32 + static_cast<uint64_t>(__ffs(m) - 1);
      m &= m - 1;
      const SlotRef x = slot_ref(a, gs);
      const DevProj& P = *x.P;
      const uint64_t pos = P.out_off + x.i;
      if (!SNC_IN_BOUNDS(a.err, 2u, pos, g.cap)) continue;
      const uint64_t pair = a.pairs[gs];
      const uint32_t s = src_node<true>(P, g.arr, static_cast<uint32_t>(pair >> 32) - P.s0);
      const uint32_t t = tgt_node<true>(P, g.arr, static_cast<uint32_t>(pair) - P.t0);
      const uint64_t old = g.key32 ? static_cast<uint64_t>(static_cast<uint32_t*>(g.keys)[pos])
                                   : static_cast<uint64_t*>(g.keys)[pos];
      const uint64_t key = pack_key(s - P.t_base, static_cast<uint32_t>(old & dmask), g.layout.delay_bits);
      if (g.key32) static_cast<uint32_t*>(g.keys)[pos] = static_cast<uint32_t>(key);
      else static_cast<uint64_t*>(g.keys)[pos] = key;
      g.vals[pos] = pack_value(t - P.t_base, static_cast<uint32_t>(g.vals[pos]));
#pragma unroll
      for (int p = 0; p < kMaxPasses; ++p) {
        if (p >= hr.n) break;
        const uint32_t d0 = static_cast<uint32_t>(old >> hr.shift[p]) & hr.mask[p];
        const uint32_t d1 = static_cast<uint32_t>(key >> hr.shift[p]) & hr.mask[p];
        if (d0 == d1) continue;
        atomicAdd(delta + p * hr.stride + d0, ~0u);  // minus one
        atomicAdd(delta + p * hr.stride + d1, 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < hr.n * hr.stride; i += blockDim.x) {
    const int32_t v = static_cast<int32_t>(delta[i]);
    if (v) atomicAdd(g.hist.global + (i / hr.stride) * kMaxRadix + (i % hr.stride), static_cast<unsigned long long>(static_cast<int64_t>(v)));
  }
}

// Spreads the super-buckets over their buckets.  A block takes a unit of
// kSplitUnit entries of one region, counts them per bucket in shared
// memory, stages them in bucket order, reserves each bucket's run with one
// global atomic and writes every run with consecutive threads.
size_t redraw_split_smem() {
  return static_cast<size_t>(kSplitUnit) * (sizeof(uint64_t) + sizeof(uint16_t)) +
         3u * (1u << kSplitBits) * sizeof(uint32_t) + 32 * sizeof(uint32_t);
}

__global__ void __launch_bounds__(kSplitThreads) redraw_bucket_split_kernel(RedrawArgs a) {
  extern __shared__ uint64_t split_smem[];
  uint64_t* stage = split_smem;                                          // entries in bucket order
  uint16_t* stage_f = reinterpret_cast<uint16_t*>(stage + kSplitUnit);  // their buckets
  uint32_t* fcnt = reinterpret_cast<uint32_t*>(stage_f + kSplitUnit);
  uint32_t* fbase = fcnt + (1u << kSplitBits);   // reserved start of each run
  uint32_t* lstart = fbase + (1u << kSplitBits);  // start of each run in the stage
  uint32_t* wsum = lstart + (1u << kSplitBits);   // warp totals of the scan
  constexpr int kPer = kSplitUnit / kSplitThreads;
  static_assert((1u << kSplitBits) == kSplitThreads, "one bucket per thread in the scan");
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint64_t u = blockIdx.x; u < a.n_split_units; u += gridDim.x) {
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.rp[mid].split_base <= u) lo = mid; else hi = mid - 1;
    }
    const RedrawProj& r = a.rp[lo];
    const uint64_t lu = u - r.split_base;
    const uint64_t rr = lu / r.split_per_super;  // region (s, lane) = s * kSuperLanes + lane
    const uint64_t part = lu - rr * r.split_per_super;
    const uint64_t s = rr / kSuperLanes;
    const int fine_shift = r.bucket_bits - r.super_bits;
    const uint32_t n_fine = 1u << fine_shift;
    const int sh = r.slot_bits + 1;
    const uint64_t rf = a.sfill[(r.super_base * kSuperLanes + rr) * kFillStride];
    const uint64_t fill = rf < r.super_cap ? rf : r.super_cap;
    const uint64_t i0 = part * kSplitUnit;
    if (i0 >= fill) continue;  // uniform over the block
    const uint32_t n = static_cast<uint32_t>(fill - i0 < kSplitUnit ? fill - i0 : kSplitUnit);
    const uint64_t* src = a.sup + r.super_off + rr * r.super_cap + i0;
    const uint64_t first = r.bucket_base + (s << fine_shift);  // first bucket of this super-bucket
    fcnt[threadIdx.x] = 0;
    uint64_t e[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = threadIdx.x + static_cast<uint32_t>(k) * kSplitThreads;
      e[k] = i < n ? src[i] : kEmpty;
    }
    __syncthreads();
    uint32_t fr[kPer];  // (bucket << 16) | rank
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      fr[k] = ~0u;
      if (e[k] == kEmpty) continue;
      const uint64_t pair = e[k] >> sh;
      const uint64_t fine = r.bucket_bits ? pair_hash(pair) >> (64 - r.bucket_bits) : 0ull;
      const uint32_t f = static_cast<uint32_t>(fine) & (n_fine - 1u);
      fr[k] = (f << 16) | atomicAdd(fcnt + f, 1u);
    }
    __syncthreads();
    // Exclusive scan of the counts (bucket = thread) and the reservations.
    const uint32_t c = fcnt[threadIdx.x];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    if (threadIdx.x < n_fine) fbase[threadIdx.x] = c ? atomicAdd(a.fill + first + threadIdx.x, c) : 0u;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < kSplitThreads / 32 ? wsum[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= static_cast<uint32_t>(o)) w += y;
      }
      if (lane < kSplitThreads / 32) wsum[lane] = w;
    }
    __syncthreads();
    lstart[threadIdx.x] = x - c + (warp ? wsum[warp - 1] : 0u);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (fr[k] == ~0u) continue;
      const uint32_t f = fr[k] >> 16;
      const uint32_t at = lstart[f] + (fr[k] & 0xFFFFu);
      if (at < kSplitUnit) {
        stage[at] = e[k];
        stage_f[at] = static_cast<uint16_t>(f);
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += kSplitThreads) {
      const uint32_t f = stage_f[i];
      const uint32_t pos = fbase[f] + (i - lstart[f]);
      if (pos < a.cap) a.ent[(first + f) * a.cap + pos] = stage[i];
      else atomicOr(a.err, kErrBounds);
    }
    __syncthreads();
  }
}

// Round 0 of the bucketed claims, one block per bucket at a time: the
// bucket's entries go into a shared-memory table where, for every pair, the
// smallest entry (the lowest slot) stays; every other claimant joins the
// pending list.  The table is written back over the bucket's region as its
// table of accepted pairs.
__global__ void __launch_bounds__(256, 4) redraw_bucket0_kernel(RedrawArgs a) {
  __shared__ __align__(16) unsigned long long tab[kBucketCap];
  constexpr int kPer = kBucketCap / 256;
  constexpr uint32_t kMask = kBucketCap - 1;
  // Entries are below 2^63, never kEmpty.  The next bucket's entries are
  // loaded while this one's table is built.
  uint64_t b = blockIdx.x;
  uint64_t mine[kPer];
  {
    const uint32_t n = b < a.n_buckets ? min(a.fill[b], a.cap) : 0u;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = threadIdx.x + static_cast<uint32_t>(k) * 256u;
      mine[k] = i < n ? a.ent[b * a.cap + i] : kEmpty;
    }
  }
  while (b < a.n_buckets) {
    const uint64_t b2 = b + gridDim.x;
    const uint32_t n2 = b2 < a.n_buckets ? min(a.fill[b2], a.cap) : 0u;
    const RedrawProj& r = a.rp[bucket_owner(a, b)];
    const int sh = r.slot_bits + 1;
    const uint64_t slot_mask = (1ull << r.slot_bits) - 1;
    for (uint32_t i = threadIdx.x; i < kBucketCap / 2; i += blockDim.x)
      reinterpret_cast<ulonglong2*>(tab)[i] = make_ulonglong2(kEmpty, kEmpty);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (mine[k] == kEmpty) continue;
      const uint64_t pair = mine[k] >> sh;
      uint32_t h = static_cast<uint32_t>(pair_hash(pair)) & kMask;
      for (uint32_t probe = 0; probe <= kMask; ++probe) {
        const uint64_t old = atomicCAS(tab + h, kEmpty, mine[k]);
        if (old == kEmpty) break;
        if ((old >> sh) == pair) {
          const uint64_t prev = atomicMin(tab + h, mine[k]);
          push_pending(a, r.slot_base + ((prev < mine[k] ? mine[k] : prev) & slot_mask));
          break;
        }
        h = (h + 1) & kMask;
      }
    }
    uint64_t nxt[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = threadIdx.x + static_cast<uint32_t>(k) * 256u;
      nxt[k] = i < n2 ? a.ent[b2 * a.cap + i] : kEmpty;
    }
    __syncthreads();
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(a.ent + b * a.cap);
    for (uint32_t i = threadIdx.x; i < kBucketCap / 2; i += blockDim.x) dst[i] = reinterpret_cast<ulonglong2*>(tab)[i];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) mine[k] = nxt[k];
    b = b2;
  }
}

// Decides the slots of round r >= 1: winners become accepted, the others are
// appended to next_pending (the order of the list is irrelevant: each slot's
// later draws depend only on the slot and the round).
__global__ void redraw_resolve_kernel(RedrawArgs a, const uint64_t* pending, uint64_t n_pending,
                                      const unsigned long long* d_count) {
  if (d_count) n_pending = *d_count;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n_pending; q += stride) {
    const uint64_t g = pending[q];
    const SlotRef x = slot_ref(a, g);
    const DevProj& P = *x.P;
    const uint64_t pair = a.pairs[g];
    const uint32_t s = static_cast<uint32_t>(pair >> 32), t = static_cast<uint32_t>(pair);
    bool ok = allowed_pair(P, a.arr, s, t);
    if (ok && !P.multapses) ok = a.bucketed ? bucket_resolve(a, *x.r, P, s, t, x.i) : resolve(a, *x.r, P, s, t, x.i);
    if (!ok) push_pending(a, g);
  }
}

__global__ void redraw_rounds_check_kernel(const unsigned long long* d_count, uint32_t* err) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *d_count != 0) atomicOr(err, kErrGraphRounds);
}

// Writes the redraw projections' connections (global pair tables): the final
// pairs with the round-0 weight and delay of each slot.  Blocks take chunks
// of kChunk slots of one projection (delay table reloaded when the
// projection changes).
__global__ void __launch_bounds__(kGenThreads) total_emit_kernel(GenArgs g, RedrawArgs a, uint64_t total_chunks) {
  extern __shared__ uint32_t smem_raw[];
  const uint32_t hw = hist_words(g);
  SmemTables tabs{smem_raw + hw, reinterpret_cast<uint16_t*>(smem_raw + hw + g.max_delay_len)};
  const BlockHist bh = block_hist_begin(g, smem_raw);
  __syncthreads();
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  int cur = -1;
  for (uint64_t c = blockIdx.x; c < total_chunks; c += gridDim.x) {
    const int lo = chunk_owner(a, c);
    const RedrawProj& r = a.rp[lo];
    const DevProj& P = a.projs[r.proj];
    if (lo != cur) {
      __syncthreads();
      load_delay_table(P, g.thr_blob, g.guide_blob, tabs);
      __syncthreads();
      cur = lo;
    }
    const uint64_t start = (c - r.chunk_base) * kChunk;
    const uint64_t end = min(start + kChunk, P.count);
    for (int win = 0; win < kChunk / (128 * (kGenThreads / 32)); ++win) {
      const uint64_t wbase = start + (static_cast<uint64_t>(warp) * (kChunk / (kGenThreads / 32))) +
                             static_cast<uint64_t>(win) * 128;
      if (wbase >= end) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t i = wbase + static_cast<uint64_t>(q) * 32 + lane;
        if (i >= end) continue;
        const uint64_t pair = a.pairs[r.slot_base + i];
        const Words W = draw(P.k0, P.k1, kTagWD, 0, kPrimaryNone, i);
        const uint32_t s = src_node<true>(P, g.arr, static_cast<uint32_t>(pair >> 32) - P.s0);
        const uint32_t t = tgt_node<true>(P, g.arr, static_cast<uint32_t>(pair) - P.t0);
        store(g, bh, P.out_off + i, s - P.t_base, conn_delay<true>(P, g.arr, tabs, i, W.x), t - P.t_base,
              conn_weight<true>(P, g.arr, i, W.z, W.w));
      }
    }
  }
  block_hist_end(g, bh);
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 counts into uint64 offsets (n + 1 entries):
// block sums, one-block scan of the sums, then per-block scans.
// ---------------------------------------------------------------------------
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane) >= o) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    uint64_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (static_cast<int>(lane) >= o) si += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
    if (lane == kScanThreads / 32 - 1) *total = si;
  }
  __syncthreads();
  const uint64_t r = incl - v + warp_sums[warp];
  __syncthreads();
  return r;
}
}  // namespace

__global__ void scan_block_sums(const uint32_t* in, uint64_t n, uint64_t* block_sums) {
  __shared__ uint64_t total;
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
  uint64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const uint64_t i = base + static_cast<uint64_t>(k) * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void scan_sums_single(uint64_t* block_sums, uint64_t n_blocks) {
  __shared__ uint64_t total;
  uint64_t carry = 0;
  for (uint64_t base = 0; base < n_blocks; base += kScanThreads) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t v = i < n_blocks ? block_sums[i] : 0;
    const uint64_t ex = block_exclusive_scan(v, &total);
    if (i < n_blocks) block_sums[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
}

__global__ void scan_apply(const uint32_t* in, uint64_t n, const uint64_t* block_offsets, uint64_t* out) {
  __shared__ uint64_t total;
  // Blocked arrangement: thread handles kScanItems consecutive entries.
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile + static_cast<uint64_t>(threadIdx.x) * kScanItems;
  uint32_t v[kScanItems];
  uint64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0u;
    s += v[k];
  }
  uint64_t run = block_exclusive_scan(s, &total) + block_offsets[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k <= n) out[base + k] = run;
    run += v[k];
  }
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* block_tmp,
                               cudaStream_t st) {
  const uint64_t n_blocks = (n + 1 + kScanTile - 1) / kScanTile;
  scan_block_sums<<<static_cast<unsigned>(n_blocks), kScanThreads, 0, st>>>(in, n, block_tmp);
  scan_sums_single<<<1, kScanThreads, 0, st>>>(block_tmp, n_blocks);
  scan_apply<<<static_cast<unsigned>(n_blocks), kScanThreads, 0, st>>>(in, n, block_tmp, out);
  return cudaGetLastError();
}

uint64_t scan_tmp_entries(uint64_t n) { return (n + 1 + kScanTile - 1) / kScanTile; }

}  // namespace snc
