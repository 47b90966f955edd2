// source_major.cu -- stable (source, delay) sort of builds generated source
// by source: a counting sort of each source's runs by delay step.
#include "source_major.h"

#include "snc.h"
#include "snc_check.cuh"

namespace snc {

bool source_major_rule(uint32_t rule) {
  return rule == SNC_ONE_TO_ONE || rule == SNC_ALL_TO_ALL || rule == SNC_FIXED_OUTDEGREE;
}

namespace {

// The run of source s in projection P: positions [start, start + len) of the
// generated arrays, in generation order (Sec. 2.1 numbering of the rule).
__device__ __forceinline__ bool run_of(const DevProj& P, uint32_t s, uint64_t& start, uint64_t& len) {
  if (P.count == 0 || s < P.s0 || s - P.s0 >= P.ns) return false;
  const uint32_t row = s - P.s0;
  if (P.rule == SNC_FIXED_OUTDEGREE) {
    len = P.k;
    start = P.out_off + static_cast<uint64_t>(row) * P.k;
  } else if (P.rule == SNC_ALL_TO_ALL) {
    // Without autapses the diagonal target of a row is skipped and later
    // rows shift back by the diagonals before them.
    const bool diag = !P.autapses && s >= P.t0 && s - P.t0 < P.nt;
    uint64_t before = 0;
    if (!P.autapses) {
      const uint32_t lo = max(P.s0, P.t0), hi = min(P.s0 + P.ns, P.t0 + P.nt);
      if (hi > lo && s > lo) before = min(s, hi) - lo;
    }
    len = P.nt - (diag ? 1u : 0u);
    start = P.out_off + static_cast<uint64_t>(row) * P.nt - before;
  } else {  // one_to_one: a projection that drops its pairs has no connections
    len = 1;
    start = P.out_off + row;
  }
  return len > 0;
}

}  // namespace

__global__ void src_major_count_kernel(SrcMajorArgs a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.n_nodes; s += stride) {
    uint64_t c = 0;
    for (int p = 0; p < a.n_proj; ++p) {
      uint64_t start, len;
      if (run_of(a.projs[p], s, start, len)) c += len;
    }
    if (c > 0xFFFFFFFFull) {
      atomicOr(a.err, kErrBounds);
      c = 0;
    }
    a.counts[s] = static_cast<uint32_t>(c);
  }
}

// One warp per source at a time (no block barriers: sources are short).
// Pass 1 counts the source's delay steps in the warp's shared-memory
// histogram; pass 2 takes its connections in generation order, 32 at a time,
// ranks equal delays by lane (match) after the delay's running offset, and
// writes every connection at the source's offset + that rank.
__global__ void __launch_bounds__(kSrcMajorThreads) src_major_sort_kernel(SrcMajorArgs a) {
  constexpr int NW = kSrcMajorThreads / 32, U = kSrcMajorItems;
  constexpr int RMAX = 1 << kSrcMajorMaxDelayBits;
  __shared__ uint32_t hist_all[NW][RMAX];  // delay counts, then running offsets
  __shared__ uint64_t run_start_all[NW][kSrcMajorMaxProj];
  __shared__ uint64_t run_pre_all[NW][kSrcMajorMaxProj + 1];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* hist = hist_all[warp];
  uint64_t* run_start = run_start_all[warp];
  uint64_t* run_pre = run_pre_all[warp];
  const uint32_t R = 1u << a.delay_bits;
  const uint32_t dmask = R - 1u;
  const uint32_t per_lane = (R + 31u) / 32u;  // histogram bins per lane in the scan
  const uint64_t total_warps = static_cast<uint64_t>(gridDim.x) * NW;
  const auto key_at = [&](uint64_t gi) -> uint64_t {
    return a.key32 ? static_cast<uint64_t>(static_cast<const uint32_t*>(a.keys_in)[gi])
                   : static_cast<const uint64_t*>(a.keys_in)[gi];
  };
  for (uint64_t s = static_cast<uint64_t>(blockIdx.x) * NW + warp; s < a.n_nodes; s += total_warps) {
    const uint64_t base = a.row_base[s];
    const uint64_t c = a.row_base[s + 1] - base;
    if (c == 0) continue;  // uniform over the warp
    // Runs: lane p looks at projection p; the runs are kept in projection
    // (Connect) order.
    uint64_t start = 0, len = 0;
    const bool has = static_cast<int>(lane) < a.n_proj &&
                     run_of(a.projs[lane], static_cast<uint32_t>(s), start, len);
    const uint32_t hm = __ballot_sync(0xffffffffu, has);
    const int n_runs = __popc(hm);
    uint64_t pre = has ? len : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= static_cast<uint32_t>(o)) pre += y;
    }
    if (has) {
      const int k = __popc(hm & lt);
      run_start[k] = start;
      run_pre[k] = pre - len;
    }
    const uint64_t total = __shfl_sync(0xffffffffu, pre, 31);
    if (lane == 0) run_pre[n_runs] = total;
    for (uint32_t d = lane; d < R; d += 32) hist[d] = 0;
    __syncwarp();
    if (total != c || n_runs == 0) {  // inconsistent plan: reported, nothing written
      if (lane == 0) atomicOr(a.err, kErrBounds);
      continue;
    }
    const auto gen_index = [&](uint64_t e) -> uint64_t {
      int k = 0;
      while (k + 1 < n_runs && run_pre[k + 1] <= e) ++k;
      return run_start[k] + (e - run_pre[k]);
    };
    // Pass 1: delay counts.
    for (uint64_t e0 = 0; e0 < c; e0 += 32u * U) {
      uint32_t d[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t e = e0 + static_cast<uint32_t>(u) * 32u + lane;
        d[u] = R;
        if (e < c) {
          const uint64_t gi = gen_index(e);
          if (SNC_IN_BOUNDS(a.err, 30u, gi, a.n)) d[u] = static_cast<uint32_t>(key_at(gi)) & dmask;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (d[u] < R) atomicAdd(hist + d[u], 1u);
    }
    __syncwarp();
    // Exclusive scan of the counts: lane l holds bins [l * per_lane, ...).
    {
      uint32_t sum = 0;
      for (uint32_t q = 0; q < per_lane; ++q) {
        const uint32_t b = lane * per_lane + q;
        if (b < R) sum += hist[b];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
      }
      uint32_t run = x - sum;
      for (uint32_t q = 0; q < per_lane; ++q) {
        const uint32_t b = lane * per_lane + q;
        if (b < R) {
          const uint32_t v = hist[b];
          hist[b] = run;
          run += v;
        }
      }
    }
    __syncwarp();
    // Pass 2: 32 connections at a time in generation order.
    for (uint64_t e0 = 0; e0 < c; e0 += 32u * U) {
      uint64_t key[U], val[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t e = e0 + static_cast<uint32_t>(u) * 32u + lane;
        key[u] = ~0ull;
        val[u] = 0;
        if (e < c) {
          const uint64_t gi = gen_index(e);
          if (SNC_IN_BOUNDS(a.err, 31u, gi, a.n)) {
            key[u] = key_at(gi);
            val[u] = a.vals_in[gi];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool ok = key[u] != ~0ull;
        const uint32_t d = ok ? (static_cast<uint32_t>(key[u]) & dmask) : R;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t old = ok ? hist[d] : 0u;
        __syncwarp();
        if (ok && static_cast<int>(lane) == __ffs(peers) - 1) hist[d] = old + __popc(peers);
        __syncwarp();
        if (!ok) continue;
        const uint64_t pos = base + old + __popc(peers & lt);
        if (!SNC_IN_BOUNDS(a.err, 32u, pos, a.n)) continue;
        if (a.key32) static_cast<uint32_t*>(a.keys_out)[pos] = static_cast<uint32_t>(key[u]);
        else static_cast<uint64_t*>(a.keys_out)[pos] = key[u];
        a.target[pos] = static_cast<uint32_t>(val[u] >> 32);
        a.weight[pos] = static_cast<uint32_t>(val[u]);
        a.delay[pos] = static_cast<uint16_t>(d);
      }
    }
    __syncwarp();
  }
}

}  // namespace snc
