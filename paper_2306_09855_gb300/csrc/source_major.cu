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
    if (c > kSrcMajorSmall) a.long_list[atomicAdd(a.n_long, 1u)] = s;
  }
}

// Sources of at most kSrcMajorSmall connections: one warp per source at a
// time (no block barriers).  Pass 1 counts the source's delay steps in the
// warp's shared-memory histogram; pass 2 takes its connections in generation
// order, 32 at a time, ranks equal delays by lane (match) after the delay's
// running offset, and writes every connection at the source's offset + that
// rank.
__global__ void __launch_bounds__(kSrcMajorThreads) src_major_small_kernel(SrcMajorArgs a) {
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
    if (c == 0 || c > kSrcMajorSmall) continue;  // uniform over the warp
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


// Sources above kSrcMajorSmall connections: one block per source at a time.
// Pass 1 counts the delay steps; pass 2 takes chunks of kSrcMajorChunk
// connections in generation order, ranks each chunk stably (warp w holds
// items [w*32*I, (w+1)*32*I) lane-interleaved, so warp, item and lane order is
// input order), stages it in shared memory in delay order and writes each
// delay's run of the chunk with consecutive threads, after the runs of the
// earlier chunks.
__global__ void __launch_bounds__(kSrcMajorThreads, 4) src_major_sort_kernel(SrcMajorArgs a) {
  constexpr int TPB = kSrcMajorThreads, IPT = kSrcMajorItems, NW = TPB / 32, CH = kSrcMajorChunk;
  constexpr int RMAX = 1 << kSrcMajorMaxDelayBits;
  constexpr int DPT = RMAX / TPB;  // delays per thread in the per-delay loops
  static_assert(CH == TPB * IPT, "chunk = block x items");
  __shared__ uint64_t run_start[kSrcMajorMaxProj];
  __shared__ uint64_t run_pre[kSrcMajorMaxProj + 1];  // connections before each run
  __shared__ int n_runs_sh;
  __shared__ uint32_t running[RMAX];   // delay counts, then next output offset per delay
  __shared__ uint32_t cstart[RMAX];    // start of each delay's run in the staged chunk
  __shared__ uint16_t wcnt[NW][RMAX];  // per-warp counts, then per-warp offsets
  __shared__ uint32_t scan_tmp[NW];
  __shared__ uint64_t skey[CH];
  __shared__ uint64_t sval[CH];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t R = 1u << a.delay_bits;
  const uint32_t dmask = R - 1u;
  const auto key_at = [&](uint64_t gi) -> uint64_t {
    return a.key32 ? static_cast<uint64_t>(static_cast<const uint32_t*>(a.keys_in)[gi])
                   : static_cast<const uint64_t*>(a.keys_in)[gi];
  };
  // Exclusive block scan of v[DPT] (delays tid*DPT ...); returns the total.
  const auto block_scan = [&](uint32_t (&v)[DPT], uint32_t* out) -> uint32_t {
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) sum += v[q];
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    if (lane == 31) scan_tmp[warp] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      if (w < static_cast<int>(warp)) before += scan_tmp[w];
      total += scan_tmp[w];
    }
    uint32_t run = before + x - sum;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      out[tid * DPT + q] = run;
      run += v[q];
    }
    __syncthreads();  // scan_tmp is reused
    return total;
  };
  const uint32_t n_long = *a.n_long;
  for (uint32_t q = blockIdx.x; q < n_long; q += gridDim.x) {
    const uint32_t s = a.long_list[q];
    const uint64_t base = a.row_base[s];
    const uint64_t c = a.row_base[s + 1] - base;
    if (c <= kSrcMajorSmall) continue;  // uniform over the block
    if (warp == 0) {
      uint64_t start = 0, len = 0;
      const bool has = static_cast<int>(lane) < a.n_proj && run_of(a.projs[lane], s, start, len);
      const uint32_t hm = __ballot_sync(0xffffffffu, has);
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
      if (lane == 31) {
        run_pre[__popc(hm)] = pre;
        n_runs_sh = __popc(hm);
        if (pre != c) atomicOr(a.err, kErrBounds);
      }
    }
    for (uint32_t d = tid; d < RMAX; d += TPB) running[d] = 0;
    __syncthreads();
    const int n_runs = n_runs_sh;
    if (n_runs == 0 || run_pre[n_runs] != c) {  // inconsistent plan: reported, nothing written
      __syncthreads();
      continue;
    }
    const auto gen_index = [&](uint64_t e) -> uint64_t {
      int k = 0;
      while (k + 1 < n_runs && run_pre[k + 1] <= e) ++k;
      return run_start[k] + (e - run_pre[k]);
    };
    // A source of one chunk is ranked, staged and written in one go (its
    // staged order is its final order); longer ones count their delays first.
    const bool one_chunk = c <= CH;
    // Pass 1: delay counts.
    for (uint64_t e0 = 0; !one_chunk && e0 < c; e0 += CH) {
      uint32_t d[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t e = e0 + static_cast<uint32_t>(j) * TPB + tid;
        d[j] = R;
        if (e < c) {
          const uint64_t gi = gen_index(e);
          if (SNC_IN_BOUNDS(a.err, 30u, gi, a.n)) d[j] = static_cast<uint32_t>(key_at(gi)) & dmask;
        }
      }
#pragma unroll
      for (int j = 0; j < IPT; ++j)
        if (d[j] < R) atomicAdd(&running[d[j]], 1u);
    }
    __syncthreads();
    if (!one_chunk) {
      uint32_t v[DPT];
#pragma unroll
      for (int q = 0; q < DPT; ++q) v[q] = running[tid * DPT + q];
      __syncthreads();
      block_scan(v, running);
    }
    // Pass 2: chunks in generation order.
    // While a chunk is ranked the staging buffer is free: it holds one
    // 32-bit lane mask per warp and delay step (the peers of an item).
    static_assert(sizeof(skey) >= sizeof(uint32_t) * NW * RMAX, "peer masks fit the key staging buffer");
    uint32_t* pmask = reinterpret_cast<uint32_t*>(skey) + warp * RMAX;
    for (uint64_t cb = 0; cb < c; cb += CH) {
      // Only the build's R delay steps of each warp's counters and masks are
      // used (R >= 2: a delay step takes at least one bit).
      for (uint32_t i = tid; i < NW * R / 2; i += TPB) {
        const uint32_t w = i / (R / 2), h = i % (R / 2);
        reinterpret_cast<uint32_t*>(&wcnt[w][0])[h] = 0u;
      }
      for (uint32_t i = tid; i < NW * R; i += TPB) reinterpret_cast<uint32_t*>(skey)[(i / R) * RMAX + i % R] = 0u;
      __syncthreads();
      uint64_t key[IPT], val[IPT];
      uint32_t rank[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t e = cb + warp * 32u * IPT + static_cast<uint32_t>(j) * 32u + lane;
        key[j] = ~0ull;
        val[j] = 0;
        if (e < c) {
          const uint64_t gi = gen_index(e);
          if (SNC_IN_BOUNDS(a.err, 31u, gi, a.n)) {
            key[j] = key_at(gi);
            val[j] = a.vals_in[gi];
          }
        }
      }
      // Peers: each lane ORs its bit into its delay's mask and reads the mask
      // back; the lowest peer advances the counter and clears the mask (the
      // match instruction costs about two SM cycles per distinct delay in the
      // warp).  A slot whose lanes hold one delay skips the masks.
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const bool ok = key[j] != ~0ull;
        const uint32_t d = ok ? (static_cast<uint32_t>(key[j]) & dmask) : R;
        uint32_t peers = 0xffffffffu;
        if (__reduce_min_sync(0xffffffffu, d) != __reduce_max_sync(0xffffffffu, d)) {
          if (ok) atomicOr(pmask + d, 1u << lane);
          __syncwarp();
          peers = ok ? pmask[d] : 0u;
        }
        const uint32_t old = ok ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (ok && static_cast<int>(lane) == __ffs(peers) - 1) {
          wcnt[warp][d] = static_cast<uint16_t>(old + __popc(peers));
          pmask[d] = 0u;
        }
        rank[j] = old + __popc(peers & lt);
        __syncwarp();
      }
      __syncthreads();
      uint32_t tot[DPT];
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const uint32_t d = tid * DPT + q;
        uint32_t r = 0;
        if (d < R) {  // the counters of unused delay steps were not cleared
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            const uint32_t cw = wcnt[w][d];
            wcnt[w][d] = static_cast<uint16_t>(r);
            r += cw;
          }
        }
        tot[q] = r;
      }
      const uint32_t n_chunk = block_scan(tot, cstart);  // includes the barriers
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (key[j] == ~0ull) continue;
        const uint32_t d = static_cast<uint32_t>(key[j]) & dmask;
        const uint32_t lp = cstart[d] + wcnt[warp][d] + rank[j];
        if (SNC_IN_BOUNDS(a.err, 33u, lp, CH)) {
          skey[lp] = key[j];
          sval[lp] = val[j];
        }
      }
      __syncthreads();
      for (uint32_t i = tid; i < n_chunk && i < CH; i += TPB) {
        const uint64_t k = skey[i];
        const uint64_t v = sval[i];
        const uint32_t d = static_cast<uint32_t>(k) & dmask;
        const uint64_t pos = base + (one_chunk ? i : running[d] + (i - cstart[d]));
        if (!SNC_IN_BOUNDS(a.err, 32u, pos, a.n)) continue;
        if (a.key32) static_cast<uint32_t*>(a.keys_out)[pos] = static_cast<uint32_t>(k);
        else static_cast<uint64_t*>(a.keys_out)[pos] = k;
        a.target[pos] = static_cast<uint32_t>(v >> 32);
        a.weight[pos] = static_cast<uint32_t>(v);
        a.delay[pos] = static_cast<uint16_t>(d);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < DPT; ++q) running[tid * DPT + q] += tot[q];
      __syncthreads();
    }
  }
}

}  // namespace snc
