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

// One block per source at a time.  Pass 1 counts the source's delay steps;
// pass 2 takes its connections in generation order, chunk by chunk, ranks
// each chunk stably per warp (warp w holds chunk items [w*32*I, (w+1)*32*I)
// lane-interleaved, so warp, item and lane order is input order) and writes
// every connection at the source's offset + its delay's running start + its
// rank.
__global__ void __launch_bounds__(kSrcMajorThreads) src_major_sort_kernel(SrcMajorArgs a) {
  constexpr int TPB = kSrcMajorThreads, IPT = kSrcMajorItems, NW = TPB / 32;
  constexpr int RMAX = 1 << kSrcMajorMaxDelayBits;
  constexpr int DPT = RMAX / TPB;  // digits per thread in the per-digit loops
  __shared__ uint64_t run_start[kSrcMajorMaxProj];
  __shared__ uint64_t run_pre[kSrcMajorMaxProj + 1];  // elements before each run
  __shared__ int n_runs;
  __shared__ uint32_t running[RMAX];                   // delay counts, then next free offset per delay
  __shared__ uint16_t wcnt[NW][RMAX];                  // per-warp counts, then per-warp offsets
  __shared__ uint32_t scan_tmp[NW];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t R = 1u << a.delay_bits;
  const uint32_t dmask = R - 1u;
  const auto key_at = [&](uint64_t gi) -> uint64_t {
    return a.key32 ? static_cast<uint64_t>(static_cast<const uint32_t*>(a.keys_in)[gi])
                   : static_cast<const uint64_t*>(a.keys_in)[gi];
  };
  // Position in the generated arrays of the source's e-th connection.
  const auto gen_index = [&](uint64_t e) -> uint64_t {
    int k = 0;
    while (k + 1 < n_runs && run_pre[k + 1] <= e) ++k;
    return run_start[k] + (e - run_pre[k]);
  };
  for (uint32_t s = blockIdx.x; s < a.n_nodes; s += gridDim.x) {
    const uint64_t base = a.row_base[s];
    const uint64_t c = a.row_base[s + 1] - base;
    if (c == 0) continue;  // uniform over the block
    if (tid == 0) {
      int k = 0;
      uint64_t pre = 0;
      for (int p = 0; p < a.n_proj; ++p) {
        uint64_t start, len;
        if (run_of(a.projs[p], s, start, len) && k < kSrcMajorMaxProj) {
          run_start[k] = start;
          run_pre[k] = pre;
          pre += len;
          ++k;
        }
      }
      run_pre[k] = pre;
      n_runs = k;
      if (pre != c) atomicOr(a.err, kErrBounds);
    }
    for (uint32_t d = tid; d < RMAX; d += TPB) running[d] = 0;
    __syncthreads();
    if (n_runs == 0 || run_pre[n_runs] != c) {  // inconsistent plan: reported, nothing written
      __syncthreads();
      continue;
    }
    // Pass 1: delay counts of the source.
    for (uint64_t e = tid; e < c; e += TPB) {
      const uint64_t gi = gen_index(e);
      if (!SNC_IN_BOUNDS(a.err, 30u, gi, a.n)) continue;
      atomicAdd(&running[static_cast<uint32_t>(key_at(gi)) & dmask], 1u);
    }
    __syncthreads();
    // Exclusive scan of the counts (DPT consecutive delays per thread).
    {
      uint32_t v[DPT];
      uint32_t sum = 0;
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        v[q] = running[tid * DPT + q];
        sum += v[q];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
      }
      if (lane == 31) scan_tmp[warp] = x;
      __syncthreads();
      uint32_t before = 0;
      for (uint32_t w = 0; w < warp; ++w) before += scan_tmp[w];
      uint32_t run = before + x - sum;
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        running[tid * DPT + q] = run;
        run += v[q];
      }
    }
    // Pass 2: chunks in generation order.
    for (uint64_t cb = 0; cb < c; cb += static_cast<uint64_t>(TPB) * IPT) {
      for (uint32_t i = tid; i < NW * RMAX / 2; i += TPB) reinterpret_cast<uint32_t*>(&wcnt[0][0])[i] = 0u;
      __syncthreads();
      uint64_t key[IPT], val[IPT];
      uint32_t rank[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t e = cb + warp * 32u * IPT + static_cast<uint32_t>(j) * 32u + lane;
        const bool ok = e < c;
        uint64_t gi = 0;
        if (ok) gi = gen_index(e);
        const bool in = ok && SNC_IN_BOUNDS(a.err, 31u, gi, a.n);
        key[j] = in ? key_at(gi) : 0ull;
        val[j] = in ? a.vals_in[gi] : 0ull;
        const uint32_t d = ok ? (static_cast<uint32_t>(key[j]) & dmask) : R;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t old = ok ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (ok && static_cast<int>(lane) == __ffs(peers) - 1) wcnt[warp][d] = static_cast<uint16_t>(old + __popc(peers));
        rank[j] = old + __popc(peers & lt);
        __syncwarp();
      }
      __syncthreads();
      uint32_t tot[DPT];
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const uint32_t d = tid * DPT + q;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint32_t cw = wcnt[w][d];
          wcnt[w][d] = static_cast<uint16_t>(r);
          r += cw;
        }
        tot[q] = r;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t e = cb + warp * 32u * IPT + static_cast<uint32_t>(j) * 32u + lane;
        if (e >= c) continue;
        const uint32_t d = static_cast<uint32_t>(key[j]) & dmask;
        const uint64_t pos = base + running[d] + wcnt[warp][d] + rank[j];
        if (!SNC_IN_BOUNDS(a.err, 32u, pos, a.n)) continue;
        if (a.key32) static_cast<uint32_t*>(a.keys_out)[pos] = static_cast<uint32_t>(key[j]);
        else static_cast<uint64_t*>(a.keys_out)[pos] = key[j];
        a.target[pos] = static_cast<uint32_t>(val[j] >> 32);
        a.weight[pos] = static_cast<uint32_t>(val[j]);
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
