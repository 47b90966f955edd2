// sort_kernels.cu -- stable LSD radix sort of (key, value) pairs with 32- or
// 64-bit keys and values: one upfront histogram of every digit, then one
// "onesweep" pass per digit (Adinets & Merrill 2022) whose tiles find their
// global offsets by decoupled look-back (Merrill & Garland 2016).
//
// The paper sorts connections by source and delay with an extension of radix
// sort (Sec. 2.2).  Here the key packs (source, delay) and the value carries
// (target, weight); the sort is stable, so connections with equal keys keep
// their generation order.
//
// Look-back status words are 64-bit: [flag:2][epoch:14][count:48].  The epoch
// changes every pass, so a stale word from an earlier pass reads as "not yet
// published" and the array never needs clearing between passes.  Every wait
// on a predecessor is bounded; on expiry the kernel sets an error bit and
// finishes its tile without waiting (the result is then wrong, the error is
// reported by snc_synchronize, and the GPU is never held).
#include <cuda_runtime.h>

#include <cstdint>

#include "digit_hist.cuh"
#include "snc_check.cuh"
#include "snc_internal.h"
#include "sort_kernels.h"

namespace snc {

namespace {

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kCountMask = (1ull << 48) - 1;
constexpr uint32_t kSpinLimit = kDefaultSpinLimit;  // bulk-copy waits

__device__ __forceinline__ void st_status(uint64_t* p, uint64_t v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ uint64_t ld_status(const uint64_t* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan over the block of one uint32 per thread; *total gets the sum.
template <int TPB>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tmp, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane) >= o) incl += y;
  }
  if (lane == 31) warp_tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = TPB / 32;
    const uint32_t s = lane < NW ? warp_tmp[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (static_cast<int>(lane) >= o) si += y;
    }
    if (lane < NW) warp_tmp[lane] = si - s;
    if (lane == NW - 1) *total = si;
  }
  __syncthreads();
  return incl - v + warp_tmp[warp];
}

}  // namespace

// ---------------------------------------------------------------------------
// Histogram of every pass's digit over all keys (shared-memory counters per
// block, merged into global 64-bit counters).
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(512) radix_hist_kernel(const K* __restrict__ keys, uint64_t n, HistPlan plan) {
  extern __shared__ uint32_t sh[];
  const HistRegs r = hist_regs(plan);
  hist_clear(sh, r);
  __syncthreads();
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  constexpr int PER = 16 / sizeof(K);  // keys per 16-byte vector
  const uint64_t vecs = n / PER;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys);
  const bool aligned = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
  if (aligned) {
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < vecs; i += stride) {
      const uint4 v = k4[i];
      const K* kv = reinterpret_cast<const K*>(&v);
#pragma unroll
      for (int j = 0; j < PER; ++j) hist_add(sh, r, static_cast<uint64_t>(kv[j]));
    }
    for (uint64_t i = vecs * PER + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
      hist_add(sh, r, static_cast<uint64_t>(keys[i]));
  } else {
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
      hist_add(sh, r, static_cast<uint64_t>(keys[i]));
  }
  __syncthreads();
  hist_flush(sh, r, plan.global);
}

HistPlan hist_plan(const SortPasses& sp, unsigned long long* global) {
  HistPlan h{};
  h.global = global;
  h.n_passes = sp.n_passes;
  h.stride = 1 << sp.kernel_bits;
  for (int p = 0; p < kMaxPasses; ++p) {
    h.shift[p] = p < sp.n_passes ? sp.shift[p] : 0;
    h.mask[p] = p < sp.n_passes ? sp.mask[p] : 0u;
  }
  return h;
}

// Exclusive scan of each pass's digit counts (one block of kDigitScanThreads
// per pass, each thread owning kMaxRadix / kDigitScanThreads consecutive
// digits).
__global__ void radix_digit_scan_kernel(const unsigned long long* __restrict__ hist, uint64_t* __restrict__ start) {
  constexpr int PER = kMaxRadix / kDigitScanThreads;
  __shared__ uint64_t wsum[kDigitScanThreads / 32];
  const int p = blockIdx.x;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned long long* h = hist + static_cast<size_t>(p) * kMaxRadix + threadIdx.x * PER;
  uint64_t v[PER];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    v[i] = h[i];
    sum += v[i];
  }
  uint64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane) >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint64_t before = 0;
  for (uint32_t w = 0; w < warp; ++w) before += wsum[w];
  uint64_t run = before + incl - sum;
  uint64_t* out = start + static_cast<size_t>(p) * kMaxRadix + threadIdx.x * PER;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    out[i] = run;
    run += v[i];
  }
}

// Writes one sorted pair, or on an unpacking last pass its target, weight
// and delay.
template <bool UNPACK, typename K, typename V>
__device__ __forceinline__ void emit_pair(const OnesweepArgs<K, V>& a, uint64_t pos, K k, V v) {
  a.keys_out[pos] = k;
  if constexpr (UNPACK && sizeof(V) == 8) {
    {
      a.unpack_target[pos] = static_cast<uint32_t>(v >> 32);
      a.unpack_weight[pos] = static_cast<uint32_t>(v);
      a.unpack_delay[pos] = static_cast<uint16_t>(static_cast<uint32_t>(k) & a.unpack_delay_mask);
      return;
    }
  }
  a.vals_out[pos] = v;
}

// ---------------------------------------------------------------------------
// One onesweep pass.  Tile = 256 threads x 16 keys; warp w ranks keys
// [w*512, (w+1)*512) of the tile lane-interleaved, so that ranking warp by
// warp and item by item preserves input order (stability).
//
// G = 1: a block ranks its tile, publishes the tile's digit counts, looks
// back over earlier tiles for its global offsets and scatters the tile.
// G > 1: a block takes a group of G consecutive tiles, first counts the
// group's digits (so that the look-back runs once per group), then ranks and
// scatters the group's tiles one after another with per-digit running
// offsets; the second read of the group's keys is meant to hit L2.
// Groups / tiles are taken from a dynamic ticket, so every predecessor has
// already started when a block waits for it.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

template <int BITS, int G, typename K, typename V>
struct Onesweep {
  static constexpr int TPB = kSortThreads, IPT = kSortItems, TILE = kSortTile;
  static constexpr int RADIX = 1 << BITS;
  static constexpr int NW = TPB / 32;
  static constexpr int GROUP = TILE * G;
  static constexpr int DPT = RADIX / TPB;  // digits per thread
  static constexpr int W = DPT >= 8 ? 2 : (DPT >= 4 ? 4 : 8);  // look-back window per round
  static constexpr int MINB = BITS <= 9 ? 3 : 2;                // resident blocks per SM
  static constexpr size_t kCntBytes = static_cast<size_t>(NW) * RADIX * sizeof(uint16_t);
  static constexpr size_t kTileBytes = static_cast<size_t>(TILE) * (sizeof(K) + sizeof(V));
  static constexpr size_t kUnion = kCntBytes > kTileBytes ? kCntBytes : kTileBytes;
  static constexpr size_t kSmem = kUnion + RADIX * sizeof(uint32_t) * 2 + RADIX * sizeof(uint64_t);
  // Peer masks (one 32-bit word per warp and digit) after the counters,
  // while ranking, when both fit the tile's staging area.
  static constexpr bool kMaskRank = kCntBytes * 3 <= kTileBytes;
};

// Sum, for each of this thread's DPT digits, the counts that groups before
// `unit` published (decoupled look-back, W predecessors per round trip).
template <int RADIX, int DPT, int W, typename A>
__device__ __forceinline__ void look_back(const A& a, uint32_t unit, uint64_t (&prefix)[DPT]) {
  const uint32_t tid = threadIdx.x;
  int32_t look[DPT];
  uint32_t pending = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    prefix[q] = 0;
    look[q] = static_cast<int32_t>(unit) - 1;
    if (unit > 0) pending |= 1u << q;
  }
  uint32_t spins = 0;
  uint32_t backoff = 32u;
  while (pending) {
    bool progress = false;
    uint64_t v[DPT][W];
#pragma unroll
    for (int q = 0; q < DPT; ++q)
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int32_t t = look[q] - w;
        v[q][w] = ((pending >> q) & 1u) && t >= 0
                      ? ld_status(a.status + static_cast<size_t>(t) * RADIX + tid * DPT + q)
                      : 0ull;
      }
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      if (!((pending >> q) & 1u)) continue;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint64_t x = v[q][w];
        const bool fresh = ((x >> 48) & 0x3FFFull) == a.epoch;
        const uint64_t flag = fresh ? (x & (3ull << 62)) : 0ull;
        if (flag == 0 || look[q] < 0) break;  // not yet published: read again next round
        progress = true;
        prefix[q] += x & kCountMask;
        if (flag == kFlagInc) {
          pending &= ~(1u << q);
          break;
        }
        --look[q];
      }
    }
    if (pending && !progress) {
      if (++spins > a.lookback_spin_limit) {
        atomicOr(a.err, kErrLookbackTimeout);
        break;
      }
      __nanosleep(backoff);  // let the other warps of the SM issue
      backoff = backoff < 1024u ? backoff * 2u : 1024u;
    } else {
      backoff = 32u;
    }
  }
}

template <int BITS, int G, bool UNPACK, typename K, typename V>
__global__ void __launch_bounds__(kSortThreads, (Onesweep<BITS, G, K, V>::MINB))
    onesweep_kernel(OnesweepArgs<K, V> a) {
  using C = Onesweep<BITS, G, K, V>;
  constexpr int RADIX = C::RADIX, NW = C::NW, TILE = C::TILE, GROUP = C::GROUP, DPT = C::DPT, W = C::W;
  constexpr int TPB = C::TPB, IPT = C::IPT;
  static_assert(RADIX % TPB == 0, "radix must be a multiple of the block size");

  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(smem);
  K* skeys = reinterpret_cast<K*>(smem);
  V* svals = reinterpret_cast<V*>(smem + static_cast<size_t>(TILE) * sizeof(K));
  uint32_t* ghist = reinterpret_cast<uint32_t*>(smem + C::kUnion);
  uint32_t* local_start = ghist + RADIX;
  uint64_t* run = reinterpret_cast<uint64_t*>(smem + C::kUnion + 2 * RADIX * sizeof(uint32_t));
  __shared__ uint32_t unit_sh;
  __shared__ uint32_t warp_tmp[32];
  __shared__ uint32_t scan_total;

  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t mask = a.mask;
  const int shift = a.shift;
  const uint32_t lt = lanemask_lt();
  const uint64_t ep = static_cast<uint64_t>(a.epoch) << 48;

  for (;;) {
    if (tid == 0) unit_sh = atomicAdd(a.tile_counter, 1u);
    if (G > 1)
      for (int i = tid; i < RADIX; i += TPB) ghist[i] = 0u;
    __syncthreads();
    const uint32_t unit = unit_sh;
    if (static_cast<uint64_t>(unit) * GROUP >= a.n) break;
    const uint64_t gbase = static_cast<uint64_t>(unit) * GROUP;
    uint64_t* st_row = a.status + static_cast<size_t>(unit) * RADIX + static_cast<size_t>(tid) * DPT;

    if (G > 1) {
      // Digit counts of the whole group (coalesced, order irrelevant).
      for (int s = 0; s < G; ++s) {
        const uint64_t tbase = gbase + static_cast<uint64_t>(s) * TILE;
        if (tbase >= a.n) break;
        uint32_t d[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const uint64_t idx = tbase + static_cast<uint64_t>(j) * TPB + tid;
          d[j] = idx < a.n ? (static_cast<uint32_t>(a.keys_in[idx] >> shift) & mask) : static_cast<uint32_t>(RADIX);
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const uint32_t d0 = __shfl_sync(0xffffffffu, d[j], 0);
          if (__all_sync(0xffffffffu, d[j] == d0)) {
            if (lane == 0 && d0 < RADIX) atomicAdd(&ghist[d0], 32u);
          } else if (d[j] < RADIX) {
            atomicAdd(&ghist[d[j]], 1u);
          }
        }
      }
      __syncthreads();
      uint32_t cnt[DPT];
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        cnt[q] = ghist[tid * DPT + q];
        if (unit != a.withhold_unit) st_status(st_row + q, (unit == 0 ? kFlagInc : kFlagAgg) | ep | cnt[q]);
      }
      uint64_t prefix[DPT];
      look_back<RADIX, DPT, W>(a, unit, prefix);
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        if (unit > 0 && unit != a.withhold_unit)
          st_status(st_row + q, kFlagInc | ep | ((prefix[q] + cnt[q]) & kCountMask));
        run[tid * DPT + q] = a.digit_start[tid * DPT + q] + prefix[q];
      }
    }

    for (int s = 0; s < G; ++s) {
      const uint64_t tbase = gbase + static_cast<uint64_t>(s) * TILE;
      if (tbase >= a.n) break;
      __syncthreads();  // previous tile's staging and run[] update are complete
      for (int i = tid; i < NW * RADIX / 2; i += TPB) reinterpret_cast<uint32_t*>(wcnt)[i] = 0u;
      if constexpr (C::kMaskRank)
        for (int i = tid; i < NW * RADIX; i += TPB) reinterpret_cast<uint32_t*>(smem + C::kCntBytes)[i] = 0u;
      __syncthreads();
      const uint64_t warp_base = tbase + static_cast<uint64_t>(warp) * 32 * IPT;
      K key[IPT];
      uint32_t rank[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
        key[j] = idx < a.n ? a.keys_in[idx] : K(0);
      }
      uint16_t* my = wcnt + static_cast<size_t>(warp) * RADIX;
      uint32_t* pmask = reinterpret_cast<uint32_t*>(smem + C::kCntBytes) + static_cast<size_t>(warp) * RADIX;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
        const bool valid = idx < a.n;
        const uint32_t d = valid ? (static_cast<uint32_t>(key[j] >> shift) & mask) : static_cast<uint32_t>(RADIX);
        uint32_t peers = 0xffffffffu;
        if constexpr (C::kMaskRank) {
          // Peers from the lane masks (as in the bulk-copy kernel below).
          if (__reduce_min_sync(0xffffffffu, d) != __reduce_max_sync(0xffffffffu, d)) {
            if (valid) atomicOr(pmask + d, 1u << lane);
            __syncwarp();
            peers = valid ? pmask[d] : 0u;
          }
        } else {
          peers = __match_any_sync(0xffffffffu, d);
        }
        const uint32_t old = valid ? my[d] : 0u;
        __syncwarp();
        if (valid && static_cast<int>(lane) == __ffs(peers) - 1) {
          my[d] = static_cast<uint16_t>(old + __popc(peers));
          if constexpr (C::kMaskRank) pmask[d] = 0u;
        }
        rank[j] = old + __popc(peers & lt);
        __syncwarp();
      }
      __syncthreads();
      // Per digit: exclusive offsets across warps and the tile total.
      uint32_t tot[DPT];
      uint32_t tsum = 0;
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint32_t c = wcnt[w * RADIX + d];
          wcnt[w * RADIX + d] = static_cast<uint16_t>(r);
          r += c;
        }
        tot[q] = r;
        tsum += r;
      }
      if (G == 1) {
        // Publish the tile's counts before the local scan, then look back.
#pragma unroll
        for (int q = 0; q < DPT; ++q)
          if (unit != a.withhold_unit) st_status(st_row + q, (unit == 0 ? kFlagInc : kFlagAgg) | ep | tot[q]);
      }
      uint32_t excl = block_excl_scan<TPB>(tsum, warp_tmp, &scan_total);
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        local_start[tid * DPT + q] = excl;
        excl += tot[q];
      }
      if (G == 1) {
        uint64_t prefix[DPT];
        look_back<RADIX, DPT, W>(a, unit, prefix);
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
          if (unit > 0 && unit != a.withhold_unit)
            st_status(st_row + q, kFlagInc | ep | ((prefix[q] + tot[q]) & kCountMask));
          run[tid * DPT + q] = a.digit_start[tid * DPT + q] + prefix[q];
        }
      }
      __syncthreads();
      uint32_t lpos[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
        const uint32_t d = static_cast<uint32_t>(key[j] >> shift) & mask;
        lpos[j] = idx < a.n ? local_start[d] + wcnt[warp * RADIX + d] + rank[j] : 0xFFFFFFFFu;
      }
      __syncthreads();  // counters are dead; the union becomes the staging area
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (lpos[j] != 0xFFFFFFFFu && SNC_IN_BOUNDS(a.err, 10u, lpos[j], TILE)) {
          const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
          skeys[lpos[j]] = key[j];
          svals[lpos[j]] = a.vals_in[idx];
        }
      }
      __syncthreads();
      const uint64_t left = a.n - tbase;
      const uint32_t valid = left < static_cast<uint64_t>(TILE) ? static_cast<uint32_t>(left) : static_cast<uint32_t>(TILE);
      for (uint32_t i = tid; i < valid; i += TPB) {
        const K k = skeys[i];
        const uint32_t d = static_cast<uint32_t>(k >> shift) & mask;
        const uint64_t pos = run[d] + (i - local_start[d]);
        if (!SNC_IN_BOUNDS(a.err, 11u + 0x100u * d, pos, a.n)) continue;
        emit_pair<UNPACK>(a, pos, k, svals[i]);
      }
      __syncthreads();  // all reads of run[] for this tile are done
#pragma unroll
      for (int q = 0; q < DPT; ++q) run[tid * DPT + q] += tot[q];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// TMA-fed onesweep pass for 8- and 9-bit digits (one look-back per tile of
// 256 threads x ITEMS keys, 2,048 to 8,192).  A persistent block takes tiles
// from the ticket; one thread issues
// two bulk copies (cp.async.bulk, completion on an mbarrier) that bring the
// tile's keys and values into shared memory, so the ranking reads keys from
// shared memory and all tile-local indices are 32-bit.  After the keys are in
// registers the key buffer is reused to stage the tile in digit order.  The
// last, partial tile is loaded with ordinary loads.  Every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbarrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// 32-bit look-back words [tile][digit] = [flag:2][count:30] for the
// bulk-copy kernel (the area is cleared before every pass, counts < 2^30).
constexpr uint32_t kAgg32 = 1u << 30;
constexpr uint32_t kInc32 = 2u << 30;
constexpr uint32_t kCount32 = (1u << 30) - 1u;

__device__ __forceinline__ void st_status32(uint32_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t*>(p) = v;
}
__device__ __forceinline__ uint32_t ld_status32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// The first tile of the sort (or of its segment) has no predecessor; the
// others look back until an inclusive value, which the first tile of their
// segment always publishes, so a look-back never leaves its segment.
template <int RADIX, int DPT, int W, typename A>
__device__ __forceinline__ void look_back32(const A& a, uint32_t unit, bool first, uint64_t (&prefix)[DPT]) {
  const uint32_t tid = threadIdx.x;
  const uint32_t* base = a.status32 + tid * DPT;
  int32_t look[DPT];
  uint32_t pending = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    prefix[q] = 0;
    look[q] = static_cast<int32_t>(unit) - 1;
    if (!first) pending |= 1u << q;
  }
  uint32_t spins = 0, backoff = 32u;
  while (pending) {
    bool progress = false;
    uint32_t v[DPT][W];
#pragma unroll
    for (int q = 0; q < DPT; ++q)
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int32_t t = look[q] - w;
        v[q][w] = ((pending >> q) & 1u) && t >= 0 ? ld_status32(base + static_cast<size_t>(t) * RADIX + q) : 0u;
      }
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      if (!((pending >> q) & 1u)) continue;
      uint32_t sum = 0;
      int used = 0;
      bool done = false;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        if (done) continue;
        const uint32_t x = v[q][w];
        if (x < kAgg32) {  // not yet published
          done = true;
          continue;
        }
        sum += x & kCount32;
        ++used;
        if (x >= kInc32) {
          pending &= ~(1u << q);
          done = true;
        }
      }
      prefix[q] += sum;
      look[q] -= used;
      progress = progress || used > 0;
    }
    if (pending && !progress) {
      if (++spins > a.lookback_spin_limit) {
        atomicOr(a.err, kErrLookbackTimeout);
        break;
      }
      __nanosleep(backoff);
      backoff = backoff < 1024u ? backoff * 2u : 1024u;
    } else {
      backoff = 32u;
    }
  }
}

template <int BITS, int ITEMS, typename K, typename V>
struct OnesweepTma {
  static constexpr int TPB = kSortThreads, IPT = ITEMS, TILE = kSortThreads * ITEMS;
  static constexpr int RADIX = 1 << BITS;
  static constexpr int NW = TPB / 32;
  static constexpr int DPT = RADIX / TPB;
  static constexpr int W = DPT >= 2 ? 4 : 8;
  static constexpr size_t kKeysBytes = static_cast<size_t>(TILE) * sizeof(K);  // input / staged keys
  static constexpr size_t kValsBytes = static_cast<size_t>(TILE) * sizeof(V);  // input / staged values
  static constexpr size_t kBufBytes = (kKeysBytes + kValsBytes + 127) / 128 * 128;
  static constexpr size_t kCntBytes = static_cast<size_t>(NW) * RADIX * sizeof(uint16_t);
  static constexpr size_t kOffCnt = kBufBytes;
  static constexpr size_t kOffLocal = kOffCnt + kCntBytes;
  static constexpr size_t kOffGlob = kOffLocal + RADIX * sizeof(uint32_t);
  static constexpr size_t kOffBar = kOffGlob + RADIX * sizeof(uint64_t);
  static constexpr size_t kSmem = kOffBar + 16;
  // Resident blocks per SM: shared memory (228 KB per SM, 1 KB reserved per
  // block) and the register target of the item count (24 and 32 -> 2,
  // 16 -> 3, 12 -> 4, 8 -> 5 blocks of 256 threads).  Larger tiles take
  // fewer look-backs per key.
  static constexpr int kFit = static_cast<int>((228u * 1024u) / (kSmem + 1024u + 256u));
  static constexpr int kRegCap = ITEMS >= 20 ? 2 : (ITEMS >= 16 ? 3 : (ITEMS >= 12 ? 4 : 5));
  static constexpr int MINB = kFit < 1 ? 1 : (kFit > kRegCap ? kRegCap : kFit);
  // Peer masks in the warp's part of the key buffer (32 * IPT keys) during
  // ranking: one 32-bit word per digit.
  static constexpr bool kMaskRank = static_cast<size_t>(RADIX) * 4u <= 32u * IPT * sizeof(K);
};

// Bounded wait for a bulk copy, with the outcome voted over the block so
// that every thread leaves together when it times out.
__device__ __forceinline__ bool tile_wait(uint64_t* bar, uint32_t parity) {
  uint32_t spins = 0;
  bool ok = true;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > kSpinLimit) {
      ok = false;
      break;
    }
  }
  return __syncthreads_and(ok) != 0;
}

// One pass.  A persistent block takes tiles from the ticket in increasing
// order and sorts each before taking the next, so the lowest unfinished tile
// is always being sorted and every look-back wait ends.
template <int BITS, int ITEMS, bool UNPACK, typename K, typename V>
__global__ void __launch_bounds__(kSortThreads, (OnesweepTma<BITS, ITEMS, K, V>::MINB))
    onesweep_tma_kernel(OnesweepArgs<K, V> a) {
  using C = OnesweepTma<BITS, ITEMS, K, V>;
  constexpr int RADIX = C::RADIX, NW = C::NW, TILE = C::TILE, DPT = C::DPT, W = C::W;
  constexpr int TPB = C::TPB, IPT = C::IPT;
  static_assert(RADIX % TPB == 0, "radix must be a multiple of the block size");
  extern __shared__ __align__(128) unsigned char smem[];
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(smem + C::kOffCnt);
  uint64_t* globm = reinterpret_cast<uint64_t*>(smem + C::kOffGlob);  // global position of local index 0
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kOffBar);
  __shared__ uint32_t ticket_sh;
  __shared__ uint32_t warp_tmp[32];
  __shared__ uint32_t scan_total;

  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t mask = a.mask;
  const int shift = a.shift;
  const uint32_t lt = lanemask_lt();
  // Tiles: consecutive TILE-key ranges of [0, n), or with segments the
  // tiles of each segment in turn (a segment's last tile may be partial).
  const uint64_t n_tiles = a.n_seg ? a.seg_tile_begin[a.n_seg] : (a.n + TILE - 1) / TILE;
  __shared__ uint64_t tile_base_sh;
  __shared__ uint32_t tile_valid_sh, tile_seg_sh, tile_first_sh;
  const auto buf_keys = [&](int b) { return reinterpret_cast<K*>(smem + b * C::kBufBytes); };
  const auto buf_vals = [&](int b) { return reinterpret_cast<V*>(smem + b * C::kBufBytes + C::kKeysBytes); };
  // Thread 0: take a ticket, locate its tile and start its bulk copy into
  // buffer b when the tile is full.
  const auto take = [&](int b) {
    const uint32_t t = atomicAdd(a.tile_counter, 1u);
    ticket_sh = t;
    if (t >= n_tiles) return;
    uint64_t tb, end;
    uint32_t seg = 0, first;
    if (a.n_seg) {
      int lo = 0, hi = a.n_seg - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.seg_tile_begin[mid] <= t) lo = mid; else hi = mid - 1;
      }
      seg = static_cast<uint32_t>(lo);
      first = a.seg_tile_begin[seg];
      tb = a.seg_begin[seg] + static_cast<uint64_t>(t - first) * TILE;
      end = a.seg_end[seg];
      first = t == first;
    } else {
      tb = static_cast<uint64_t>(t) * TILE;
      end = a.n;
      first = t == 0;
    }
    const uint32_t valid = end - tb < static_cast<uint64_t>(TILE) ? static_cast<uint32_t>(end - tb) : TILE;
    tile_base_sh = tb;
    tile_valid_sh = valid;
    tile_seg_sh = seg;
    tile_first_sh = first;
    if (valid == TILE) {
      fence_proxy_async_smem();  // earlier generic accesses to the buffer come first
      mbar_arrive_expect_tx(bars + b, static_cast<uint32_t>(C::kKeysBytes + C::kValsBytes));
      bulk_load(buf_keys(b), a.keys_in + tb, static_cast<uint32_t>(C::kKeysBytes), bars + b);
      bulk_load(buf_vals(b), a.vals_in + tb, static_cast<uint32_t>(C::kValsBytes), bars + b);
    }
  };

  if (tid == 0) {
    mbar_init(bars, 1);
    fence_mbarrier_init();
    take(0);
  }
  __syncthreads();
  uint32_t cur = ticket_sh;
  uint32_t parity = 0;
  K* skeys = buf_keys(0);
  V* vin = buf_vals(0);  // input values, then the staged values

  for (;;) {
    if (cur >= n_tiles) break;
    for (int i = tid; i < NW * RADIX / 2; i += TPB) reinterpret_cast<uint32_t*>(wcnt)[i] = 0u;
    __syncthreads();
    const uint32_t unit = cur;
    const uint64_t tbase = tile_base_sh;
    const uint32_t valid = tile_valid_sh;
    const bool first_tile = tile_first_sh != 0;  // first tile of [0, n) or of its segment
    const uint64_t* digit_start = a.digit_start + static_cast<size_t>(tile_seg_sh) * a.seg_digit_stride;
    if (valid == TILE) {
      if (!tile_wait(bars, parity)) {
        // Give the copies in flight a second bounded chance to land, then leave.
        if (tid == 0) atomicOr(a.err, kErrLookbackTimeout);
        uint32_t spins = 0;
        while (!mbar_try_wait(bars, parity) && ++spins < kSpinLimit) {
        }
        break;
      }
      parity ^= 1u;
    } else {
      for (uint32_t i = tid; i < valid; i += TPB) {
        skeys[i] = a.keys_in[tbase + i];
        vin[i] = a.vals_in[tbase + i];
      }
      __syncthreads();
    }

    // Rank within the warp.  An item's rank is its digit's count so far in
    // the warp plus the lanes of its slot that hold the same digit and come
    // before it (its peers).  The match instruction finds peers at a cost
    // that grows with the number of distinct digits in the warp (about two
    // SM cycles each, 60+ for random digits, and it saturates the SM's
    // divergence unit); when the warp's part of the key buffer can hold one
    // 32-bit lane mask per digit, the keys go to registers and the peers are
    // collected there instead: each lane ORs its bit into its digit's mask,
    // reads the mask back, and the lowest peer clears it.  A slot whose lanes
    // all hold one digit (structured networks) skips the masks.
    const uint32_t wbase = warp * 32u * IPT;
    K key[IPT];
    uint32_t rank[IPT];
    uint16_t* my = wcnt + static_cast<size_t>(warp) * RADIX;
    if constexpr (C::kMaskRank) {
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t li = wbase + static_cast<uint32_t>(j) * 32u + lane;
        key[j] = li < valid ? skeys[li] : K(0);
      }
      uint32_t* pmask = reinterpret_cast<uint32_t*>(skeys + wbase);  // this warp's keys are in registers now
      __syncwarp();
#pragma unroll
      for (int i = static_cast<int>(lane); i < RADIX; i += 32) pmask[i] = 0u;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t li = wbase + static_cast<uint32_t>(j) * 32u + lane;
        const bool ok = li < valid;
        const uint32_t d = ok ? (static_cast<uint32_t>(key[j] >> shift) & mask) : static_cast<uint32_t>(RADIX);
        uint32_t peers = 0xffffffffu;
        if (__reduce_min_sync(0xffffffffu, d) != __reduce_max_sync(0xffffffffu, d)) {
          if (ok) atomicOr(pmask + d, 1u << lane);
          __syncwarp();
          peers = ok ? pmask[d] : 0u;
        }
        const uint32_t old = ok ? my[d] : 0u;
        __syncwarp();
        if (ok && static_cast<int>(lane) == __ffs(peers) - 1) {
          my[d] = static_cast<uint16_t>(old + __popc(peers));
          pmask[d] = 0u;
        }
        rank[j] = old + __popc(peers & lt);
        __syncwarp();
      }
    } else {
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t li = wbase + static_cast<uint32_t>(j) * 32u + lane;
        const bool ok = li < valid;
        key[j] = ok ? skeys[li] : K(0);
        const uint32_t d = ok ? (static_cast<uint32_t>(key[j] >> shift) & mask) : static_cast<uint32_t>(RADIX);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        // Every lane reads its digit's counter (peers read the same word),
        // then the lowest peer advances it past the whole peer set.
        const uint32_t old = ok ? my[d] : 0u;
        __syncwarp();
        if (ok && static_cast<int>(lane) == __ffs(peers) - 1) my[d] = static_cast<uint16_t>(old + __popc(peers));
        rank[j] = old + __popc(peers & lt);
        __syncwarp();
      }
    }
    __syncthreads();
    // Per digit (this thread's DPT digits): the tile's count, then, after the
    // block scan, each warp's first staging position (digit start plus the
    // counts of the warps before it) in place of its count, so that staging
    // reads one offset per key.
    uint32_t tot[DPT];
    uint32_t tsum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      uint32_t r = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) r += wcnt[w * RADIX + d];
      tot[q] = r;
      tsum += r;
    }
    uint32_t* st_row = a.status32 + static_cast<size_t>(unit) * RADIX + static_cast<size_t>(tid) * DPT;
#pragma unroll
    for (int q = 0; q < DPT; ++q)
      if (unit != a.withhold_unit) st_status32(st_row + q, (first_tile ? kInc32 : kAgg32) | tot[q]);
    uint32_t excl = block_excl_scan<TPB>(tsum, warp_tmp, &scan_total);
    uint32_t my_start[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      my_start[q] = excl;
      uint32_t run = excl;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = wcnt[w * RADIX + d];
        wcnt[w * RADIX + d] = static_cast<uint16_t>(run);
        run += c;
      }
      excl += tot[q];
    }
    __syncthreads();
    // Stage the tile in digit order while the predecessors publish.  The
    // keys are in registers, so the key buffer takes the staged keys; the
    // values are then read in input order into registers and, after a
    // barrier, scattered into their own buffer in digit order, so that the
    // output loop reads both buffers sequentially.
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t li = wbase + static_cast<uint32_t>(j) * 32u + lane;
      if (li < valid) {
        const uint32_t d = static_cast<uint32_t>(key[j] >> shift) & mask;
        const uint32_t lp = wcnt[warp * RADIX + d] + rank[j];
        rank[j] = lp;
        if (SNC_IN_BOUNDS(a.err, 10u, lp, TILE)) skeys[lp] = key[j];
      }
    }
    V val[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t li = wbase + static_cast<uint32_t>(j) * 32u + lane;
      val[j] = li < valid ? vin[li] : V(0);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t li = wbase + static_cast<uint32_t>(j) * 32u + lane;
      if (li < valid && SNC_IN_BOUNDS(a.err, 10u, rank[j], TILE)) vin[rank[j]] = val[j];
    }
    uint64_t prefix[DPT];
    look_back32<RADIX, DPT, W>(a, unit, first_tile, prefix);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      if (!first_tile && unit != a.withhold_unit)
        st_status32(st_row + q, kInc32 | static_cast<uint32_t>((prefix[q] + tot[q]) & kCount32));
      globm[d] = digit_start[d] + prefix[q] - my_start[q];
    }
    __syncthreads();
    if (valid == TILE) {
      // Full tile: all shared-memory reads first, then the stores, so that
      // the stores of one thread are in flight together.
      K kk[IPT];
      V vv[IPT];
      uint64_t pp[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        kk[j] = skeys[tid + j * TPB];
        vv[j] = vin[tid + j * TPB];
      }
#pragma unroll
      for (int j = 0; j < IPT; ++j)
        pp[j] = globm[static_cast<uint32_t>(kk[j] >> shift) & mask] + tid + static_cast<uint32_t>(j * TPB);
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (SNC_IN_BOUNDS(a.err, 11u, pp[j], a.n)) emit_pair<UNPACK>(a, pp[j], kk[j], vv[j]);
      }
    } else {
      for (uint32_t i = tid; i < valid; i += TPB) {
        const K k = skeys[i];
        const uint32_t d = static_cast<uint32_t>(k >> shift) & mask;
        const uint64_t pos = globm[d] + i;
        if (!SNC_IN_BOUNDS(a.err, 11u + 0x100u * d, pos, a.n)) continue;
        emit_pair<UNPACK>(a, pos, k, vin[i]);
      }
    }
    __syncthreads();  // the tile's buffers and counters are free again
    if (tid == 0) take(0);
    __syncthreads();
    cur = ticket_sh;
  }
}

template <int BITS, int ITEMS, bool UNPACK, typename K, typename V>
cudaError_t launch_onesweep_tma_u(const OnesweepArgs<K, V>& a, int sms, cudaStream_t st) {
  using C = OnesweepTma<BITS, ITEMS, K, V>;
  // Set on every launch: the attribute is per function and device, and
  // builds may run on several threads and devices.
  cudaError_t e = cudaFuncSetAttribute(onesweep_tma_kernel<BITS, ITEMS, UNPACK, K, V>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(C::kSmem));
  if (e != cudaSuccess) return e;
  const uint64_t tiles = (a.n + C::TILE - 1) / C::TILE;
  const uint64_t resident = static_cast<uint64_t>(C::MINB) * sms;
  const uint64_t grid = tiles < resident ? tiles : resident;
  onesweep_tma_kernel<BITS, ITEMS, UNPACK, K, V><<<static_cast<unsigned>(grid), C::TPB, C::kSmem, st>>>(a);
  return cudaGetLastError();
}

// The unpacking variant exists for 64-bit values only (the build's sort).
template <int BITS, int ITEMS, typename K, typename V>
cudaError_t launch_onesweep_tma(const OnesweepArgs<K, V>& a, int sms, cudaStream_t st) {
  if constexpr (sizeof(V) == 8) {
    if (a.unpack_target) return launch_onesweep_tma_u<BITS, ITEMS, true, K, V>(a, sms, st);
  }
  return launch_onesweep_tma_u<BITS, ITEMS, false, K, V>(a, sms, st);
}

template <int BITS, typename K, typename V>
cudaError_t launch_onesweep_tma_sel(const SortPasses& sp, const OnesweepArgs<K, V>& a, int sms, cudaStream_t st) {
  if (sp.items == 8) return launch_onesweep_tma<BITS, 8, K, V>(a, sms, st);
  if (sp.items == 12) return launch_onesweep_tma<BITS, 12, K, V>(a, sms, st);
  if (sp.items == 24) return launch_onesweep_tma<BITS, 24, K, V>(a, sms, st);
  if (sp.items == 32) return launch_onesweep_tma<BITS, 32, K, V>(a, sms, st);
  return launch_onesweep_tma<BITS, 16, K, V>(a, sms, st);
}

template <int BITS, int G, bool UNPACK, typename K, typename V>
cudaError_t launch_onesweep_u(const OnesweepArgs<K, V>& a, int sms, cudaStream_t st) {
  using C = Onesweep<BITS, G, K, V>;
  // Set on every launch: the attribute is per function and device, and
  // builds may run on several threads and devices.
  cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<BITS, G, UNPACK, K, V>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(C::kSmem));
  if (e != cudaSuccess) return e;
  const uint64_t units = (a.n + C::GROUP - 1) / C::GROUP;
  const uint64_t resident = static_cast<uint64_t>(C::MINB) * sms;
  const uint64_t grid = units < resident ? units : resident;
  onesweep_kernel<BITS, G, UNPACK, K, V><<<static_cast<unsigned>(grid), C::TPB, C::kSmem, st>>>(a);
  return cudaGetLastError();
}

template <int BITS, int G, typename K, typename V>
cudaError_t launch_onesweep(const OnesweepArgs<K, V>& a, int sms, cudaStream_t st) {
  if constexpr (sizeof(V) == 8) {
    if (a.unpack_target) return launch_onesweep_u<BITS, G, true, K, V>(a, sms, st);
  }
  return launch_onesweep_u<BITS, G, false, K, V>(a, sms, st);
}

// Keys per look-back unit: one tile of the bulk-copy kernel, or a group of
// 4096-key tiles.
int onesweep_group(const SortPasses& sp) {
  if (sp.group_tiles == 0 && sp.kernel_bits <= 9) return kSortThreads * (sp.items > 0 ? sp.items : kSortItems);
  return kSortTile * (sp.group_tiles > 0 ? sp.group_tiles : 1);
}

template <int BITS, typename K, typename V>
cudaError_t launch_onesweep_g(const SortPasses& sp, int group_tiles, const OnesweepArgs<K, V>& a, int sms,
                              cudaStream_t st) {
  switch (group_tiles) {
    case 0:
      if (BITS <= 9) return launch_onesweep_tma_sel<(BITS <= 9 ? BITS : 9), K, V>(sp, a, sms, st);
      return launch_onesweep<BITS, 1, K, V>(a, sms, st);
    case 1: return launch_onesweep<BITS, 1, K, V>(a, sms, st);
    case 4: return launch_onesweep<BITS, 4, K, V>(a, sms, st);
    case 8: return launch_onesweep<BITS, 8, K, V>(a, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename K, typename V>
cudaError_t launch_onesweep_bits(const SortPasses& sp, int group_tiles, const OnesweepArgs<K, V>& a, int sms,
                                 cudaStream_t st) {
  switch (sp.kernel_bits) {
    case 8: return launch_onesweep_g<8, K, V>(sp, group_tiles, a, sms, st);
    case 9: return launch_onesweep_g<9, K, V>(sp, group_tiles, a, sms, st);
    case 10: return launch_onesweep_g<10, K, V>(sp, group_tiles, a, sms, st);
    case 11: return launch_onesweep_g<11, K, V>(sp, group_tiles, a, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

// Process-wide sort tuning (set by snc_set_tuning / the autotuner).  Digits
// of up to 9 bits: plan_passes takes the fewest passes and the narrowest
// even widths, so 9-bit digits are used only where they save a pass (e.g. 3
// passes instead of 4 for a 25-bit key; a 24-bit key keeps three 8-bit
// passes).  32 keys per thread: 8,192-key tiles, two blocks per SM, about
// half the look-backs per key of 16.
SortTuning g_sort_tuning{9, 0, 32};
WaitTest g_wait_test{kDefaultSpinLimit, 0xFFFFFFFFu};

// Digit plan: the fewest passes of at most max_bits bits, widths as even as
// possible, the kernel's digit width the widest of them (at least 8).
SortPasses plan_passes(int key_bits) { return plan_passes(key_bits, g_sort_tuning); }

SortPasses plan_passes(int key_bits, const SortTuning& tune) {
  SortPasses sp{};
  const int max_bits = tune.max_digit_bits < 8 ? 8 : (tune.max_digit_bits > 11 ? 11 : tune.max_digit_bits);
  sp.n_passes = (key_bits + max_bits - 1) / max_bits;
  if (sp.n_passes < 1) sp.n_passes = 1;
  int shift = 0;
  int widest = 0;
  for (int p = 0; p < sp.n_passes; ++p) {
    const int remaining = key_bits - shift;
    const int w = (remaining + (sp.n_passes - p) - 1) / (sp.n_passes - p);
    sp.shift[p] = shift;
    sp.mask[p] = (w >= 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);
    shift += w;
    if (w > widest) widest = w;
  }
  sp.kernel_bits = widest < 8 ? 8 : widest;
  sp.group_tiles = (tune.group_tiles == 0 || tune.group_tiles == 1 || tune.group_tiles == 4) ? tune.group_tiles : 8;
  sp.items = (tune.items == 8 || tune.items == 12 || tune.items == 24 || tune.items == 32) ? tune.items : 16;
  return sp;
}

namespace {
// Digit counters / offsets: [pass][kMaxRadix] for one range, or
// [segment][pass][radix] for a segmented sort.
size_t digit_entries(const SortPasses& sp, int n_seg) {
  const size_t one = static_cast<size_t>(kMaxPasses) * kMaxRadix;
  const size_t seg = static_cast<size_t>(n_seg) * sp.n_passes * (1u << sp.kernel_bits);
  return seg > one ? seg : one;
}
}  // namespace

size_t sort_scratch_bytes(uint64_t n, const SortPasses& sp, uint64_t n_tiles, int n_seg) {
  uint64_t groups = (n + onesweep_group(sp) - 1) / onesweep_group(sp);
  if (n_tiles > groups) groups = n_tiles;
  const size_t status = static_cast<size_t>(groups ? groups : 1) * (1u << sp.kernel_bits) * sizeof(uint64_t);
  const size_t digits = digit_entries(sp, n_seg) * sizeof(uint64_t);
  const size_t counters = 64 * sizeof(uint32_t);
  return status + 2 * digits + counters + 4 * 256;
}

namespace {
size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
}

// Sorts n (key, value) pairs stably on the planned digits.  Pass 0 reads
// (keys_in, vals_in); the passes alternate between (keys_tmp, vals_tmp) and
// (keys_out, vals_out) so that the last one writes (keys_out, vals_out):
// with an even number of passes pass 0 writes keys_tmp.  keys_tmp may
// therefore alias keys_in (and vals_tmp vals_in) only for an odd number of
// passes (pass 0 has read the input completely before pass 1 writes it);
// an aliased even-pass plan is rejected.  keys_tmp is unused for one pass.
// scratch: sort_scratch_bytes(n, sp) bytes of device memory.
// pass_events (optional, n_passes + 1 events): recorded after the histogram
// and after each pass.
SortScratch sort_scratch_layout(void* scratch, uint64_t n, const SortPasses& sp, uint64_t n_tiles, int n_seg) {
  SortScratch l{};
  const int group = onesweep_group(sp);
  uint64_t groups = (n + group - 1) / group;
  if (n_tiles > groups) groups = n_tiles;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  l.status_bytes = static_cast<size_t>(groups ? groups : 1) * (1u << sp.kernel_bits) * sizeof(uint64_t);
  l.status = reinterpret_cast<uint64_t*>(p);
  p += align256(l.status_bytes);
  l.hist_bytes = digit_entries(sp, n_seg) * sizeof(unsigned long long);
  l.hist = reinterpret_cast<unsigned long long*>(p);
  p += align256(l.hist_bytes);
  l.start = reinterpret_cast<uint64_t*>(p);
  p += align256(digit_entries(sp, n_seg) * sizeof(uint64_t));
  l.counters = reinterpret_cast<uint32_t*>(p);
  return l;
}

// ---------------------------------------------------------------------------
// Segmented sorts: digit counts per segment (keys read once, shared-memory
// counters flushed whenever the block moves to another segment) and their
// exclusive scans, offset by each segment's first position.
// ---------------------------------------------------------------------------
struct SegHistArgs {
  int n_passes;
  int shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
  uint32_t radix;           // counters per (segment, pass)
  int n_seg;
  const uint64_t* begin;
  const uint64_t* end;
  const uint32_t* tile_begin;
  uint64_t n_tiles;
  uint32_t tile;            // keys per tile
  uint32_t tiles_per_block;
  unsigned long long* hist; // [segment][pass][radix]
};

template <typename K>
__global__ void __launch_bounds__(256) seg_hist_kernel(const K* __restrict__ keys, SegHistArgs h) {
  extern __shared__ uint32_t sh[];
  const uint32_t nc = static_cast<uint32_t>(h.n_passes) * h.radix;
  const auto flush = [&](int seg) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
      const uint32_t v = sh[i];
      if (v) atomicAdd(&h.hist[static_cast<size_t>(seg) * nc + i], static_cast<unsigned long long>(v));
      sh[i] = 0u;
    }
    __syncthreads();
  };
  for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) sh[i] = 0u;
  for (uint64_t t0 = static_cast<uint64_t>(blockIdx.x) * h.tiles_per_block; t0 < h.n_tiles;
       t0 += static_cast<uint64_t>(gridDim.x) * h.tiles_per_block) {
    const uint64_t t1 = t0 + h.tiles_per_block < h.n_tiles ? t0 + h.tiles_per_block : h.n_tiles;
    int lo = 0, hi = h.n_seg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (h.tile_begin[mid] <= t0) lo = mid; else hi = mid - 1;
    }
    int seg = lo;
    __syncthreads();
    for (uint64_t t = t0; t < t1; ++t) {
      if (t >= h.tile_begin[seg + 1]) {
        flush(seg);
        while (t >= h.tile_begin[seg + 1]) ++seg;
      }
      const uint64_t tb = h.begin[seg] + (t - h.tile_begin[seg]) * h.tile;
      const uint64_t te = tb + h.tile < h.end[seg] ? tb + h.tile : h.end[seg];
      for (uint64_t i = tb + threadIdx.x; i < te; i += blockDim.x) {
        const uint64_t k = static_cast<uint64_t>(keys[i]);
#pragma unroll
        for (int p = 0; p < kMaxPasses; ++p)
          if (p < h.n_passes) atomicAdd(&sh[p * h.radix + (static_cast<uint32_t>(k >> h.shift[p]) & h.mask[p])], 1u);
      }
    }
    flush(seg);
  }
}

// start[s][p][d] = begin[s] + sum of the counts of digits below d.  One
// block of 256 threads per (segment, pass).
__global__ void __launch_bounds__(256) seg_digit_scan_kernel(const unsigned long long* __restrict__ hist,
                                                             uint64_t* __restrict__ start, uint32_t radix,
                                                             int n_passes, const uint64_t* __restrict__ begin) {
  __shared__ uint64_t wsum[8];
  const int seg = blockIdx.x / n_passes;
  const size_t row = static_cast<size_t>(blockIdx.x) * radix;
  const uint32_t per = radix / 256u;  // 1 or 2 digits per thread
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t v0 = hist[row + threadIdx.x * per];
  uint64_t v1 = per > 1 ? hist[row + threadIdx.x * per + 1] : 0ull;
  const uint64_t sum = v0 + v1;
  uint64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane) >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint64_t before = begin[seg];
  for (uint32_t w = 0; w < warp; ++w) before += wsum[w];
  const uint64_t run = before + incl - sum;
  start[row + threadIdx.x * per] = run;
  if (per > 1) start[row + threadIdx.x * per + 1] = run + v0;
}

template <typename K, typename V>
cudaError_t radix_sort_run(const K* keys_in, const V* vals_in, K* keys_out, V* vals_out, K* keys_tmp, V* vals_tmp,
                           uint64_t n, const SortPasses& sp, void* scratch, uint32_t* err, cudaStream_t st,
                           cudaEvent_t* pass_events, bool hist_ready, const SortUnpack* unpack, bool* fused,
                           const SortSegments* segs) {
  if (fused) *fused = false;
  const int n_seg = segs ? segs->n_seg : 0;
  // Segments are sorted by the bulk-copy kernel only (8-9 bit digits, 30-bit
  // look-back counts: every segment below 2^30 keys, 16-byte aligned arrays).
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (n_seg && (sp.group_tiles != 0 || sp.kernel_bits > 9 || segs->max_len >= (1ull << 30) || !al16(keys_in) ||
                !al16(vals_in) || !al16(keys_out) || !al16(vals_out) || !al16(keys_tmp) || !al16(vals_tmp)))
    return cudaErrorInvalidValue;
  // The pass kernels shift keys by up to the key width minus one.
  if (static_cast<size_t>(sp.shift[sp.n_passes - 1]) >= 8 * sizeof(K)) return cudaErrorInvalidValue;
  if (n == 0) {
    if (pass_events)
      for (int i = 0; i <= sp.n_passes; ++i) cudaEventRecord(pass_events[i], st);
    return cudaSuccess;
  }
  const int group = onesweep_group(sp);
  const uint64_t groups = (n + group - 1) / group;
  if (groups > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  if ((sp.n_passes % 2 == 0) && (static_cast<const void*>(keys_tmp) == static_cast<const void*>(keys_in) ||
                                 static_cast<const void*>(vals_tmp) == static_cast<const void*>(vals_in)))
    return cudaErrorInvalidValue;
  const uint64_t n_tiles_seg = n_seg ? segs->n_tiles : 0;
  const SortScratch lay = sort_scratch_layout(scratch, n, sp, n_tiles_seg, n_seg);
  uint64_t* status = lay.status;
  const size_t status_bytes = lay.status_bytes;
  unsigned long long* hist = lay.hist;
  uint64_t* start = lay.start;
  uint32_t* counters = lay.counters;

  cudaError_t e;
  if ((e = cudaMemsetAsync(status, 0, status_bytes, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counters, 0, 64 * sizeof(uint32_t), st)) != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t radix = 1u << sp.kernel_bits;
  if (n_seg) {
    if ((e = cudaMemsetAsync(hist, 0, lay.hist_bytes, st)) != cudaSuccess) return e;
    SegHistArgs h{};
    h.n_passes = sp.n_passes;
    for (int p = 0; p < kMaxPasses; ++p) {
      h.shift[p] = p < sp.n_passes ? sp.shift[p] : 0;
      h.mask[p] = p < sp.n_passes ? sp.mask[p] : 0u;
    }
    h.radix = radix;
    h.n_seg = n_seg;
    h.begin = segs->begin;
    h.end = segs->end;
    h.tile_begin = segs->tile_begin;
    h.n_tiles = segs->n_tiles;
    h.tile = static_cast<uint32_t>(onesweep_group(sp));
    h.tiles_per_block = 16;
    h.hist = hist;
    const size_t hsm = static_cast<size_t>(sp.n_passes) * radix * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(seg_hist_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(hsm))) != cudaSuccess)
      return e;
    const uint64_t blocks = (segs->n_tiles + h.tiles_per_block - 1) / h.tiles_per_block;
    seg_hist_kernel<K><<<static_cast<unsigned>(blocks ? blocks : 1), 256, hsm, st>>>(keys_in, h);
    seg_digit_scan_kernel<<<static_cast<unsigned>(n_seg * sp.n_passes), 256, 0, st>>>(hist, start, radix, sp.n_passes,
                                                                                     segs->begin);
  } else if (!hist_ready) {
    if ((e = cudaMemsetAsync(hist, 0, static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(unsigned long long),
                             st)) != cudaSuccess)
      return e;
    const HistPlan plan = hist_plan(sp, hist);
    const size_t hist_smem = hist_smem_bytes(plan);
    // Set on every launch: the attribute is per function and device, and
    // builds may run on several threads and devices.
    e = cudaFuncSetAttribute(radix_hist_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kMaxPasses * kMaxRadix * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    radix_hist_kernel<K><<<sms * 2, 512, hist_smem, st>>>(keys_in, n, plan);
  }
  if (!n_seg) radix_digit_scan_kernel<<<sp.n_passes, kDigitScanThreads, 0, st>>>(hist, start);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (pass_events) cudaEventRecord(pass_events[0], st);

  // The bulk-copy kernel needs 16-byte aligned arrays and counts below 2^30
  // (30-bit look-back words); fall back otherwise.
  const auto aligned16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  int group_tiles = sp.group_tiles;
  if (group_tiles == 0 && !n_seg &&
      (n >= (1ull << 30) || !(aligned16(keys_in) && aligned16(vals_in) && aligned16(keys_out) &&
                              aligned16(vals_out) && (sp.n_passes < 2 || (aligned16(keys_tmp) && aligned16(vals_tmp))))))
    group_tiles = 1;
  const uint64_t tile32 = onesweep_group(sp);  // the bulk-copy kernel's tile
  const uint64_t tiles32 = n_seg ? n_tiles_seg : (n + tile32 - 1) / tile32;
  const size_t status32_bytes = static_cast<size_t>(tiles32) * (1u << sp.kernel_bits) * 4u;
  const K* kin = keys_in;
  const V* vin = vals_in;
  for (int pass = 0; pass < sp.n_passes; ++pass) {
    const bool to_out = ((sp.n_passes - 1 - pass) & 1) == 0;
    K* kout = to_out ? keys_out : keys_tmp;
    V* vout = to_out ? vals_out : vals_tmp;
    OnesweepArgs<K, V> a{};
    a.keys_in = kin;
    a.vals_in = vin;
    a.keys_out = kout;
    a.vals_out = vout;
    a.n = n;
    a.shift = sp.shift[pass];
    a.mask = sp.mask[pass];
    a.digit_start = start + static_cast<size_t>(pass) * (n_seg ? radix : kMaxRadix);
    a.n_seg = n_seg;
    if (n_seg) {
      a.seg_begin = segs->begin;
      a.seg_end = segs->end;
      a.seg_tile_begin = segs->tile_begin;
      a.seg_digit_stride = static_cast<uint64_t>(sp.n_passes) * radix;
    }
    a.status = status;
    a.tile_counter = counters + pass;
    a.epoch = static_cast<uint32_t>(pass + 1);
    a.err = err;
    a.lookback_spin_limit = g_wait_test.lookback_spin_limit;
    a.withhold_unit = g_wait_test.withhold_unit;
    a.status32 = reinterpret_cast<uint32_t*>(status);
    if (sizeof(V) == 8 && unpack && pass == sp.n_passes - 1) {
      a.unpack_target = unpack->target;
      a.unpack_weight = unpack->weight;
      a.unpack_delay = unpack->delay;
      a.unpack_delay_mask = unpack->delay_mask;
      if (fused) *fused = true;
    }
    if (group_tiles == 0 && (e = cudaMemsetAsync(status, 0, status32_bytes, st)) != cudaSuccess) return e;
    // The bulk-copy kernel runs each pass at that pass's own digit width
    // (at least 8 bits): a narrower radix ranks faster.  Digit starts and
    // status words keep the plan's widest stride.
    SortPasses sp_pass = sp;
    if (group_tiles == 0) {
      const int w = __builtin_popcount(sp.mask[pass]);
      sp_pass.kernel_bits = w < 8 ? 8 : w;
    }
    if ((e = launch_onesweep_bits<K, V>(sp_pass, group_tiles, a, sms, st)) != cudaSuccess) return e;
    if (pass_events) cudaEventRecord(pass_events[pass + 1], st);
    kin = kout;
    vin = vout;
  }
  return cudaSuccess;
}

template cudaError_t radix_sort_run<uint64_t, uint32_t>(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*,
                                                        uint64_t*, uint32_t*, uint64_t, const SortPasses&, void*,
                                                        uint32_t*, cudaStream_t, cudaEvent_t*, bool,
                                                        const SortUnpack*, bool*, const SortSegments*);
template cudaError_t radix_sort_run<uint32_t, uint64_t>(const uint32_t*, const uint64_t*, uint32_t*, uint64_t*,
                                                        uint32_t*, uint64_t*, uint64_t, const SortPasses&, void*,
                                                        uint32_t*, cudaStream_t, cudaEvent_t*, bool,
                                                        const SortUnpack*, bool*, const SortSegments*);
template cudaError_t radix_sort_run<uint64_t, uint64_t>(const uint64_t*, const uint64_t*, uint64_t*, uint64_t*,
                                                        uint64_t*, uint64_t*, uint64_t, const SortPasses&, void*,
                                                        uint32_t*, cudaStream_t, cudaEvent_t*, bool,
                                                        const SortUnpack*, bool*, const SortSegments*);

}  // namespace snc
