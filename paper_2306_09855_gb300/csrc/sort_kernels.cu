// sort_kernels.cu -- stable LSD radix sort of (64-bit key, 32-bit value)
// pairs: one upfront histogram of every digit, then one "onesweep" pass per
// digit (Adinets & Merrill 2022) whose tiles find their global offsets by
// decoupled look-back (Merrill & Garland 2016).
//
// The paper sorts connections by source and delay with an extension of radix
// sort (Sec. 2.2); here the key also carries the target, and the sort is a
// plain stable LSD sort over the packed key's bits.
//
// Look-back status words are 64-bit: [flag:2][epoch:14][count:48].  The epoch
// changes every pass, so a stale word from an earlier pass reads as "not yet
// published" and the array never needs clearing between passes.  Every wait
// on a predecessor is bounded; on expiry the kernel sets an error bit and
// finishes its tile without waiting (the result is then wrong, the error is
// reported by snc_synchronize, and the GPU is never held).
#include <cuda_runtime.h>

#include <cstdint>

#include "snc_check.cuh"
#include "snc_internal.h"
#include "sort_kernels.h"

namespace snc {

namespace {

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kCountMask = (1ull << 48) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

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
// block, merged into global 64-bit counters).  A warp whose 32 keys share a
// digit adds 32 once instead of 32 conflicting atomics.
// ---------------------------------------------------------------------------
__global__ void radix_hist_kernel(const uint64_t* __restrict__ keys, uint64_t n, SortPasses sp,
                                  unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t sh[];
  const int bins = sp.n_passes * kMaxRadix;
  for (int i = threadIdx.x; i < bins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps_total = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (uint64_t base = gw * 32; base < n; base += warps_total * 32) {
    const uint64_t i = base + lane;
    const bool valid = i < n;
    const uint64_t key = valid ? keys[i] : 0ull;
    for (int p = 0; p < sp.n_passes; ++p) {
      const uint32_t d = static_cast<uint32_t>(key >> sp.shift[p]) & sp.mask[p];
      const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
      const bool all_valid = base + 32 <= n;
      if (__all_sync(0xffffffffu, d == d0) && all_valid) {
        if (lane == 0) atomicAdd(&sh[p * kMaxRadix + d], 32u);
      } else if (valid) {
        atomicAdd(&sh[p * kMaxRadix + d], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < bins; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], static_cast<unsigned long long>(sh[i]));
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

// ---------------------------------------------------------------------------
// One onesweep pass.  Tile = TPB threads x IPT keys; warp w owns keys
// [w*32*IPT, (w+1)*32*IPT) of the tile, lane-interleaved, so that ranking
// warp by warp and item by item preserves input order (stability).
// ---------------------------------------------------------------------------
template <int BITS, int TPB, int IPT>
__global__ void __launch_bounds__(TPB) onesweep_kernel(OnesweepArgs a) {
  constexpr int RADIX = 1 << BITS;
  constexpr int NW = TPB / 32;
  constexpr int TILE = TPB * IPT;
  constexpr int DPT = RADIX / TPB;  // digits per thread
  static_assert(RADIX % TPB == 0, "radix must be a multiple of the block size");
  constexpr size_t kCntBytes = static_cast<size_t>(NW) * RADIX * sizeof(uint16_t);
  constexpr size_t kTileBytes = static_cast<size_t>(TILE) * (sizeof(uint64_t) + sizeof(uint32_t));
  constexpr size_t kUnion = kCntBytes > kTileBytes ? kCntBytes : kTileBytes;

  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(smem);
  uint64_t* skeys = reinterpret_cast<uint64_t*>(smem);
  uint32_t* svals = reinterpret_cast<uint32_t*>(smem + static_cast<size_t>(TILE) * sizeof(uint64_t));
  uint32_t* local_start = reinterpret_cast<uint32_t*>(smem + kUnion);
  uint64_t* glob = reinterpret_cast<uint64_t*>(smem + kUnion + RADIX * sizeof(uint32_t));
  __shared__ uint32_t tile_sh;
  __shared__ uint32_t warp_tmp[32];
  __shared__ uint32_t scan_total;

  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) tile_sh = atomicAdd(a.tile_counter, 1u);
  for (int i = tid; i < NW * RADIX / 2; i += TPB) reinterpret_cast<uint32_t*>(wcnt)[i] = 0u;
  __syncthreads();
  const uint32_t tile = tile_sh;
  const uint64_t tile_base = static_cast<uint64_t>(tile) * TILE;
  const uint64_t warp_base = tile_base + static_cast<uint64_t>(warp) * 32 * IPT;
  const uint32_t mask = a.mask;
  const int shift = a.shift;

  uint64_t key[IPT];
  uint32_t rank[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
    key[j] = idx < a.n ? a.keys_in[idx] : 0ull;
  }

  // Rank within the warp: peers with an equal digit share one counter update.
  uint16_t* my = wcnt + static_cast<size_t>(warp) * RADIX;
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
    const bool valid = idx < a.n;
    const uint32_t d = valid ? (static_cast<uint32_t>(key[j] >> shift) & mask) : static_cast<uint32_t>(RADIX);
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (static_cast<int>(lane) == leader && valid) {
      old = my[d];
      my[d] = static_cast<uint16_t>(old + __popc(peers));
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[j] = old + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();

  // Per digit: exclusive offsets across warps and the tile total.
  uint32_t tot[DPT];
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int d = tid * DPT + q;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = wcnt[w * RADIX + d];
      wcnt[w * RADIX + d] = static_cast<uint16_t>(run);
      run += c;
    }
    tot[q] = run;
  }
  // Publish this tile's counts before looking back.
  uint64_t* st_row = a.status + static_cast<size_t>(tile) * RADIX + static_cast<size_t>(tid) * DPT;
  const uint64_t ep = static_cast<uint64_t>(a.epoch) << 48;
#pragma unroll
  for (int q = 0; q < DPT; ++q) st_status(st_row + q, (tile == 0 ? kFlagInc : kFlagAgg) | ep | tot[q]);

  // Tile-local exclusive scan over digits.
  uint32_t tsum = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) tsum += tot[q];
  uint32_t run = block_excl_scan<TPB>(tsum, warp_tmp, &scan_total);
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    local_start[tid * DPT + q] = run;
    run += tot[q];
  }

  // Decoupled look-back, all of this thread's digits in flight together.
  uint64_t prefix[DPT];
  int64_t look[DPT];
  uint32_t pending = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    prefix[q] = 0;
    look[q] = static_cast<int64_t>(tile) - 1;
    if (tile > 0) pending |= 1u << q;
  }
  uint32_t spins = 0;
  while (pending) {
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      if (!(pending & (1u << q))) continue;
      if (!SNC_IN_BOUNDS(a.err, 12u, static_cast<uint64_t>(look[q]), static_cast<uint64_t>(tile))) {
        pending &= ~(1u << q);
        continue;
      }
      const uint64_t v = ld_status(a.status + static_cast<size_t>(look[q]) * RADIX + tid * DPT + q);
      const bool fresh = ((v >> 48) & 0x3FFFull) == a.epoch;
      const uint64_t flag = fresh ? (v & (3ull << 62)) : 0ull;
      if (flag == 0) continue;
      prefix[q] += v & kCountMask;
      if (flag == kFlagInc) pending &= ~(1u << q);
      else --look[q];
    }
    if (pending && ++spins > kSpinLimit) {
      atomicOr(a.err, kErrLookbackTimeout);
      break;
    }
  }
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int d = tid * DPT + q;
    if (tile > 0) st_status(st_row + q, kFlagInc | ep | ((prefix[q] + tot[q]) & kCountMask));
    glob[d] = a.digit_start[d] + prefix[q] - local_start[d];
  }
  __syncthreads();

  // Local positions; then the tile is staged in digit order.
  uint32_t lpos[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
    const uint32_t d = static_cast<uint32_t>(key[j] >> shift) & mask;
    lpos[j] = idx < a.n ? local_start[d] + wcnt[warp * RADIX + d] + rank[j] : 0xFFFFFFFFu;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if (lpos[j] != 0xFFFFFFFFu && SNC_IN_BOUNDS(a.err, 10u, lpos[j], TILE)) {
      const uint64_t idx = warp_base + static_cast<uint64_t>(j) * 32 + lane;
      skeys[lpos[j]] = key[j];
      svals[lpos[j]] = a.vals_in[idx];
    }
  }
  __syncthreads();
  const uint64_t left = a.n - tile_base;
  const uint32_t valid = left < static_cast<uint64_t>(TILE) ? static_cast<uint32_t>(left) : static_cast<uint32_t>(TILE);
  for (uint32_t i = tid; i < valid; i += TPB) {
    const uint64_t k = skeys[i];
    const uint32_t d = static_cast<uint32_t>(k >> shift) & mask;
    const uint64_t pos = glob[d] + i;
    if (!SNC_IN_BOUNDS(a.err, 11u + 0x100u * d, pos, a.n)) continue;
    a.keys_out[pos] = k;
    a.vals_out[pos] = svals[i];
  }
}

template <int BITS, int TPB, int IPT>
size_t onesweep_smem() {
  constexpr int RADIX = 1 << BITS;
  constexpr int NW = TPB / 32;
  constexpr int TILE = TPB * IPT;
  constexpr size_t cnt = static_cast<size_t>(NW) * RADIX * sizeof(uint16_t);
  constexpr size_t tilebytes = static_cast<size_t>(TILE) * (sizeof(uint64_t) + sizeof(uint32_t));
  constexpr size_t u = cnt > tilebytes ? cnt : tilebytes;
  return u + RADIX * sizeof(uint32_t) + RADIX * sizeof(uint64_t);
}

template <int BITS, int TPB, int IPT>
cudaError_t launch_onesweep(const OnesweepArgs& a, uint32_t n_tiles, cudaStream_t st) {
  const size_t sm = onesweep_smem<BITS, TPB, IPT>();
  static bool configured = false;  // per process; attribute is per function
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<BITS, TPB, IPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  onesweep_kernel<BITS, TPB, IPT><<<n_tiles, TPB, sm, st>>>(a);
  return cudaGetLastError();
}

// Tile shape per digit width.
int onesweep_tile(int bits) {
  switch (bits) {
    case 8: return 256 * 16;
    case 9: return 256 * 16;
    case 10: return 256 * 16;
    default: return 512 * 12;
  }
}

cudaError_t launch_onesweep_bits(int bits, const OnesweepArgs& a, uint32_t n_tiles, cudaStream_t st) {
  switch (bits) {
    case 8: return launch_onesweep<8, 256, 16>(a, n_tiles, st);
    case 9: return launch_onesweep<9, 256, 16>(a, n_tiles, st);
    case 10: return launch_onesweep<10, 256, 16>(a, n_tiles, st);
    case 11: return launch_onesweep<11, 512, 12>(a, n_tiles, st);
    default: return cudaErrorInvalidValue;
  }
}

// Digit plan: the fewest passes of at most 11 bits, widths as even as
// possible, the kernel's digit width the widest of them (at least 8).
SortPasses plan_passes(int key_bits) {
  SortPasses sp{};
  sp.n_passes = (key_bits + 10) / 11;
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
  return sp;
}

size_t sort_scratch_bytes(uint64_t n, const SortPasses& sp) {
  const uint64_t tiles = (n + onesweep_tile(sp.kernel_bits) - 1) / onesweep_tile(sp.kernel_bits);
  const size_t status = static_cast<size_t>(tiles ? tiles : 1) * (1u << sp.kernel_bits) * sizeof(uint64_t);
  const size_t hist = static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(unsigned long long);
  const size_t start = static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(uint64_t);
  const size_t counters = 64 * sizeof(uint32_t);
  return status + hist + start + counters + 4 * 256;
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
cudaError_t radix_sort_run(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                           uint64_t* keys_tmp, uint32_t* vals_tmp, uint64_t n, const SortPasses& sp, void* scratch,
                           uint32_t* err, cudaStream_t st, cudaEvent_t* pass_events) {
  if (n == 0) {
    if (pass_events)
      for (int i = 0; i <= sp.n_passes; ++i) cudaEventRecord(pass_events[i], st);
    return cudaSuccess;
  }
  const int tile = onesweep_tile(sp.kernel_bits);
  const uint64_t tiles = (n + tile - 1) / tile;
  if (tiles > 0xFFFFFFFFull) return cudaErrorInvalidValue;
  if ((sp.n_passes % 2 == 0) && (static_cast<const void*>(keys_tmp) == static_cast<const void*>(keys_in) ||
                                 static_cast<const void*>(vals_tmp) == static_cast<const void*>(vals_in)))
    return cudaErrorInvalidValue;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  const size_t status_bytes = static_cast<size_t>(tiles) * (1u << sp.kernel_bits) * sizeof(uint64_t);
  uint64_t* status = reinterpret_cast<uint64_t*>(p);
  p += align256(status_bytes);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(p);
  p += align256(static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(unsigned long long));
  uint64_t* start = reinterpret_cast<uint64_t*>(p);
  p += align256(static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(uint64_t));
  uint32_t* counters = reinterpret_cast<uint32_t*>(p);

  cudaError_t e;
  if ((e = cudaMemsetAsync(status, 0, status_bytes, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(hist, 0, static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(unsigned long long), st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(counters, 0, 64 * sizeof(uint32_t), st)) != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t hist_smem = static_cast<size_t>(sp.n_passes) * kMaxRadix * sizeof(uint32_t);
  static bool hist_configured = false;
  if (!hist_configured) {
    e = cudaFuncSetAttribute(radix_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kMaxPasses * kMaxRadix * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    hist_configured = true;
  }
  radix_hist_kernel<<<sms * 2, 512, hist_smem, st>>>(keys_in, n, sp, hist);
  radix_digit_scan_kernel<<<sp.n_passes, kDigitScanThreads, 0, st>>>(hist, start);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (pass_events) cudaEventRecord(pass_events[0], st);

  const uint64_t* kin = keys_in;
  const uint32_t* vin = vals_in;
  for (int pass = 0; pass < sp.n_passes; ++pass) {
    const bool to_out = ((sp.n_passes - 1 - pass) & 1) == 0;
    uint64_t* kout = to_out ? keys_out : keys_tmp;
    uint32_t* vout = to_out ? vals_out : vals_tmp;
    OnesweepArgs a{};
    a.keys_in = kin;
    a.vals_in = vin;
    a.keys_out = kout;
    a.vals_out = vout;
    a.n = n;
    a.shift = sp.shift[pass];
    a.mask = sp.mask[pass];
    a.digit_start = start + static_cast<size_t>(pass) * kMaxRadix;
    a.status = status;
    a.tile_counter = counters + pass;
    a.epoch = static_cast<uint32_t>(pass + 1);
    a.err = err;
    if ((e = launch_onesweep_bits(sp.kernel_bits, a, static_cast<uint32_t>(tiles), st)) != cudaSuccess) return e;
    if (pass_events) cudaEventRecord(pass_events[pass + 1], st);
    kin = kout;
    vin = vout;
  }
  return cudaSuccess;
}

}  // namespace snc
