// index_kernels.cu -- unpacking of the sorted (key, value) pairs into
// target / delay / weight arrays, and the group index of Sec. 2.2.
//
// A connection starts a group when its source or its delay differs from the
// previous connection's.  group_first[g] is the position of the g-th group
// start (a stream compaction over per-block counts), row_ptr[i] the first
// connection of source i and group_ptr[i] = p_i = sum_{j<i} G_j the first
// group of source i (both found by binary search, one thread per node).  A
// batch's networks are separate segments of the arrays, each with its own
// row_ptr and group_ptr.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>

#include "index_kernels.h"
#include "snc_check.cuh"
#include "snc_internal.h"

namespace snc {

// Unpack of the sorted pairs and group starts.  Block b covers positions
// [b * kIndexTile, (b + 1) * kIndexTile); thread t of a block owns the
// kIndexItems consecutive positions starting at t * kIndexItems.  Writes
// target, delay and weight (vector stores), one bit per position in
// `starts` (bit i of the bitmap <-> position i) and the number of group
// starts of the block.  A group starts where the (source, delay) key
// changes.
// KEYS_ONLY: the sort's last pass wrote target, delay and weight, so only the
// keys are read (at up to eight blocks per SM, for more loads in flight).
template <typename K, bool KEYS_ONLY>
__global__ void __launch_bounds__(kIndexThreads, KEYS_ONLY ? 8 : 1) index_unpack_kernel(IndexArgs a) {
  __shared__ uint32_t warp_cnt[kIndexThreads / 32];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const K* keys = static_cast<const K*>(a.keys);
  const uint32_t delay_mask = (1u << a.delay_bits) - 1u;
  const uint64_t n_blocks = (a.n + kIndexTile - 1) / kIndexTile;
  constexpr int KPV = 16 / sizeof(K);  // keys per 16-byte vector
  for (uint64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const uint64_t base = blk * kIndexTile + static_cast<uint64_t>(tid) * kIndexItems;
    K key[kIndexItems];
    uint64_t val[kIndexItems];
    const bool full = base + kIndexItems <= a.n;
    if (full) {
      const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
      for (int k = 0; k < kIndexItems / KPV; ++k) {
        const uint4 v = __ldg(k4 + k);
        const K* kv = reinterpret_cast<const K*>(&v);
#pragma unroll
        for (int j = 0; j < KPV; ++j) key[k * KPV + j] = kv[j];
      }
      if (!KEYS_ONLY) {
        const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(a.vals + base);
#pragma unroll
        for (int k = 0; k < kIndexItems / 2; ++k) {
          const ulonglong2 v = __ldg(v2 + k);
          val[2 * k] = v.x;
          val[2 * k + 1] = v.y;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < kIndexItems; ++k) {
        key[k] = base + k < a.n ? __ldg(keys + base + k) : K(0);
        val[k] = base + k < a.n && !KEYS_ONLY ? __ldg(a.vals + base + k) : 0ull;
      }
    }
    // Predecessor of this thread's first key: the previous lane's last key,
    // or one extra load for lane 0.
    K prev = __shfl_up_sync(0xffffffffu, key[kIndexItems - 1], 1);
    if (lane == 0) prev = (base > 0 && base < a.n) ? __ldg(keys + base - 1) : K(0);
    uint32_t bits = 0;
    if (a.n_seg) {
      // The network of each position: positions outside every network
      // (alignment gaps) start nothing; a network's first position starts a
      // group.
      int lo = 0, hi = a.n_seg - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.seg_begin[mid] <= base) lo = mid; else hi = mid - 1;
      }
      int seg = lo;
#pragma unroll
      for (int k = 0; k < kIndexItems; ++k) {
        const uint64_t q = base + k;
        while (seg + 1 < a.n_seg && q >= a.seg_begin[seg + 1]) ++seg;
        const K before = k == 0 ? prev : key[k - 1];
        const bool real = q >= a.seg_begin[seg] && q < a.seg_end[seg];
        const bool start = real && (q == a.seg_begin[seg] || key[k] != before);
        bits |= (start ? 1u : 0u) << k;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kIndexItems; ++k) {
        const uint64_t q = base + k;
        const K before = k == 0 ? prev : key[k - 1];
        const bool start = q < a.n && (q == 0 || key[k] != before);
        bits |= (start ? 1u : 0u) << k;
      }
    }
    if (KEYS_ONLY) {
      // target, weight and delay were written by the sort's last pass
    } else if (full) {
      uint32_t tv[kIndexItems], wv[kIndexItems];
      uint16_t dv[kIndexItems];
#pragma unroll
      for (int k = 0; k < kIndexItems; ++k) {
        tv[k] = static_cast<uint32_t>(val[k] >> 32);
        wv[k] = static_cast<uint32_t>(val[k]);
        dv[k] = static_cast<uint16_t>(static_cast<uint32_t>(key[k]) & delay_mask);
      }
      uint4* t4 = reinterpret_cast<uint4*>(a.target + base);
      uint4* w4 = reinterpret_cast<uint4*>(a.weight + base);
#pragma unroll
      for (int k = 0; k < kIndexItems / 4; ++k) {
        t4[k] = make_uint4(tv[4 * k], tv[4 * k + 1], tv[4 * k + 2], tv[4 * k + 3]);
        w4[k] = make_uint4(wv[4 * k], wv[4 * k + 1], wv[4 * k + 2], wv[4 * k + 3]);
      }
      uint4* d4 = reinterpret_cast<uint4*>(a.delay + base);
#pragma unroll
      for (int k = 0; k < kIndexItems / 8; ++k)
        d4[k] = make_uint4(dv[8 * k] | (static_cast<uint32_t>(dv[8 * k + 1]) << 16),
                           dv[8 * k + 2] | (static_cast<uint32_t>(dv[8 * k + 3]) << 16),
                           dv[8 * k + 4] | (static_cast<uint32_t>(dv[8 * k + 5]) << 16),
                           dv[8 * k + 6] | (static_cast<uint32_t>(dv[8 * k + 7]) << 16));
    } else {
#pragma unroll
      for (int k = 0; k < kIndexItems; ++k)
        if (base + k < a.n) {
          a.target[base + k] = static_cast<uint32_t>(val[k] >> 32);
          a.weight[base + k] = static_cast<uint32_t>(val[k]);
          a.delay[base + k] = static_cast<uint16_t>(static_cast<uint32_t>(key[k]) & delay_mask);
        }
    }
    // Bitmap: kIndexItems (= 8) bits per thread, four threads per word.
    static_assert(kIndexItems == 8, "bitmap assembly assumes one byte per thread");
    const uint32_t b1 = __shfl_down_sync(0xffffffffu, bits, 1);
    const uint32_t b2 = __shfl_down_sync(0xffffffffu, bits, 2);
    const uint32_t b3 = __shfl_down_sync(0xffffffffu, bits, 3);
    if ((lane & 3u) == 0) a.starts[blk * (kIndexTile / 32) + tid / 4] = bits | (b1 << 8) | (b2 << 16) | (b3 << 24);
    uint32_t c = __popc(bits);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) warp_cnt[warp] = c;
    __syncthreads();
    if (tid == 0) {
      uint32_t total = 0;
      for (int w = 0; w < kIndexThreads / 32; ++w) total += warp_cnt[w];
      a.block_counts[blk] = total;
    }
    __syncthreads();
  }
}

// group_first[g] = position of the g-th group start, from the bitmap and the
// exclusive scan of the per-block counts.  One bitmap word (32 positions)
// per thread: a block of 256 threads covers four unpack blocks, two warps
// each.
__global__ void __launch_bounds__(kIndexThreads) index_groups_kernel(IndexArgs a) {
  constexpr uint32_t kWords = kIndexTile / 32;  // bitmap words per unpack block
  static_assert(kWords == 64 && kIndexThreads % kWords == 0, "two warps per unpack block");
  __shared__ uint32_t warp_tmp[kIndexThreads / 32];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t n_blocks = (a.n + kIndexTile - 1) / kIndexTile;
  const uint64_t n_words = n_blocks * kWords;
  for (uint64_t w0 = static_cast<uint64_t>(blockIdx.x) * kIndexThreads; w0 < n_words;
       w0 += static_cast<uint64_t>(gridDim.x) * kIndexThreads) {
    const uint64_t w = w0 + tid;
    uint32_t bits = w < n_words ? a.starts[w] : 0u;
    const uint32_t c = __popc(bits);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (static_cast<int>(lane) >= o) incl += y;
    }
    if (lane == 31) warp_tmp[warp] = incl;
    __syncthreads();
    if (bits) {
      const uint32_t before = (warp & 1u) ? warp_tmp[warp - 1] : 0u;
      uint64_t g = a.block_offsets[w / kWords] + before + incl - c;
      const uint64_t q0 = w * 32u;
      do {
        const uint32_t b = __ffs(bits) - 1;
        bits &= bits - 1;
        if (g < a.group_cap) a.group_first[g] = q0 + b;
        else atomicOr(a.err, kErrBounds);
        ++g;
      } while (bits);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && tid == 0) *a.n_groups = a.block_offsets[n_blocks];
}

// One thread per (network m, local node i = 0 .. n_nodes_m): the network's
// CSR offset of i (first position of its segment whose source is >= i) and
// the groups before it.
template <typename K>
__global__ void member_index_kernel(MemberIndexArgs a) {
  const uint64_t e = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= a.n_entries) return;
  int lo = 0, hi = a.n_members - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.local_base[mid] <= e) lo = mid; else hi = mid - 1;
  }
  const int m = lo;
  const uint64_t i = e - a.local_base[m];
  const K* keys = static_cast<const K*>(a.keys);
  const uint64_t sb = a.seg_begin[m];
  uint64_t l = sb, h = a.seg_end[m];
  while (l < h) {
    const uint64_t mid = (l + h) >> 1;
    if ((static_cast<uint64_t>(keys[mid]) >> a.delay_bits) < i) l = mid + 1; else h = mid;
  }
  a.row_local[e] = l - sb;
  const uint64_t ng = *a.n_groups < a.group_cap ? *a.n_groups : a.group_cap;
  const auto first_group_at = [&](uint64_t pos) {
    uint64_t gl = 0, gh = ng;
    while (gl < gh) {
      const uint64_t mid = (gl + gh) >> 1;
      if (a.group_first[mid] < pos) gl = mid + 1; else gh = mid;
    }
    return gl;
  };
  const uint64_t g0 = first_group_at(sb);
  a.group_local[e] = first_group_at(l) - g0;
  if (i == 0) a.gfirst[m] = g0;
  if (e == 0) a.gfirst[a.n_members] = ng;
}

cudaError_t launch_index_unpack(const IndexArgs& a, unsigned grid, cudaStream_t st) {
  if (a.key32)
    a.unpacked ? index_unpack_kernel<uint32_t, true><<<grid, kIndexThreads, 0, st>>>(a)
               : index_unpack_kernel<uint32_t, false><<<grid, kIndexThreads, 0, st>>>(a);
  else
    a.unpacked ? index_unpack_kernel<uint64_t, true><<<grid, kIndexThreads, 0, st>>>(a)
               : index_unpack_kernel<uint64_t, false><<<grid, kIndexThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_member_index(const MemberIndexArgs& a, cudaStream_t st) {
  const unsigned grid = static_cast<unsigned>((a.n_entries + 255) / 256);
  if (a.key32)
    member_index_kernel<uint32_t><<<grid, 256, 0, st>>>(a);
  else
    member_index_kernel<uint64_t><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

__global__ void rebase_group_first_kernel(uint64_t* group_first, const uint64_t* n_groups, uint64_t group_cap,
                                          const uint64_t* gfirst, const uint64_t* seg_begin, int n_members) {
  const uint64_t ng = *n_groups < group_cap ? *n_groups : group_cap;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < ng; g += stride) {
    int lo = 0, hi = n_members - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (gfirst[mid] <= g) lo = mid; else hi = mid - 1;
    }
    group_first[g] -= seg_begin[lo];
  }
}

// Source of every connection from row_ptr (for host copies): one warp per
// node writes its row with coalesced stores.
__global__ void expand_sources_kernel(const uint64_t* row_ptr, uint64_t n_nodes, uint32_t* src) {
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t i = warp; i < n_nodes; i += n_warps) {
    const uint64_t b = row_ptr[i], e = row_ptr[i + 1];
    for (uint64_t q = b + lane; q < e; q += 32) src[q] = static_cast<uint32_t>(i);
  }
}

// Target shards: flags[i] = 1 when connection i's target (the value's high
// word) lies in [first, first + count).
__global__ void shard_flag_kernel(const uint64_t* vals, uint64_t n, uint32_t first, uint32_t count, uint32_t* flags) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t t = static_cast<uint32_t>(vals[i] >> 32);
    flags[i] = (t >= first && t - first < count) ? 1u : 0u;
  }
}

// Keeps the flagged connections, in generation order, at their scanned
// positions (offsets = exclusive scan of the flags).
__global__ void shard_compact_kernel(const void* keys_in, const uint64_t* vals_in, int key32, uint64_t n,
                                     const uint64_t* offsets, uint32_t first, uint32_t count, void* keys_out,
                                     uint64_t* vals_out) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t v = vals_in[i];
    const uint32_t t = static_cast<uint32_t>(v >> 32);
    if (!(t >= first && t - first < count)) continue;
    const uint64_t o = offsets[i];
    if (key32) static_cast<uint32_t*>(keys_out)[o] = static_cast<const uint32_t*>(keys_in)[i];
    else static_cast<uint64_t*>(keys_out)[o] = static_cast<const uint64_t*>(keys_in)[i];
    vals_out[o] = v;
  }
}

// In-place unpack of a build sorted in place (COPASS block sort): windows
// [x0, x1) in increasing order; take copies a window's keys and values into
// a temporary block, put writes its targets as uint32 over the value array,
// its weight bits over the key array and its delay steps into their own
// array.  Position x writes bytes [4x, 4x + 4) of each array, which hold
// pairs at positions <= x: already taken, so nothing is read after it was
// overwritten.
template <typename K>
__global__ void unpack_take_kernel(const K* __restrict__ keys, const uint64_t* __restrict__ vals, uint64_t x0,
                                   uint64_t x1, K* __restrict__ tk, uint64_t* __restrict__ tv) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t x = x0 + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < x1; x += stride) {
    tk[x - x0] = keys[x];
    tv[x - x0] = vals[x];
  }
}

template <typename K>
__global__ void unpack_put_kernel(uint32_t* __restrict__ weight, uint32_t* __restrict__ target,
                                  uint16_t* __restrict__ delay, uint64_t x0, uint64_t x1, const K* __restrict__ tk,
                                  const uint64_t* __restrict__ tv, uint32_t delay_mask) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t x = x0 + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < x1; x += stride) {
    const uint64_t v = tv[x - x0];
    target[x] = static_cast<uint32_t>(v >> 32);
    weight[x] = static_cast<uint32_t>(v);
    delay[x] = static_cast<uint16_t>(static_cast<uint32_t>(tk[x - x0]) & delay_mask);
  }
}

cudaError_t unpack_in_place(void* keys, int key32, uint64_t* vals, uint64_t n, uint64_t window, void* tk,
                            uint64_t* tv, uint32_t delay_mask, uint16_t* delay, int sms, cudaStream_t st) {
  for (uint64_t x0 = 0; x0 < n; x0 += window) {
    const uint64_t x1 = x0 + window < n ? x0 + window : n;
    const unsigned grid = static_cast<unsigned>(
        std::max<uint64_t>(1, std::min<uint64_t>((x1 - x0 + 255) / 256, static_cast<uint64_t>(sms) * 8)));
    if (key32) {
      unpack_take_kernel<uint32_t><<<grid, 256, 0, st>>>(static_cast<const uint32_t*>(keys), vals, x0, x1,
                                                         static_cast<uint32_t*>(tk), tv);
      unpack_put_kernel<uint32_t><<<grid, 256, 0, st>>>(static_cast<uint32_t*>(keys), reinterpret_cast<uint32_t*>(vals),
                                                        delay, x0, x1, static_cast<const uint32_t*>(tk), tv, delay_mask);
    } else {
      unpack_take_kernel<uint64_t><<<grid, 256, 0, st>>>(static_cast<const uint64_t*>(keys), vals, x0, x1,
                                                         static_cast<uint64_t*>(tk), tv);
      unpack_put_kernel<uint64_t><<<grid, 256, 0, st>>>(static_cast<uint32_t*>(keys), reinterpret_cast<uint32_t*>(vals),
                                                        delay, x0, x1, static_cast<const uint64_t*>(tk), tv, delay_mask);
    }
  }
  return cudaGetLastError();
}

}  // namespace snc
