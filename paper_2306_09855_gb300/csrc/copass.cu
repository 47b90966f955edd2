// copass.cu -- COPASS block sort (Appendix A): the sorted runs of an array
// divided in blocks are partitioned, block by block, by a common threshold,
// the left partitions gathered and sorted into the block's place and the
// right partitions shifted to the end of the array.  Working memory: two
// blocks and the radix sort's scratch for one block.
#include "copass.h"

#include <algorithm>
#include <vector>

#include "snc_internal.h"

namespace snc {

namespace {

constexpr int kT = kCopassMaxRuns;  // threads of the partition kernel: one per run

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Run tables in device memory, one entry per run (kCopassMaxRuns each).
struct RunTable {
  uint64_t* len;    // remaining pairs of each run
  uint64_t* cum;    // exclusive prefix of len: run i starts at first + cum[i]
  uint64_t* part;   // its share of the current output block (left partition)
  uint64_t* pre;    // exclusive prefix of part: its place in the auxiliary block
  uint64_t* shift;  // how far its right partition moves: sum of part over later runs
};

__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kT / 2; s > 0; s >>= 1) {
    if (static_cast<int>(threadIdx.x) < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const uint64_t r = red[0];
  __syncthreads();
  return r;
}

// Exclusive prefix over the threads (Hillis-Steele in shared memory).
__device__ __forceinline__ uint64_t block_excl(uint64_t v, uint64_t* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 1; s < kT; s <<= 1) {
    const uint64_t add = static_cast<int>(threadIdx.x) >= s ? red[threadIdx.x - s] : 0ull;
    __syncthreads();
    red[threadIdx.x] += add;
    __syncthreads();
  }
  const uint64_t r = red[threadIdx.x] - v;
  __syncthreads();
  return r;
}

template <typename K>
__device__ __forceinline__ uint64_t count_below(const K* a, uint64_t n, K t, bool upper) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (upper ? a[mid] <= t : a[mid] < t) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The COPASS partition of the remaining runs (Appendix A, "The COPASS
// partition algorithm"), one thread per run: lo / hi are the counts of
// elements <= the lower and < the upper threshold; each iteration takes the
// run with the widest open interval (the lowest such run), its middle
// element as the trial threshold t~, and the counts below t~ (mu_lo: < t~,
// mu_hi: <= t~) in every run: t~ is the threshold (case 1), the new upper
// threshold (case 2) or the new lower one (case 3).  Last steps: with every
// interval at most one wide, the undecided elements (at index lo) are taken
// in ascending (value, run) order; with t~ the threshold, its copies are
// shared out in run order.  Both give ties to lower runs, so the left
// partitions are the first m pairs of the stable order.
template <typename K>
__global__ void __launch_bounds__(kT) copass_partition_kernel(const K* __restrict__ keys, uint64_t first, int k,
                                                              uint64_t m, RunTable t, uint32_t* err) {
  __shared__ uint64_t red[kT];
  __shared__ uint64_t s_lo[kT], s_hi[kT];
  __shared__ K s_val[kT];
  __shared__ uint64_t s_width[kT];
  __shared__ int s_arg[kT];
  const int i = threadIdx.x;
  const bool act = i < k;
  const uint64_t len = act ? t.len[i] : 0ull;
  const uint64_t cum = block_excl(len, red);
  const uint64_t total = block_sum(len, red);
  const K* run = keys + first + cum;
  uint64_t lo = 0, hi = len, part = 0;
  if (m == 0 || m >= total) {
    part = m == 0 ? 0ull : len;
  } else {
    bool done = false;
    for (uint32_t iter = 0; !done; ++iter) {
      if (iter > (1u << 20)) {  // far above any run count times the key width
        if (i == 0) atomicOr(err, kErrBounds);
        part = lo;
        break;
      }
      // The run with the widest open interval (lowest index among equals).
      s_width[i] = hi - lo;
      s_arg[i] = i;
      __syncthreads();
      for (int s = kT / 2; s > 0; s >>= 1) {
        if (i < s) {
          const uint64_t a = s_width[i], b = s_width[i + s];
          if (b > a || (b == a && s_arg[i + s] < s_arg[i])) {
            s_width[i] = b;
            s_arg[i] = s_arg[i + s];
          }
        }
        __syncthreads();
      }
      const uint64_t widest = s_width[0];
      const int l = s_arg[0];
      s_lo[i] = lo;
      s_hi[i] = hi;
      __syncthreads();
      const uint64_t sum_lo = block_sum(lo, red);
      if (widest <= 1) {
        // Last step, case 1: the undecided elements by (value, run).
        const bool cand = act && hi == lo + 1;
        s_val[i] = cand ? run[lo] : K(0);
        __syncthreads();
        const uint64_t d = m - sum_lo;
        uint64_t rank = 0;
        if (cand)
          for (int j = 0; j < k; ++j)
            if (s_hi[j] == s_lo[j] + 1 && (s_val[j] < s_val[i] || (s_val[j] == s_val[i] && j < i))) ++rank;
        part = lo + ((cand && rank < d) ? 1u : 0u);
        done = true;
        break;
      }
      const uint64_t mid = (s_lo[l] + s_hi[l]) / 2;
      __syncthreads();
      // Every thread reads the trial threshold from run l.
      uint64_t cum_l;
      {
        red[i] = cum;
        __syncthreads();
        cum_l = red[l];
        __syncthreads();
      }
      const K tv = keys[first + cum_l + mid];
      const uint64_t mul = act ? count_below(run, len, tv, false) : 0ull;
      const uint64_t muh = act ? count_below(run, len, tv, true) : 0ull;
      const uint64_t s_mul = block_sum(mul, red);
      const uint64_t s_muh = block_sum(muh, red);
      if (s_mul <= m && m <= s_muh) {
        // Last step, case 2: t~ is the threshold; its copies in run order.
        const uint64_t eq = muh - mul;
        const uint64_t before = block_excl(eq, red);
        const uint64_t d = m - s_mul;
        const uint64_t take = d > before ? (d - before < eq ? d - before : eq) : 0ull;
        part = mul + take;
        done = true;
        break;
      }
      if (m < s_mul) hi = mul;  // case 2: the threshold lies below t~
      else lo = muh;            // case 3: it lies above
    }
  }
  const uint64_t pre = block_excl(part, red);
  const uint64_t all = block_sum(part, red);
  if (act) {
    t.cum[i] = cum;
    t.part[i] = part;
    t.pre[i] = pre;
    t.shift[i] = all - pre - part;  // parts of the runs after this one
  }
  if (i == 0 && all != m) atomicOr(err, kErrBounds);
}

// The run holding position g of the remaining pairs (cum ascending).
__device__ __forceinline__ int run_of(const uint64_t* cum, int k, uint64_t g) {
  int lo = 0, hi = k - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cum[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Left partitions into the auxiliary block, in run order.
template <typename K, typename V>
__global__ void copass_gather_kernel(const K* __restrict__ keys, const V* __restrict__ vals, uint64_t first, int k,
                                     RunTable t, uint64_t m, K* __restrict__ ak, V* __restrict__ av) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < m; g += stride) {
    const int i = run_of(t.pre, k, g);
    const uint64_t src = first + t.cum[i] + (g - t.pre[i]);
    ak[g] = keys[src];
    av[g] = vals[src];
  }
}

// One window [x0, x1) of the right shift: its right-partition pairs into
// the temporary block (take), then to their new places (put).  Windows are
// handled from the end of the array, so every place a window writes is
// either inside it (already taken) or after it (already moved away).
template <typename K, typename V>
__global__ void copass_take_kernel(const K* __restrict__ keys, const V* __restrict__ vals, uint64_t first, int k,
                                   RunTable t, uint64_t x0, uint64_t x1, K* __restrict__ tk, V* __restrict__ tv) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t x = x0 + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < x1; x += stride) {
    const uint64_t g = x - first;
    const int i = run_of(t.cum, k, g);
    if (g - t.cum[i] < t.part[i]) continue;  // a left pair, already gathered
    tk[x - x0] = keys[x];
    tv[x - x0] = vals[x];
  }
}

template <typename K, typename V>
__global__ void copass_put_kernel(K* __restrict__ keys, V* __restrict__ vals, uint64_t first, int k, RunTable t,
                                  uint64_t x0, uint64_t x1, const K* __restrict__ tk, const V* __restrict__ tv) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t x = x0 + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < x1; x += stride) {
    const uint64_t g = x - first;
    const int i = run_of(t.cum, k, g);
    if (g - t.cum[i] < t.part[i]) continue;
    keys[x + t.shift[i]] = tk[x - x0];
    vals[x + t.shift[i]] = tv[x - x0];
  }
}

// After a round: every run keeps its right partition.
__global__ void copass_commit_kernel(RunTable t, int k) {
  const int i = threadIdx.x;
  if (i < k) t.len[i] -= t.part[i];
}

struct CopassLayout {
  void* ak;
  void* av;
  void* tk;
  void* tv;
  void* sort_scratch;
  RunTable runs;
};

CopassLayout copass_layout(void* scratch, uint64_t block, int kb, int vb, const SortPasses& sp) {
  CopassLayout l{};
  unsigned char* p = static_cast<unsigned char*>(scratch);
  l.ak = p;
  p += align256(block * kb);
  l.av = p;
  p += align256(block * vb);
  l.tk = p;
  p += align256(block * kb);
  l.tv = p;
  p += align256(block * vb);
  l.sort_scratch = p;
  p += align256(sort_scratch_bytes(block, sp));
  uint64_t* r = reinterpret_cast<uint64_t*>(p);
  l.runs = RunTable{r, r + kT, r + 2 * kT, r + 3 * kT, r + 4 * kT};
  return l;
}

}  // namespace

size_t copass_scratch_bytes(uint64_t block, int key_bytes, int val_bytes, const SortPasses& sp) {
  return 2 * align256(block * key_bytes) + 2 * align256(block * val_bytes) + align256(sort_scratch_bytes(block, sp)) +
         5 * kT * sizeof(uint64_t);
}

template <typename K, typename V>
cudaError_t copass_sort_run(K* keys, V* vals, uint64_t n, uint64_t block, const SortPasses& sp, void* scratch,
                            uint32_t* err, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (block == 0 || block % kCopassAlign != 0) return cudaErrorInvalidValue;
  const uint64_t nb = (n + block - 1) / block;
  if (nb > static_cast<uint64_t>(kCopassMaxRuns)) return cudaErrorInvalidValue;
  const CopassLayout L = copass_layout(scratch, block, sizeof(K), sizeof(V), sp);
  K* ak = static_cast<K*>(L.ak);
  V* av = static_cast<V*>(L.av);
  K* tk = static_cast<K*>(L.tk);
  V* tv = static_cast<V*>(L.tv);
  const int k = static_cast<int>(nb);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  // 1. Every block sorted on its own (into the auxiliary block, then back).
  std::vector<uint64_t> len(kT, 0);
  for (uint64_t b = 0; b < nb; ++b) {
    const uint64_t off = b * block, cnt = std::min<uint64_t>(block, n - off);
    len[b] = cnt;
    if ((e = radix_sort_run<K, V>(keys + off, vals + off, ak, av, tk, tv, cnt, sp, L.sort_scratch, err, st,
                                  nullptr)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(keys + off, ak, cnt * sizeof(K), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(vals + off, av, cnt * sizeof(V), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  }
  if (nb == 1) return cudaSuccess;
  if ((e = cudaMemcpyAsync(L.runs.len, len.data(), kT * sizeof(uint64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  // The host copy of len must stay valid until the copy ran.
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const auto grid = [&](uint64_t items) {
    return static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>((items + 255) / 256, sms * 8ull)));
  };
  // 2. Output blocks in order.
  for (uint64_t o = 0; o + 1 < nb; ++o) {
    const uint64_t first = o * block, size = std::min<uint64_t>(block, n - first);
    copass_partition_kernel<K><<<1, kT, 0, st>>>(keys, first, k, size, L.runs, err);
    copass_gather_kernel<K, V><<<grid(size), 256, 0, st>>>(keys, vals, first, k, L.runs, size, ak, av);
    for (uint64_t x1 = n; x1 > first;) {
      const uint64_t x0 = x1 - first > block ? x1 - block : first;
      copass_take_kernel<K, V><<<grid(x1 - x0), 256, 0, st>>>(keys, vals, first, k, L.runs, x0, x1, tk, tv);
      copass_put_kernel<K, V><<<grid(x1 - x0), 256, 0, st>>>(keys, vals, first, k, L.runs, x0, x1, tk, tv);
      x1 = x0;
    }
    copass_commit_kernel<<<1, kT, 0, st>>>(L.runs, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // The auxiliary block, sorted, becomes block o (its place is free now).
    if ((e = radix_sort_run<K, V>(ak, av, keys + first, vals + first, tk, tv, size, sp, L.sort_scratch, err, st,
                                  nullptr)) != cudaSuccess)
      return e;
  }
  // The last block holds the rest, the largest keys: already sorted runs
  // merged into it by the last round's shift, sorted once more in place.
  {
    const uint64_t first = (nb - 1) * block, size = n - first;
    if ((e = cudaMemcpyAsync(ak, keys + first, size * sizeof(K), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(av, vals + first, size * sizeof(V), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = radix_sort_run<K, V>(ak, av, keys + first, vals + first, tk, tv, size, sp, L.sort_scratch, err, st,
                                  nullptr)) != cudaSuccess)
      return e;
  }
  return cudaGetLastError();
}

template cudaError_t copass_sort_run<uint64_t, uint32_t>(uint64_t*, uint32_t*, uint64_t, uint64_t, const SortPasses&,
                                                         void*, uint32_t*, cudaStream_t);
template cudaError_t copass_sort_run<uint32_t, uint64_t>(uint32_t*, uint64_t*, uint64_t, uint64_t, const SortPasses&,
                                                         void*, uint32_t*, cudaStream_t);
template cudaError_t copass_sort_run<uint64_t, uint64_t>(uint64_t*, uint64_t*, uint64_t, uint64_t, const SortPasses&,
                                                         void*, uint32_t*, cudaStream_t);

}  // namespace snc
