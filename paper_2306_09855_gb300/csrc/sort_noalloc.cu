// sort_noalloc.cu -- snc_radix_sort_pairs_noalloc: the radix sort of
// snc_radix_sort_pairs for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: for example a simulation loop that
// has handed all of the device's memory to its own pool, or latency-bound
// code that cannot afford the implicit device synchronisation cudaMalloc and
// cudaFree may cause.  This entry point therefore takes all its working
// memory from one file-scope device array, g_sort_scratch, which every GPU
// that loads the library holds (kNoAllocScratchBytes) until the process
// exits.  The caller still passes the input and output buffers.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress while
// that device is current and caches it; that first call should therefore
// come before any stream capture.  Every call shares the array: two calls
// whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/snc.h"
#include "snc_internal.h"
#include "sort_kernels.h"

namespace snc {
void set_last_error(const char* msg);
}

namespace snc {
namespace {

constexpr uint64_t kNoAllocMaxPairs = SNC_NOALLOC_MAX_PAIRS;
constexpr size_t kNoAllocScratchBytes = 8u << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

// Layout inside the array: [ping-pong keys | ping-pong values | error word |
// sort scratch (look-back words, histograms, digit offsets, tile counters)].
constexpr size_t kTmpKeysBytes = kNoAllocMaxPairs * sizeof(uint64_t);
constexpr size_t kTmpValsBytes = kNoAllocMaxPairs * sizeof(uint32_t);
constexpr size_t kErrOffset = kTmpKeysBytes + kTmpValsBytes;
constexpr size_t kSortOffset = kErrOffset + 256;
constexpr SortTuning kNoAllocTuning{9, 0, 32};
// Worst case of the fixed plan: 64-bit keys take eight passes of 8 bits, and
// the status words of 2^19 / 8,192 tiles, two digit tables and the tickets
// must fit after the ping-pong buffers.
constexpr size_t kWorstTiles = (kNoAllocMaxPairs + 8191) / 8192;
constexpr size_t kWorstSortScratch = kWorstTiles * 512 * sizeof(uint64_t) + 2 * 8 * 2048 * sizeof(uint64_t) + 4096;
static_assert(kSortOffset + kWorstSortScratch <= kNoAllocScratchBytes, "no-allocation scratch too small");

__device__ __align__(256) static unsigned char g_sort_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

snc_status fail(snc_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

// Device address of g_sort_scratch on the current device (looked up once).
cudaError_t scratch_address(int dev, unsigned char** out) {
  unsigned char* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (p) {
    *out = p;
    return cudaSuccess;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  p = g_scratch_addr[dev].load(std::memory_order_relaxed);
  if (!p) {
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_sort_scratch);
    if (e != cudaSuccess) return e;
    p = static_cast<unsigned char*>(addr);
    g_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return cudaSuccess;
}

}  // namespace

}  // namespace snc

extern "C" snc_status snc_radix_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in,
                                                   uint64_t* keys_out, uint32_t* vals_out, uint64_t n,
                                                   int key_bits, void* stream) {
  return snc::abi_guard([&]() -> snc_status {
    using namespace snc;
    if (key_bits < 1 || key_bits > 64) return fail(SNC_ERR_INVALID_ARG, "key_bits outside [1, 64]");
    if (n > kNoAllocMaxPairs) {
      char msg[160];
      snprintf(msg, sizeof msg, "n = %llu exceeds the %llu pairs the no-allocation sort holds",
               static_cast<unsigned long long>(n), static_cast<unsigned long long>(kNoAllocMaxPairs));
      return fail(SNC_ERR_INVALID_ARG, msg);
    }
    if (n == 0) return SNC_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return fail(SNC_ERR_INVALID_ARG, "null buffer");
    // A fixed plan (digits of at most 9 bits, 8,192-key tiles), whatever the
    // process-wide tuning: its scratch fits the array for every n and key
    // width this entry point accepts (a wider tuned digit would need 2,048
    // look-back words per tile).
    const SortPasses sp = plan_passes(key_bits, kNoAllocTuning);
    if (kSortOffset + sort_scratch_bytes(n, sp) > kNoAllocScratchBytes)
      return fail(SNC_ERR_UNSUPPORTED, "sort scratch does not fit the static array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(SNC_ERR_CUDA, "no usable current device");
    unsigned char* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return fail(SNC_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t* keys_tmp = reinterpret_cast<uint64_t*>(base);
    uint32_t* vals_tmp = reinterpret_cast<uint32_t*>(base + kTmpKeysBytes);
    uint32_t* err = reinterpret_cast<uint32_t*>(base + kErrOffset);
    // The error word keeps the previous call's contents: clear it first (the
    // sort clears its own look-back words, histograms and counters).
    e = cudaMemsetAsync(err, 0, 256, st);
    if (e == cudaSuccess)
      e = radix_sort_run(keys_in, vals_in, keys_out, vals_out, keys_tmp, vals_tmp, n, sp, base + kSortOffset, err, st,
                         nullptr);
    // Wait for the sort and read its error word (a bounded device wait that
    // expired leaves the output unsorted).
    uint32_t bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SNC_ERR_CUDA, cudaGetErrorString(e));
    if (bits & kErrLookbackTimeout) return fail(SNC_ERR_TIMEOUT, "a look-back wait expired on the device");
    if (bits) return fail(SNC_ERR_CUDA, "device error bits set by the sort");
    return SNC_OK;
  });
}
