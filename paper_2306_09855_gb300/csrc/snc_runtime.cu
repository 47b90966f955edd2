// snc_runtime.cu -- the C ABI: context, Create / Connect bookkeeping and the
// calibration (Finalize) driver that queues the generation, sort and index
// kernels on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/snc.h"
#include "gen_kernels.h"
#include "index_kernels.h"
#include "snc_internal.h"
#include "sort_kernels.h"
#include "source_major.h"
#include "deliver.h"
#include "arrays.h"
#include "copass.h"

using namespace snc;

namespace {

constexpr int kMaxEvents = 4 + kMaxPasses + 2;
int g_gen_blocks_per_sm = 8;
thread_local std::string g_last_error = "no error";

struct DevBuf {
  void* p;
  size_t bytes;
};

// Page-locked host memory is recycled for the whole process: freeing it
// (cudaFreeHost) would synchronize the device and stall builds running on
// other streams when a context is destroyed.
// Bounds a graph-recorded build fixes (snc_set_graph_test).
struct GraphTest {
  double bernoulli_sd = 10.0;
  double bernoulli_slack = 32.0;
  uint32_t redraw_rounds = 0;  // 0: computed from the density
};
GraphTest g_graph_test;

class PinnedPool {
 public:
  static size_t round_size(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
  }
  void* get(size_t bytes) {
    const size_t cls = round_size(bytes);
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto& v = free_[cls];
      if (!v.empty()) {
        void* p = v.back();
        v.pop_back();
        return p;
      }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, cls) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    free_[round_size(bytes)].push_back(p);
  }

 private:
  std::mutex mu_;
  std::map<size_t, std::vector<void*>> free_;
};

PinnedPool& pinned_pool() {
  static PinnedPool* pool = new PinnedPool();  // lives as long as the process
  return *pool;
}

// Device memory of one build (a context, or all members of a batch), shared
// by the member contexts and released when the last of them is destroyed.
struct Storage {
  snc_allocator alloc{};
  bool custom_alloc = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<DevBuf> bufs;
  uint64_t live_bytes = 0, peak_bytes = 0;
  cudaEvent_t ev[kMaxEvents] = {};
  int n_ev = 0;
  bool events_ok = false;
  uint64_t* h_pinned = nullptr;  // small pinned staging area
  size_t h_pinned_words = 0;
  uint32_t* d_err = nullptr;
  uint64_t* d_n_groups = nullptr;
  // Batches: per-member first connection / first group, read back at sync.
  uint64_t* d_bases = nullptr;  // [2 * (members + 1)] on the device
  uint64_t* h_bases = nullptr;  // pinned copy
  size_t h_bases_words = 0;
  // Graph builds with pairwise_bernoulli projections: each network's
  // connection count is drawn on the device at every replay; the build
  // copies the counts here (pinned), read at sync.
  uint64_t* h_real = nullptr;
  size_t h_real_words = 0;
  bool real_counts = false;
  int n_members = 1;
  uint64_t n_total = 0;  // connections of the whole build
  bool synced = false;
  uint32_t err_bits = 0;
  uint64_t n_groups = 0;
  // Host -> device copies go through pinned staging chunks that live as long
  // as the build, so that a recorded graph can replay them.
  std::vector<std::pair<unsigned char*, size_t>> stage_chunks;  // (memory, capacity)
  size_t stage_used = 0;    // bytes used in the last chunk
  size_t stage_total = 0;   // bytes staged by the current build
  // Graph builds (snc_batch_finalize_graph): mode 1 keeps every buffer of
  // the first build (no frees) and records the allocation order; mode 2 hands
  // the recorded buffers out again while the same build is captured.
  int mode = 0;
  bool capturing = false;
  std::vector<DevBuf> rec;
  size_t rec_pos = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t own_stream = nullptr;  // graph builds run on a stream of their own
  struct SeedSite {
    DevProj* host;  // staged copy of a projection record
    int member;
    uint32_t local;
  };
  std::vector<SeedSite> seed_sites;
  uint64_t generation = 0;  // bumped by every replay: member views are refreshed

  void* stage(const void* src, size_t bytes) {
    const size_t need = (bytes + 15) & ~static_cast<size_t>(15);
    if (stage_chunks.empty() || stage_used + need > stage_chunks.back().second) {
      if (capturing) return nullptr;  // reserved before the capture
      const size_t cap = PinnedPool::round_size(std::max<size_t>(need, 1u << 20));
      void* p = pinned_pool().get(cap);
      if (!p) return nullptr;
      stage_chunks.push_back({static_cast<unsigned char*>(p), cap});
      stage_used = 0;
    }
    unsigned char* dst = stage_chunks.back().first + stage_used;
    std::memcpy(dst, src, bytes);
    stage_used += need;
    stage_total += need;
    return dst;
  }
  bool reserve_stage(size_t bytes) {
    const size_t cap = PinnedPool::round_size(std::max<size_t>(bytes, 1u << 20));
    void* p = pinned_pool().get(cap);
    if (!p) return false;
    stage_chunks.push_back({static_cast<unsigned char*>(p), cap});
    stage_used = 0;
    return true;
  }

  void* get(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (mode == 2) {  // replaying the recorded allocation order
      if (rec_pos >= rec.size() || rec[rec_pos].bytes != bytes) return nullptr;
      return rec[rec_pos++].p;
    }
    void* p = nullptr;
    if (custom_alloc) {
      p = alloc.alloc(bytes, stream, alloc.user);
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {
      // The kernels use vector and bulk copies that need aligned arrays.
      if (custom_alloc) alloc.free(p, bytes, stream, alloc.user);
      return nullptr;
    }
    if (p) {
      bufs.push_back({p, bytes});
      live_bytes += bytes;
      if (live_bytes > peak_bytes) peak_bytes = live_bytes;
      if (mode == 1) rec.push_back({p, bytes});
    }
    return p;
  }
  void put(void* p) {
    if (!p || mode != 0) return;  // graph builds keep every buffer
    for (size_t i = 0; i < bufs.size(); ++i) {
      if (bufs[i].p == p) {
        if (custom_alloc)
          alloc.free(p, bufs[i].bytes, stream, alloc.user);
        else
          cudaFreeAsync(p, stream);
        live_bytes -= bufs[i].bytes;
        bufs.erase(bufs.begin() + static_cast<long>(i));
        return;
      }
    }
  }
  bool init_host(size_t words) {
    for (int i = 0; i < kMaxEvents; ++i) {
      if (cudaEventCreate(&ev[i]) != cudaSuccess) {
        cudaGetLastError();
        for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
        return false;
      }
    }
    events_ok = true;
    h_pinned = static_cast<uint64_t*>(pinned_pool().get(words * sizeof(uint64_t)));
    if (!h_pinned) return false;
    h_pinned_words = words;
    return true;
  }
  ~Storage() {
    cudaSetDevice(device);
    cudaStreamSynchronize(stream);
    if (gexec) cudaGraphExecDestroy(gexec);
    mode = 0;
    while (!bufs.empty()) put(bufs.back().p);
    cudaStreamSynchronize(stream);
    if (own_stream) cudaStreamDestroy(own_stream);
    if (events_ok)
      for (int i = 0; i < kMaxEvents; ++i) cudaEventDestroy(ev[i]);
    pinned_pool().put(h_pinned, h_pinned_words * sizeof(uint64_t));
    pinned_pool().put(h_bases, h_bases_words * sizeof(uint64_t));
    pinned_pool().put(h_real, h_real_words * sizeof(uint64_t));
    for (auto& ch : stage_chunks) pinned_pool().put(ch.first, ch.second);
    cudaGetLastError();
  }
};

}  // namespace

struct snc_ctx {
  snc_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 148;
  uint64_t n_nodes = 0;
  std::vector<Projection> projs;
  bool finalized = false;
  std::string err = "no error";
  std::shared_ptr<Storage> store;
  // Position of this context in its build (member 0 of one for a plain
  // finalize; a batch concatenates its members' nodes).
  int member = 0;
  uint64_t node_base = 0;
  int sort_stages = 0;  // timed sort stages of the last build (radix passes, or 1 for the source-major sort)
  // Target shard: keep only the connections whose target is in
  // [shard_first, shard_first + shard_n) (snc_set_target_shard).
  bool sharded = false;
  uint32_t shard_first = 0, shard_n = 0;
  // COPASS block sort (snc_set_block_sort): blocks of this many connections,
  // 0 = the out-of-place radix sort.
  uint64_t block_sort = 0;
  // Results: device views; for batch members resolved at synchronize (and
  // again after every graph replay of the build).
  bool view_ready = false;
  uint64_t view_gen = 0;
  uint64_t seg_begin = 0;  // first position of this network's connections in the build's arrays
  uint64_t seg_count = 0;
  uint64_t n_syn = 0;
  uint64_t n_groups = 0;
  uint64_t group_cap = 0;
  uint64_t* row_ptr = nullptr;
  uint64_t* group_ptr = nullptr;
  uint32_t* target_all = nullptr;
  uint16_t* delay_all = nullptr;
  float* weight_all = nullptr;
  uint64_t* group_first_all = nullptr;
  uint32_t* target = nullptr;
  uint16_t* delay = nullptr;
  float* weight = nullptr;
  uint64_t* group_first = nullptr;
  KeyLayout layout{1, 1, 1};
  SortPasses passes{};
  snc_stats stats{};
};

namespace {

snc_status fail(snc_ctx* c, snc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_last_error = buf;
  return st;
}

#define SNC_CUDA(c, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail((c), SNC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void* dev_alloc(snc_ctx* c, size_t bytes) {
  void* p = c->store->get(bytes);
  c->stats.device_bytes_peak = c->store->peak_bytes;
  return p;
}

void dev_free(snc_ctx* c, void* p) { c->store->put(p); }

// Calls on a finished network (delivery, host copies) free their temporary
// buffers when they end, also on a graph-built network, whose store
// otherwise keeps every buffer it hands out.
class CallScope {
 public:
  explicit CallScope(snc_ctx* c) : s_(*c->store), saved_(s_.mode) { s_.mode = 0; }
  ~CallScope() { s_.mode = saved_; }
  CallScope(const CallScope&) = delete;
  CallScope& operator=(const CallScope&) = delete;

 private:
  Storage& s_;
  int saved_;
};

// Host -> device copy through the build's pinned staging area; *staged
// receives the staged host copy.
cudaError_t upload(snc_ctx* c, void* dst, const void* src, size_t bytes, void** staged = nullptr) {
  if (bytes == 0) return cudaSuccess;
  void* h = c->store->stage(src, bytes);
  if (!h) return cudaErrorMemoryAllocation;
  if (staged) *staged = h;
  c->stats.h2d_bytes += bytes;
  return cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, c->store->stream);
}

int bit_width(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

bool is_sampler(const Projection& p) {
  return p.rule.kind == SNC_PAIRWISE_BERNOULLI ||
         ((p.rule.kind == SNC_FIXED_INDEGREE || p.rule.kind == SNC_FIXED_OUTDEGREE) && !p.rule.allow_multapses);
}

bool is_total_redraw(const Projection& p) {
  return p.rule.kind == SNC_FIXED_TOTAL_NUMBER && (!p.rule.allow_multapses || !p.rule.allow_autapses);
}

// Validation and sizing of one Connect call (readings of Sec. 2.1 / Sec. 4).
// The node lists, the rule's limits and the count are checked as for a call
// with explicit arrays (arrays.cpp), here with both lists given as ranges.
snc_status plan_projection(snc_ctx* c, Projection& p, const ConnectArrays& arrays = ConnectArrays{}) {
  const snc_conn_rule& r = p.rule;
  ArrayPlan lists;
  std::string why;
  const snc_status cs = check_connect_arrays(static_cast<uint32_t>(c->n_nodes), c->cfg.dt_ms, p.src, p.tgt, r,
                                             arrays, &lists, &why);
  if (cs != SNC_OK) return fail(c, cs, "connect: %s", why.c_str());
  p.exact_count = r.kind != SNC_PAIRWISE_BERNOULLI;  // Bernoulli counts are drawn at finalize
  p.count = lists.count;
  // The library's own copy of the arrays (the caller's are read during the
  // call only).
  if (arrays.src_ids) {
    p.src_list = true;
    p.src_ids.assign(arrays.src_ids, arrays.src_ids + p.src.n);
    p.src.first = 0;
  }
  if (arrays.tgt_ids) {
    p.tgt_list = true;
    p.tgt_ids.assign(arrays.tgt_ids, arrays.tgt_ids + p.tgt.n);
    p.tgt.first = 0;
  }
  if (arrays.weights) {
    p.w_bits.resize(arrays.n_conn);
    std::memcpy(p.w_bits.data(), arrays.weights, arrays.n_conn * sizeof(float));
  }
  if (arrays.delays_ms) p.d_steps = std::move(lists.steps);
  const snc_dist& wd = p.syn.weight;
  const snc_dist& dd = p.syn.delay_ms;
  if ((wd.kind != SNC_DIST_CONST && wd.kind != SNC_DIST_NORMAL) ||
      (dd.kind != SNC_DIST_CONST && dd.kind != SNC_DIST_NORMAL))
    return fail(c, SNC_ERR_INVALID_ARG, "unknown distribution kind");
  if ((wd.kind == SNC_DIST_NORMAL && !(wd.std >= 0.0)) || (dd.kind == SNC_DIST_NORMAL && !(dd.std >= 0.0)))
    return fail(c, SNC_ERR_INVALID_ARG, "negative standard deviation");
  if (!std::isfinite(wd.mean) || !std::isfinite(dd.mean)) return fail(c, SNC_ERR_INVALID_ARG, "non-finite mean");
  // Delay: given per connection, constant step or threshold table (Sec. 2.1:
  // round(d / dt), >= 1).
  if (!p.d_steps.empty()) {
    p.d_table = false;
    p.d_const = 1;
    p.max_step = std::max<uint32_t>(1, lists.max_step);
  } else if (arrays.delays_ms) {  // zero numbered connections
    p.d_table = false;
    p.d_const = 1;
    p.max_step = 1;
  } else if (dd.kind == SNC_DIST_CONST || dd.std == 0.0) {
    uint32_t step = 1;
    if (delay_step_of(dd.mean, c->cfg.dt_ms, &step) != SNC_OK)
      return fail(c, SNC_ERR_UNSUPPORTED, "delay above 65535 steps");
    p.d_table = false;
    p.d_const = step;
    p.max_step = p.d_const;
  } else {
    const int st = delay_thresholds(dd.mean, dd.std, c->cfg.dt_ms, p.d_thr, p.d_base);
    if (st != SNC_OK) return fail(c, static_cast<snc_status>(st), "delay distribution outside the table limits");
    if (static_cast<uint64_t>(p.d_base) + p.d_thr.size() > 65535)
      return fail(c, SNC_ERR_UNSUPPORTED, "delay above 65535 steps");
    p.d_table = true;
    p.max_step = p.d_base + static_cast<uint32_t>(p.d_thr.size());
  }
  if (r.kind == SNC_PAIRWISE_BERNOULLI) {
    for (int s = 0; s < 2; ++s) {
      const uint64_t cand = (s == 1 && p.src.n > 0) ? p.src.n - 1u : (s == 1 ? 0 : p.src.n);
      const int st = binomial_thresholds(cand, r.p, p.b_thr[s], p.b_base[s]);
      if (st != SNC_OK) return fail(c, static_cast<snc_status>(st), "binomial table outside limits");
    }
  }
  if (is_sampler(p)) {
    const uint64_t n_other = (r.kind == SNC_FIXED_OUTDEGREE) ? p.tgt.n : p.src.n;
    if (n_other > kSamplerMaxNodes)
      return fail(c, SNC_ERR_UNSUPPORTED, "sampler range of %llu nodes above the bitmap limit %llu",
                  static_cast<unsigned long long>(n_other), static_cast<unsigned long long>(kSamplerMaxNodes));
  }
  return SNC_OK;
}

}  // namespace

namespace snc {
// Lets other translation units report context-free failures through
// snc_last_error(NULL).
void set_last_error(const char* msg) { g_last_error = msg; }

snc_status abi_exception(const char* what) noexcept {
  try {
    g_last_error = std::string("host resources exhausted: ") + what;
  } catch (...) {
  }
  return SNC_ERR_OOM;
}

snc_status estimate_build(const snc_ctx* c, BuildEstimate* e) {
  if (!c || !e) return SNC_ERR_INVALID_ARG;
  uint64_t n = 0, redraw_slots = 0, redraw_table = 0, primaries = 0;
  uint32_t max_step = 1;
  for (const Projection& p : c->projs) {
    max_step = std::max(max_step, p.max_step);
    if (p.rule.kind == SNC_PAIRWISE_BERNOULLI) {
      // Hard bound: every target draws at most base + table length sources
      // (Sec. 4 reading of the Bernoulli rule); the estimate takes the mean
      // plus ten standard deviations of the total when that is lower.
      const uint64_t hard = static_cast<uint64_t>(p.tgt.n) *
                            std::max(p.b_base[0] + p.b_thr[0].size(), p.b_base[1] + p.b_thr[1].size());
      const double mean = static_cast<double>(p.tgt.n) * p.src.n * p.rule.p;
      const double soft = mean + 10.0 * std::sqrt(mean * (1.0 - p.rule.p)) + 1024.0;
      n += std::min<uint64_t>(hard, static_cast<uint64_t>(soft));
      primaries += p.tgt.n;
    } else {
      n += p.count;
      if (is_sampler(p)) primaries += (p.rule.kind == SNC_FIXED_OUTDEGREE) ? p.src.n : p.tgt.n;
      if (is_total_redraw(p)) {
        redraw_slots += p.count;
        if (!p.rule.allow_multapses) {
          uint64_t cap = 1;
          while (cap < 2 * p.count + 64) cap <<= 1;
          redraw_table += 2 * cap;  // keys and (when not packed) values
        }
      }
    }
  }
  const uint64_t N = c->n_nodes;
  const uint64_t gc = std::max<uint64_t>(1, std::min<uint64_t>(n, N * (static_cast<uint64_t>(max_step) + 1)));
  KeyLayout lay{std::max(1, bit_width(N > 0 ? N - 1 : 0)), std::max(1, bit_width(max_step)),
                std::max(1, bit_width(N > 0 ? N - 1 : 0))};
  const uint64_t scratch = sort_scratch_bytes(n, plan_passes(lay.total_bits()));
  const uint64_t pair = (lay.key32() ? 4 : 8) + 8;  // key + (target, weight) value
  // Generation and sort: two key/value buffers, sort scratch, the redraw
  // lists and tables, per-primary offsets.
  const uint64_t gen = 2 * pair * n + scratch +
                       std::max<uint64_t>(34 * redraw_slots + 8 * redraw_table + 16 * (primaries + 1), 2 * n);
  // Index: sorted keys, targets and weights (in the value buffer) and delays
  // (or, when the sort could not unpack, separate target / weight arrays),
  // group starts, row and group pointers (twice for batch members), scans.
  const uint64_t index = (pair + 10) * n + n / 8 + 8 * gc + 32 * (N + 1) + 16 * (primaries + 1);
  // Allocation granularity and the small per-build arrays.
  const uint64_t slack = 96ull << 20;
  e->n_syn = n;
  e->peak_bytes = std::max(gen, index) + slack;
  if (c->block_sort && !c->sharded) {
    // COPASS block sort: one key/value buffer, the delays, two blocks of
    // working memory and one block's sort scratch; the unpack works in place.
    const uint64_t blk = c->block_sort;
    const SortPasses sp = plan_passes(lay.total_bits());
    const uint64_t base = pair * n + 2 * n;
    const uint64_t sort = base + copass_scratch_bytes(blk, lay.key32() ? 4 : 8, 8, sp);
    const uint64_t gen1 = pair * n + std::max<uint64_t>(34 * redraw_slots + 8 * redraw_table + 16 * (primaries + 1), 0);
    const uint64_t idx1 = base + n / 8 + 8 * gc + 32 * (N + 1) + 16 * (primaries + 1) + pair * blk;
    e->peak_bytes = std::max(std::max(gen1, sort), idx1) + slack;
  }
  e->resident_bytes = 10 * n + 8 * gc + 32 * (N + 1) + slack;
  e->n_nodes = N;
  e->max_step = max_step;
  return SNC_OK;
}

void rebind_build(snc_ctx* c, cudaStream_t stream, const snc_allocator* alloc) {
  c->stream = stream;
  c->cfg.stream = stream;
  c->store->stream = stream;
  if (alloc) {
    c->store->alloc = *alloc;
    c->store->custom_alloc = true;
  }
}

uint64_t storage_live_bytes(const snc_ctx* c) { return c->store ? c->store->live_bytes : 0; }
int ctx_device(const snc_ctx* c) { return c->device; }
bool ctx_finalized(const snc_ctx* c) { return c->finalized; }
bool ctx_sharded(const snc_ctx* c) { return c->sharded; }
}  // namespace snc

extern "C" {

snc_status snc_create(const snc_config* cfg, snc_ctx** out) {
  return snc::abi_guard([&]() -> snc_status {
    if (!cfg || !out) return fail(nullptr, SNC_ERR_INVALID_ARG, "snc_create: null argument");
    if (!(cfg->dt_ms > 0.0) || !std::isfinite(cfg->dt_ms)) return fail(nullptr, SNC_ERR_INVALID_ARG, "dt must be > 0");
    if (cfg->allocator && (!cfg->allocator->alloc || !cfg->allocator->free))
      return fail(nullptr, SNC_ERR_INVALID_ARG, "allocator without alloc/free");
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
      cudaGetLastError();
      return fail(nullptr, SNC_ERR_CUDA, "cannot select device %d", cfg->device);
    }
    std::unique_ptr<snc_ctx> owner(new (std::nothrow) snc_ctx());  // freed if anything below throws
    snc_ctx* c = owner.get();
    if (!c) return fail(nullptr, SNC_ERR_OOM, "out of host memory");
    c->cfg = *cfg;
    c->device = cfg->device;
    c->stream = static_cast<cudaStream_t>(cfg->stream);
    c->store = std::make_shared<Storage>();
    c->store->device = c->device;
    c->store->stream = c->stream;
    if (cfg->allocator) {
      c->store->alloc = *cfg->allocator;
      c->store->custom_alloc = true;
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (!c->store->init_host(64)) return fail(nullptr, SNC_ERR_CUDA, "event / pinned staging allocation failed");
    *out = owner.release();
    return SNC_OK;
  });
}

snc_status snc_destroy(snc_ctx* c) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return SNC_OK;
    cudaSetDevice(c->device);
    c->store.reset();  // the build's memory goes with its last member
    cudaGetLastError();
    delete c;
    return SNC_OK;
  });
}

snc_status snc_create_population(snc_ctx* c, uint32_t n, uint32_t* first_id) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    if (c->finalized) return fail(c, SNC_ERR_STATE, "create_population after finalize");
    if (c->n_nodes + n > 0xFFFFFFFFull) return fail(c, SNC_ERR_INVALID_ARG, "more than 2^32 - 1 nodes");
    if (first_id) *first_id = static_cast<uint32_t>(c->n_nodes);
    c->n_nodes += n;
    return SNC_OK;
  });
}

snc_status snc_connect(snc_ctx* c, snc_range src, snc_range tgt, const snc_conn_rule* rule,
                       const snc_syn_spec* syn, uint32_t* proj_id) {
  return snc_connect_arrays(c, src, tgt, rule, syn, nullptr, proj_id);
}

snc_status snc_connect_arrays(snc_ctx* c, snc_range src, snc_range tgt, const snc_conn_rule* rule,
                              const snc_syn_spec* syn, const snc_conn_arrays* arrays, uint32_t* proj_id) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    if (!rule || !syn) return fail(c, SNC_ERR_INVALID_ARG, "connect: null rule or synapse spec");
    if (c->finalized) return fail(c, SNC_ERR_STATE, "connect after finalize");
    Projection p;
    p.src = src;
    p.tgt = tgt;
    p.rule = *rule;
    p.syn = *syn;
    ConnectArrays ca;
    if (arrays) {
      ca.src_ids = arrays->src_ids;
      ca.tgt_ids = arrays->tgt_ids;
      ca.weights = arrays->weights;
      ca.delays_ms = arrays->delays_ms;
      ca.n_conn = arrays->n_conn;
    }
    const snc_status st = plan_projection(c, p, ca);
    if (st != SNC_OK) return st;
    if (proj_id) *proj_id = static_cast<uint32_t>(c->projs.size());
    c->projs.push_back(std::move(p));
    return SNC_OK;
  });
}

}  // extern "C"

namespace {

// Calibration of one build: a single context, or the members of a batch
// whose nodes are concatenated (member m's node i is global node
// node_base[m] + i).  Every draw is keyed by the member's seed and the
// projection's index within its member, so each member's result equals its
// own single build.  All device work runs on the first member's stream and
// memory; the members share the result storage.
snc_status finalize_build(snc_ctx* const* members, int n_members) {
  snc_ctx* c = members[0];
  SNC_CUDA(c, cudaSetDevice(c->device));
  Storage& S = *c->store;
  cudaStream_t st = c->stream;
  // Stage timers (not while the build is being captured into a graph).
  const auto mark = [&]() {
    if (!S.capturing) cudaEventRecord(S.ev[S.n_ev++], st);
  };
  if (!S.capturing) S.n_ev = 0;
  mark();
  S.seed_sites.clear();
  S.stage_total = 0;

  // The union of the members' projections.
  struct UnionProj {
    const Projection* p;
    const snc_ctx* owner;
    uint32_t base;
    uint32_t local;
    int member;
  };
  std::vector<uint64_t> node_base(static_cast<size_t>(n_members) + 1, 0);
  uint64_t max_nodes = 0;
  std::vector<UnionProj> ups;
  for (int m = 0; m < n_members; ++m) {
    node_base[m + 1] = node_base[m] + members[m]->n_nodes;
    max_nodes = std::max<uint64_t>(max_nodes, members[m]->n_nodes);
    for (size_t i = 0; i < members[m]->projs.size(); ++i)
      ups.push_back({&members[m]->projs[i], members[m], static_cast<uint32_t>(node_base[m]), static_cast<uint32_t>(i), m});
  }
  const uint64_t total_nodes = node_base[n_members];
  if (total_nodes > 0xFFFFFFFFull) return fail(c, SNC_ERR_UNSUPPORTED, "more than 2^32 - 1 nodes in one build");

  // Target shard.  A projection whose primary node is the target
  // (one_to_one, all_to_all, fixed_indegree, pairwise_bernoulli) keeps only
  // the targets inside the shard: its node range shrinks to them and its
  // draws stay keyed by the whole network's primary index (prim_shift), so it
  // generates exactly its share and nothing else.  fixed_outdegree and
  // fixed_total_number draw their targets, and a call with explicit arrays
  // has no contiguous target range, so these are generated whole and the
  // connections onto other targets are filtered out after generation.
  std::vector<Projection> shard_projs;
  std::vector<uint32_t> prim_shift(ups.size(), 0);
  bool shard_filter = false;
  if (n_members == 1 && c->sharded) {
    shard_projs.reserve(ups.size());
    for (size_t i = 0; i < ups.size(); ++i) {
      Projection q = *ups[i].p;
      const int kind = q.rule.kind;
      if (!q.has_arrays() && (kind == SNC_ONE_TO_ONE || kind == SNC_ALL_TO_ALL || kind == SNC_FIXED_INDEGREE ||
                              kind == SNC_PAIRWISE_BERNOULLI)) {
        const uint64_t f = c->shard_first, e = f + c->shard_n;
        const uint64_t t0 = q.tgt.first, t1 = t0 + q.tgt.n;
        const uint64_t lo = std::max(f, t0), hi = std::min(e, t1);
        const uint32_t shift = hi > lo ? static_cast<uint32_t>(lo - t0) : 0u;
        const uint32_t nt = hi > lo ? static_cast<uint32_t>(hi - lo) : 0u;
        q.tgt.first = static_cast<uint32_t>(t0) + shift;
        q.tgt.n = nt;
        if (kind == SNC_ONE_TO_ONE) {  // pair i = (s0 + i, t0 + i)
          q.src.first += shift;
          q.src.n = nt;
        }
        ArrayPlan lists;
        std::string why;
        if (check_connect_arrays(static_cast<uint32_t>(c->n_nodes), c->cfg.dt_ms, q.src, q.tgt, q.rule,
                                 ConnectArrays{}, &lists, &why) != SNC_OK)
          return fail(c, SNC_ERR_INVALID_ARG, "target shard: %s", why.c_str());
        q.count = lists.count;
        prim_shift[i] = shift;
      } else {
        shard_filter = true;
      }
      shard_projs.push_back(std::move(q));
    }
    for (size_t i = 0; i < ups.size(); ++i) ups[i].p = &shard_projs[i];
  }

  // A graph build cannot read the pairwise_bernoulli counts back (a replay
  // draws new ones): each such projection gets a capacity, and the positions
  // its draw leaves free hold a padding key above every real key (all ones,
  // with one more source bit so that no node has that source).
  const bool graph_build = S.mode != 0;
  bool graph_pad = false;
  for (const UnionProj& u : ups) graph_pad = graph_pad || (graph_build && u.p->rule.kind == SNC_PAIRWISE_BERNOULLI);

  // Key layout: network-local source | delay step (the target is in the value).
  uint32_t max_step = 1;
  for (const UnionProj& u : ups) max_step = std::max(max_step, u.p->max_step);
  c->layout.src_bits = std::max(1, bit_width(graph_pad ? max_nodes : (max_nodes > 0 ? max_nodes - 1 : 0)));
  c->layout.tgt_bits = std::max(1, bit_width(max_nodes > 0 ? max_nodes - 1 : 0));
  c->layout.delay_bits = std::max(1, bit_width(max_step));
  if (c->layout.total_bits() > 64)
    return fail(c, SNC_ERR_UNSUPPORTED, "packed key of %d bits exceeds 64", c->layout.total_bits());

  // Table blobs: thresholds (uint32) and their guides (uint16 x 257).
  const size_t np = ups.size();
  std::vector<uint64_t> cnt(np);
  std::vector<uint32_t> thr_blob;
  std::vector<uint16_t> guide_blob;
  std::vector<DevProj> dp(np);
  uint32_t max_delay_len = 0, max_binom_len = 0;
  auto add_table = [&](const std::vector<uint32_t>& t, uint32_t& off, uint32_t& goff) {
    off = static_cast<uint32_t>(thr_blob.size());
    thr_blob.insert(thr_blob.end(), t.begin(), t.end());
    goff = static_cast<uint32_t>(guide_blob.size());
    guide_blob.resize(guide_blob.size() + kDelayGuide);
    guide_table(t, guide_blob.data() + goff);
  };
  for (size_t i = 0; i < np; ++i) {
    const Projection& p = *ups[i].p;
    DevProj& d = dp[i];
    std::memset(&d, 0, sizeof d);
    cnt[i] = p.count;
    d.s0 = p.src.first + ups[i].base;
    d.ns = p.src.n;
    d.t0 = p.tgt.first + ups[i].base;
    d.nt = p.tgt.n;
    d.t_base = ups[i].base;
    d.prim_shift = prim_shift[i];
    d.rule = static_cast<uint32_t>(p.rule.kind);
    d.autapses = p.rule.allow_autapses ? 1u : 0u;
    d.multapses = p.rule.allow_multapses ? 1u : 0u;
    d.k0 = static_cast<uint32_t>(ups[i].owner->cfg.seed);
    d.k1 = static_cast<uint32_t>(ups[i].owner->cfg.seed >> 32) ^ ups[i].local;
    d.k = p.rule.k;
    division_magic(d.k, &d.k_mul, &d.k_sh1, &d.k_sh2);
    d.w_normal = (p.syn.weight.kind == SNC_DIST_NORMAL) ? 1u : 0u;
    d.w_mean = static_cast<float>(p.syn.weight.mean);
    d.w_std = static_cast<float>(p.syn.weight.std);
    d.d_const = p.d_const;
    d.d_table = p.d_table ? 1u : 0u;
    if (p.d_table) {
      d.d_base = p.d_base;
      d.d_len = static_cast<uint32_t>(p.d_thr.size());
      add_table(p.d_thr, d.d_off, d.d_goff);
      max_delay_len = std::max(max_delay_len, d.d_len);
    }
    if (p.rule.kind == SNC_PAIRWISE_BERNOULLI) {
      for (int s = 0; s < 2; ++s) {
        d.b_base[s] = static_cast<uint32_t>(p.b_base[s]);
        d.b_len[s] = static_cast<uint32_t>(p.b_thr[s].size());
        add_table(p.b_thr[s], d.b_off[s], d.b_goff[s]);
        max_binom_len = std::max(max_binom_len, d.b_len[s]);
      }
    }
  }
  if (thr_blob.empty()) thr_blob.push_back(0);
  if (guide_blob.empty()) guide_blob.resize(kDelayGuide, 0);

  // Explicit arrays (Sec. 2.1): node ids, weights and delay steps of every
  // call that gave them, plus what the kernels need to skip autapses on
  // lists: the position of each primary's node in the list it draws from
  // (per-primary rules), the kept pairs (one_to_one) and the dropped pairs
  // of each source row (all_to_all).
  std::vector<uint32_t> id_blob;
  std::vector<uint16_t> step_blob;
  std::vector<uint64_t> off_blob;
  bool any_lists = false;
  for (size_t i = 0; i < np; ++i) {
    const Projection& p = *ups[i].p;
    DevProj& d = dp[i];
    d.src_list = d.tgt_list = d.w_list = d.d_list = d.self_list = d.row_list = d.drop_list = kNoList;
    if (!p.has_arrays()) continue;
    any_lists = any_lists || p.has_lists();
    const auto append = [&](const std::vector<uint32_t>& v) {
      const uint64_t off = id_blob.size();
      id_blob.insert(id_blob.end(), v.begin(), v.end());
      return off;
    };
    if (p.src_list) d.src_list = append(p.src_ids);
    if (p.tgt_list) d.tgt_list = append(p.tgt_ids);
    if (!p.w_bits.empty()) d.w_list = append(p.w_bits);
    if (!p.d_steps.empty()) {
      d.d_list = step_blob.size();
      step_blob.insert(step_blob.end(), p.d_steps.begin(), p.d_steps.end());
    }
    if (!p.has_lists() || p.rule.allow_autapses) continue;
    const auto src_at = [&](uint32_t a) { return p.src_list ? p.src_ids[a] : p.src.first + a; };
    const auto tgt_at = [&](uint32_t b) { return p.tgt_list ? p.tgt_ids[b] : p.tgt.first + b; };
    const int kind = p.rule.kind;
    if (kind == SNC_FIXED_INDEGREE || kind == SNC_FIXED_OUTDEGREE || kind == SNC_PAIRWISE_BERNOULLI) {
      // The list drawn from holds distinct ids here (checked at Connect).
      const bool out = kind == SNC_FIXED_OUTDEGREE;
      const uint32_t n_other = out ? p.tgt.n : p.src.n, n_prim = out ? p.src.n : p.tgt.n;
      std::unordered_map<uint32_t, uint32_t> where;
      where.reserve(n_other * 2u + 1u);
      for (uint32_t k = 0; k < n_other; ++k) where.emplace(out ? tgt_at(k) : src_at(k), k);
      std::vector<uint32_t> self(n_prim, kNoPosition);
      for (uint32_t b = 0; b < n_prim; ++b) {
        const auto it = where.find(out ? src_at(b) : tgt_at(b));
        if (it != where.end()) self[b] = it->second;
      }
      d.self_list = append(self);
    } else if (kind == SNC_ONE_TO_ONE) {
      std::vector<uint32_t> kept;
      kept.reserve(p.src.n);
      for (uint32_t k = 0; k < p.src.n; ++k)
        if (src_at(k) != tgt_at(k)) kept.push_back(k);
      d.row_list = append(kept);
    } else if (kind == SNC_ALL_TO_ALL) {
      std::unordered_map<uint32_t, std::vector<uint32_t>> at;  // target id -> its positions, ascending
      for (uint32_t b = 0; b < p.tgt.n; ++b) at[tgt_at(b)].push_back(b);
      std::vector<uint32_t> drops;
      d.row_list = off_blob.size();
      uint64_t run = 0;
      for (uint32_t a = 0; a < p.src.n; ++a) {
        off_blob.push_back(run);
        const auto it = at.find(src_at(a));
        if (it == at.end()) continue;
        drops.insert(drops.end(), it->second.begin(), it->second.end());
        run += it->second.size();
      }
      off_blob.push_back(run);
      d.drop_list = append(drops);
    }
  }
  if (id_blob.empty()) id_blob.push_back(0);
  if (step_blob.empty()) step_blob.push_back(0);
  if (off_blob.empty()) off_blob.push_back(0);

  uint32_t* d_thr = static_cast<uint32_t*>(dev_alloc(c, thr_blob.size() * sizeof(uint32_t)));
  uint16_t* d_guide = static_cast<uint16_t*>(dev_alloc(c, guide_blob.size() * sizeof(uint16_t)));
  DevProj* d_proj = static_cast<DevProj*>(dev_alloc(c, std::max<size_t>(1, np) * sizeof(DevProj)));
  S.d_err = static_cast<uint32_t*>(dev_alloc(c, 8 * sizeof(uint64_t)));
  S.d_n_groups = static_cast<uint64_t*>(dev_alloc(c, sizeof(uint64_t)));
  uint32_t* d_ids = static_cast<uint32_t*>(dev_alloc(c, id_blob.size() * sizeof(uint32_t)));
  uint16_t* d_steps = static_cast<uint16_t*>(dev_alloc(c, step_blob.size() * sizeof(uint16_t)));
  uint64_t* d_offs = static_cast<uint64_t*>(dev_alloc(c, off_blob.size() * sizeof(uint64_t)));
  if (!d_thr || !d_guide || !d_proj || !S.d_err || !S.d_n_groups || !d_ids || !d_steps || !d_offs)
    return fail(c, SNC_ERR_OOM, "device allocation failed (tables)");
  SNC_CUDA(c, upload(c, d_thr, thr_blob.data(), thr_blob.size() * sizeof(uint32_t)));
  SNC_CUDA(c, upload(c, d_guide, guide_blob.data(), guide_blob.size() * sizeof(uint16_t)));
  SNC_CUDA(c, upload(c, d_ids, id_blob.data(), id_blob.size() * sizeof(uint32_t)));
  SNC_CUDA(c, upload(c, d_steps, step_blob.data(), step_blob.size() * sizeof(uint16_t)));
  SNC_CUDA(c, upload(c, d_offs, off_blob.data(), off_blob.size() * sizeof(uint64_t)));
  const ArrayBlobs arrays{d_ids, d_steps, d_offs};
  SNC_CUDA(c, cudaMemsetAsync(S.d_err, 0, 8 * sizeof(uint64_t), st));
  SNC_CUDA(c, cudaMemsetAsync(S.d_n_groups, 0, sizeof(uint64_t), st));

  // Count phase: per-target counts of every pairwise Bernoulli projection in
  // one launch, one scan, one read-back of the per-projection totals.
  uint64_t* d_prim_off = nullptr;
  uint32_t* d_bern_list = nullptr;    // graph_pad: the Bernoulli projections and their drawn totals
  uint64_t* d_bern_totals = nullptr;
  std::vector<uint32_t> bern;
  std::vector<uint64_t> bern_prefix(1, 0);
  for (size_t i = 0; i < np; ++i)
    if (ups[i].p->rule.kind == SNC_PAIRWISE_BERNOULLI) {
      dp[i].prim_off = bern_prefix.back();
      bern.push_back(static_cast<uint32_t>(i));
      bern_prefix.push_back(bern_prefix.back() + ups[i].p->tgt.n);
    }
  if (!bern.empty()) {
    const uint64_t n_targets = bern_prefix.back();
    const int nb = static_cast<int>(bern.size());
    // The count kernel reads these records: their staged copy is a seed site
    // too (a graph replay draws the counts with the new seeds).
    void* h_counted = nullptr;
    SNC_CUDA(c, upload(c, d_proj, dp.data(), np * sizeof(DevProj), &h_counted));
    for (size_t i = 0; i < np; ++i)
      S.seed_sites.push_back({static_cast<DevProj*>(h_counted) + i, ups[i].member, ups[i].local});
    d_prim_off = static_cast<uint64_t*>(dev_alloc(c, (n_targets + 1) * sizeof(uint64_t)));
    uint32_t* d_counts = static_cast<uint32_t*>(dev_alloc(c, (n_targets + 1) * sizeof(uint32_t)));
    uint64_t* d_scan_tmp = static_cast<uint64_t*>(dev_alloc(c, (scan_tmp_entries(n_targets) + 1) * sizeof(uint64_t)));
    uint32_t* d_blist = static_cast<uint32_t*>(dev_alloc(c, bern.size() * sizeof(uint32_t)));
    uint64_t* d_bprefix = static_cast<uint64_t*>(dev_alloc(c, bern_prefix.size() * sizeof(uint64_t)));
    uint64_t* d_totals = static_cast<uint64_t*>(dev_alloc(c, bern.size() * sizeof(uint64_t)));
    if (!d_prim_off || !d_counts || !d_scan_tmp || !d_blist || !d_bprefix || !d_totals)
      return fail(c, SNC_ERR_OOM, "device allocation failed (counts)");
    SNC_CUDA(c, upload(c, d_blist, bern.data(), bern.size() * sizeof(uint32_t)));
    SNC_CUDA(c, upload(c, d_bprefix, bern_prefix.data(), bern_prefix.size() * sizeof(uint64_t)));
    const unsigned cgrid =
        static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>((n_targets + 255) / 256, c->sms * 16ull)));
    bernoulli_count_kernel<<<cgrid, 256, 0, st>>>(d_proj, d_blist, d_bprefix, nb, d_thr, d_guide, arrays, d_counts);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
    SNC_CUDA(c, exclusive_scan_u32(d_counts, n_targets, d_prim_off, d_scan_tmp, st));
    c->stats.kernel_launches += 3;
    segment_totals_kernel<<<(nb + 255) / 256, 256, 0, st>>>(d_prim_off, d_bprefix, nb, d_totals);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
    if (graph_pad) {
      // Capacity: the total is a sum of Binomial counts over at most ns * nt
      // pairs; mean + 10 sd + 32 is exceeded with probability below e^-48
      // (Bernstein), and a replay that does exceed it reports an error.
      for (size_t bi = 0; bi < bern.size(); ++bi) {
        const Projection& p = *ups[bern[bi]].p;
        const double pairs = static_cast<double>(p.src.n) * static_cast<double>(p.tgt.n);
        const double q = std::min(1.0, std::max(0.0, p.rule.p));
        const double bound = std::ceil(pairs * q + g_graph_test.bernoulli_sd * std::sqrt(pairs * q * (1.0 - q)) +
                                       g_graph_test.bernoulli_slack);
        cnt[bern[bi]] = static_cast<uint64_t>(std::min(bound, pairs));
      }
      d_bern_list = d_blist;
      d_bern_totals = d_totals;
    } else {
      std::vector<uint64_t> totals(bern.size());
      SNC_CUDA(c, cudaMemcpyAsync(totals.data(), d_totals, bern.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
      c->stats.d2h_bytes += bern.size() * sizeof(uint64_t);
      SNC_CUDA(c, cudaStreamSynchronize(st));
      for (size_t bi = 0; bi < bern.size(); ++bi) cnt[bern[bi]] = totals[bi];
      dev_free(c, d_blist);
      dev_free(c, d_totals);
    }
    dev_free(c, d_counts);
    dev_free(c, d_scan_tmp);
    dev_free(c, d_bprefix);
  }
  mark();

  // Output offsets and generation chunks.  A batch's networks are segments
  // of the arrays, each starting on a multiple of 4 positions (the sort's
  // bulk copies need 16-byte aligned tiles); the few positions between
  // segments belong to no network.
  uint64_t off = 0;
  std::vector<DevProj> direct;
  std::vector<size_t> direct_src;  // union index of each direct projection
  uint64_t chunk = 0;
  std::vector<uint64_t> seg_begin(n_members, 0), seg_end(n_members, 0);
  int cur_m = -1;
  const auto open_member = [&](int m) {
    if (cur_m >= 0) seg_end[cur_m] = off;
    while (cur_m < m) {
      ++cur_m;
      if (n_members > 1) off = (off + 3) & ~3ull;
      seg_begin[cur_m] = off;
      seg_end[cur_m] = off;
    }
  };
  uint64_t n_conn = 0;
  for (size_t i = 0; i < np; ++i) {
    const Projection& p = *ups[i].p;
    DevProj& d = dp[i];
    if (ups[i].member != cur_m) open_member(ups[i].member);
    n_conn += cnt[i];
    d.count = cnt[i];
    d.out_off = off;
    off += cnt[i];
    if (cnt[i] == 0 || is_sampler(p) || is_total_redraw(p)) continue;
    if (p.rule.kind == SNC_ALL_TO_ALL) {
      d.chunks_per_row = (p.tgt.n + kChunk - 1) / kChunk;
      d.row_len = p.tgt.n;
      d.n_chunks = static_cast<uint64_t>(p.src.n) * d.chunks_per_row;
    } else {
      d.n_chunks = (cnt[i] + kChunk - 1) / kChunk;
    }
    d.chunk_begin = chunk;
    chunk += d.n_chunks;
    direct.push_back(d);
    direct_src.push_back(i);
  }
  open_member(n_members - 1);
  seg_end[n_members - 1] = off;
  const uint64_t n_total = off;  // positions, with the gaps between networks
  // The projection records carry the Philox keys: their staged copies are
  // where a graph replay puts new seeds.
  if (np > 0) {
    void* h = nullptr;
    SNC_CUDA(c, upload(c, d_proj, dp.data(), np * sizeof(DevProj), &h));
    for (size_t i = 0; i < np; ++i)
      S.seed_sites.push_back({static_cast<DevProj*>(h) + i, ups[i].member, ups[i].local});
  }
  DevProj* d_direct = nullptr;
  if (!direct.empty()) {
    d_direct = static_cast<DevProj*>(dev_alloc(c, direct.size() * sizeof(DevProj)));
    if (!d_direct) return fail(c, SNC_ERR_OOM, "device allocation failed (projections)");
    void* h = nullptr;
    SNC_CUDA(c, upload(c, d_direct, direct.data(), direct.size() * sizeof(DevProj), &h));
    for (size_t k = 0; k < direct.size(); ++k)
      S.seed_sites.push_back({static_cast<DevProj*>(h) + k, ups[direct_src[k]].member, ups[direct_src[k]].local});
  }

  // Buffers: generated keys/values, the sort's second buffer, outputs.
  uint64_t n = n_total;  // connections; a target shard keeps fewer after generation
  const bool segmented = n_members > 1;
  const bool sharded = !segmented && c->sharded;
  // A single network whose projections all generate source by source
  // (one_to_one, all_to_all, fixed_outdegree) is sorted per source by delay
  // step instead of by radix passes.
  // It pays when sources average at least 64 connections (one_to_one stays
  // on the radix sort, measured faster there) and at most two chunks, or up
  // to 32 chunks when there are at least 16 sources per resident block (a
  // source is one block's work, so fewer would leave blocks idle at the
  // end; 2 x 10,000 all_to_all rows of 20,000: 4.2 ms instead of 6.1 ms for
  // three radix passes).
  const uint64_t per_source = n / std::max<uint64_t>(1, total_nodes);
  const uint64_t long_rows_min_sources = 16ull * 4ull * static_cast<uint64_t>(c->sms);
  bool src_major = !segmented && !sharded && np > 0 && np <= static_cast<size_t>(kSrcMajorMaxProj) &&
                   c->layout.delay_bits <= kSrcMajorMaxDelayBits && per_source >= 64 &&
                   (per_source <= 2 * static_cast<uint64_t>(kSrcMajorChunk) ||
                    (per_source <= 32 * static_cast<uint64_t>(kSrcMajorChunk) && total_nodes >= long_rows_min_sources));
  for (size_t i = 0; i < np && src_major; ++i) src_major = source_major_rule(dp[i].rule);
  if (any_lists) src_major = false;  // sources of a list are not generated in node order
  if (segmented) {
    for (int m = 0; m < n_members; ++m)
      if (seg_end[m] - seg_begin[m] >= (1ull << 30))
        return fail(c, SNC_ERR_UNSUPPORTED, "batch: network %d has 2^30 connections or more; build it alone", m);
    // One launch per pass sorts every network as a segment: bulk-copy pass
    // kernel (8-9 bit digits), digit counts per segment from the keys.
    SortTuning tune = g_sort_tuning;
    tune.max_digit_bits = std::min(tune.max_digit_bits, 9);
    tune.group_tiles = 0;
    c->passes = plan_passes(c->layout.total_bits(), tune);
  } else {
    c->passes = plan_passes(c->layout.total_bits());
  }
  // Segment tables (device): begin, end, first tile of each network.
  const uint64_t seg_tile = static_cast<uint64_t>(onesweep_group(c->passes));
  std::vector<uint32_t> tile_begin(n_members + 1, 0);
  for (int m = 0; m < n_members; ++m)
    tile_begin[m + 1] = tile_begin[m] + static_cast<uint32_t>((seg_end[m] - seg_begin[m] + seg_tile - 1) / seg_tile);
  uint64_t* d_seg = static_cast<uint64_t*>(dev_alloc(c, 2 * static_cast<size_t>(n_members) * sizeof(uint64_t)));
  uint32_t* d_tile_begin = static_cast<uint32_t*>(dev_alloc(c, (static_cast<size_t>(n_members) + 1) * sizeof(uint32_t)));
  if (!d_seg || !d_tile_begin) return fail(c, SNC_ERR_OOM, "device allocation failed (segments)");
  SNC_CUDA(c, upload(c, d_seg, seg_begin.data(), n_members * sizeof(uint64_t)));
  SNC_CUDA(c, upload(c, d_seg + n_members, seg_end.data(), n_members * sizeof(uint64_t)));
  SNC_CUDA(c, upload(c, d_tile_begin, tile_begin.data(), (n_members + 1) * sizeof(uint32_t)));
  // graph_pad: the index sees each network's real positions only ([begin,
  // begin + drawn count)); the sort sorts whole segments, padding last.
  uint64_t* d_seg_real = d_seg;
  uint64_t* d_real_count = nullptr;
  if (graph_pad) {
    std::vector<uint64_t> fixed(n_members, 0);
    std::vector<uint32_t> bern_member;
    for (size_t i = 0; i < np; ++i)
      if (ups[i].p->rule.kind != SNC_PAIRWISE_BERNOULLI) fixed[ups[i].member] += cnt[i];
    for (uint32_t i : bern) bern_member.push_back(static_cast<uint32_t>(ups[i].member));
    d_seg_real = static_cast<uint64_t*>(dev_alloc(c, 2 * static_cast<size_t>(n_members) * sizeof(uint64_t)));
    d_real_count = static_cast<uint64_t*>(dev_alloc(c, static_cast<size_t>(n_members) * sizeof(uint64_t)));
    uint64_t* d_fixed = static_cast<uint64_t*>(dev_alloc(c, static_cast<size_t>(n_members) * sizeof(uint64_t)));
    uint32_t* d_bern_member = static_cast<uint32_t*>(dev_alloc(c, bern_member.size() * sizeof(uint32_t)));
    if (!d_seg_real || !d_real_count || !d_fixed || !d_bern_member)
      return fail(c, SNC_ERR_OOM, "device allocation failed (network counts)");
    SNC_CUDA(c, upload(c, d_seg_real, seg_begin.data(), n_members * sizeof(uint64_t)));
    SNC_CUDA(c, upload(c, d_fixed, fixed.data(), n_members * sizeof(uint64_t)));
    SNC_CUDA(c, upload(c, d_bern_member, bern_member.data(), bern_member.size() * sizeof(uint32_t)));
    member_real_kernel<<<(n_members + 255) / 256, 256, 0, st>>>(d_bern_totals, d_bern_member,
                                                                static_cast<int>(bern.size()), d_fixed, d_seg_real,
                                                                d_seg + n_members, n_members, d_seg_real + n_members,
                                                                d_real_count);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
  }
  const bool key32 = c->layout.key32();
  const size_t key_bytes = key32 ? sizeof(uint32_t) : sizeof(uint64_t);
  // COPASS block sort (Appendix A): the pairs are sorted in place in blocks,
  // so there is no second key/value buffer, only two blocks of working
  // memory; the sorted pairs are then unpacked in place.
  const uint64_t block = c->block_sort;
  const bool block_sorted = block > 0 && !segmented && !sharded;
  if (block_sorted && (n + block - 1) / block > static_cast<uint64_t>(kCopassMaxRuns))
    return fail(c, SNC_ERR_INVALID_ARG, "block sort: %llu connections need more than %d blocks of %llu",
                static_cast<unsigned long long>(n), kCopassMaxRuns, static_cast<unsigned long long>(block));
  if (block_sorted) src_major = false;
  void* keys_a = dev_alloc(c, n * key_bytes);
  uint64_t* vals_a = static_cast<uint64_t*>(dev_alloc(c, n * sizeof(uint64_t)));
  void* keys_b = block_sorted ? nullptr : dev_alloc(c, n * key_bytes);
  uint64_t* vals_b = block_sorted ? nullptr : static_cast<uint64_t*>(dev_alloc(c, n * sizeof(uint64_t)));
  const uint64_t n_seg_tiles = tile_begin[n_members];
  void* sort_scratch = dev_alloc(c, block_sorted ? copass_scratch_bytes(block, static_cast<int>(key_bytes), 8, c->passes)
                                    : segmented  ? sort_scratch_bytes(n, c->passes, n_seg_tiles, n_members)
                                                 : sort_scratch_bytes(n, c->passes));
  if (!keys_a || !vals_a || (!block_sorted && (!keys_b || !vals_b)) || !sort_scratch)
    return fail(c, SNC_ERR_OOM, "device allocation failed (%llu connections)", static_cast<unsigned long long>(n));

  // The generation kernels count the sort's digits as they write the keys
  // (a segmented sort counts per segment itself).
  const SortScratch sort_lay = segmented ? sort_scratch_layout(sort_scratch, n, c->passes, n_seg_tiles, n_members)
                                         : sort_scratch_layout(sort_scratch, n, c->passes);
  // (A target shard that filters counts the digits of the kept connections
  // in the sort.)
  const bool gen_counts = !segmented && !src_major && !shard_filter && !block_sorted;
  if (gen_counts)
    SNC_CUDA(c, cudaMemsetAsync(sort_lay.hist, 0,
                                static_cast<size_t>(kMaxPasses) * kMaxRadix * sizeof(unsigned long long), st));
  const HistPlan hplan = hist_plan(c->passes, gen_counts ? sort_lay.hist : nullptr);
  const size_t hist_bytes = hist_smem_bytes(hplan);

  // Generation.
  GenArgs g{};
  g.projs = d_direct;
  g.n_proj = static_cast<int>(direct.size());
  g.total_chunks = chunk;
  g.thr_blob = d_thr;
  g.guide_blob = d_guide;
  g.max_delay_len = max_delay_len;
  g.layout = c->layout;
  g.keys = keys_a;
  g.vals = vals_a;
  g.key32 = key32 ? 1 : 0;
  g.cap = n;
  g.err = S.d_err;
  g.hist = hplan;
  g.arr = arrays;
  const size_t table_smem =
      hist_bytes + static_cast<size_t>(max_delay_len) * sizeof(uint32_t) + kDelayGuide * sizeof(uint16_t) + 16;
  if (chunk > 0) {
    // Set on every launch: the attribute is per function and device, and
    // builds may run on several threads and devices.
    SNC_CUDA(c, cudaFuncSetAttribute(gen_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    const uint64_t grid = std::min<uint64_t>(chunk, static_cast<uint64_t>(c->sms) * g_gen_blocks_per_sm);
    gen_direct_kernel<<<static_cast<unsigned>(grid), kGenThreads, table_smem, st>>>(g);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
  }
  // Samplers (in/out-degree without multapses, Bernoulli subsets): one launch.
  {
    std::vector<uint32_t> slist;
    std::vector<uint64_t> sprefix(1, 0);
    uint32_t max_other = 1, max_len = 0;
    for (size_t i = 0; i < np; ++i) {
      const Projection& p = *ups[i].p;
      if (cnt[i] == 0 || !is_sampler(p)) continue;
      const bool out_deg = p.rule.kind == SNC_FIXED_OUTDEGREE;
      slist.push_back(static_cast<uint32_t>(i));
      sprefix.push_back(sprefix.back() + (out_deg ? p.src.n : p.tgt.n));
      max_other = std::max<uint32_t>(max_other, out_deg ? p.tgt.n : p.src.n);
      max_len = std::max(max_len, dp[i].d_len);
    }
    if (!slist.empty()) {
      uint32_t* d_slist = static_cast<uint32_t*>(dev_alloc(c, slist.size() * sizeof(uint32_t)));
      uint64_t* d_sprefix = static_cast<uint64_t*>(dev_alloc(c, sprefix.size() * sizeof(uint64_t)));
      if (!d_slist || !d_sprefix) return fail(c, SNC_ERR_OOM, "device allocation failed (sampler list)");
      SNC_CUDA(c, upload(c, d_slist, slist.data(), slist.size() * sizeof(uint32_t)));
      SNC_CUDA(c, upload(c, d_sprefix, sprefix.data(), sprefix.size() * sizeof(uint64_t)));
      SamplerArgs s{};
      s.gen = g;
      s.projs = d_proj;
      s.list = d_slist;
      s.prim_prefix = d_sprefix;
      s.n_list = static_cast<int>(slist.size());
      s.thr_blob = d_thr;
      s.guide_blob = d_guide;
      s.max_delay_len = max_len;
      // Per-warp areas in whole 16-byte units (the bitmap is cleared with
      // 16-byte stores).
      s.table_words = (max_len + (kDelayGuide + 1) / 2 + 1 + 3u) & ~3u;
      s.bitmap_words = ((max_other + 31u) / 32u + 3u) & ~3u;
      s.prim_offsets = d_prim_off;
      s.err = S.d_err;
      const size_t per_warp = static_cast<size_t>(s.bitmap_words + s.table_words) * sizeof(uint32_t);
      const int warps = static_cast<int>(std::min<size_t>(8, (kSamplerSmem - hist_bytes - 16) / per_warp));
      if (warps < 1) return fail(c, SNC_ERR_UNSUPPORTED, "sampler bitmap does not fit shared memory");
      const size_t smem = hist_bytes + static_cast<size_t>(warps) * per_warp + 16;
      // Set on every launch: the attribute is per function and device, and
      // builds may run on several threads and devices.
      SNC_CUDA(c, cudaFuncSetAttribute(sampler_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSamplerSmem)));
      const uint64_t want_blocks = (sprefix.back() + warps - 1) / warps;
      const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(want_blocks, static_cast<uint64_t>(c->sms) * 16));
      sampler_kernel<<<static_cast<unsigned>(grid), 32 * warps, smem, st>>>(s);
      ++c->stats.kernel_launches;
      SNC_CUDA(c, cudaGetLastError());
      dev_free(c, d_slist);
      dev_free(c, d_sprefix);
    }
  }
  if (graph_pad && !bern.empty()) {
    const uint64_t pad_key = (c->layout.total_bits() >= 64) ? ~0ull : ((1ull << c->layout.total_bits()) - 1ull);
    const dim3 pgrid(static_cast<unsigned>(std::max<uint64_t>(1, static_cast<uint64_t>(c->sms))),
                     static_cast<unsigned>(std::min<size_t>(bern.size(), 65535)));
    bern_pad_kernel<<<pgrid, 256, 0, st>>>(g, d_proj, d_bern_list, static_cast<int>(bern.size()), d_bern_totals,
                                           pad_key);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
  }
  // fixed_total_number with redraws: all such projections together, one
  // read-back of the pending count per round (a graph build: a fixed number
  // of rounds with the count on the device).
  {
    std::vector<RedrawProj> rps;
    uint64_t n_slots = 0, n_table = 0, n_chunks_r = 0;
    bool any_vals = false;
    uint32_t max_len = 0;
    for (size_t i = 0; i < np; ++i) {
      const Projection& p = *ups[i].p;
      if (cnt[i] == 0 || !is_total_redraw(p)) continue;
      const uint64_t N = cnt[i];
      RedrawProj r{};
      r.proj = static_cast<uint32_t>(i);
      r.slot_base = n_slots;
      r.chunk_base = n_chunks_r;
      r.table_off = n_table;
      r.slot_bits = std::max(1, bit_width(N - 1));
      r.t_bits = bit_width(p.tgt.n > 0 ? p.tgt.n - 1u : 0u);
      if (!p.rule.allow_multapses) {
        uint64_t cap = 1;
        while (cap < 2 * N + 64) cap <<= 1;
        // One word per entry when (source, target, slot) fit in 63 bits.
        const int s_bits = bit_width(p.src.n > 0 ? p.src.n - 1u : 0u);
        r.packed = (s_bits + r.t_bits + r.slot_bits + 1 <= 63) ? 1 : 0;
        any_vals = any_vals || !r.packed;
        r.table_mask = cap - 1;
        n_table += cap;
      }
      n_slots += N;
      n_chunks_r += (N + kChunk - 1) / kChunk;
      max_len = std::max(max_len, dp[i].d_len);
      rps.push_back(r);
    }
    // Claims go to buckets of about kBucketMean pairs, each settled in a
    // shared-memory table, when every pair table would be packed; else to
    // one global hash table per projection.
    bool bucketed = !rps.empty();
    uint64_t n_buckets = 0;
    for (RedrawProj& r : rps) {
      const Projection& p = *ups[r.proj].p;
      if (!p.rule.allow_multapses && !r.packed) bucketed = false;
    }
    uint64_t n_super = 0, sup_entries = 0, n_split_units = 0;
    uint32_t max_super = 1;
    if (bucketed) {
      for (RedrawProj& r : rps) {
        const Projection& p = *ups[r.proj].p;
        if (p.rule.allow_multapses) continue;
        const uint64_t want = (cnt[r.proj] + kBucketMean - 1) / kBucketMean;
        int bits = 0;
        while ((1ull << bits) < want) ++bits;
        if (bits - kSplitBits > kMaxSuperBits) bucketed = false;  // above 2^31 slots: global tables
      }
    }
    if (bucketed) {
      n_table = 0;
      for (RedrawProj& r : rps) {
        const Projection& p = *ups[r.proj].p;
        r.bucket_base = n_buckets;
        r.super_base = n_super;
        r.super_off = sup_entries;
        r.split_base = n_split_units;
        if (p.rule.allow_multapses) continue;
        const uint64_t N = cnt[r.proj];
        const uint64_t want = (N + kBucketMean - 1) / kBucketMean;
        int bits = 0;
        while ((1ull << bits) < want) ++bits;
        r.bucket_bits = bits;
        r.n_buckets = 1ull << bits;
        n_buckets += r.n_buckets;
        // Super-buckets of up to 2^kSplitBits buckets, kSuperLanes regions
        // each (one per residue of the chunk index).  A region holds the mean
        // share of its lane's slots plus 16 standard deviations of the
        // binomial count.
        r.super_bits = bits > kSplitBits ? bits - kSplitBits : 0;
        const uint64_t n_sup = 1ull << r.super_bits;
        const uint64_t chunks = (N + kChunk - 1) / kChunk;
        const uint64_t lane_slots = std::min<uint64_t>(N, (chunks + kSuperLanes - 1) / kSuperLanes * kChunk);
        const double mean = static_cast<double>(lane_slots) / static_cast<double>(n_sup);
        r.super_cap = std::min<uint64_t>(lane_slots, static_cast<uint64_t>(mean + 16.0 * std::sqrt(mean)) + 64);
        r.split_base = n_split_units;
        r.split_per_super = std::max<uint64_t>(1, (r.super_cap + kSplitUnit - 1) / kSplitUnit);
        n_split_units += n_sup * kSuperLanes * r.split_per_super;
        n_super += n_sup;
        sup_entries += n_sup * kSuperLanes * r.super_cap;
        max_super = std::max<uint32_t>(max_super, static_cast<uint32_t>(n_sup));
      }
    }
    if (!rps.empty()) {
      RedrawArgs a{};
      a.projs = d_proj;
      a.arr = arrays;
      a.n = static_cast<int>(rps.size());
      a.n_slots = n_slots;
      a.err = S.d_err;
      RedrawProj* d_rp = static_cast<RedrawProj*>(dev_alloc(c, rps.size() * sizeof(RedrawProj)));
      a.pairs = static_cast<uint64_t*>(dev_alloc(c, n_slots * sizeof(uint64_t)));
      a.lost = bucketed ? nullptr : static_cast<uint8_t*>(dev_alloc(c, n_slots));
      uint64_t* pend_a = static_cast<uint64_t*>(dev_alloc(c, n_slots * sizeof(uint64_t)));
      uint64_t* pend_b = static_cast<uint64_t*>(dev_alloc(c, n_slots * sizeof(uint64_t)));
      // Two pending counters: a graph build keeps each round's count on the
      // device (the round reads one, fills the other).
      a.n_next = static_cast<unsigned long long*>(dev_alloc(c, 2 * sizeof(unsigned long long)));
      if (!d_rp || !a.pairs || (!bucketed && !a.lost) || !pend_a || !pend_b || !a.n_next)
        return fail(c, SNC_ERR_OOM, "device allocation failed (redraw lists)");
      if (n_table > 0) {
        a.table_keys = static_cast<uint64_t*>(dev_alloc(c, n_table * sizeof(uint64_t)));
        if (!a.table_keys) return fail(c, SNC_ERR_OOM, "device allocation failed (pair table)");
        SNC_CUDA(c, cudaMemsetAsync(a.table_keys, 0xFF, n_table * sizeof(uint64_t), st));
        if (any_vals) {
          a.table_vals = static_cast<uint64_t*>(dev_alloc(c, n_table * sizeof(uint64_t)));
          if (!a.table_vals) return fail(c, SNC_ERR_OOM, "device allocation failed (pair table)");
          SNC_CUDA(c, cudaMemsetAsync(a.table_vals, 0xFF, n_table * sizeof(uint64_t), st));
        }
      }
      if (bucketed && n_buckets > 0) {
        a.bucketed = 1;
        a.cap = kBucketCap;
        a.n_buckets = n_buckets;
        a.ent = static_cast<uint64_t*>(dev_alloc(c, n_buckets * kBucketCap * sizeof(uint64_t)));
        a.fill = static_cast<uint32_t*>(dev_alloc(c, n_buckets * sizeof(uint32_t)));
        if (!a.ent || !a.fill) return fail(c, SNC_ERR_OOM, "device allocation failed (claim buckets)");
        SNC_CUDA(c, cudaMemsetAsync(a.fill, 0, n_buckets * sizeof(uint32_t), st));
        a.n_super = n_super;
        a.max_super = max_super;
        a.n_split_units = n_split_units;
        const uint64_t sfill_words = n_super * kSuperLanes * kFillStride;
        a.sup = static_cast<uint64_t*>(dev_alloc(c, sup_entries * sizeof(uint64_t)));
        a.sfill = static_cast<uint32_t*>(dev_alloc(c, sfill_words * sizeof(uint32_t)));
        if (!a.sup || !a.sfill)
          return fail(c, SNC_ERR_OOM, "device allocation failed (claim super-buckets)");
        SNC_CUDA(c, cudaMemsetAsync(a.sfill, 0, sfill_words * sizeof(uint32_t), st));
      } else if (bucketed) {
        a.bucketed = 1;  // autapse redraws only: no pair tables
      }
      if (a.bucketed) {
        const uint64_t words = (n_slots + 31) / 32;
        a.moved = static_cast<uint32_t*>(dev_alloc(c, words * sizeof(uint32_t)));
        if (!a.moved) return fail(c, SNC_ERR_OOM, "device allocation failed (redraw marks)");
        SNC_CUDA(c, cudaMemsetAsync(a.moved, 0, words * sizeof(uint32_t), st));
      }
      a.rp = d_rp;
      SNC_CUDA(c, upload(c, d_rp, rps.data(), rps.size() * sizeof(RedrawProj)));
      if (a.lost) SNC_CUDA(c, cudaMemsetAsync(a.lost, 0, n_slots, st));
      SNC_CUDA(c, cudaMemsetAsync(a.n_next, 0, sizeof(unsigned long long), st));
      a.next_pending = pend_a;
      const auto grid_for = [&](uint64_t items) {
        return static_cast<unsigned>(
            std::max<uint64_t>(1, std::min<uint64_t>((items + 255) / 256, static_cast<uint64_t>(c->sms) * 16)));
      };
      const unsigned bucket_grid = static_cast<unsigned>(
          std::max<uint64_t>(1, std::min<uint64_t>(n_buckets, static_cast<uint64_t>(c->sms) * 6)));
      GenArgs ge = g;
      ge.max_delay_len = max_len;
      const unsigned eg = static_cast<unsigned>(
          std::min<uint64_t>(n_chunks_r, static_cast<uint64_t>(c->sms) * g_gen_blocks_per_sm));
      if (a.bucketed) {
        // Round 0 writes every slot's connection; the slots that redraw are
        // rewritten after the last round.
        const size_t dsm = redraw_draw_smem(ge, a);
        SNC_CUDA(c, cudaFuncSetAttribute(redraw_draw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(dsm)));
        redraw_draw_kernel<<<eg, kGenThreads, dsm, st>>>(ge, a, n_chunks_r);
      } else {
        redraw_round0_kernel<<<grid_for(n_slots), 256, 0, st>>>(a);
      }
      ++c->stats.kernel_launches;
      if (a.bucketed) {
        // Round-0 losers go straight to the pending list.
        if (n_buckets > 0) {
          const unsigned split_grid = static_cast<unsigned>(
              std::max<uint64_t>(1, std::min<uint64_t>(n_split_units, static_cast<uint64_t>(c->sms) * 2)));
          const size_t ssm = redraw_split_smem();
          SNC_CUDA(c, cudaFuncSetAttribute(redraw_bucket_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(ssm)));
          redraw_bucket_split_kernel<<<split_grid, kSplitThreads, ssm, st>>>(a);
          redraw_bucket0_kernel<<<bucket_grid, 256, 0, st>>>(a);
          c->stats.kernel_launches += 2;
        }
      } else {
        redraw_collect_kernel<<<grid_for(n_slots), 256, 0, st>>>(a);
        ++c->stats.kernel_launches;
      }
      SNC_CUDA(c, cudaGetLastError());
      uint64_t* pending = pend_a;
      uint64_t* next = pend_b;
      // A pending slot redraws until its pair is free: it fails a round with
      // probability at most q (the share of pairs already taken, or of pairs
      // joining a node to itself), so after R rounds about n_slots * q^R
      // remain.  A graph build records R rounds chosen for 10^-12 (a replay
      // with slots still pending after the last one reports TIMEOUT); a plain
      // build runs R rounds chosen for 10^-15 the same way when R <= 64, so
      // that finalize does not wait on the host for the pending counts, and
      // otherwise reads the count back after every round.
      double q = 0.0;
      for (const RedrawProj& r : rps) {
        const Projection& p = *ups[r.proj].p;
        const double pairs = std::max(1.0, static_cast<double>(p.src.n) * static_cast<double>(p.tgt.n));
        double f = p.rule.allow_autapses ? 0.0 : 1.0 / std::max(1u, std::min(p.src.n, p.tgt.n));
        if (!p.rule.allow_multapses) f += static_cast<double>(cnt[r.proj]) / pairs;
        q = std::max(q, std::min(f, 1.0));
      }
      const double decades = graph_build ? 12.0 : 15.0;
      const double need = (std::log(static_cast<double>(n_slots) + 1.0) + decades * std::log(10.0)) /
                          std::max(1e-9, -std::log(std::max(q, 1e-300)));
      const bool device_rounds = graph_build || (q < 1.0 && need <= 64.0);
      if (device_rounds) {
        if (q >= 1.0 || need > 512.0)
          return fail(c, SNC_ERR_UNSUPPORTED,
                      "graph build: fixed_total_number without multapses at this density needs host-driven rounds");
        const uint32_t rounds = g_graph_test.redraw_rounds ? g_graph_test.redraw_rounds
                                                           : static_cast<uint32_t>(std::max(2.0, std::ceil(need)));
        unsigned long long* cur_n = a.n_next;  // round 0 filled pend_a and this counter
        unsigned long long* nxt_n = a.n_next + 1;
        for (uint32_t round = 1; round <= rounds; ++round) {
          RedrawArgs ar = a;
          ar.next_pending = next;
          ar.n_next = nxt_n;
          SNC_CUDA(c, cudaMemsetAsync(nxt_n, 0, sizeof(unsigned long long), st));
          redraw_claim_kernel<<<grid_for(n_slots), 256, 0, st>>>(ar, pending, 0, round, cur_n);
          redraw_resolve_kernel<<<grid_for(n_slots), 256, 0, st>>>(ar, pending, 0, cur_n);
          c->stats.kernel_launches += 2;
          SNC_CUDA(c, cudaGetLastError());
          std::swap(pending, next);
          std::swap(cur_n, nxt_n);
        }
        redraw_rounds_check_kernel<<<1, 32, 0, st>>>(cur_n, S.d_err);
        ++c->stats.kernel_launches;
        SNC_CUDA(c, cudaGetLastError());
      }
      for (uint32_t round = 1; !device_rounds; ++round) {
        SNC_CUDA(c, cudaMemcpyAsync(S.h_pinned, a.n_next, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        c->stats.d2h_bytes += sizeof(uint64_t);
        SNC_CUDA(c, cudaStreamSynchronize(st));
        const uint64_t n_pend = S.h_pinned[0];
        if (n_pend == 0) break;
        if (round > 0xFFFFFFu) return fail(c, SNC_ERR_TIMEOUT, "fixed_total_number: redraw rounds exhausted");
        if (n_pend > n_slots) return fail(c, SNC_ERR_CUDA, "fixed_total_number: pending list overflow (internal error)");
        a.next_pending = next;
        SNC_CUDA(c, cudaMemsetAsync(a.n_next, 0, sizeof(unsigned long long), st));
        redraw_claim_kernel<<<grid_for(n_pend), 256, 0, st>>>(a, pending, n_pend, round, nullptr);
        redraw_resolve_kernel<<<grid_for(n_pend), 256, 0, st>>>(a, pending, n_pend, nullptr);
        c->stats.kernel_launches += 2;
        SNC_CUDA(c, cudaGetLastError());
        std::swap(pending, next);
      }
      if (a.bucketed) {
        const uint64_t words = (n_slots + 31) / 32;
        const size_t psm = hist_bytes > 0 ? hist_bytes : 16;
        redraw_patch_kernel<<<grid_for(words), 256, psm, st>>>(ge, a);
      } else {
        const size_t tsm =
            hist_bytes + static_cast<size_t>(max_len) * sizeof(uint32_t) + kDelayGuide * sizeof(uint16_t) + 16;
        // Set on every launch: the attribute is per function and device, and
        // builds may run on several threads and devices.
        SNC_CUDA(c, cudaFuncSetAttribute(total_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        total_emit_kernel<<<eg, kGenThreads, tsm, st>>>(ge, a, n_chunks_r);
      }
      ++c->stats.kernel_launches;
      SNC_CUDA(c, cudaGetLastError());
      dev_free(c, d_rp);
      dev_free(c, a.pairs);
      dev_free(c, a.lost);
      dev_free(c, pend_a);
      dev_free(c, pend_b);
      dev_free(c, a.n_next);
      dev_free(c, a.table_keys);
      dev_free(c, a.table_vals);
      dev_free(c, a.ent);
      dev_free(c, a.fill);
      dev_free(c, a.moved);
      dev_free(c, a.sup);
      dev_free(c, a.sfill);
    }
  }
  mark();
  // The array blobs are read by generation only.
  dev_free(c, d_ids);
  dev_free(c, d_steps);
  dev_free(c, d_offs);

  // Target shard with fixed_outdegree or fixed_total_number projections:
  // keep the connections whose target is in the shard, in generation order
  // (so the stable sort below gives the full network's order restricted to
  // them), compacted into the second buffer pair.
  if (shard_filter && n > 0) {
    uint32_t* flags = static_cast<uint32_t*>(dev_alloc(c, (n + 1) * sizeof(uint32_t)));
    uint64_t* offs = static_cast<uint64_t*>(dev_alloc(c, (n + 1) * sizeof(uint64_t)));
    uint64_t* tmp = static_cast<uint64_t*>(dev_alloc(c, (scan_tmp_entries(n) + 1) * sizeof(uint64_t)));
    if (!flags || !offs || !tmp) return fail(c, SNC_ERR_OOM, "device allocation failed (target shard)");
    const unsigned fg = static_cast<unsigned>(
        std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, static_cast<uint64_t>(c->sms) * 16)));
    shard_flag_kernel<<<fg, 256, 0, st>>>(vals_a, n, c->shard_first, c->shard_n, flags);
    SNC_CUDA(c, exclusive_scan_u32(flags, n, offs, tmp, st));
    shard_compact_kernel<<<fg, 256, 0, st>>>(keys_a, vals_a, key32 ? 1 : 0, n, offs, c->shard_first, c->shard_n,
                                             keys_b, vals_b);
    SNC_CUDA(c, cudaGetLastError());
    c->stats.kernel_launches += 5;
    SNC_CUDA(c, cudaMemcpyAsync(S.h_pinned, offs + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    c->stats.d2h_bytes += sizeof(uint64_t);
    SNC_CUDA(c, cudaStreamSynchronize(st));
    n = S.h_pinned[0];
    seg_end[0] = seg_begin[0] + n;
    SNC_CUDA(c, upload(c, d_seg + n_members, seg_end.data(), sizeof(uint64_t)));  // the index reads the end
    std::swap(keys_a, keys_b);
    std::swap(vals_a, vals_b);
    dev_free(c, flags);
    dev_free(c, offs);
    dev_free(c, tmp);
  }

  // Stable sort by (source, delay): equal keys keep generation order.  The
  // passes ping-pong between the two buffers; the result lands in
  // (keys_b, vals_b) for an odd number of passes and back in (keys_a,
  // vals_a) for an even number.
  const bool odd = !block_sorted && (src_major || (c->passes.n_passes & 1) != 0);
  void* keys_res = odd ? keys_b : keys_a;
  uint64_t* vals_res = odd ? vals_b : vals_a;
  void* keys_oth = odd ? keys_a : keys_b;
  uint64_t* vals_oth = odd ? vals_a : vals_b;
  // The last pass writes target and weight over the result value buffer
  // (which it no longer needs) and the delays into their own array.
  uint16_t* u_delay = static_cast<uint16_t*>(dev_alloc(c, n * sizeof(uint16_t)));
  if (!u_delay) return fail(c, SNC_ERR_OOM, "device allocation failed (delays)");
  SortUnpack unpack{};
  unpack.target = reinterpret_cast<uint32_t*>(vals_res);
  unpack.weight = reinterpret_cast<uint32_t*>(vals_res) + n;
  unpack.delay = u_delay;
  unpack.delay_mask = (1u << c->layout.delay_bits) - 1u;
  bool fused = false;
  SortSegments segs{};
  segs.n_seg = n_members;
  segs.begin = d_seg;
  segs.end = d_seg + n_members;
  segs.tile_begin = d_tile_begin;
  segs.n_tiles = n_seg_tiles;
  for (int m = 0; m < n_members; ++m) segs.max_len = std::max(segs.max_len, seg_end[m] - seg_begin[m]);
  const SortSegments* seg_arg = segmented ? &segs : nullptr;
  if (block_sorted) {
    // Sorted in place (keys_a, vals_a); one timed sort stage.
    mark();
    if (key32)
      SNC_CUDA(c, copass_sort_run(static_cast<uint32_t*>(keys_a), vals_a, n, block, c->passes, sort_scratch, S.d_err, st));
    else
      SNC_CUDA(c, copass_sort_run(static_cast<uint64_t*>(keys_a), vals_a, n, block, c->passes, sort_scratch, S.d_err, st));
    mark();
    c->stats.kernel_launches += 2 * ((n + block - 1) / block) * (static_cast<uint64_t>(c->passes.n_passes) + 4);
    c->stats.n_passes = c->passes.n_passes;
    c->stats.source_major = 0;
    c->sort_stages = 1;
  } else if (src_major) {
    const uint64_t nn = total_nodes;
    uint32_t* sm_counts = static_cast<uint32_t*>(dev_alloc(c, (nn + 1) * sizeof(uint32_t)));
    uint64_t* sm_base = static_cast<uint64_t*>(dev_alloc(c, (nn + 1) * sizeof(uint64_t)));
    uint64_t* sm_tmp = static_cast<uint64_t*>(dev_alloc(c, (scan_tmp_entries(nn) + 1) * sizeof(uint64_t)));
    uint32_t* sm_long = static_cast<uint32_t*>(dev_alloc(c, (nn + 1) * sizeof(uint32_t)));
    if (!sm_counts || !sm_base || !sm_tmp || !sm_long)
      return fail(c, SNC_ERR_OOM, "device allocation failed (source offsets)");
    SNC_CUDA(c, cudaMemsetAsync(sm_long + nn, 0, sizeof(uint32_t), st));
    SrcMajorArgs sa{};
    sa.projs = d_proj;
    sa.n_proj = static_cast<int>(np);
    sa.n_nodes = static_cast<uint32_t>(nn);
    sa.counts = sm_counts;
    sa.row_base = sm_base;
    sa.keys_in = keys_a;
    sa.vals_in = vals_a;
    sa.key32 = key32 ? 1 : 0;
    sa.delay_bits = c->layout.delay_bits;
    sa.keys_out = keys_res;
    sa.target = unpack.target;
    sa.weight = unpack.weight;
    sa.delay = unpack.delay;
    sa.n = n;
    sa.err = S.d_err;
    sa.long_list = sm_long;
    sa.n_long = sm_long + nn;
    const unsigned cg = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>((nn + 255) / 256, c->sms * 8ull)));
    src_major_count_kernel<<<cg, 256, 0, st>>>(sa);
    SNC_CUDA(c, exclusive_scan_u32(sm_counts, nn, sm_base, sm_tmp, st));
    mark();
    // Short sources one warp each, the others one block each.
    const uint64_t warps = kSrcMajorThreads / 32;
    const unsigned wg = static_cast<unsigned>(
        std::max<uint64_t>(1, std::min<uint64_t>((nn + warps - 1) / warps, c->sms * 4ull)));
    src_major_small_kernel<<<wg, kSrcMajorThreads, 0, st>>>(sa);
    const unsigned bg = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(nn, c->sms * 4ull)));
    src_major_sort_kernel<<<bg, kSrcMajorThreads, 0, st>>>(sa);
    SNC_CUDA(c, cudaGetLastError());
    mark();
    fused = true;
    c->stats.kernel_launches += 6;  // count, three scan kernels, two sorts
    c->stats.n_passes = 0;
    c->stats.source_major = 1;
    c->sort_stages = 1;
    dev_free(c, sm_counts);
    dev_free(c, sm_base);
    dev_free(c, sm_tmp);
    dev_free(c, sm_long);
  } else if (key32)
    SNC_CUDA(c, radix_sort_run(static_cast<const uint32_t*>(keys_a), vals_a, static_cast<uint32_t*>(keys_res), vals_res,
                               static_cast<uint32_t*>(keys_oth), vals_oth, n, c->passes, sort_scratch, S.d_err, st,
                               S.capturing ? nullptr : S.ev + S.n_ev, /*hist_ready=*/!shard_filter, &unpack, &fused, seg_arg));
  else
    SNC_CUDA(c, radix_sort_run(static_cast<const uint64_t*>(keys_a), vals_a, static_cast<uint64_t*>(keys_res), vals_res,
                               static_cast<uint64_t*>(keys_oth), vals_oth, n, c->passes, sort_scratch, S.d_err, st,
                               S.capturing ? nullptr : S.ev + S.n_ev, /*hist_ready=*/!shard_filter, &unpack, &fused, seg_arg));
  if (!src_major && !block_sorted) {
    if (!S.capturing) S.n_ev += c->passes.n_passes + 1;
    if (n > 0) c->stats.kernel_launches += static_cast<uint64_t>(c->passes.n_passes) + 1;
    c->stats.n_passes = c->passes.n_passes;
    c->stats.source_major = 0;
    c->sort_stages = c->passes.n_passes;
  }
  c->stats.key_bits = c->layout.total_bits();
  dev_free(c, sort_scratch);
  dev_free(c, keys_oth);
  dev_free(c, vals_oth);

  // Index: unpack target / delay / weight, group starts, row_ptr and p_i.
  const uint64_t n_delay_values = max_step;
  const uint64_t group_cap = std::max<uint64_t>(1, std::min<uint64_t>(n, total_nodes * n_delay_values));
  // (A block-sorted build unpacks in place after the index: targets over
  // the value array, weights over the key array.)
  uint32_t* u_target = fused          ? unpack.target
                       : block_sorted ? reinterpret_cast<uint32_t*>(vals_res)
                                      : static_cast<uint32_t*>(dev_alloc(c, n * sizeof(uint32_t)));
  float* u_weight = fused          ? reinterpret_cast<float*>(unpack.weight)
                    : block_sorted ? static_cast<float*>(keys_res)
                                   : static_cast<float*>(dev_alloc(c, n * sizeof(float)));
  uint64_t* u_group_first = static_cast<uint64_t*>(dev_alloc(c, group_cap * sizeof(uint64_t)));
  // Per-network CSR and group offsets: network m's n_nodes_m + 1 entries
  // start at local_base[m].
  std::vector<uint64_t> local_base(n_members, 0);
  for (int m = 1; m < n_members; ++m) local_base[m] = local_base[m - 1] + members[m - 1]->n_nodes + 1;
  const uint64_t n_local = total_nodes + static_cast<uint64_t>(n_members);
  uint64_t* u_row_ptr = static_cast<uint64_t*>(dev_alloc(c, n_local * sizeof(uint64_t)));
  uint64_t* u_group_ptr = static_cast<uint64_t*>(dev_alloc(c, n_local * sizeof(uint64_t)));
  uint64_t* d_local_base = static_cast<uint64_t*>(dev_alloc(c, n_members * sizeof(uint64_t)));
  S.d_bases = static_cast<uint64_t*>(dev_alloc(c, (static_cast<size_t>(n_members) + 1) * sizeof(uint64_t)));
  const uint64_t iblocks = (n + kIndexTile - 1) / kIndexTile;
  uint32_t* starts = static_cast<uint32_t*>(dev_alloc(c, (iblocks * (kIndexTile / 32) + 1) * sizeof(uint32_t)));
  uint32_t* bcounts = static_cast<uint32_t*>(dev_alloc(c, (iblocks + 1) * sizeof(uint32_t)));
  uint64_t* boffsets = static_cast<uint64_t*>(dev_alloc(c, (iblocks + 1) * sizeof(uint64_t)));
  uint64_t* iscan = static_cast<uint64_t*>(dev_alloc(c, (scan_tmp_entries(iblocks) + 1) * sizeof(uint64_t)));
  if (!u_target || !u_delay || !u_weight || !u_group_first || !u_row_ptr || !u_group_ptr || !d_local_base ||
      !S.d_bases || !starts || !bcounts || !boffsets || !iscan)
    return fail(c, SNC_ERR_OOM, "device allocation failed (index)");
  if (n > 0) {
    IndexArgs ia{};
    ia.keys = keys_res;
    ia.vals = vals_res;
    ia.key32 = key32 ? 1 : 0;
    ia.unpacked = (fused || block_sorted) ? 1 : 0;
    ia.n = n;
    ia.delay_bits = c->layout.delay_bits;
    ia.target = u_target;
    ia.delay = u_delay;
    ia.weight = reinterpret_cast<uint32_t*>(u_weight);
    ia.starts = starts;
    ia.block_counts = bcounts;
    ia.block_offsets = boffsets;
    ia.group_first = u_group_first;
    ia.group_cap = group_cap;
    ia.n_groups = S.d_n_groups;
    ia.err = S.d_err;
    ia.n_seg = (segmented || graph_pad) ? n_members : 0;
    ia.seg_begin = d_seg_real;
    ia.seg_end = d_seg_real + n_members;
    const unsigned igrid = static_cast<unsigned>(std::min<uint64_t>(iblocks, static_cast<uint64_t>(c->sms) * 8));
    SNC_CUDA(c, launch_index_unpack(ia, igrid, st));
    ++c->stats.kernel_launches;
    SNC_CUDA(c, exclusive_scan_u32(bcounts, iblocks, boffsets, iscan, st));
    c->stats.kernel_launches += 3;
    index_groups_kernel<<<igrid, kIndexThreads, 0, st>>>(ia);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
  }
  SNC_CUDA(c, upload(c, d_local_base, local_base.data(), n_members * sizeof(uint64_t)));
  if (n == 0) SNC_CUDA(c, cudaMemsetAsync(S.d_n_groups, 0, sizeof(uint64_t), st));
  MemberIndexArgs mi{};
  mi.keys = keys_res;
  mi.key32 = key32 ? 1 : 0;
  mi.delay_bits = c->layout.delay_bits;
  mi.n_members = n_members;
  mi.seg_begin = d_seg_real;
  mi.seg_end = d_seg_real + n_members;
  mi.local_base = d_local_base;
  mi.n_entries = n_local;
  mi.group_first = u_group_first;
  mi.group_cap = group_cap;
  mi.n_groups = S.d_n_groups;
  mi.row_local = u_row_ptr;
  mi.group_local = u_group_ptr;
  mi.gfirst = S.d_bases;
  SNC_CUDA(c, launch_member_index(mi, st));
  ++c->stats.kernel_launches;
  if (segmented) {
    // group_first relative to each network's first connection.
    rebase_group_first_kernel<<<static_cast<unsigned>(std::max<uint64_t>(
                                    1, std::min<uint64_t>((group_cap + 255) / 256, static_cast<uint64_t>(c->sms) * 8))),
                                256, 0, st>>>(u_group_first, S.d_n_groups, group_cap, S.d_bases, d_seg, n_members);
    ++c->stats.kernel_launches;
    SNC_CUDA(c, cudaGetLastError());
  }
  if (block_sorted && n > 0) {
    // The index has read the keys: unpack in place, one block at a time.
    void* utk = dev_alloc(c, block * key_bytes);
    uint64_t* utv = static_cast<uint64_t*>(dev_alloc(c, block * sizeof(uint64_t)));
    if (!utk || !utv) return fail(c, SNC_ERR_OOM, "device allocation failed (unpack block)");
    SNC_CUDA(c, unpack_in_place(keys_res, key32 ? 1 : 0, vals_res, n, block, utk, utv,
                                (1u << c->layout.delay_bits) - 1u, u_delay, c->sms, st));
    c->stats.kernel_launches += 2 * ((n + block - 1) / block);
    dev_free(c, utk);
    dev_free(c, utv);
  }
  // First group of every network (and the total) for the views.
  if (!S.h_bases) {
    S.h_bases_words = static_cast<size_t>(n_members) + 1;
    S.h_bases = static_cast<uint64_t*>(pinned_pool().get(S.h_bases_words * sizeof(uint64_t)));
    if (!S.h_bases) return fail(c, SNC_ERR_OOM, "pinned allocation failed (views)");
  }
  SNC_CUDA(c, cudaMemcpyAsync(S.h_bases, S.d_bases, (static_cast<size_t>(n_members) + 1) * sizeof(uint64_t),
                              cudaMemcpyDeviceToHost, st));
  c->stats.d2h_bytes += (static_cast<size_t>(n_members) + 1) * sizeof(uint64_t);
  S.real_counts = graph_pad;
  if (graph_pad) {
    if (!S.h_real) {
      S.h_real_words = static_cast<size_t>(n_members);
      S.h_real = static_cast<uint64_t*>(pinned_pool().get(S.h_real_words * sizeof(uint64_t)));
      if (!S.h_real) return fail(c, SNC_ERR_OOM, "pinned allocation failed (views)");
    }
    SNC_CUDA(c, cudaMemcpyAsync(S.h_real, d_real_count, static_cast<size_t>(n_members) * sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, st));
    c->stats.d2h_bytes += static_cast<size_t>(n_members) * sizeof(uint64_t);
  }
  mark();
  dev_free(c, starts);
  dev_free(c, bcounts);
  dev_free(c, boffsets);
  dev_free(c, iscan);
  if (!block_sorted) dev_free(c, keys_res);       // a block-sorted build keeps its weights there
  if (!fused && !block_sorted) dev_free(c, vals_res);  // else it holds the targets (and weights)
  dev_free(c, d_direct);
  dev_free(c, d_prim_off);
  dev_free(c, d_seg);
  dev_free(c, d_tile_begin);
  dev_free(c, d_local_base);
  dev_free(c, d_bern_list);
  dev_free(c, d_bern_totals);

  S.n_members = n_members;
  S.n_total = n_conn;
  S.synced = false;
  for (int m = 0; m < n_members; ++m) {
    snc_ctx* x = members[m];
    if (m > 0) x->store = c->store;
    x->member = m;
    x->node_base = node_base[m];
    x->layout = c->layout;
    x->passes = c->passes;
    x->sort_stages = c->sort_stages;
    x->group_cap = group_cap;
    x->target_all = u_target;
    x->delay_all = u_delay;
    x->weight_all = u_weight;
    x->group_first_all = u_group_first;
    x->row_ptr = u_row_ptr + local_base[m];
    x->group_ptr = u_group_ptr + local_base[m];
    x->seg_begin = seg_begin[m];
    x->seg_count = seg_end[m] - seg_begin[m];
    x->view_ready = false;
    x->finalized = true;
    if (m > 0) x->stats = c->stats;
  }
  return SNC_OK;
}

}  // namespace

extern "C" {

snc_status snc_finalize(snc_ctx* c) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    if (c->finalized) return fail(c, SNC_ERR_STATE, "finalize called twice");
    if (c->sharded && c->block_sort)
      return fail(c, SNC_ERR_INVALID_ARG, "a target shard is built with the out-of-place sort");
    if (c->sharded && static_cast<uint64_t>(c->shard_first) + c->shard_n > c->n_nodes)
      return fail(c, SNC_ERR_INVALID_ARG, "target shard [%u, %u + %u) outside the %llu nodes", c->shard_first,
                  c->shard_first, c->shard_n, static_cast<unsigned long long>(c->n_nodes));
    return finalize_build(&c, 1);
  });
}

snc_status snc_set_block_sort(snc_ctx* c, uint64_t block) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    if (c->finalized) return fail(c, SNC_ERR_STATE, "set_block_sort after finalize");
    if (block % kCopassAlign != 0)
      return fail(c, SNC_ERR_INVALID_ARG, "block sort: block of %llu is not a multiple of %llu",
                  static_cast<unsigned long long>(block), static_cast<unsigned long long>(kCopassAlign));
    c->block_sort = block;
    return SNC_OK;
  });
}

snc_status snc_set_target_shard(snc_ctx* c, uint32_t first, uint32_t n) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    if (c->finalized) return fail(c, SNC_ERR_STATE, "set_target_shard after finalize");
    c->sharded = true;
    c->shard_first = first;
    c->shard_n = n;
    return SNC_OK;
  });
}

snc_status snc_batch_finalize(snc_ctx* const* ctxs, int n) {
  return snc::abi_guard([&]() -> snc_status {
    if (!ctxs || n <= 0) return fail(nullptr, SNC_ERR_INVALID_ARG, "batch: no contexts");
    for (int i = 0; i < n; ++i) {
      if (!ctxs[i]) return fail(nullptr, SNC_ERR_INVALID_ARG, "batch: null context");
      if (ctxs[i]->finalized) return fail(ctxs[i], SNC_ERR_STATE, "batch: context already finalized");
      if (ctxs[i]->device != ctxs[0]->device) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: contexts on different devices");
      if (ctxs[i]->sharded) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: a target shard is built alone");
      if (ctxs[i]->block_sort) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: a block-sorted build is built alone");
      for (int j = 0; j < i; ++j)
        if (ctxs[j] == ctxs[i]) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: context listed twice");
    }
    const snc_status st = finalize_build(ctxs, n);
    if (st != SNC_OK)
      for (int i = 1; i < n; ++i) ctxs[i]->err = ctxs[0]->err;
    return st;
  });
}

namespace {
// A graph build replays the recorded device work with every size fixed:
// pairwise_bernoulli projections get capacities, total-number redraws a
// fixed number of rounds (finalize_build); a target shard reads its kept
// count back before the sort and is built alone.
bool graph_eligible(const snc_ctx* c) { return !c->sharded; }
}  // namespace

snc_status snc_batch_finalize_graph(snc_ctx* const* ctxs, int n) {
  return snc::abi_guard([&]() -> snc_status {
    if (!ctxs || n <= 0) return fail(nullptr, SNC_ERR_INVALID_ARG, "batch: no contexts");
    for (int i = 0; i < n; ++i) {
      if (!ctxs[i]) return fail(nullptr, SNC_ERR_INVALID_ARG, "batch: null context");
      if (ctxs[i]->finalized) return fail(ctxs[i], SNC_ERR_STATE, "batch: context already finalized");
      if (ctxs[i]->device != ctxs[0]->device) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: contexts on different devices");
      if (ctxs[i]->sharded) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: a target shard is built alone");
      if (ctxs[i]->block_sort) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: a block-sorted build is built alone");
      for (int j = 0; j < i; ++j)
        if (ctxs[j] == ctxs[i]) return fail(ctxs[i], SNC_ERR_INVALID_ARG, "batch: context listed twice");
      if (!graph_eligible(ctxs[i]))
        return fail(ctxs[i], SNC_ERR_UNSUPPORTED, "graph build: a target shard is built alone");
    }
    snc_ctx* c = ctxs[0];
    Storage& S = *c->store;
    SNC_CUDA(c, cudaSetDevice(c->device));
    // A stream of the build's own (the legacy default stream cannot be
    // captured), ordered after the work already queued on the caller's.
    cudaStream_t own = nullptr;
    SNC_CUDA(c, cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    S.own_stream = own;
    cudaEvent_t ready = nullptr;
    SNC_CUDA(c, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaEventRecord(ready, c->stream);
    cudaStreamWaitEvent(own, ready, 0);
    cudaEventDestroy(ready);
    for (int i = 0; i < n; ++i) snc::rebind_build(ctxs[i], own, nullptr);
    // First build: runs now and keeps every buffer, recording their order.
    S.mode = 1;
    S.rec.clear();
    snc_status st = finalize_build(ctxs, n);
    if (st != SNC_OK) {
      for (int i = 1; i < n; ++i) ctxs[i]->err = ctxs[0]->err;
      return st;
    }
    // Second pass over the same plan, captured: the same buffers in the same
    // order, copies from a fresh staging chunk that the graph keeps reading.
    if (!S.reserve_stage(S.stage_total + 4096)) return fail(c, SNC_ERR_OOM, "pinned staging allocation failed");
    S.mode = 2;
    S.rec_pos = 0;
    S.capturing = true;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(S.stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      st = finalize_build(ctxs, n);
      const cudaError_t e2 = cudaStreamEndCapture(S.stream, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    S.capturing = false;
    S.mode = 1;
    if (e == cudaSuccess && st == SNC_OK) e = cudaGraphInstantiate(&S.gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      S.gexec = nullptr;
      return fail(c, SNC_ERR_CUDA, "graph capture of the build failed: %s", cudaGetErrorString(e));
    }
    if (st != SNC_OK) return st;
    return SNC_OK;
  });
}

snc_status snc_batch_rebuild(snc_ctx* ctx, const uint64_t* seeds, int n) {
  return snc::abi_guard([&]() -> snc_status {
    if (!ctx || !seeds) return fail(ctx, SNC_ERR_INVALID_ARG, "rebuild: null argument");
    if (!ctx->finalized || !ctx->store || !ctx->store->gexec)
      return fail(ctx, SNC_ERR_STATE, "rebuild: the context was not built by snc_batch_finalize_graph");
    Storage& S = *ctx->store;
    if (n != S.n_members) return fail(ctx, SNC_ERR_INVALID_ARG, "rebuild: %d seeds for %d networks", n, S.n_members);
    SNC_CUDA(ctx, cudaSetDevice(ctx->device));
    // The replayed copies read the staged records: the previous build must be done.
    SNC_CUDA(ctx, cudaStreamSynchronize(S.stream));
    for (const Storage::SeedSite& site : S.seed_sites) {
      const uint64_t seed = seeds[site.member];
      site.host->k0 = static_cast<uint32_t>(seed);
      site.host->k1 = static_cast<uint32_t>(seed >> 32) ^ site.local;
    }
    ctx->cfg.seed = seeds[ctx->member];
    S.synced = false;
    ++S.generation;
    SNC_CUDA(ctx, cudaGraphLaunch(S.gexec, S.stream));
    ++ctx->stats.kernel_launches;
    return SNC_OK;
  });
}

snc_status snc_synchronize(snc_ctx* c) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    SNC_CUDA(c, cudaSetDevice(c->device));
    Storage& S = *c->store;
    SNC_CUDA(c, cudaStreamSynchronize(S.stream));
    if (!c->finalized) return SNC_OK;
    if (!S.synced) {
      SNC_CUDA(c, cudaMemcpyAsync(S.h_pinned + 4, S.d_err, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost, S.stream));
      SNC_CUDA(c, cudaMemcpyAsync(S.h_pinned + 1, S.d_n_groups, sizeof(uint64_t), cudaMemcpyDeviceToHost, S.stream));
      c->stats.d2h_bytes += 5 * sizeof(uint64_t);
      SNC_CUDA(c, cudaStreamSynchronize(S.stream));
      S.err_bits = static_cast<uint32_t>(S.h_pinned[4] & 0xFFFFFFFFu);
      S.n_groups = S.h_pinned[1];
      S.synced = true;
    }
    if (!c->view_ready || c->view_gen != S.generation) {
      const uint64_t g0 = S.h_bases[c->member], g1 = S.h_bases[c->member + 1];
      c->n_syn = S.real_counts ? S.h_real[c->member] : c->seg_count;
      c->n_groups = g1 - g0;
      c->target = c->target_all + c->seg_begin;
      c->delay = c->delay_all + c->seg_begin;
      c->weight = c->weight_all + c->seg_begin;
      c->group_first = c->group_first_all + g0;
      c->view_ready = true;
      c->view_gen = S.generation;
    }
    const uint32_t err = S.err_bits;
    if (err & kErrLookbackTimeout) return fail(c, SNC_ERR_TIMEOUT, "a look-back wait expired on the device");
    if (err & kErrSamplerBound) return fail(c, SNC_ERR_TIMEOUT, "a sampler exceeded its attempt bound");
    if (err & kErrGraphRounds)
      return fail(c, SNC_ERR_TIMEOUT, "fixed_total_number: redraws still pending after the last device-counted round");
    if (err & kErrGraphCapacity)
      return fail(c, SNC_ERR_UNSUPPORTED, "graph replay: a pairwise_bernoulli projection drew past its capacity");
    if (err & kErrBounds) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(S.h_pinned + 4);
      return fail(c, SNC_ERR_CUDA, "a device index check failed (site %u, index %llu, limit %llu)", w[2],
                  static_cast<unsigned long long>(w[4] | (static_cast<uint64_t>(w[5]) << 32)),
                  static_cast<unsigned long long>(w[6] | (static_cast<uint64_t>(w[7]) << 32)));
    }
    return SNC_OK;
  });
}

snc_status snc_get_connections(snc_ctx* c, snc_conn_view* out) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c || !out) return fail(c, SNC_ERR_INVALID_ARG, "null argument");
    if (!c->finalized) return fail(c, SNC_ERR_STATE, "get_connections before finalize");
    const snc_status st = snc_synchronize(c);
    if (st != SNC_OK) return st;
    out->n_syn = c->n_syn;
    out->n_nodes = c->n_nodes;
    out->n_groups = c->n_groups;
    out->row_ptr = c->row_ptr;
    out->target = c->target;
    out->delay = c->delay;
    out->weight = c->weight;
    out->group_ptr = c->group_ptr;
    out->group_first = c->group_first;
    return SNC_OK;
  });
}

snc_status snc_deliver(snc_ctx* c, const uint32_t* src, const uint32_t* grp, const float* mult,
                       uint64_t n_spikes, float* input) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
    if (!c->finalized) return fail(c, SNC_ERR_STATE, "deliver before finalize");
    snc_conn_view v{};
    snc_status s = snc_get_connections(c, &v);  // synchronizes and resolves the views
    if (s != SNC_OK) return s;
    if (n_spikes == 0) return SNC_OK;
    if (!src || !grp || !mult || !input) return fail(c, SNC_ERR_INVALID_ARG, "null spike array or input");
    CallScope scope(c);
    cudaStream_t st = c->store->stream;
    uint32_t* sizes = static_cast<uint32_t*>(dev_alloc(c, (n_spikes + 1) * sizeof(uint32_t)));
    uint64_t* offsets = static_cast<uint64_t*>(dev_alloc(c, (n_spikes + 1) * sizeof(uint64_t)));
    uint64_t* tmp = static_cast<uint64_t*>(dev_alloc(c, (scan_tmp_entries(n_spikes) + 1) * sizeof(uint64_t)));
    uint64_t* first = static_cast<uint64_t*>(dev_alloc(c, n_spikes * sizeof(uint64_t)));
    uint32_t* err = static_cast<uint32_t*>(dev_alloc(c, 8 * sizeof(uint32_t)));
    if (!sizes || !offsets || !tmp || !first || !err) {
      for (void* p : {static_cast<void*>(sizes), static_cast<void*>(offsets), static_cast<void*>(tmp),
                      static_cast<void*>(first), static_cast<void*>(err)})
        dev_free(c, p);
      return fail(c, SNC_ERR_OOM, "device allocation failed (spike array)");
    }
    SNC_CUDA(c, cudaMemsetAsync(err, 0, 8 * sizeof(uint32_t), st));
    DeliverArgs a{};
    a.src = src;
    a.grp = grp;
    a.mult = mult;
    a.n_spikes = n_spikes;
    a.row_ptr = v.row_ptr;
    a.group_ptr = v.group_ptr;
    a.group_first = v.group_first;
    a.target = v.target;
    a.weight = v.weight;
    a.n_nodes = v.n_nodes;
    a.n_syn = v.n_syn;
    a.sizes = sizes;
    a.first = first;
    a.offsets = offsets;
    a.input = input;
    a.err = err;
    const unsigned g1 = static_cast<unsigned>(
        std::max<uint64_t>(1, std::min<uint64_t>((n_spikes + 255) / 256, static_cast<uint64_t>(c->sms) * 16)));
    deliver_size_kernel<<<g1, 256, 0, st>>>(a);
    SNC_CUDA(c, exclusive_scan_u32(sizes, n_spikes, offsets, tmp, st));
    deliver_kernel<<<static_cast<unsigned>(c->sms) * 8, kDeliverThreads, 0, st>>>(a);
    SNC_CUDA(c, cudaGetLastError());
    c->stats.kernel_launches += 5;
    uint32_t* h_err = reinterpret_cast<uint32_t*>(c->store->h_pinned + 12);
    SNC_CUDA(c, cudaMemcpyAsync(h_err, err, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    SNC_CUDA(c, cudaStreamSynchronize(st));
    const uint32_t bits = h_err[0];
    dev_free(c, sizes);
    dev_free(c, offsets);
    dev_free(c, tmp);
    dev_free(c, first);
    dev_free(c, err);
    if (bits & kErrBounds) return fail(c, SNC_ERR_INVALID_ARG, "a spike array entry names no connection group");
    return SNC_OK;
  });
}

namespace {
// Host copies of a finalized network, queued on the context's stream; the
// caller has synchronized (errors, counts of the views) and checked the
// capacities.
snc_status queue_connection_copies(snc_ctx* c, uint32_t* src, uint32_t* tgt, uint16_t* delay, float* weight) {
  const uint64_t n = c->n_syn;
  CallScope scope(c);
  cudaStream_t st = c->store->stream;
  if (src && n > 0) {
    uint32_t* d_src = static_cast<uint32_t*>(dev_alloc(c, n * sizeof(uint32_t)));
    if (!d_src) return fail(c, SNC_ERR_OOM, "device allocation failed (source expansion)");
    if (c->n_nodes > 0) {
      const uint64_t blocks = std::min<uint64_t>((c->n_nodes + 7) / 8, static_cast<uint64_t>(c->sms) * 16);
      expand_sources_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(c->row_ptr, c->n_nodes, d_src);
      ++c->stats.kernel_launches;
    }
    SNC_CUDA(c, cudaGetLastError());
    SNC_CUDA(c, cudaMemcpyAsync(src, d_src, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    dev_free(c, d_src);  // stream-ordered: after the copy
  }
  if (tgt && n > 0) SNC_CUDA(c, cudaMemcpyAsync(tgt, c->target, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (delay && n > 0) SNC_CUDA(c, cudaMemcpyAsync(delay, c->delay, n * sizeof(uint16_t), cudaMemcpyDeviceToHost, st));
  if (weight && n > 0) SNC_CUDA(c, cudaMemcpyAsync(weight, c->weight, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  c->stats.d2h_bytes += n * ((src ? 4 : 0) + (tgt ? 4 : 0) + (delay ? 2 : 0) + (weight ? 4 : 0));
  return SNC_OK;
}

snc_status queue_index_copies(snc_ctx* c, uint64_t* row_ptr, uint64_t* group_ptr, uint64_t* group_first) {
  cudaStream_t st = c->store->stream;
  const size_t rows = (c->n_nodes + 1) * sizeof(uint64_t);
  if (row_ptr) SNC_CUDA(c, cudaMemcpyAsync(row_ptr, c->row_ptr, rows, cudaMemcpyDeviceToHost, st));
  if (group_ptr) SNC_CUDA(c, cudaMemcpyAsync(group_ptr, c->group_ptr, rows, cudaMemcpyDeviceToHost, st));
  if (group_first && c->n_groups > 0)
    SNC_CUDA(c, cudaMemcpyAsync(group_first, c->group_first, c->n_groups * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  c->stats.d2h_bytes += (row_ptr ? rows : 0) + (group_ptr ? rows : 0) + (group_first ? c->n_groups * sizeof(uint64_t) : 0);
  return SNC_OK;
}

// The build done and its errors reported (snc_synchronize), before a copy.
snc_status ready_for_copy(snc_ctx* c, const char* what) {
  if (!c) return fail(nullptr, SNC_ERR_INVALID_ARG, "null context");
  if (!c->finalized) return fail(c, SNC_ERR_STATE, "%s before finalize", what);
  return snc_synchronize(c);
}
}  // namespace

snc_status snc_copy_connections(snc_ctx* c, uint32_t* src, uint32_t* tgt, uint16_t* delay, float* weight,
                                uint64_t cap) {
  return snc::abi_guard([&]() -> snc_status {
    snc_status s = ready_for_copy(c, "copy_connections");
    if (s != SNC_OK) return s;
    if (cap < c->n_syn) return fail(c, SNC_ERR_INVALID_ARG, "capacity below the number of connections");
    s = queue_connection_copies(c, src, tgt, delay, weight);
    if (s != SNC_OK) return s;
    SNC_CUDA(c, cudaStreamSynchronize(c->store->stream));
    return SNC_OK;
  });
}

snc_status snc_copy_index(snc_ctx* c, uint64_t* row_ptr, uint64_t* group_ptr, uint64_t* group_first,
                          uint64_t group_cap) {
  return snc::abi_guard([&]() -> snc_status {
    snc_status s = ready_for_copy(c, "copy_index");
    if (s != SNC_OK) return s;
    if (group_first && group_cap < c->n_groups) return fail(c, SNC_ERR_INVALID_ARG, "group capacity below n_groups");
    s = queue_index_copies(c, row_ptr, group_ptr, group_first);
    if (s != SNC_OK) return s;
    SNC_CUDA(c, cudaStreamSynchronize(c->store->stream));
    return SNC_OK;
  });
}

snc_status snc_copy_network_async(snc_ctx* c, uint32_t* tgt, uint16_t* delay, float* weight, uint64_t cap,
                                  uint64_t* row_ptr, uint64_t* group_ptr, uint64_t* group_first,
                                  uint64_t group_cap) {
  return snc::abi_guard([&]() -> snc_status {
    // The build's errors and counts first, so that nothing is queued when an
    // argument is refused; then the copies, without waiting for them.
    snc_status s = ready_for_copy(c, "copy_network_async");
    if (s != SNC_OK) return s;
    if (cap < c->n_syn) return fail(c, SNC_ERR_INVALID_ARG, "capacity below the number of connections");
    if (group_first && group_cap < c->n_groups) return fail(c, SNC_ERR_INVALID_ARG, "group capacity below n_groups");
    s = queue_connection_copies(c, nullptr, tgt, delay, weight);
    if (s != SNC_OK) return s;
    return queue_index_copies(c, row_ptr, group_ptr, group_first);
  });
}

snc_status snc_stage_times(snc_ctx* c, float* ms, int max_stages, int* n_stages, int* n_passes) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c || !ms || max_stages < 0) return fail(c, SNC_ERR_INVALID_ARG, "null argument");
    if (!c->finalized) return fail(c, SNC_ERR_STATE, "no finalize has run");
    Storage& S = *c->store;
    SNC_CUDA(c, cudaStreamSynchronize(S.stream));
    int k = 0;
    for (int i = 1; i < S.n_ev && k < max_stages; ++i, ++k) {
      float t = 0.f;
      SNC_CUDA(c, cudaEventElapsedTime(&t, S.ev[i - 1], S.ev[i]));
      ms[k] = t;
    }
    if (n_stages) *n_stages = k;
    if (n_passes) *n_passes = c->sort_stages;
    return SNC_OK;
  });
}

snc_status snc_radix_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                uint32_t* vals_out, uint64_t n, int key_bits, void* stream) {
  return snc::abi_guard([&]() -> snc_status {
    if (key_bits < 1 || key_bits > 64) return fail(nullptr, SNC_ERR_INVALID_ARG, "key_bits outside [1, 64]");
    if (n == 0) return SNC_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return fail(nullptr, SNC_ERR_INVALID_ARG, "null buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const SortPasses sp = plan_passes(key_bits);
    const size_t scratch_bytes = sort_scratch_bytes(n, sp);
    void* scratch = nullptr;
    uint64_t* ktmp = nullptr;
    uint32_t* vtmp = nullptr;
    uint32_t* err = nullptr;
    auto release = [&]() {
      if (scratch) cudaFreeAsync(scratch, st);
      if (ktmp) cudaFreeAsync(ktmp, st);
      if (vtmp) cudaFreeAsync(vtmp, st);
      if (err) cudaFreeAsync(err, st);
    };
    if (cudaMallocAsync(&scratch, scratch_bytes, st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&err), 256, st) != cudaSuccess ||
        (sp.n_passes > 1 && (cudaMallocAsync(reinterpret_cast<void**>(&ktmp), n * sizeof(uint64_t), st) != cudaSuccess ||
                             cudaMallocAsync(reinterpret_cast<void**>(&vtmp), n * sizeof(uint32_t), st) != cudaSuccess))) {
      cudaGetLastError();
      release();
      return fail(nullptr, SNC_ERR_OOM, "sort scratch allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(err, 0, 256, st);
    if (e == cudaSuccess) e = radix_sort_run(keys_in, vals_in, keys_out, vals_out, ktmp, vtmp, n, sp, scratch, err, st, nullptr);
    // The device error word tells whether a bounded wait expired (the output
    // is then not sorted): read it once the queued work is done.
    uint32_t bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, st);
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, SNC_ERR_CUDA, "radix sort: %s", cudaGetErrorString(e));
    if (bits & kErrLookbackTimeout) return fail(nullptr, SNC_ERR_TIMEOUT, "radix sort: a look-back wait expired on the device");
    if (bits) return fail(nullptr, SNC_ERR_CUDA, "radix sort: device error bits 0x%x", bits);
    return SNC_OK;
  });
}

snc_status snc_block_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t n, int key_bits, uint64_t block,
                                void* stream) {
  return snc::abi_guard([&]() -> snc_status {
    if (key_bits < 1 || key_bits > 64) return fail(nullptr, SNC_ERR_INVALID_ARG, "key_bits outside [1, 64]");
    if (n == 0) return SNC_OK;
    if (!keys || !vals) return fail(nullptr, SNC_ERR_INVALID_ARG, "null buffer");
    if (block == 0 || block % kCopassAlign != 0)
      return fail(nullptr, SNC_ERR_INVALID_ARG, "block of %llu is not a positive multiple of %llu",
                  static_cast<unsigned long long>(block), static_cast<unsigned long long>(kCopassAlign));
    if ((n + block - 1) / block > static_cast<uint64_t>(kCopassMaxRuns))
      return fail(nullptr, SNC_ERR_INVALID_ARG, "%llu pairs need more than %d blocks of %llu",
                  static_cast<unsigned long long>(n), kCopassMaxRuns, static_cast<unsigned long long>(block));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const SortPasses sp = plan_passes(key_bits);
    void* scratch = nullptr;
    uint32_t* err = nullptr;
    if (cudaMallocAsync(&scratch, copass_scratch_bytes(block, 8, 4, sp), st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&err), 256, st) != cudaSuccess) {
      cudaGetLastError();
      if (scratch) cudaFreeAsync(scratch, st);
      if (err) cudaFreeAsync(err, st);
      return fail(nullptr, SNC_ERR_OOM, "block sort working memory allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(err, 0, 256, st);
    if (e == cudaSuccess) e = copass_sort_run(keys, vals, n, block, sp, scratch, err, st);
    uint32_t bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, SNC_ERR_CUDA, "block sort: %s", cudaGetErrorString(e));
    if (bits & kErrLookbackTimeout) return fail(nullptr, SNC_ERR_TIMEOUT, "block sort: a look-back wait expired");
    if (bits) return fail(nullptr, SNC_ERR_CUDA, "block sort: device error bits 0x%x", bits);
    return SNC_OK;
  });
}

snc_status snc_set_wait_test(uint32_t lookback_spin_limit, uint32_t withhold_tile) {
  return snc::abi_guard([&]() -> snc_status {
    g_wait_test.lookback_spin_limit = lookback_spin_limit ? lookback_spin_limit : kDefaultSpinLimit;
    g_wait_test.withhold_unit = withhold_tile;
    return SNC_OK;
  });
}

snc_status snc_set_graph_test(double bernoulli_sd, double bernoulli_slack, uint32_t redraw_rounds) {
  return snc::abi_guard([&]() -> snc_status {
    if (!(bernoulli_sd >= 0.0) || !(bernoulli_slack >= 0.0))
      return fail(nullptr, SNC_ERR_INVALID_ARG, "graph test: negative capacity margin");
    g_graph_test.bernoulli_sd = bernoulli_sd;
    g_graph_test.bernoulli_slack = bernoulli_slack;
    g_graph_test.redraw_rounds = redraw_rounds;
    return SNC_OK;
  });
}

snc_status snc_set_tuning(const snc_tuning* t) {
  return snc::abi_guard([&]() -> snc_status {
    if (!t) return fail(nullptr, SNC_ERR_INVALID_ARG, "null tuning");
    if (t->sort_digit_bits < 8 || t->sort_digit_bits > 11)
      return fail(nullptr, SNC_ERR_INVALID_ARG, "sort_digit_bits outside [8, 11]");
    if (t->sort_group_tiles != 0 && t->sort_group_tiles != 1 && t->sort_group_tiles != 4 && t->sort_group_tiles != 8)
      return fail(nullptr, SNC_ERR_INVALID_ARG, "sort_group_tiles must be 0, 1, 4 or 8");
    if (t->gen_blocks_per_sm < 1 || t->gen_blocks_per_sm > 32)
      return fail(nullptr, SNC_ERR_INVALID_ARG, "gen_blocks_per_sm outside [1, 32]");
    if (t->sort_items != 8 && t->sort_items != 12 && t->sort_items != 16 && t->sort_items != 24 && t->sort_items != 32)
      return fail(nullptr, SNC_ERR_INVALID_ARG, "sort_items must be 8, 12, 16, 24 or 32");
    if (t->reserved[0] || t->reserved[1] || t->reserved[2] || t->reserved[3])
      return fail(nullptr, SNC_ERR_INVALID_ARG, "reserved tuning fields must be 0");
    g_sort_tuning.max_digit_bits = t->sort_digit_bits;
    g_sort_tuning.group_tiles = t->sort_group_tiles;
    g_sort_tuning.items = t->sort_items;
    g_gen_blocks_per_sm = t->gen_blocks_per_sm;
    return SNC_OK;
  });
}

snc_status snc_get_tuning(snc_tuning* t) {
  return snc::abi_guard([&]() -> snc_status {
    if (!t) return fail(nullptr, SNC_ERR_INVALID_ARG, "null tuning");
    t->sort_digit_bits = g_sort_tuning.max_digit_bits;
    t->sort_group_tiles = g_sort_tuning.group_tiles;
    t->gen_blocks_per_sm = g_gen_blocks_per_sm;
    t->sort_items = g_sort_tuning.items;
    t->reserved[0] = t->reserved[1] = t->reserved[2] = t->reserved[3] = 0;
    return SNC_OK;
  });
}

snc_status snc_get_stats(const snc_ctx* c, snc_stats* out) {
  return snc::abi_guard([&]() -> snc_status {
    if (!c || !out) return fail(nullptr, SNC_ERR_INVALID_ARG, "null argument");
    *out = c->stats;
    return SNC_OK;
  });
}

const char* snc_last_error(const snc_ctx* c) {
  if (c) return c->err.c_str();
  return g_last_error.c_str();
}

}  // extern "C"
