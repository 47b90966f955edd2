// snc_server.cpp -- the served form: admission of construction requests
// under a device-memory budget, concurrent builds on worker threads and
// streams, small requests grouped into batched builds, results resident
// until released (include/snc_server.h).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/snc_server.h"
#include "snc_internal.h"

namespace snc {
void set_last_error(const char* msg);
}

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Memory of one finalize call (one network, or the members of a batch): it
// is freed when the last of its networks is released.
struct Group {
  uint64_t resident_bytes = 0;
  int live = 0;
};

struct Job {
  uint64_t ticket = 0;
  snc_ctx* ctx = nullptr;
  snc_job_state state = SNC_JOB_QUEUED;
  snc_status status = SNC_OK;
  std::string error;
  snc::BuildEstimate est{};
  Clock::time_point t_submit, t_start, t_done;
  int batch_size = 1;
  std::shared_ptr<Group> group;
};

int bits_of(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

void* pool_alloc(size_t bytes, void* stream, void* user) {
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, static_cast<cudaMemPool_t>(user), static_cast<cudaStream_t>(stream)) !=
      cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pool_free(void* p, size_t, void* stream, void*) { cudaFreeAsync(p, static_cast<cudaStream_t>(stream)); }

}  // namespace

namespace snc {

size_t admit_from_front(const AdmitRequest* q, size_t n, const AdmitLimits& lim, uint64_t* reserve) {
  *reserve = 0;
  if (n == 0 || lim.reserved_bytes + q[0].peak_bytes > lim.budget_bytes) return 0;
  uint64_t res = q[0].peak_bytes, syn = q[0].n_syn;
  uint64_t nodes = q[0].n_nodes, max_nodes = q[0].n_nodes;
  uint32_t max_step = q[0].max_step;
  size_t take = 1;
  const uint64_t small = lim.batch_max_syn / 2;
  if (lim.batch_max_nets > 1 && q[0].n_syn <= small && !q[0].alone) {
    while (take < n && static_cast<int>(take) < lim.batch_max_nets) {
      const AdmitRequest& j = q[take];
      if (j.n_syn > small || syn + j.n_syn > lim.batch_max_syn || j.alone) break;
      if (lim.reserved_bytes + res + j.peak_bytes > lim.budget_bytes) break;
      const uint64_t n2 = nodes + j.n_nodes, m2 = std::max(max_nodes, j.n_nodes);
      const uint32_t d2 = std::max(max_step, j.max_step);
      if (n2 > 0xFFFFFFFFull || bits_of(n2 - 1) + bits_of(m2 - 1) + bits_of(d2) > 64) break;
      ++take;
      res += j.peak_bytes;
      syn += j.n_syn;
      nodes = n2;
      max_nodes = m2;
      max_step = d2;
    }
  }
  *reserve = res;
  return take;
}

}  // namespace snc

struct snc_server {
  snc_server_config cfg{};
  cudaMemPool_t pool = nullptr;
  snc_allocator alloc{};
  cudaStream_t release_stream = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;

  std::mutex mu;
  std::condition_variable cv_work;  // queue changed, memory freed, or stop
  std::condition_variable cv_done;  // a request finished
  bool stop = false;
  uint64_t next_ticket = 1;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::deque<Job*> queue;
  std::deque<uint64_t> finished;  // not yet reported by wait_any
  snc_server_stats st{};
  std::mutex release_mu;

  // Takes the next build off the queue if it fits (mu held).
  std::vector<Job*> take_build() {
    std::vector<Job*> out;
    if (queue.empty()) return out;
    // The admission looks at the first batch_max_nets requests at most.
    std::vector<snc::AdmitRequest> front;
    const size_t look = std::min<size_t>(queue.size(), static_cast<size_t>(std::max(1, cfg.batch_max_nets)));
    for (size_t i = 0; i < look; ++i) {
      const Job* j = queue[i];
      // (Target shards are built alone.)
      front.push_back({j->est.peak_bytes, j->est.n_syn, j->est.n_nodes, j->est.max_step, snc::ctx_sharded(j->ctx)});
    }
    uint64_t reserve = 0;
    const snc::AdmitLimits lim{cfg.hbm_budget_bytes, st.reserved_bytes, cfg.batch_max_syn, cfg.batch_max_nets};
    const size_t take = snc::admit_from_front(front.data(), front.size(), lim, &reserve);
    for (size_t i = 0; i < take; ++i) {
      out.push_back(queue.front());
      queue.pop_front();
    }
    if (out.empty()) return out;
    const Clock::time_point now = Clock::now();
    for (Job* j : out) {
      j->state = SNC_JOB_RUNNING;
      j->t_start = now;
      j->batch_size = static_cast<int>(out.size());
    }
    st.reserved_bytes += reserve;
    st.peak_reserved_bytes = std::max(st.peak_reserved_bytes, st.reserved_bytes);
    st.queued -= out.size();
    st.running += out.size();
    return out;
  }

  void worker(int w) {
    cudaSetDevice(cfg.device);
    cudaStream_t s = streams[w];
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      std::vector<Job*> build;
      cv_work.wait(lk, [&] {
        if (stop) return true;
        build = take_build();
        return !build.empty();
      });
      if (build.empty()) return;  // stopping with nothing admitted
      lk.unlock();
      std::vector<snc_ctx*> ctxs;
      for (Job* j : build) {
        snc::rebind_build(j->ctx, s, &alloc);
        ctxs.push_back(j->ctx);
      }
      snc_status status = ctxs.size() == 1 ? snc_finalize(ctxs[0])
                                           : snc_batch_finalize(ctxs.data(), static_cast<int>(ctxs.size()));
      std::string err = status == SNC_OK ? "" : snc_last_error(ctxs[0]);
      std::vector<snc_status> each(ctxs.size(), status);
      uint64_t built = 0;
      if (status == SNC_OK) {
        for (size_t i = 0; i < ctxs.size(); ++i) {
          snc_conn_view v{};
          each[i] = snc_get_connections(ctxs[i], &v);  // waits for the device work
          if (each[i] == SNC_OK) built += v.n_syn;
          else if (err.empty()) err = snc_last_error(ctxs[i]);
        }
      } else {
        cudaStreamSynchronize(s);
        cudaGetLastError();
      }
      const Clock::time_point done = Clock::now();
      // The worker's stream takes the next build: later calls on these
      // contexts (views, copies, release) use the server's idle stream.
      for (snc_ctx* c : ctxs) snc::rebind_build(c, release_stream, nullptr);
      auto group = std::make_shared<Group>();
      group->resident_bytes = snc::storage_live_bytes(ctxs[0]);
      group->live = static_cast<int>(build.size());
      lk.lock();
      uint64_t reserve = 0;
      for (size_t i = 0; i < build.size(); ++i) {
        Job* j = build[i];
        reserve += j->est.peak_bytes;
        j->t_done = done;
        j->group = group;
        j->status = each[i];
        j->state = each[i] == SNC_OK ? SNC_JOB_DONE : SNC_JOB_FAILED;
        if (each[i] != SNC_OK) {
          j->error = err;
          ++st.failed;
        } else {
          ++st.completed;
        }
        finished.push_back(j->ticket);
      }
      st.reserved_bytes -= reserve;
      st.reserved_bytes += group->resident_bytes;
      st.resident_bytes += group->resident_bytes;
      st.peak_reserved_bytes = std::max(st.peak_reserved_bytes, st.reserved_bytes);
      st.running -= build.size();
      ++st.builds;
      if (build.size() > 1) ++st.batched_builds;
      st.connections_built += built;
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

namespace {
snc_status server_fail(snc_status s, const char* msg) {
  snc::set_last_error(msg);
  return s;
}
}  // namespace

extern "C" {

snc_status snc_estimate_build(const snc_ctx* ctx, uint64_t* peak_bytes, uint64_t* resident_bytes, uint64_t* n_syn) {
  return snc::abi_guard([&]() -> snc_status {
    if (!ctx || !peak_bytes || !resident_bytes || !n_syn)
      return server_fail(SNC_ERR_INVALID_ARG, "snc_estimate_build: null argument");
    snc::BuildEstimate e{};
    const snc_status s = snc::estimate_build(ctx, &e);
    if (s != SNC_OK) return server_fail(s, "snc_estimate_build failed");
    *peak_bytes = e.peak_bytes;
    *resident_bytes = e.resident_bytes;
    *n_syn = e.n_syn;
    return SNC_OK;
  });
}

snc_status snc_server_create(const snc_server_config* cfg, snc_server** out) {
  return snc::abi_guard([&]() -> snc_status {
    if (!cfg || !out) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_create: null argument");
    if (cfg->hbm_budget_bytes == 0 || cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->batch_max_nets < 1 ||
        cfg->batch_max_nets > 256 || cfg->reserved != 0)
      return server_fail(SNC_ERR_INVALID_ARG, "snc_server_create: configuration out of range");
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
      cudaGetLastError();
      return server_fail(SNC_ERR_CUDA, "snc_server_create: cannot select the device");
    }
    std::unique_ptr<snc_server> srv(new (std::nothrow) snc_server());
    if (!srv) return server_fail(SNC_ERR_OOM, "out of host memory");
    srv->cfg = *cfg;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = cfg->device;
    if (cudaMemPoolCreate(&srv->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return server_fail(SNC_ERR_CUDA, "snc_server_create: memory pool creation failed");
    }
    // Keep freed memory in the pool up to the budget instead of returning it
    // to the driver at every synchronization.
    uint64_t keep = cfg->hbm_budget_bytes;
    cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    srv->alloc.alloc = pool_alloc;
    srv->alloc.free = pool_free;
    srv->alloc.user = srv->pool;
    if (cudaStreamCreateWithFlags(&srv->release_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      cudaMemPoolDestroy(srv->pool);
      return server_fail(SNC_ERR_CUDA, "snc_server_create: stream creation failed");
    }
    for (int i = 0; i < cfg->max_slots; ++i) {
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        for (cudaStream_t x : srv->streams) cudaStreamDestroy(x);
        cudaStreamDestroy(srv->release_stream);
        cudaMemPoolDestroy(srv->pool);
        return server_fail(SNC_ERR_CUDA, "snc_server_create: stream creation failed");
      }
      srv->streams.push_back(s);
    }
    snc_server* p = srv.release();
    try {
      for (int i = 0; i < cfg->max_slots; ++i) p->workers.emplace_back([p, i] { p->worker(i); });
    } catch (...) {
      snc_server_destroy(p);  // joins the workers already started and frees the rest
      throw;
    }
    *out = p;
    return SNC_OK;
  });
}

snc_status snc_server_destroy(snc_server* srv) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv) return SNC_OK;
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (std::thread& t : srv->workers) t.join();
    cudaSetDevice(srv->cfg.device);
    for (auto& kv : srv->jobs) {
      Job& j = *kv.second;
      if (j.ctx) {
        snc::rebind_build(j.ctx, srv->release_stream, nullptr);
        snc_destroy(j.ctx);
      }
    }
    srv->jobs.clear();
    cudaStreamSynchronize(srv->release_stream);
    for (cudaStream_t s : srv->streams) cudaStreamDestroy(s);
    cudaStreamDestroy(srv->release_stream);
    cudaMemPoolDestroy(srv->pool);
    cudaGetLastError();
    delete srv;
    return SNC_OK;
  });
}

snc_status snc_server_submit(snc_server* srv, snc_ctx* ctx, uint64_t* ticket) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv || !ctx || !ticket) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_submit: null argument");
    if (snc::ctx_finalized(ctx)) return server_fail(SNC_ERR_STATE, "snc_server_submit: context already finalized");
    if (snc::ctx_device(ctx) != srv->cfg.device)
      return server_fail(SNC_ERR_INVALID_ARG, "snc_server_submit: context on another device");
    auto job = std::make_unique<Job>();
    if (snc::estimate_build(ctx, &job->est) != SNC_OK)
      return server_fail(SNC_ERR_INVALID_ARG, "snc_server_submit: estimate failed");
    if (job->est.peak_bytes > srv->cfg.hbm_budget_bytes)
      return server_fail(SNC_ERR_INVALID_ARG, "snc_server_submit: the request alone exceeds the memory budget");
    job->ctx = ctx;
    job->t_submit = Clock::now();
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      if (srv->stop) return server_fail(SNC_ERR_STATE, "snc_server_submit: server is shutting down");
      job->ticket = srv->next_ticket++;
      *ticket = job->ticket;
      srv->queue.push_back(job.get());
      srv->jobs.emplace(job->ticket, std::move(job));
      ++srv->st.submitted;
      ++srv->st.queued;
    }
    srv->cv_work.notify_one();
    return SNC_OK;
  });
}

snc_status snc_server_poll(snc_server* srv, uint64_t ticket, snc_job_state* state, snc_conn_view* view) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv || !state) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_poll: null argument");
    snc_ctx* ctx = nullptr;
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      auto it = srv->jobs.find(ticket);
      if (it == srv->jobs.end()) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_poll: unknown ticket");
      Job& j = *it->second;
      *state = j.state;
      if (j.state == SNC_JOB_FAILED) return server_fail(j.status, j.error.c_str());
      if (j.state != SNC_JOB_DONE || !view) return SNC_OK;
      ctx = j.ctx;
    }
    return snc_get_connections(ctx, view);
  });
}

snc_status snc_server_wait_any(snc_server* srv, int timeout_ms, uint64_t* ticket) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv || !ticket) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_wait_any: null argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] { return !srv->finished.empty(); };
    if (timeout_ms < 0)
      srv->cv_done.wait(lk, ready);
    else
      srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (srv->finished.empty()) {
      *ticket = 0;
      return SNC_OK;
    }
    *ticket = srv->finished.front();
    srv->finished.pop_front();
    return SNC_OK;
  });
}

snc_status snc_server_context(snc_server* srv, uint64_t ticket, snc_ctx** ctx) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv || !ctx) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_context: null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_context: unknown ticket");
    *ctx = it->second->ctx;
    return SNC_OK;
  });
}

snc_status snc_server_times(snc_server* srv, uint64_t ticket, snc_job_times* out) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv || !out) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_times: null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_times: unknown ticket");
    const Job& j = *it->second;
    if (j.state != SNC_JOB_DONE && j.state != SNC_JOB_FAILED)
      return server_fail(SNC_ERR_STATE, "snc_server_times: request not finished");
    std::memset(out, 0, sizeof *out);
    out->queued_ms = ms_between(j.t_submit, j.t_start);
    out->build_ms = ms_between(j.t_start, j.t_done);
    out->latency_ms = ms_between(j.t_submit, j.t_done);
    out->batch_size = j.batch_size;
    return SNC_OK;
  });
}

snc_status snc_server_release(snc_server* srv, uint64_t ticket) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_release: null server");
    std::unique_ptr<Job> job;
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      auto it = srv->jobs.find(ticket);
      if (it == srv->jobs.end()) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_release: unknown ticket");
      if (it->second->state != SNC_JOB_DONE && it->second->state != SNC_JOB_FAILED)
        return server_fail(SNC_ERR_STATE, "snc_server_release: request still queued or running");
      job = std::move(it->second);
      srv->jobs.erase(it);
    }
    // The build's stream may be running another build by now: free on the
    // server's release stream (the build itself has finished).
    bool last = false;
    {
      std::lock_guard<std::mutex> rl(srv->release_mu);
      cudaSetDevice(srv->cfg.device);
      last = --job->group->live == 0;
      // Only the last network of a build frees memory; the others leave the
      // shared storage (and its stream) untouched for their siblings.
      if (last) snc::rebind_build(job->ctx, srv->release_stream, nullptr);
      snc_destroy(job->ctx);
      job->ctx = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      ++srv->st.released;
      if (last) {
        srv->st.reserved_bytes -= job->group->resident_bytes;
        srv->st.resident_bytes -= job->group->resident_bytes;
      }
    }
    if (last) srv->cv_work.notify_all();
    return SNC_OK;
  });
}

snc_status snc_server_get_stats(snc_server* srv, snc_server_stats* out) {
  return snc::abi_guard([&]() -> snc_status {
    if (!srv || !out) return server_fail(SNC_ERR_INVALID_ARG, "snc_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    return SNC_OK;
  });
}

}  // extern "C"
