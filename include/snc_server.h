/*
 * snc_server.h -- served form of libsnc: construction requests that arrive
 * over time are admitted under a device-memory budget, built concurrently on
 * the GPU and kept resident until the caller releases them.
 *
 * The paper builds one network per process (Sec. 2.6); its discussion of
 * parameter scans and repeated construction (Sec. 4) motivates building many
 * networks back to back on one device.  Each request is an ordinary snc_ctx
 * (populations created and Connect calls made, not finalized); the server
 * finalizes it exactly as snc_finalize would, so a network built through the
 * server is identical to the same context finalized on its own.
 *
 * Scheduling:
 *   - Requests are admitted in submission order.  A request is admitted when
 *     a build slot is free and its estimated peak device memory, added to the
 *     memory already reserved (peaks of builds in progress plus the actual
 *     size of resident networks), stays within the budget.
 *   - Up to `max_slots` builds run at the same time, each on its own host
 *     worker thread and CUDA stream, so their kernels and host round trips
 *     overlap on the device.
 *   - Small requests waiting back to back in the queue are built together by
 *     one batched finalize (snc_batch_finalize), up to `batch_max_nets`
 *     networks and `batch_max_syn` estimated connections per batch; a
 *     target shard (snc_set_target_shard) is always built alone.
 *   - Device memory comes from a memory pool owned by the server (its
 *     contexts' own allocator settings are replaced); a released network's
 *     memory returns to that pool.
 *
 * Thread safety: every snc_server_* call may be made from any host thread.
 * A submitted context belongs to the server: after snc_server_submit the
 * caller must not destroy, connect or finalize it; once the request is DONE
 * the caller may use the read-only calls (snc_get_connections,
 * snc_copy_connections, snc_get_stats, snc_stage_times) on it until
 * snc_server_release.
 */
#ifndef SNC_SERVER_H
#define SNC_SERVER_H

#include "snc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snc_server snc_server;

typedef struct {
  uint64_t hbm_budget_bytes; /* device memory the server may reserve (> 0)          */
  int device;                /* CUDA device of every request                        */
  int max_slots;             /* concurrent builds (worker threads), 1..64           */
  int batch_max_nets;        /* networks per batched build (1 = no batching), <= 256 */
  int reserved;              /* must be 0                                           */
  uint64_t batch_max_syn;    /* connections (estimated) per batched build; requests  */
                             /* above half of it are built alone                     */
} snc_server_config;

/* Request states reported by snc_server_poll. */
typedef enum {
  SNC_JOB_QUEUED = 0,  /* waiting for a slot or for memory            */
  SNC_JOB_RUNNING = 1, /* being built                                 */
  SNC_JOB_DONE = 2,    /* built; views valid until snc_server_release */
  SNC_JOB_FAILED = 3   /* the build failed; the status says why       */
} snc_job_state;

/* Times of one request, milliseconds of the host steady clock. */
typedef struct {
  double queued_ms;  /* submit -> admitted                          */
  double build_ms;   /* admitted -> built (device work finished)    */
  double latency_ms; /* submit -> built                             */
  int batch_size;    /* networks in the build that carried it       */
  int reserved;
} snc_job_times;

typedef struct {
  uint64_t submitted, completed, failed, released;
  uint64_t queued, running;         /* requests now waiting / being built         */
  uint64_t builds, batched_builds;  /* finalize calls; of them with >1 network     */
  uint64_t reserved_bytes;          /* budget now reserved                        */
  uint64_t resident_bytes;          /* device memory of built, unreleased networks */
  uint64_t peak_reserved_bytes;
  uint64_t connections_built;
} snc_server_stats;

/* Starts the worker threads and the memory pool.
 * INVALID_ARG: null pointers, budget 0, max_slots outside 1..64,
 * batch_max_nets outside 1..256, reserved != 0.  CUDA: device setup failed. */
snc_status snc_server_create(const snc_server_config* cfg, snc_server** out);

/* Waits for builds in progress, then destroys every context the server holds
 * (queued, built or failed) and the pool.  NULL is a no-op. */
snc_status snc_server_destroy(snc_server* srv);

/* Queues ctx for building and returns its ticket (> 0).  The server owns ctx
 * from here on.  INVALID_ARG: null pointers, a context on another device, a
 * request whose estimated peak memory exceeds the whole budget (the context
 * is then left to the caller).  STATE: ctx already finalized or the server
 * is shutting down. */
snc_status snc_server_submit(snc_server* srv, snc_ctx* ctx, uint64_t* ticket);

/* Non-blocking state of a request.  With state DONE and view != NULL, *view
 * receives the device views (as snc_get_connections).  For FAILED the
 * build's status is returned and snc_last_error(NULL) has its reason.
 * INVALID_ARG: unknown or released ticket. */
snc_status snc_server_poll(snc_server* srv, uint64_t ticket, snc_job_state* state, snc_conn_view* view);

/* Blocks until some request not yet reported by this call is DONE or FAILED,
 * or until timeout_ms passes (negative: no limit).  *ticket = the finished
 * request, 0 on timeout.  Every request is reported once, in completion
 * order.  INVALID_ARG: null ticket pointer. */
snc_status snc_server_wait_any(snc_server* srv, int timeout_ms, uint64_t* ticket);

/* The request's context (to call the read-only functions on once DONE).
 * INVALID_ARG: unknown or released ticket. */
snc_status snc_server_context(snc_server* srv, uint64_t ticket, snc_ctx** ctx);

/* Queue, build and total latency of a finished request.
 * INVALID_ARG: unknown ticket; STATE: not finished yet. */
snc_status snc_server_times(snc_server* srv, uint64_t ticket, snc_job_times* out);

/* Frees a finished request's network and its budget reservation (a network
 * built in a batch frees its memory when the last network of that batch is
 * released).  INVALID_ARG: unknown ticket; STATE: still queued or running. */
snc_status snc_server_release(snc_server* srv, uint64_t ticket);

/* Counters of the server.  INVALID_ARG on null pointers. */
snc_status snc_server_get_stats(snc_server* srv, snc_server_stats* out);

/* Estimated device memory of finalizing ctx: the peak during the build and
 * the part that stays resident, and the estimated connection count (exact
 * except for pairwise_bernoulli, whose estimate is an upper bound with
 * overwhelming probability).  INVALID_ARG: null pointers. */
snc_status snc_estimate_build(const snc_ctx* ctx, uint64_t* peak_bytes, uint64_t* resident_bytes,
                              uint64_t* n_syn);

#ifdef __cplusplus
}
#endif

#endif /* SNC_SERVER_H */
