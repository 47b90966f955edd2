/*
 * snc.h -- C ABI of libsnc: construction of spiking-network connectivity
 * directly in GPU memory (Golosio et al., "Runtime Construction of
 * Large-Scale Spiking Neuronal Network Models on GPU Devices",
 * arXiv 2306.09855).
 *
 * The calls follow the paper's statement of the problem (Sec. 2.1, 2.6):
 * populations are created (Create), connected by high-level rules
 * (Connect(sources, targets, conn_dict, syn_dict)), and the calibration
 * phase (triggered by Simulate in the paper, snc_finalize here) generates the
 * connections, sorts them by source and delay and builds the group index that
 * spike delivery reads (Sec. 2.2).
 *
 * Conventions for every call:
 *   - Every function returns an snc_status; nothing throws or aborts across
 *     the ABI.  snc_last_error() gives a human-readable reason for the last
 *     failing call on a context.
 *   - Node ids are uint32, connection counts and offsets uint64.
 *   - Device pointers are plain CUDA device addresses of the context's device;
 *     host pointers are ordinary host memory.
 *   - A context is not thread-safe; distinct contexts may be used from
 *     distinct threads.
 */
#ifndef SNC_H
#define SNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snc_ctx snc_ctx;

typedef enum {
  SNC_OK = 0,
  SNC_ERR_INVALID_ARG = 1, /* bad argument or rule parameters (checked up front) */
  SNC_ERR_STATE = 2,       /* call not allowed in the context's current state    */
  SNC_ERR_OOM = 3,         /* device or host allocation failed                   */
  SNC_ERR_CUDA = 4,        /* a CUDA runtime call failed                         */
  SNC_ERR_TIMEOUT = 5,     /* a bounded device wait or redraw loop gave up       */
  SNC_ERR_UNSUPPORTED = 6  /* valid request outside this build's limits          */
} snc_status;

/* Connection rules.  Sec. 2.1 defines one_to_one, all_to_all,
 * fixed_indegree, fixed_outdegree and fixed_total_number (each with
 * multapses); Sec. 4 names pairwise_bernoulli and the option to forbid
 * autapses and multapses. */
typedef enum {
  SNC_ONE_TO_ONE = 0,
  SNC_ALL_TO_ALL = 1,
  SNC_FIXED_INDEGREE = 2,
  SNC_FIXED_OUTDEGREE = 3,
  SNC_FIXED_TOTAL_NUMBER = 4,
  SNC_PAIRWISE_BERNOULLI = 5
} snc_rule_kind;

/* A contiguous node range [first, first + n) (Sec. 2.1: "both the source-node
 * group and the target-node group contain nodes with consecutive indexes"). */
typedef struct {
  uint32_t first;
  uint32_t n;
} snc_range;

/* conn_dict of Sec. 2.1.  k: K of fixed_indegree / fixed_outdegree, or the
 * total N of fixed_total_number.  p: probability of pairwise_bernoulli.
 * allow_autapses / allow_multapses: nonzero to allow (the paper's only mode). */
typedef struct {
  int32_t kind; /* snc_rule_kind */
  int32_t allow_autapses;
  int32_t allow_multapses;
  int32_t reserved;
  uint64_t k;
  double p;
} snc_conn_rule;

typedef enum { SNC_DIST_CONST = 0, SNC_DIST_NORMAL = 1 } snc_dist_kind;

/* A constant value (std ignored) or a normal distribution N(mean, std). */
typedef struct {
  int32_t kind; /* snc_dist_kind */
  int32_t reserved;
  double mean;
  double std;
} snc_dist;

/* syn_dict of Sec. 2.1: weights (any unit) and delays in milliseconds.  The
 * delay becomes an integer number of time steps, round(d / dt), at least 1. */
typedef struct {
  snc_dist weight;
  snc_dist delay_ms;
} snc_syn_spec;

/* Optional device-memory provider.  alloc returns a 256-byte aligned device
 * pointer of at least `bytes` usable in stream order on `stream` (NULL on
 * failure); free releases it in stream order.  Used for every device buffer
 * of a context. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} snc_allocator;

typedef struct {
  uint64_t seed;    /* seed of the counter-based random stream                */
  double dt_ms;     /* simulation time step (ms) > 0                           */
  int32_t device;   /* CUDA device ordinal                                     */
  int32_t reserved;
  void* stream;     /* cudaStream_t for all device work; NULL = default stream */
  const snc_allocator* allocator; /* NULL: cudaMallocAsync / cudaFreeAsync    */
} snc_config;

/* Device views of a finalized network, sorted stably by (source, delay
 * step) (Sec. 2.2 sorts by these two keys): connections with equal source and
 * delay keep their generation order (the order of the Connect calls, then
 * the rule's connection numbering of Sec. 2.1), so targets are NOT ascending
 * within a group.  Arrays live on the context's device and stay valid until
 * snc_destroy.
 *   row_ptr[n_nodes + 1]: connections of source i are [row_ptr[i], row_ptr[i+1])
 *   target, delay (time steps >= 1), weight: [n_syn]
 *   group_ptr[n_nodes + 1]: p_i of Sec. 2.2 (groups of source i are
 *     [group_ptr[i], group_ptr[i+1]); entry n_nodes = n_groups)
 *   group_first[n_groups]: index of the first connection of each group
 *     (a group = consecutive connections with equal source and delay). */
typedef struct {
  uint64_t n_syn;
  uint64_t n_nodes;
  uint64_t n_groups;
  const uint64_t* row_ptr;
  const uint32_t* target;
  const uint16_t* delay;
  const float* weight;
  const uint64_t* group_ptr;
  const uint64_t* group_first;
} snc_conn_view;

/* Creates a context on cfg->device.  *out receives the handle (owned by the
 * caller, released with snc_destroy).  INVALID_ARG: null pointers, dt <= 0;
 * CUDA: the device cannot be selected. */
snc_status snc_create(const snc_config* cfg, snc_ctx** out);

/* Releases every buffer of the context (after waiting for its stream). */
snc_status snc_destroy(snc_ctx* ctx);

/* Create (Sec. 2.6, node creation): appends n nodes with contiguous global
 * ids; *first_id receives the first.  STATE after snc_finalize;
 * INVALID_ARG when the total would exceed 2^32 - 1 nodes. */
snc_status snc_create_population(snc_ctx* ctx, uint32_t n, uint32_t* first_id);

/* Connect (Sec. 2.1): records one projection from `src` to `tgt` with the
 * given rule and synapse specification; *proj_id (may be NULL) receives its
 * index.  Host-side only: validates and sizes the projection.
 * INVALID_ARG: range outside the created nodes, one_to_one with unequal
 * sizes, K or N larger than the candidates when multapses are forbidden,
 * probability outside [0, 1], std < 0, unknown rule or distribution.
 * UNSUPPORTED: delay above 65535 steps or threshold table too long.
 * STATE: after snc_finalize. */
snc_status snc_connect(snc_ctx* ctx, snc_range src, snc_range tgt, const snc_conn_rule* rule,
                       const snc_syn_spec* syn, uint32_t* proj_id);

/* Explicit node lists and per-connection values of one Connect call
 * (Sec. 2.1: sources and targets may be given as arrays of node ids, the
 * rule's index formulas then giving positions in the arrays; weights and
 * delays may be given per connection by arrays as long as the number of
 * connections).  Every pointer is host memory, read during the call only
 * (the library keeps its own copy); NULL leaves that part as in snc_connect.
 *   src_ids: src.n node ids in place of the range src (src.first ignored);
 *   tgt_ids: tgt.n node ids in place of the range tgt (tgt.first ignored);
 *   weights: n_conn weights in place of the weight distribution;
 *   delays_ms: n_conn delays (ms) in place of the delay distribution, each
 *     rounded to floor(d / dt + 1/2) steps, at least one.
 * Element i of weights / delays_ms belongs to connection number i of the
 * rule's numbering (one_to_one i; all_to_all a * Nt + b; fixed_indegree
 * b * K + j; fixed_outdegree a * K + j; fixed_total_number the slot); a
 * number whose pair is dropped as an autapse leaves its element unused;
 * pairwise_bernoulli takes no per-connection arrays (its count is drawn).
 * Positions and random draws are those of ranges of the same lengths, so
 * listing the ids of a range gives the range's network; an autapse is a pair
 * of equal node ids.  With multapses forbidden both lists must hold distinct
 * ids; with autapses forbidden so must the list a per-primary rule draws
 * from (sources of fixed_indegree and pairwise_bernoulli, targets of
 * fixed_outdegree). */
typedef struct {
  const uint32_t* src_ids;
  const uint32_t* tgt_ids;
  const float* weights;
  const float* delays_ms;
  uint64_t n_conn; /* elements of weights / delays_ms */
} snc_conn_arrays;

/* Connect with explicit arrays (Sec. 2.1), otherwise as snc_connect (arrays
 * may be NULL: then it is snc_connect).  INVALID_ARG in addition: an id at or
 * above the created nodes, a repeated id where distinct ids are required,
 * n_conn different from the rule's numbered connections, a non-finite delay,
 * per-connection arrays with pairwise_bernoulli.  UNSUPPORTED: a delay above
 * 65535 steps.  STATE after snc_finalize. */
snc_status snc_connect_arrays(snc_ctx* ctx, snc_range src, snc_range tgt, const snc_conn_rule* rule,
                              const snc_syn_spec* syn, const snc_conn_arrays* arrays, uint32_t* proj_id);

/* Calibration (Sec. 2.2, 2.6): generates every connection on the device,
 * sorts them stably by (source, delay step) and builds the CSR and group
 * index.
 * Work is queued on the context's stream; the call blocks only for the
 * small device->host reads that size variable-count rules (pairwise_bernoulli
 * counts; the pending counts of each redraw round of fixed_total_number
 * without multapses or autapses when it needs more than 64 rounds: below
 * that, the rounds are counted on the device and a redraw still pending
 * after the last one, probability below 10^-15, is reported as TIMEOUT by
 * snc_synchronize).  After it, snc_connect returns STATE.  UNSUPPORTED:
 * packed key wider than 64 bits or a sampler range beyond the shared-memory
 * bitmap. */
snc_status snc_finalize(snc_ctx* ctx);

/* Batched calibration (no counterpart in the paper, which builds one network
 * at a time; useful for parameter scans): finalizes n unfinalized contexts
 * of one device together, with one launch per stage for all of them.  The
 * members' nodes are concatenated internally; every random draw stays keyed
 * by the member's own seed and projection index, so each member's result is
 * identical to what snc_finalize would give it alone.  All device work runs
 * on ctxs[0]'s stream with ctxs[0]'s allocator; the members share the result
 * memory, which is released when the last of them is destroyed.  Views and
 * copies of each member work as for a single build.
 * INVALID_ARG: empty list, null or repeated context, different devices.
 * STATE: a context already finalized.  Other errors as snc_finalize. */
snc_status snc_batch_finalize(snc_ctx* const* ctxs, int n);

/* The same batched build, recorded as a CUDA graph so that the networks can
 * be rebuilt with new seeds by replaying the recorded device work
 * (snc_batch_rebuild): repeated trials of one model, as in the paper's
 * validation over many seeds (Sec. 2.7), or parameter scans over seeds.
 * The first build runs immediately and gives the same result as
 * snc_batch_finalize.  The build keeps all its temporary buffers (its peak
 * device memory stays allocated).  Stage timers report the first build.
 * Every rule is accepted.  Counts that a seed decides are kept on the
 * device: a pairwise_bernoulli projection is given a capacity of mean + 10
 * standard deviations + 32 of its Binomial total over ns * nt pairs (the
 * positions its draw leaves free are sorted past the network's connections
 * and are not part of any view), and fixed_total_number without autapses or
 * multapses runs a fixed number of redraw rounds, chosen so that a slot is
 * still pending after the last one with probability below 10^-12.
 * UNSUPPORTED: a total-number projection without multapses so dense that
 * the number of rounds would exceed 512.  Other errors as
 * snc_batch_finalize; CUDA if the capture fails. */
snc_status snc_batch_finalize_graph(snc_ctx* const* ctxs, int n);

/* Rebuilds every network of ctx's graph build (ctx: any member) with
 * seeds[m] for member m (n = number of members, in the order given to
 * snc_batch_finalize_graph), in place: the views keep their addresses;
 * connection counts (of networks with pairwise_bernoulli projections), group
 * counts and contents change, and the views follow at the next
 * snc_synchronize or snc_get_connections.
 * Asynchronous on the build's stream; waits for the previous build first.
 * Result = snc_batch_finalize of the same contexts with those seeds.
 * STATE: not a graph build.  INVALID_ARG: null pointers or n mismatch.
 * A replay that exceeds a bound fixed when the graph was recorded is
 * reported by the next snc_synchronize: UNSUPPORTED for a pairwise_bernoulli
 * total above its capacity, TIMEOUT for redraws still pending after the last
 * recorded round (both far less likely than 10^-12 per replay). */
snc_status snc_batch_rebuild(snc_ctx* ctx, const uint64_t* seeds, int n);

/* Waits for the context's queued work and reports device-side failures
 * (TIMEOUT for a bounded wait that expired, CUDA for a launch error). */
snc_status snc_synchronize(snc_ctx* ctx);

/* Fills *out with device views of the finalized network (no copy).
 * Synchronizes first.  STATE before snc_finalize. */
snc_status snc_get_connections(snc_ctx* ctx, snc_conn_view* out);

/* Copies the finalized network to host arrays of capacity `cap` (each may be
 * NULL to skip it): src, tgt (uint32), delay (uint16, steps), weight (float),
 * in sorted order.  INVALID_ARG when cap < n_syn. */
snc_status snc_copy_connections(snc_ctx* ctx, uint32_t* src, uint32_t* tgt, uint16_t* delay,
                                float* weight, uint64_t cap);

/* Copies the finalized network's index to host arrays (each may be NULL):
 * row_ptr and group_ptr (p_i) of n_nodes + 1 entries, group_first of
 * group_cap >= n_groups entries (Sec. 2.2).  With the target / delay /
 * weight arrays of snc_copy_connections this is the whole network (the
 * sources are implicit in row_ptr).  INVALID_ARG when group_cap < n_groups
 * and group_first is given. */
snc_status snc_copy_index(snc_ctx* ctx, uint64_t* row_ptr, uint64_t* group_ptr, uint64_t* group_first,
                          uint64_t group_cap);

/* The copies of snc_copy_connections (tgt, delay, weight; cap entries) and
 * snc_copy_index (row_ptr, group_ptr, group_first; group_cap entries) of one
 * finalized network, queued on the context's stream without waiting for
 * them.  Each array may be NULL to skip it; the arrays are caller-owned host
 * memory, page-locked for the copies to run while the host goes on (a
 * pageable array makes the call wait for its copy).  The call waits for the
 * build itself and reports its errors (as snc_synchronize); the arrays hold
 * the network once a later snc_synchronize(ctx) has returned SNC_OK, and
 * must not be read, written or freed before, nor the context destroyed
 * (snc_destroy waits for the copies).  Lets a caller copy one network while
 * the next one builds on another stream.  STATE before snc_finalize;
 * INVALID_ARG when cap < n_syn or group_cap < n_groups with group_first
 * given, before any copy is queued. */
snc_status snc_copy_network_async(snc_ctx* ctx, uint32_t* tgt, uint16_t* delay, float* weight, uint64_t cap,
                                  uint64_t* row_ptr, uint64_t* group_ptr, uint64_t* group_first,
                                  uint64_t group_cap);

/* Target shard (Sec. 4 names target-distributed construction as future
 * work): the build keeps only the connections whose target node is in
 * [first, first + n).  Every draw is keyed by (projection, node, slot), so a
 * rank that builds its shard regenerates exactly the connections the whole
 * network would give it, with no exchange between ranks; the shard's
 * connections come in the whole network's (source, delay, generation)
 * order, indexed over all source nodes.  Before snc_finalize (STATE after);
 * INVALID_ARG at snc_finalize when the range exceeds the nodes, and in a
 * batch (graph builds included): a shard is built alone. */
snc_status snc_set_target_shard(snc_ctx* ctx, uint32_t first, uint32_t n);

/* Spike delivery through the index (Sec. 2.3, the spike array).  Entry e of
 * the spike array names a source node src[e] (network-local id), the index
 * grp[e] of one of its connection groups (0 = the group of its smallest
 * delay; the source's groups are group_first[group_ptr[src] ...
 * group_ptr[src + 1] - 1]) and a multiplicity mult[e].  For every connection
 * of that group, weight * mult[e] is added to input[target]; input holds
 * n_nodes floats and is accumulated into, not cleared.  All four arrays are
 * device memory; the additions run on the context's stream in no fixed
 * order (fp32 atomics).  Synchronous: returns when the delivery is done.
 * INVALID_ARG when an entry names no group (the other entries are still
 * delivered), STATE before snc_finalize. */
snc_status snc_deliver(snc_ctx* ctx, const uint32_t* src, const uint32_t* grp, const float* mult,
                       uint64_t n_spikes, float* input);

/* Device time of each finalize stage (ms) after snc_synchronize:
 * [0] count, [1] generate, [2] histogram, [3..3+P) sort passes, then index.
 * *n_stages receives the number written (at most max_stages); *n_passes the
 * number of sort stages P: the radix passes, or 1 when the build was sorted
 * per source (snc_stats.source_major; [2] is then the per-source offsets and
 * [3] the per-source sort).  STATE before a finalize has completed. */
snc_status snc_stage_times(snc_ctx* ctx, float* ms, int max_stages, int* n_stages, int* n_passes);

/* Process-wide kernel parameters (the autotuner's knobs).  They change
 * speed only, never results: every draw is keyed by (projection, node, slot)
 * and the sort is stable whatever its digit width. */
typedef struct {
  int32_t sort_digit_bits;   /* widest radix digit: 8..11 bits              */
  int32_t sort_group_tiles;  /* 4096-key tiles per look-back unit: 1, 4, 8;
                              * 0 = one tile, loaded by bulk copy (8-9 bit digits) */
  int32_t gen_blocks_per_sm; /* generation grid = SMs x this (1..32)        */
  int32_t sort_items;        /* bulk-copy pass: keys per thread, 8, 12, 16, 24 or 32 */
  int32_t reserved[4];       /* must be 0                                    */
} snc_tuning;

/* Sets the parameters for later snc_finalize / sort calls of this process.
 * INVALID_ARG for values outside the ranges above. */
snc_status snc_set_tuning(const snc_tuning* t);

/* Reads the current parameters. */
snc_status snc_get_tuning(snc_tuning* t);

/* Counters of the last snc_finalize (and later copies) on a context. */
typedef struct {
  uint64_t kernel_launches; /* kernels this library launched                 */
  uint64_t h2d_bytes;       /* host -> device bytes copied                    */
  uint64_t d2h_bytes;       /* device -> host bytes copied                    */
  int32_t n_passes;         /* radix passes of the sort (0: source-major sort) */
  int32_t key_bits;         /* width of the packed (source, delay step) sort key */
  uint64_t device_bytes_peak; /* largest total of live device buffers          */
  int32_t source_major;     /* 1: every projection generates source by source
                             * (one_to_one, all_to_all, fixed_outdegree), so
                             * the sort was a per-source counting sort by
                             * delay step instead of radix passes            */
  int32_t reserved;
} snc_stats;

/* Fills *out with the context's counters.  INVALID_ARG on null pointers. */
snc_status snc_get_stats(const snc_ctx* ctx, snc_stats* out);

/* Stable LSD radix sort of n (key, value) pairs on the low `key_bits` bits of
 * the keys (Sec. 2.2 sorts connections with an extension of radix sort; this
 * is the same onesweep sort used by snc_finalize, exposed on its own).
 * keys_in / vals_in: device input (unchanged); keys_out / vals_out: device
 * output; the four buffers must not overlap.  stream: cudaStream_t (NULL =
 * default stream).  Scratch is allocated with cudaMallocAsync on `stream`
 * and released in stream order.  The call waits for the sort on `stream`
 * and reads its device error word, so a failure on the device is reported
 * here: TIMEOUT when a bounded look-back wait expired (the output is then not
 * sorted), CUDA for a launch or copy failure or another device error bit.
 * INVALID_ARG: null pointers with n > 0, key_bits outside [1, 64].
 * OOM: the scratch allocation failed. */
snc_status snc_radix_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                uint32_t* vals_out, uint64_t n, int key_bits, void* stream);

/* COPASS block sort (Appendix A of the paper: "COnstrained PArtition of
 * Sorted Subarrays"): sorts n (key, value) pairs stably on the low key_bits
 * bits of the keys, IN PLACE in keys / vals (device memory), keeping the
 * array's division in blocks of `block` pairs: every block is sorted, then
 * for each block in turn the remaining sorted blocks are partitioned by a
 * common threshold so that their left partitions hold that block's share,
 * which is gathered, the rest shifted to the end, and sorted into place.
 * Working memory: two blocks of pairs plus the radix sort's scratch for one
 * block (cudaMallocAsync on `stream`), instead of a second copy of all n
 * pairs; the price is about twice the data movement of snc_radix_sort_pairs.
 * block: a multiple of 1024, at most 256 blocks (n <= 256 * block).  The
 * call waits for the sort and reads its device error word (TIMEOUT: a
 * bounded look-back wait expired; CUDA: launch failure or another error
 * bit).  INVALID_ARG: null pointers with n > 0, key_bits outside [1, 64],
 * block not a multiple of 1024 or too small for n.  OOM: working memory. */
snc_status snc_block_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t n, int key_bits, uint64_t block,
                                void* stream);

/* Builds ctx with the COPASS block sort (blocks of `block` connections, a
 * multiple of 1024; 0 = the out-of-place radix sort, the default), for
 * networks whose out-of-place sort would not fit the device: the sort then
 * works in place with two blocks of working memory, and the sorted pairs are
 * unpacked in place (targets over the value array, weights over the key
 * array), so the build's peak device memory falls from about 26.5 to about
 * 14 bytes per connection plus 24 bytes per block connection.  Results are
 * identical to the default build.  Before snc_finalize (STATE after);
 * INVALID_ARG at snc_finalize for a target shard, in a batch, or when the
 * network needs more than 256 blocks. */
snc_status snc_set_block_sort(snc_ctx* ctx, uint64_t block);

/* Largest n accepted by snc_radix_sort_pairs_noalloc. */
#define SNC_NOALLOC_MAX_PAIRS (1u << 19)

/* The sort of snc_radix_sort_pairs for callers that must not allocate device
 * memory (no counterpart in the paper).  Examples: a simulation loop that has
 * handed all of the GPU's memory to its own pool, or latency-bound code that
 * cannot afford the device synchronisation cudaMalloc / cudaFree may cause.
 * It calls no allocator: its working memory (look-back words, histograms,
 * the ping-pong buffers and an error word) is one 8 MiB file-scope device
 * array that every GPU loading the library holds until the process exits.
 * Arguments, layout and result are those of snc_radix_sort_pairs; the caller
 * passes the input and output buffers.
 * Limits and rules:
 *   - n <= SNC_NOALLOC_MAX_PAIRS, else INVALID_ARG (nothing is queued);
 *   - it sorts with a fixed digit plan (digits of at most 9 bits), whatever
 *     snc_set_tuning chose for the other sorts, so that its scratch fits the
 *     array for every accepted n and key width; UNSUPPORTED (scratch does
 *     not fit) is kept as a guard and cannot occur with that plan;
 *   - the first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     The address is cached per device ordinal for the process: calls after
 *     cudaDeviceReset (which reloads the module) are not supported;
 *   - every call shares the one array: calls whose work can overlap on the
 *     GPU (other streams, other host threads) race and must be serialised
 *     by the caller.  Each call clears what it needs before use.
 * The call waits for the sort on `stream` and reads the array's error word:
 * TIMEOUT when a bounded look-back wait expired (the output is then not
 * sorted), CUDA for a launch or copy failure or another device error bit. */
snc_status snc_radix_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                        uint32_t* vals_out, uint64_t n, int key_bits, void* stream);

/* Test support for the bounded device waits (no counterpart in the paper).
 * Every wait of the sort's decoupled look-back is bounded; this call lets a
 * test make such a wait expire without faulting or holding the GPU, to check
 * that the expiry is reported as TIMEOUT and that later calls work.
 * lookback_spin_limit: polling rounds of each look-back wait before it gives
 * up (0 = the built-in bound, about 4e6 rounds with back-off);
 * withhold_tile: the tile (of each sort pass) that never publishes its
 * look-back words, so that every later tile's wait runs to its bound
 * (0xFFFFFFFF = none, the default).  Process-wide, for sorts queued after the
 * call (snc_finalize, the batched forms and the stand-alone sorts).  A
 * timed-out tile still writes only inside its output arrays.  Reset with
 * snc_set_wait_test(0, 0xFFFFFFFF). */
snc_status snc_set_wait_test(uint32_t lookback_spin_limit, uint32_t withhold_tile);

/* Test support for the bounds a graph-recorded build fixes when it is
 * recorded (snc_batch_finalize_graph; no counterpart in the paper): the
 * capacity of each pairwise_bernoulli projection is its Binomial mean +
 * bernoulli_sd standard deviations + bernoulli_slack (defaults 10 and 32),
 * and fixed_total_number without multapses runs redraw_rounds rounds (0 =
 * the number computed from the density, the default).  Smaller values let a
 * test make a replay exceed them: the replay then writes only inside its
 * arrays and the next snc_synchronize reports UNSUPPORTED (a Bernoulli total
 * above its capacity) or TIMEOUT (redraws still pending).  Process-wide, for
 * graph builds recorded after the call; redraw_rounds also sets the rounds of
 * plain builds that count their redraw rounds on the device (snc_finalize).
 * INVALID_ARG: a negative value.
 * Reset with snc_set_graph_test(10, 32, 0). */
snc_status snc_set_graph_test(double bernoulli_sd, double bernoulli_slack, uint32_t redraw_rounds);

/* Readable description of the last failure on ctx (or of the last
 * context-free failure when ctx is NULL).  Never NULL. */
const char* snc_last_error(const snc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SNC_H */
