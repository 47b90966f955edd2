/*
 * snc_oracle.c -- plain, slow CPU oracle for spiking-network connectivity
 * construction (arXiv 2306.09855, "Runtime Construction of Large-Scale
 * Spiking Neuronal Network Models on GPU Devices").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table generator with the CUDA
 * path: every formula below is written from the paper and from the bit-level
 * random-stream contract that both sides implement independently.
 *
 * What it computes, in the paper's order:
 *   1. node ids: contiguous, 0-based, in population-creation order (Sec. 2.1);
 *   2. connections of each Connect call in the rule's own numbering
 *      i_newconns (Sec. 2.1, Eqs. 2-3 and the per-rule index formulas), on
 *      node ranges or on explicit node-id arrays (the formulas then give
 *      positions in the arrays);
 *   3. weight and integer delay of every connection, drawn or given per
 *      connection by arrays (Sec. 2.1, last paragraph: delay = round(d / dt),
 *      at least one step);
 *   4. a stable sort by (source, delay) (Sec. 2.2: source first, delay
 *      second; connections equal in both keep their generation order);
 *   5. the group index: a connection starts a group when its source or its
 *      delay differs from the previous one; G_i groups per source and
 *      p_i = sum_{j<i} G_j (Sec. 2.2, Eq. for p_i).
 *
 * Precision: index, delay and count decisions are integer; the threshold
 * tables that turn a 32-bit uniform into a delay step or a binomial count
 * are evaluated in IEEE double with the operation order the contract fixes;
 * weights are evaluated in double and rounded once to float.
 *
 * Parity status of each function is stated at its definition.  Compile with
 * -O2 -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Status codes (same meaning as the public library's, values fixed here).  */
enum {
  OR_OK = 0,
  OR_ERR_INVALID_ARG = 1,
  OR_ERR_STATE = 2,
  OR_ERR_OOM = 3,
  OR_ERR_CUDA = 4,
  OR_ERR_TIMEOUT = 5,
  OR_ERR_UNSUPPORTED = 6
};

/* Connection rules (Sec. 2.1 list, plus pairwise Bernoulli from Sec. 4). */
enum {
  OR_ONE_TO_ONE = 0,
  OR_ALL_TO_ALL = 1,
  OR_FIXED_INDEGREE = 2,
  OR_FIXED_OUTDEGREE = 3,
  OR_FIXED_TOTAL_NUMBER = 4,
  OR_PAIRWISE_BERNOULLI = 5
};

enum { OR_DIST_CONST = 0, OR_DIST_NORMAL = 1 };

/* Stream tags of the random-number contract. */
#define OR_TAG_WD 0u    /* weight + delay (+ one endpoint) of a slot   */
#define OR_TAG_IDX 1u   /* endpoint draws, four per call                */
#define OR_TAG_COUNT 2u /* per-target Bernoulli count                   */
#define OR_TAG_DEDUP 3u /* redraws of fixed_total_number, round >= 1    */
#define OR_PRIMARY_NONE 0xFFFFFFFFu

#define OR_MAX_DELAY_STEP 65535u
#define OR_MAX_TABLE 16384
#define OR_MAX_ROUND 0xFFFFFFu

/* One Connect call.  Mirrors the argument list of Connect(sources, targets,
 * conn_dict, syn_dict) in Sec. 2.1.  Sources and targets are contiguous node
 * ranges, or explicit arrays of node ids (Sec. 2.1: the index formulas then
 * give positions in the arrays, src_n / tgt_n their lengths).  Weights and
 * delays follow their distributions, or per-connection arrays (Sec. 2.1)
 * whose element i belongs to connection number i_newconns = i of the rule's
 * own numbering (w_arr, d_arr in ms; n_arr elements; NULL = none). */
typedef struct {
  uint32_t src_first, src_n, tgt_first, tgt_n;
  int32_t rule;
  int32_t allow_autapses, allow_multapses;
  int32_t pad0;
  uint64_t k;   /* K for in/out-degree, N for total number */
  double p;     /* pairwise Bernoulli probability */
  int32_t w_kind, d_kind;
  double w_mean, w_std;
  double d_mean, d_std; /* milliseconds */
  const uint32_t* src_ids; /* src_n ids, or NULL for the range */
  const uint32_t* tgt_ids; /* tgt_n ids, or NULL for the range */
  const float* w_arr;
  const float* d_arr;
  uint64_t n_arr;
} or_proj;

/* Node id at position a of the source list and at position b of the target
 * list (a range: first + position). */
static uint32_t src_node(const or_proj* pj, uint32_t a) {
  return pj->src_ids ? pj->src_ids[a] : pj->src_first + a;
}

static uint32_t tgt_node(const or_proj* pj, uint32_t b) {
  return pj->tgt_ids ? pj->tgt_ids[b] : pj->tgt_first + b;
}

typedef struct {
  uint64_t seed;
  double dt;
  uint32_t n_nodes;
  uint32_t n_proj;
} or_net;

/* ======================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random       */
/* numbers: as easy as 1, 2, 3").  Ten rounds of the 4x32 Philox S-box:     */
/* two 32x32->64 multiplications by fixed odd constants, the high halves    */
/* xor-ed with the other counter words and the round key; the key is        */
/* bumped by two Weyl constants between rounds.                             */
/* Pinned against the cuRAND host-side PHILOX4_32_10 generator (a black-box */
/* library routine) in tests/test_oracle_rng.py.                            */
/* ======================================================================== */
static void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c[1] ^ k0;
    uint32_t n1 = (uint32_t)prod1;
    uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c[3] ^ k1;
    uint32_t n3 = (uint32_t)prod0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
  }
}

/* Exported for the Philox pin: n counters (4 words each) -> 4n words. */
void or_philox(const uint32_t* counters, uint32_t k0, uint32_t k1, uint64_t n,
               uint32_t* out) {
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t c[4] = {counters[4 * i], counters[4 * i + 1], counters[4 * i + 2],
                     counters[4 * i + 3]};
    philox4x32_10(c, k0, k1);
    memcpy(out + 4 * i, c, sizeof c);
  }
}

/* The contract's stream: key = (seed lo, seed hi xor projection index);
 * counter = (slot lo, primary node, tag | round << 8, slot hi). */
static void draw(const or_net* net, uint32_t proj, uint32_t tag, uint32_t round,
                 uint32_t primary, uint64_t slot, uint32_t out[4]) {
  uint32_t k0 = (uint32_t)net->seed;
  uint32_t k1 = (uint32_t)(net->seed >> 32) ^ proj;
  out[0] = (uint32_t)slot;
  out[1] = primary;
  out[2] = tag | (round << 8);
  out[3] = (uint32_t)(slot >> 32);
  philox4x32_10(out, k0, k1);
}

/* rand(N) of Sec. 2.1: a uniform integer in [0, N) from one 32-bit word,
 * taken as floor(u * N / 2^32). */
static uint32_t rand_below(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* A random endpoint in a range of n nodes; when `skip` is set the node with
 * local index skip_local (the other endpoint itself) is left out, so an
 * autapse can never be drawn. */
static uint32_t draw_endpoint(uint32_t u, uint32_t n, int skip, uint32_t skip_local) {
  if (!skip) return rand_below(u, n);
  uint32_t r = rand_below(u, n - 1u);
  if (r >= skip_local) r += 1u;
  return r;
}

/* ======================================================================== */
/* Threshold tables: value(u) = base + #{ i : T[i] <= u } for a uniform      */
/* 32-bit word u, where T[i] = floor(2^32 * F(base + i)) and F is the CDF    */
/* of the integer variable.  Entries with T = 0 are folded into `base`;      */
/* the table ends before the first entry equal to 2^32.                      */
/* ======================================================================== */

/* Delay steps, Sec. 2.1: step = max(1, round(d / dt)) with d ~ N(mu, sigma).
 * P(step <= k) = P(d < (k + 1/2) dt) = Phi(((k + 1/2) dt - mu) / sigma) for
 * k >= 1, so the clip to one step is built in.
 * Pinned by tests/test_oracle_tables.py against scipy.stats.norm.cdf and by
 * a chi-square test of sampled steps. */
int or_delay_table(double mu, double sigma, double dt, uint32_t* thr, int cap,
                   uint32_t* base, int* len) {
  if (!(dt > 0.0) || !(sigma > 0.0) || !isfinite(mu) || !isfinite(sigma)) return OR_ERR_INVALID_ARG;
  uint32_t k = 1;
  uint64_t t = 0;
  for (;; ++k) {
    if (k > OR_MAX_DELAY_STEP) return OR_ERR_UNSUPPORTED;
    double x = (((double)k + 0.5) * dt - mu) / sigma;
    double phi = 0.5 * erfc(-x * M_SQRT1_2);
    t = (uint64_t)floor(ldexp(phi, 32));
    if (t > 0) break;
  }
  *base = k;
  int n = 0;
  while (t < (1ull << 32)) {
    if (n >= cap || n >= OR_MAX_TABLE) return OR_ERR_UNSUPPORTED;
    thr[n++] = (uint32_t)t;
    ++k;
    if (k > OR_MAX_DELAY_STEP) return OR_ERR_UNSUPPORTED;
    double x = (((double)k + 0.5) * dt - mu) / sigma;
    double phi = 0.5 * erfc(-x * M_SQRT1_2);
    t = (uint64_t)floor(ldexp(phi, 32));
  }
  *len = n;
  return OR_OK;
}

/* Binomial(n, p) counts for the pairwise Bernoulli rule (Sec. 4 names the
 * rule; the count of a target is the number of successes in its n
 * independent trials).  The pmf is built outward from the mode by the ratio
 * recurrence pmf(k+1)/pmf(k) = (n-k)/(k+1) * p/(1-p), truncated where it
 * falls below 1e-20 of the mode, normalised by its ascending sum.
 * Pinned by tests/test_oracle_tables.py against scipy.stats.binom.cdf. */
int or_binom_table(uint64_t n, double p, uint32_t* thr, int cap, uint64_t* base,
                   int* len) {
  *len = 0;
  if (!(p >= 0.0) || !(p <= 1.0)) return OR_ERR_INVALID_ARG;
  if (n == 0 || p == 0.0) {
    *base = 0;
    return OR_OK;
  }
  if (p == 1.0) {
    *base = n;
    return OR_OK;
  }
  double r = p / (1.0 - p);
  uint64_t mode = (uint64_t)floor(((double)n + 1.0) * p);
  if (mode > n) mode = n;
  /* Upward and downward ratio walks from the mode. */
  int cap_walk = 4 * OR_MAX_TABLE;
  double* up = (double*)malloc(sizeof(double) * (size_t)cap_walk);
  double* dn = (double*)malloc(sizeof(double) * (size_t)cap_walk);
  if (!up || !dn) {
    free(up);
    free(dn);
    return OR_ERR_OOM;
  }
  int n_up = 0, n_dn = 0;
  double w = 1.0;
  for (uint64_t k = mode; k < n; ++k) {
    double nxt = (w * ((double)(n - k) / (double)(k + 1))) * r;
    if (nxt < 1e-20) break;
    if (n_up >= cap_walk) {
      free(up);
      free(dn);
      return OR_ERR_UNSUPPORTED;
    }
    up[n_up++] = nxt;
    w = nxt;
  }
  w = 1.0;
  for (uint64_t k = mode; k > 0; --k) {
    double nxt = (w * ((double)k / (double)(n - k + 1))) / r;
    if (nxt < 1e-20) break;
    if (n_dn >= cap_walk) {
      free(up);
      free(dn);
      return OR_ERR_UNSUPPORTED;
    }
    dn[n_dn++] = nxt;
    w = nxt;
  }
  /* Ascending order: dn reversed, the mode, then up. */
  uint64_t lo = mode - (uint64_t)n_dn;
  int span = n_dn + 1 + n_up;
  double* pmf = (double*)malloc(sizeof(double) * (size_t)span);
  if (!pmf) {
    free(up);
    free(dn);
    return OR_ERR_OOM;
  }
  for (int i = 0; i < n_dn; ++i) pmf[i] = dn[n_dn - 1 - i];
  pmf[n_dn] = 1.0;
  for (int i = 0; i < n_up; ++i) pmf[n_dn + 1 + i] = up[i];
  free(up);
  free(dn);
  double total = 0.0;
  for (int i = 0; i < span; ++i) total += pmf[i];
  double cum = 0.0;
  int found_base = 0;
  int cnt = 0;
  int status = OR_OK;
  for (int i = 0; i < span; ++i) {
    cum += pmf[i];
    uint64_t t = (uint64_t)floor(ldexp(cum / total, 32));
    if (t >= (1ull << 32)) break;
    if (t == 0) continue;
    if (!found_base) {
      *base = lo + (uint64_t)i;
      found_base = 1;
    }
    if (cnt >= cap || cnt >= OR_MAX_TABLE) {
      status = OR_ERR_UNSUPPORTED;
      break;
    }
    thr[cnt++] = (uint32_t)t;
  }
  if (!found_base) {
    /* All mass in one value: the first k whose cumulative reaches 2^32. */
    cum = 0.0;
    for (int i = 0; i < span; ++i) {
      cum += pmf[i];
      if ((uint64_t)floor(ldexp(cum / total, 32)) >= (1ull << 32)) {
        *base = lo + (uint64_t)i;
        break;
      }
    }
  }
  free(pmf);
  *len = cnt;
  return status;
}

static uint64_t table_value(uint64_t base, const uint32_t* thr, int len, uint32_t u) {
  uint64_t v = base;
  for (int i = 0; i < len; ++i)
    if (thr[i] <= u) v += 1;
  return v;
}

/* Weight of one connection: constant, or normal by the Box-Muller transform
 * (one cosine branch) of two 24-bit uniforms u1 in (0, 1], u2 in [0, 1).
 * Evaluated in double, rounded once to float.
 * Pinned by tests/test_oracle_tables.py: moments, a Kolmogorov-Smirnov test
 * against the normal CDF, and the closed-form values at u2 = 0 and u1 = 1. */
float or_normal_weight(double mu, double sigma, uint32_t w2, uint32_t w3) {
  double u1 = ((double)(w2 >> 8) + 1.0) * 0x1p-24;
  double u2 = (double)(w3 >> 8) * 0x1p-24;
  double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
  return (float)(mu + sigma * z);
}

/* Vector form of or_normal_weight for distribution tests. */
void or_normal_weights(double mu, double sigma, const uint32_t* w2, const uint32_t* w3, uint64_t n,
                       float* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = or_normal_weight(mu, sigma, w2[i], w3[i]);
}

/* ======================================================================== */
/* Per-projection state the generators need.                                */
/* ======================================================================== */
typedef struct {
  uint32_t d_const; /* delay step when the delay is constant   */
  uint32_t d_base;
  int d_len;
  uint32_t* d_thr;
  double dt;        /* for per-connection delays in ms          */
  /* Bernoulli tables for the two possible numbers of candidates. */
  uint64_t b_base[2];
  int b_len[2];
  uint32_t* b_thr[2];
  /* Explicit id arrays: position of each node in the source (0) and target
   * (1) array, OR_ABSENT where it is not listed. */
  uint32_t* pos[2];
} or_tables;

#define OR_ABSENT 0xFFFFFFFFu

static void free_tables(or_tables* t) {
  free(t->d_thr);
  free(t->b_thr[0]);
  free(t->b_thr[1]);
  free(t->pos[0]);
  free(t->pos[1]);
  memset(t, 0, sizeof *t);
}

/* Sec. 2.1: a delay in ms becomes round(d / dt) steps, at least one.  Round
 * half up, in double.  Non-finite delays are INVALID_ARG, steps above the
 * 16-bit delay field UNSUPPORTED. */
static int delay_step_ms(double d, double dt, uint32_t* step) {
  if (!isfinite(d)) return OR_ERR_INVALID_ARG;
  double q = floor(d / dt + 0.5);
  if (!(q == q)) return OR_ERR_INVALID_ARG;
  if (q < 1.0) q = 1.0;
  if (q > (double)OR_MAX_DELAY_STEP) return OR_ERR_UNSUPPORTED;
  *step = (uint32_t)q;
  return OR_OK;
}

/* Number of position pairs (a, b) whose nodes coincide,
 * #{(a, b) : src_node(a) == tgt_node(b)}: the autapses among all pairs.
 * For two ranges it is the length of their overlap. */
static int equal_pairs(const or_net* net, const or_proj* pj, uint64_t* out) {
  if (!pj->src_ids && !pj->tgt_ids) {
    uint64_t a0 = pj->src_first, a1 = (uint64_t)pj->src_first + pj->src_n;
    uint64_t b0 = pj->tgt_first, b1 = (uint64_t)pj->tgt_first + pj->tgt_n;
    uint64_t lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
    *out = hi > lo ? hi - lo : 0;
    return OR_OK;
  }
  uint64_t* in_src = (uint64_t*)calloc(net->n_nodes ? net->n_nodes : 1, sizeof(uint64_t));
  if (!in_src) return OR_ERR_OOM;
  for (uint32_t a = 0; a < pj->src_n; ++a) in_src[src_node(pj, a)] += 1;
  uint64_t n = 0;
  for (uint32_t b = 0; b < pj->tgt_n; ++b) n += in_src[tgt_node(pj, b)];
  free(in_src);
  *out = n;
  return OR_OK;
}

/* 1 if some id appears twice in ids[0..n), ids all below n_nodes. */
static int has_duplicates(const uint32_t* ids, uint32_t n, uint32_t n_nodes, int* dup) {
  unsigned char* seen = (unsigned char*)calloc(n_nodes ? n_nodes : 1, 1);
  if (!seen) return OR_ERR_OOM;
  *dup = 0;
  for (uint32_t i = 0; i < n && !*dup; ++i) {
    if (seen[ids[i]]) *dup = 1;
    seen[ids[i]] = 1;
  }
  free(seen);
  return OR_OK;
}

/* Position of `node` in the source (which = 0) or target (1) list, or -1. */
static int64_t position_of(const or_proj* pj, const or_tables* t, int which, uint32_t node) {
  const uint32_t* ids = which ? pj->tgt_ids : pj->src_ids;
  if (ids) return t->pos[which][node] == OR_ABSENT ? -1 : (int64_t)t->pos[which][node];
  uint32_t first = which ? pj->tgt_first : pj->src_first;
  uint32_t n = which ? pj->tgt_n : pj->src_n;
  return node >= first && node - first < n ? (int64_t)(node - first) : -1;
}

static int make_tables(const or_net* net, const or_proj* pj, or_tables* t) {
  memset(t, 0, sizeof *t);
  t->dt = net->dt;
  for (int which = 0; which < 2; ++which) {
    const uint32_t* ids = which ? pj->tgt_ids : pj->src_ids;
    uint32_t n = which ? pj->tgt_n : pj->src_n;
    if (!ids) continue;
    t->pos[which] = (uint32_t*)malloc(sizeof(uint32_t) * (net->n_nodes ? net->n_nodes : 1));
    if (!t->pos[which]) return OR_ERR_OOM;
    for (uint32_t v = 0; v < net->n_nodes; ++v) t->pos[which][v] = OR_ABSENT;
    for (uint32_t i = 0; i < n; ++i) t->pos[which][ids[i]] = i;
  }
  if (pj->d_arr) {
    /* per-connection delays: converted one by one (delay_at) */
  } else if (pj->d_kind == OR_DIST_CONST || (pj->d_kind == OR_DIST_NORMAL && pj->d_std == 0.0)) {
    int st = delay_step_ms(pj->d_mean, net->dt, &t->d_const);
    if (st) return st;
  } else if (pj->d_kind == OR_DIST_NORMAL) {
    t->d_thr = (uint32_t*)malloc(sizeof(uint32_t) * OR_MAX_TABLE);
    if (!t->d_thr) return OR_ERR_OOM;
    int st = or_delay_table(pj->d_mean, pj->d_std, net->dt, t->d_thr, OR_MAX_TABLE,
                            &t->d_base, &t->d_len);
    if (st) return st;
    if ((uint64_t)t->d_base + (uint64_t)t->d_len > OR_MAX_DELAY_STEP) return OR_ERR_UNSUPPORTED;
  } else {
    return OR_ERR_INVALID_ARG;
  }
  if (pj->w_kind != OR_DIST_CONST && pj->w_kind != OR_DIST_NORMAL) return OR_ERR_INVALID_ARG;
  if (pj->rule == OR_PAIRWISE_BERNOULLI) {
    for (int s = 0; s < 2; ++s) {
      uint64_t cand = (uint64_t)pj->src_n - (uint64_t)s;
      if (s == 1 && pj->src_n == 0) cand = 0;
      t->b_thr[s] = (uint32_t*)malloc(sizeof(uint32_t) * OR_MAX_TABLE);
      if (!t->b_thr[s]) return OR_ERR_OOM;
      int st = or_binom_table(cand, pj->p, t->b_thr[s], OR_MAX_TABLE, &t->b_base[s], &t->b_len[s]);
      if (st) return st;
    }
  }
  return OR_OK;
}

static uint16_t delay_of(const or_tables* t, uint32_t u) {
  if (t->d_thr == NULL) return (uint16_t)t->d_const;
  return (uint16_t)table_value(t->d_base, t->d_thr, t->d_len, u);
}

static float weight_of(const or_proj* pj, uint32_t w2, uint32_t w3) {
  if (pj->w_kind == OR_DIST_CONST) return (float)pj->w_mean;
  return or_normal_weight(pj->w_mean, pj->w_std, w2, w3);
}

/* Delay and weight of connection number inew: the per-connection array's
 * element inew when there is one (checked before generation), else the
 * distribution's value from the slot's WD words. */
static uint16_t delay_at(const or_proj* pj, const or_tables* t, uint64_t inew, uint32_t u) {
  if (pj->d_arr) {
    uint32_t step = 1;
    delay_step_ms((double)pj->d_arr[inew], t->dt, &step);
    return (uint16_t)step;
  }
  return delay_of(t, u);
}

static float weight_at(const or_proj* pj, uint64_t inew, uint32_t w2, uint32_t w3) {
  return pj->w_arr ? pj->w_arr[inew] : weight_of(pj, w2, w3);
}

/* Output sink: arrays in generation order. */
typedef struct {
  uint32_t* src;
  uint32_t* tgt;
  uint16_t* delay;
  float* weight;
  uint64_t pos;
  uint64_t cap;
} or_sink;

static int emit(or_sink* out, uint32_t s, uint32_t t, uint16_t d, float w) {
  if (out->src) {
    if (out->pos >= out->cap) return OR_ERR_INVALID_ARG;
    out->src[out->pos] = s;
    out->tgt[out->pos] = t;
    out->delay[out->pos] = d;
    out->weight[out->pos] = w;
  }
  out->pos += 1;
  return OR_OK;
}

/* Weight and delay of slot `slot` of primary node `primary`, connection
 * number inew. */
static int emit_wd(const or_net* net, uint32_t proj, const or_proj* pj, const or_tables* t,
                   uint32_t primary, uint64_t slot, uint64_t inew, uint32_t s, uint32_t tg,
                   or_sink* out) {
  uint32_t w[4];
  draw(net, proj, OR_TAG_WD, 0, primary, slot, w);
  return emit(out, s, tg, delay_at(pj, t, inew, w[0]), weight_at(pj, inew, w[2], w[3]));
}

/* ------------------------------------------------------------------------ */
/* Sampling without replacement: the first `want` distinct values among the  */
/* attempts a = 0, 1, 2, ... of primary node `primary`, attempt a using word */
/* (a mod 4) of IDX draw floor(a / 4).  When more than half of the           */
/* candidates are wanted, the (candidates - want) excluded values are chosen */
/* by the same rule and the kept values are listed in ascending order.       */
/* Result: `want` local indices in slot order.                               */
/* Pinned by tests/test_oracle_rules.py: every k-subset of a small range is  */
/* equally frequent (chi-square), no duplicates, exact counts.               */
/* ------------------------------------------------------------------------ */
static int sample_distinct(const or_net* net, uint32_t proj, uint32_t primary, uint32_t n,
                           int skip, uint32_t skip_local, uint64_t want, uint32_t* sel) {
  uint64_t cand = (uint64_t)n - (skip ? 1u : 0u);
  if (want > cand) return OR_ERR_INVALID_ARG;
  if (want == 0) return OR_OK;
  int complement = 2 * want > cand;
  uint64_t need = complement ? cand - want : want;
  unsigned char* mark = (unsigned char*)calloc(n, 1);
  if (!mark) return OR_ERR_OOM;
  uint64_t got = 0;
  uint32_t w[4];
  for (uint64_t a = 0; got < need; ++a) {
    draw(net, proj, OR_TAG_IDX, 0, primary, a / 4, w);
    uint32_t r = draw_endpoint(w[a % 4], n, skip, skip_local);
    if (!mark[r]) {
      mark[r] = 1;
      if (!complement) sel[got] = r;
      ++got;
    }
  }
  if (complement) {
    uint64_t j = 0;
    for (uint32_t r = 0; r < n; ++r) {
      if (skip && r == skip_local) continue;
      if (!mark[r]) sel[j++] = r;
    }
  }
  free(mark);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Open-addressing set of (source, target) pairs for fixed_total_number     */
/* without multapses.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t* slots;
  uint64_t mask;
} pair_set;

static int pair_set_init(pair_set* ps, uint64_t n) {
  uint64_t cap = 16;
  while (cap < 2 * n + 16) cap <<= 1;
  ps->slots = (uint64_t*)malloc(sizeof(uint64_t) * cap);
  if (!ps->slots) return OR_ERR_OOM;
  for (uint64_t i = 0; i < cap; ++i) ps->slots[i] = ~0ull;
  ps->mask = cap - 1;
  return OR_OK;
}

/* Returns 1 if inserted, 0 if it was present. */
static int pair_set_insert(pair_set* ps, uint64_t key) {
  uint64_t h = key * 0x9E3779B97F4A7C15ull;
  uint64_t i = (h >> 17) & ps->mask;
  for (;;) {
    if (ps->slots[i] == ~0ull) {
      ps->slots[i] = key;
      return 1;
    }
    if (ps->slots[i] == key) return 0;
    i = (i + 1) & ps->mask;
  }
}

/* ======================================================================== */
/* The rules (Sec. 2.1 index formulas; Sec. 4 for Bernoulli and for the      */
/* autapse / multapse prohibitions).                                         */
/* ======================================================================== */

/* The connections of primary node b of a per-primary rule, in slot order:
 *   all_to_all:  primary = target b, slot a = source index (i = a*Nt + b is
 *                the paper's numbering; emitted per target here only for
 *                sampled checks);
 *   indegree:    primary = target b, s = source at rand(Ns), K slots,
 *                connection number i = b*K + j;
 *   outdegree:   primary = source b, t = target at rand(Nt), K slots,
 *                i = b*K + j;
 *   bernoulli:   primary = target b, count ~ Binomial(candidates, p), then
 *                that many distinct sources.
 * With autapses off the primary's own node, if the other list holds it (at
 * one position: such lists are checked to hold distinct ids), is left out
 * of the draws. */
static int gen_primary(const or_net* net, uint32_t proj, const or_proj* pj,
                       const or_tables* t, uint32_t b, uint32_t* sel, or_sink* out) {
  const uint32_t Ns = pj->src_n, Nt = pj->tgt_n;
  int st = OR_OK;
  if (pj->rule == OR_ALL_TO_ALL) {
    for (uint32_t a = 0; a < Ns && !st; ++a) {
      uint32_t s = src_node(pj, a), tg = tgt_node(pj, b);
      if (!pj->allow_autapses && s == tg) continue;
      st = emit_wd(net, proj, pj, t, b, a, (uint64_t)a * Nt + b, s, tg, out);
    }
    return st;
  }
  if (pj->rule == OR_PAIRWISE_BERNOULLI) {
    uint32_t node = tgt_node(pj, b);
    int64_t q = pj->allow_autapses ? -1 : position_of(pj, t, 0, node);
    int skip = q >= 0;
    uint32_t skip_local = skip ? (uint32_t)q : 0;
    uint32_t w[4];
    draw(net, proj, OR_TAG_COUNT, 0, b, 0, w);
    uint64_t nb = table_value(t->b_base[skip], t->b_thr[skip], t->b_len[skip], w[0]);
    st = sample_distinct(net, proj, b, Ns, skip, skip_local, nb, sel);
    /* no per-connection arrays for this rule (the count is drawn) */
    for (uint64_t j = 0; j < nb && !st; ++j)
      st = emit_wd(net, proj, pj, t, b, j, 0, src_node(pj, sel[j]), node, out);
    return st;
  }
  /* fixed_indegree / fixed_outdegree */
  int indeg = pj->rule == OR_FIXED_INDEGREE;
  uint32_t n_other = indeg ? Ns : Nt;
  uint64_t K = pj->k;
  uint32_t node = indeg ? tgt_node(pj, b) : src_node(pj, b);
  int64_t q = pj->allow_autapses ? -1 : position_of(pj, t, indeg ? 0 : 1, node);
  int skip = q >= 0;
  uint32_t skip_local = skip ? (uint32_t)q : 0;
  if (pj->allow_multapses) {
    for (uint64_t j = 0; j < K && !st; ++j) {
      uint32_t w[4];
      draw(net, proj, OR_TAG_WD, 0, b, j, w);
      uint32_t r = draw_endpoint(w[1], n_other, skip, skip_local);
      uint32_t other = indeg ? src_node(pj, r) : tgt_node(pj, r);
      uint32_t s = indeg ? other : node, tg = indeg ? node : other;
      uint64_t inew = (uint64_t)b * K + j;
      st = emit(out, s, tg, delay_at(pj, t, inew, w[0]), weight_at(pj, inew, w[2], w[3]));
    }
  } else {
    st = sample_distinct(net, proj, b, n_other, skip, skip_local, K, sel);
    for (uint64_t j = 0; j < K && !st; ++j) {
      uint32_t other = indeg ? src_node(pj, sel[j]) : tgt_node(pj, sel[j]);
      uint32_t s = indeg ? other : node, tg = indeg ? node : other;
      st = emit_wd(net, proj, pj, t, b, j, (uint64_t)b * K + j, s, tg, out);
    }
  }
  return st;
}

/* fixed_total_number: slot i draws the source at position rand(Ns) and the
 * target at position rand(Nt) (source from word 1 of its WD draw, target
 * from word i mod 4 of IDX draw floor(i/4)).  A slot whose pair is not
 * allowed (an autapse when autapses are off; with multapses off, a pair
 * already held by an accepted slot or drawn this round by a lower pending
 * slot) redraws in round r = 1, 2, ... from words 0 and 1 of its DEDUP draw
 * of that round, until every slot holds an allowed pair.  Visiting the
 * pending slots in ascending order with a running set of accepted pairs
 * applies exactly that rule.  Slot i is connection number i. */
static int gen_total_number(const or_net* net, uint32_t proj, const or_proj* pj,
                            const or_tables* t, or_sink* out) {
  const uint32_t Ns = pj->src_n, Nt = pj->tgt_n;
  uint64_t N = pj->k;
  if (N == 0) return OR_OK;
  int st = OR_OK;
  uint32_t* ps = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint32_t* pt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint64_t* pending = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
  pair_set set = {0, 0};
  if (!ps || !pt || !pending) st = OR_ERR_OOM;
  if (!st && !pj->allow_multapses) st = pair_set_init(&set, N);
  uint64_t n_pending = 0;
  for (uint64_t i = 0; i < N && !st; ++i) {
    uint32_t w[4], x[4];
    draw(net, proj, OR_TAG_WD, 0, OR_PRIMARY_NONE, i, w);
    draw(net, proj, OR_TAG_IDX, 0, OR_PRIMARY_NONE, i / 4, x);
    ps[i] = src_node(pj, rand_below(w[1], Ns));
    pt[i] = tgt_node(pj, rand_below(x[i % 4], Nt));
    int ok = pj->allow_autapses || ps[i] != pt[i];
    if (ok && !pj->allow_multapses) ok = pair_set_insert(&set, ((uint64_t)ps[i] << 32) | pt[i]);
    if (!ok) pending[n_pending++] = i;
  }
  for (uint32_t round = 1; n_pending > 0 && !st; ++round) {
    if (round > OR_MAX_ROUND) {
      st = OR_ERR_TIMEOUT;
      break;
    }
    uint64_t still = 0;
    for (uint64_t q = 0; q < n_pending; ++q) {
      uint64_t i = pending[q];
      uint32_t w[4];
      draw(net, proj, OR_TAG_DEDUP, round, OR_PRIMARY_NONE, i, w);
      ps[i] = src_node(pj, rand_below(w[0], Ns));
      pt[i] = tgt_node(pj, rand_below(w[1], Nt));
      int ok = pj->allow_autapses || ps[i] != pt[i];
      if (ok && !pj->allow_multapses) ok = pair_set_insert(&set, ((uint64_t)ps[i] << 32) | pt[i]);
      if (!ok) pending[still++] = i;
    }
    n_pending = still;
  }
  for (uint64_t i = 0; i < N && !st; ++i)
    st = emit_wd(net, proj, pj, t, OR_PRIMARY_NONE, i, i, ps[i], pt[i], out);
  free(ps);
  free(pt);
  free(pending);
  free(set.slots);
  return st;
}

static int gen_projection(const or_net* net, uint32_t proj, const or_proj* pj,
                          const or_tables* t, or_sink* out) {
  const uint32_t Ns = pj->src_n, Nt = pj->tgt_n;
  int st = OR_OK;
  switch (pj->rule) {
    case OR_ONE_TO_ONE:
      /* i = 0 .. N-1: source and target at position i; with autapses off a
       * pair with s == t is dropped (its number i stays unused). */
      for (uint32_t i = 0; i < Ns && !st; ++i) {
        uint32_t s = src_node(pj, i), tg = tgt_node(pj, i);
        if (!pj->allow_autapses && s == tg) continue;
        st = emit_wd(net, proj, pj, t, i, 0, i, s, tg, out);
      }
      return st;
    case OR_ALL_TO_ALL:
      /* i = a * Nt + b: source at position floor(i / Nt), target at
       * position i mod Nt; the draw of connection (a, b) is keyed by
       * primary = target b, slot = a. */
      for (uint32_t a = 0; a < Ns && !st; ++a)
        for (uint32_t b = 0; b < Nt && !st; ++b) {
          uint32_t s = src_node(pj, a), tg = tgt_node(pj, b);
          if (!pj->allow_autapses && s == tg) continue;
          st = emit_wd(net, proj, pj, t, b, a, (uint64_t)a * Nt + b, s, tg, out);
        }
      return st;
    case OR_FIXED_TOTAL_NUMBER:
      return gen_total_number(net, proj, pj, t, out);
    case OR_FIXED_INDEGREE:
    case OR_FIXED_OUTDEGREE:
    case OR_PAIRWISE_BERNOULLI: {
      uint32_t n_primary = pj->rule == OR_FIXED_OUTDEGREE ? Ns : Nt;
      uint64_t sel_n = pj->rule == OR_PAIRWISE_BERNOULLI ? (uint64_t)Ns + 1 : pj->k + 1;
      uint32_t* sel = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)sel_n);
      if (!sel) return OR_ERR_OOM;
      for (uint32_t b = 0; b < n_primary && !st; ++b) st = gen_primary(net, proj, pj, t, b, sel, out);
      free(sel);
      return st;
    }
    default:
      return OR_ERR_INVALID_ARG;
  }
}

/* Connections the rule numbers (i_newconns = 0 .. count-1), before autapse
 * drops: the length a per-connection weight or delay array must have. */
static uint64_t numbered_count(const or_proj* pj) {
  switch (pj->rule) {
    case OR_ONE_TO_ONE: return pj->src_n;
    case OR_ALL_TO_ALL: return (uint64_t)pj->src_n * pj->tgt_n;
    case OR_FIXED_INDEGREE: return (uint64_t)pj->tgt_n * pj->k;
    case OR_FIXED_OUTDEGREE: return (uint64_t)pj->src_n * pj->k;
    default: return pj->k;
  }
}

/* Argument checks done by Connect before anything is generated.
 * Explicit id arrays: every id below n_nodes; with multapses off both
 * arrays hold distinct ids (so distinct positions are distinct nodes); with
 * autapses off, the list a per-primary rule draws from (sources of
 * in-degree and Bernoulli, targets of out-degree) holds distinct ids (so
 * the primary's own node sits at one position).  Per-connection arrays:
 * not for pairwise_bernoulli (its count is drawn), numbered_count()
 * elements, delays finite and at most 65535 steps. */
int or_check_projection(const or_net* net, const or_proj* pj) {
  if (!(net->dt > 0.0)) return OR_ERR_INVALID_ARG;
  for (int which = 0; which < 2; ++which) {
    const uint32_t* ids = which ? pj->tgt_ids : pj->src_ids;
    uint32_t first = which ? pj->tgt_first : pj->src_first;
    uint32_t n = which ? pj->tgt_n : pj->src_n;
    if (!ids) {
      if ((uint64_t)first + n > net->n_nodes) return OR_ERR_INVALID_ARG;
      continue;
    }
    for (uint32_t i = 0; i < n; ++i)
      if (ids[i] >= net->n_nodes) return OR_ERR_INVALID_ARG;
    int draws_here = which ? pj->rule == OR_FIXED_OUTDEGREE
                           : pj->rule == OR_FIXED_INDEGREE || pj->rule == OR_PAIRWISE_BERNOULLI;
    if (!pj->allow_multapses || (!pj->allow_autapses && draws_here)) {
      int dup = 0;
      int st = has_duplicates(ids, n, net->n_nodes, &dup);
      if (st) return st;
      if (dup) return OR_ERR_INVALID_ARG;
    }
  }
  uint64_t ov = 0;
  int st = equal_pairs(net, pj, &ov);
  if (st) return st;
  switch (pj->rule) {
    case OR_ONE_TO_ONE:
      if (pj->src_n != pj->tgt_n) return OR_ERR_INVALID_ARG;
      break;
    case OR_ALL_TO_ALL:
      break;
    case OR_FIXED_INDEGREE:
    case OR_FIXED_OUTDEGREE: {
      int indeg = pj->rule == OR_FIXED_INDEGREE;
      uint64_t n_other = indeg ? pj->src_n : pj->tgt_n;
      uint64_t n_primary = indeg ? pj->tgt_n : pj->src_n;
      if (pj->k == 0 || n_primary == 0) break;
      if (pj->k > 0xFFFFFFFFull) return OR_ERR_INVALID_ARG;
      /* The fewest candidates any primary node has. */
      uint64_t least = n_other;
      if (!pj->allow_autapses && ov > 0) least = n_other - 1;
      if (least == 0) return OR_ERR_INVALID_ARG;
      if (!pj->allow_multapses && pj->k > least) return OR_ERR_INVALID_ARG;
      break;
    }
    case OR_FIXED_TOTAL_NUMBER: {
      if (pj->k == 0) break;
      uint64_t pairs = (uint64_t)pj->src_n * pj->tgt_n;
      uint64_t allowed = pairs - (pj->allow_autapses ? 0 : ov);
      if (allowed == 0) return OR_ERR_INVALID_ARG;
      if (!pj->allow_multapses && pj->k > allowed) return OR_ERR_INVALID_ARG;
      break;
    }
    case OR_PAIRWISE_BERNOULLI:
      if (!(pj->p >= 0.0 && pj->p <= 1.0)) return OR_ERR_INVALID_ARG;
      if (pj->w_arr || pj->d_arr) return OR_ERR_INVALID_ARG;
      break;
    default:
      return OR_ERR_INVALID_ARG;
  }
  if (pj->w_arr || pj->d_arr) {
    if (pj->n_arr != numbered_count(pj)) return OR_ERR_INVALID_ARG;
    for (uint64_t i = 0; pj->d_arr && i < pj->n_arr; ++i) {
      uint32_t step;
      st = delay_step_ms((double)pj->d_arr[i], net->dt, &step);
      if (st) return st;
    }
  }
  if (pj->d_kind != OR_DIST_CONST && pj->d_kind != OR_DIST_NORMAL) return OR_ERR_INVALID_ARG;
  if (pj->w_kind != OR_DIST_CONST && pj->w_kind != OR_DIST_NORMAL) return OR_ERR_INVALID_ARG;
  if (pj->d_kind == OR_DIST_NORMAL && !(pj->d_std >= 0.0)) return OR_ERR_INVALID_ARG;
  if (pj->w_kind == OR_DIST_NORMAL && !(pj->w_std >= 0.0)) return OR_ERR_INVALID_ARG;
  if (!isfinite(pj->d_mean) || !isfinite(pj->w_mean)) return OR_ERR_INVALID_ARG;
  return OR_OK;
}

/* Generate every projection in Connect order.  With null output arrays it
 * only counts.  per_proj (optional) receives each projection's count. */
int or_generate(const or_net* net, const or_proj* projs, uint32_t* src, uint32_t* tgt,
                uint16_t* delay, float* weight, uint64_t cap, uint64_t* n_out,
                uint64_t* per_proj) {
  or_sink out = {src, tgt, delay, weight, 0, cap};
  for (uint32_t p = 0; p < net->n_proj; ++p) {
    int st = or_check_projection(net, &projs[p]);
    if (st) return st;
  }
  for (uint32_t p = 0; p < net->n_proj; ++p) {
    or_tables t;
    uint64_t before = out.pos;
    int st = make_tables(net, &projs[p], &t);
    if (!st) st = gen_projection(net, p, &projs[p], &t, &out);
    free_tables(&t);
    if (st) return st;
    if (per_proj) per_proj[p] = out.pos - before;
  }
  *n_out = out.pos;
  return OR_OK;
}

/* The connections of one primary node of one projection, in slot order
 * (one_to_one: the pair i; all_to_all, indegree, Bernoulli: a target;
 * outdegree: a source).  Every draw is a function of (projection, primary,
 * slot), so this equals the matching run of or_generate's output; it lets
 * tests check sampled nodes of networks too large for the full oracle. */
int or_generate_primary(const or_net* net, const or_proj* projs, uint32_t proj,
                        uint32_t primary, uint32_t* src, uint32_t* tgt, uint16_t* delay,
                        float* weight, uint64_t cap, uint64_t* n_out) {
  if (proj >= net->n_proj) return OR_ERR_INVALID_ARG;
  const or_proj* pj = &projs[proj];
  int st = or_check_projection(net, pj);
  if (st) return st;
  uint32_t n_primary = pj->rule == OR_FIXED_OUTDEGREE || pj->rule == OR_ONE_TO_ONE ? pj->src_n
                                                                                   : pj->tgt_n;
  if (pj->rule == OR_FIXED_TOTAL_NUMBER) return OR_ERR_UNSUPPORTED;
  if (primary >= n_primary) return OR_ERR_INVALID_ARG;
  or_tables t;
  or_sink out = {src, tgt, delay, weight, 0, cap};
  st = make_tables(net, pj, &t);
  if (!st) {
    if (pj->rule == OR_ONE_TO_ONE) {
      uint32_t s = src_node(pj, primary), tg = tgt_node(pj, primary);
      if (pj->allow_autapses || s != tg)
        st = emit_wd(net, proj, pj, &t, primary, 0, primary, s, tg, &out);
    } else {
      uint64_t sel_n = pj->rule == OR_PAIRWISE_BERNOULLI || pj->rule == OR_ALL_TO_ALL
                           ? (uint64_t)pj->src_n + 1
                           : pj->k + 1;
      uint32_t* sel = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)sel_n);
      if (!sel) st = OR_ERR_OOM;
      if (!st) st = gen_primary(net, proj, pj, &t, primary, sel, &out);
      free(sel);
    }
  }
  free_tables(&t);
  *n_out = out.pos;
  return st;
}

/* ======================================================================== */
/* Sort and index (Sec. 2.2).                                                */
/* ======================================================================== */
typedef struct {
  uint32_t s, t;
  uint16_t d;
  float w;
  uint64_t gen; /* position in generation order: makes the sort stable */
} or_rec;

static int cmp_rec(const void* x, const void* y) {
  const or_rec* a = (const or_rec*)x;
  const or_rec* b = (const or_rec*)y;
  if (a->s != b->s) return a->s < b->s ? -1 : 1;
  if (a->d != b->d) return a->d < b->d ? -1 : 1;
  if (a->gen != b->gen) return a->gen < b->gen ? -1 : 1;
  return 0;
}

/* Sorts the n connections (in place) by source, then delay (the two keys
 * of Sec. 2.2), connections with equal source and delay in generation order
 * (a stable sort); then builds
 *   row_ptr[i]  = number of connections with source < i,   i = 0..n_nodes;
 *   group_first = positions q where q == 0 or (s, d)[q] != (s, d)[q-1];
 *   group_ptr[i] = p_i = sum_{j<i} G_j, G_j the groups of source j.
 * group_first must hold n entries; *n_groups receives the group count.
 * Pinned by tests/test_oracle_sort_index.py against numpy's stable lexsort,
 * bincount and a per-source distinct-delay count. */
int or_sort_index(uint32_t n_nodes, uint64_t n, uint32_t* src, uint32_t* tgt, uint16_t* delay,
                  float* weight, uint64_t* row_ptr, uint64_t* group_ptr,
                  uint64_t* group_first, uint64_t* n_groups) {
  or_rec* r = (or_rec*)malloc(sizeof(or_rec) * (n ? (size_t)n : 1));
  if (!r) return OR_ERR_OOM;
  for (uint64_t q = 0; q < n; ++q) {
    if (src[q] >= n_nodes || tgt[q] >= n_nodes) {
      free(r);
      return OR_ERR_INVALID_ARG;
    }
    r[q].s = src[q];
    r[q].t = tgt[q];
    r[q].d = delay[q];
    r[q].w = weight[q];
    r[q].gen = q;
  }
  qsort(r, (size_t)n, sizeof(or_rec), cmp_rec);
  for (uint64_t q = 0; q < n; ++q) {
    src[q] = r[q].s;
    tgt[q] = r[q].t;
    delay[q] = r[q].d;
    weight[q] = r[q].w;
  }
  free(r);
  /* CSR offsets by source. */
  for (uint32_t i = 0; i <= n_nodes; ++i) row_ptr[i] = 0;
  for (uint64_t q = 0; q < n; ++q) row_ptr[src[q] + 1] += 1;
  for (uint32_t i = 0; i < n_nodes; ++i) row_ptr[i + 1] += row_ptr[i];
  /* Group starts, G_i and p_i. */
  uint64_t g = 0;
  for (uint32_t i = 0; i <= n_nodes; ++i) group_ptr[i] = 0;
  for (uint64_t q = 0; q < n; ++q) {
    int start = q == 0 || src[q] != src[q - 1] || delay[q] != delay[q - 1];
    if (start) {
      group_first[g++] = q;
      group_ptr[src[q] + 1] += 1; /* G_i */
    }
  }
  for (uint32_t i = 0; i < n_nodes; ++i) group_ptr[i + 1] += group_ptr[i];
  *n_groups = g;
  return OR_OK;
}

/* ======================================================================== */
/* COPASS block sort (Appendix A): an array divided in k blocks is sorted    */
/* keeping its block structure, with an auxiliary array of one block.        */
/* ======================================================================== */

/* Elements of sorted run a[0..n) that are <= t (upper = 1) or < t (upper = 0):
 * a binary search. */
static uint64_t count_below(const uint64_t* a, uint64_t n, uint64_t t, int upper) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (upper ? a[mid] <= t : a[mid] < t) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* The COPASS partition (Appendix A, "The COPASS partition algorithm"): k
 * runs run[i][0..len[i]), each sorted ascending, and 0 <= m <= sum len[i].
 * Finds left-partition sizes part[i] with sum part[i] = m such that every
 * element of a left partition is <= every element of a right partition.
 * The iteration keeps lo[i] = #{elements <= t_lo} and hi[i] = #{elements <
 * t_hi} with sum lo < m < sum hi; each step takes the run l with the widest
 * open interval, its middle element t~ as a trial threshold, and the counts
 * mu_lo = #{< t~}, mu_hi = #{<= t~}: t~ is the threshold (case 1), or it
 * becomes t_hi (case 2) or t_lo (case 3).  When every interval is at most
 * one wide (last step, case 1) the undecided elements, one per run, at
 * index lo[i] (the paper prints S_{i, m-bar}; the element between the two
 * counts is S_{i, m-underbar} = S_{i, m-bar - 1}), are taken in ascending
 * order of (value, run) until the left partitions hold m.  When t~ is the
 * threshold (last step, case 2) the elements equal to it are shared out in
 * run order.  Ties go to lower runs in both last steps, so that the runs'
 * order (the original positions) decides among equal keys: the left
 * partitions are the first m elements of the stable sort of the
 * concatenated runs.  Keys are integers here, so the paper's initial
 * thresholds min - 1 and max + 1 are replaced by "below every element" and
 * "above every element" (no overflow); the counts they give, 0 and len[i],
 * are what the paper derives from them. */
int or_copass_partition(const uint64_t* const* run, const uint64_t* len, uint32_t k, uint64_t m,
                        uint64_t* part) {
  uint64_t total = 0;
  for (uint32_t i = 0; i < k; ++i) total += len[i];
  if (m > total) return OR_ERR_INVALID_ARG;
  uint64_t* lo = (uint64_t*)calloc(k ? k : 1, sizeof(uint64_t));
  uint64_t* hi = (uint64_t*)calloc(k ? k : 1, sizeof(uint64_t));
  uint64_t* mul = (uint64_t*)calloc(k ? k : 1, sizeof(uint64_t));
  uint64_t* muh = (uint64_t*)calloc(k ? k : 1, sizeof(uint64_t));
  if (!lo || !hi || !mul || !muh) {
    free(lo); free(hi); free(mul); free(muh);
    return OR_ERR_OOM;
  }
  for (uint32_t i = 0; i < k; ++i) hi[i] = len[i];
  int st = OR_OK;
  if (m == 0 || m == total) {  /* the trivial partitions */
    for (uint32_t i = 0; i < k; ++i) part[i] = m == 0 ? 0 : len[i];
    goto done;
  }
  for (;;) {
    uint32_t l = 0;
    uint64_t widest = 0;
    for (uint32_t i = 0; i < k; ++i)
      if (hi[i] - lo[i] > widest) {
        widest = hi[i] - lo[i];
        l = i;
      }
    uint64_t sum_lo = 0;
    for (uint32_t i = 0; i < k; ++i) sum_lo += lo[i];
    if (widest <= 1) {
      /* Last step, case 1: undecided elements in ascending (value, run). */
      uint64_t d = m - sum_lo;
      for (uint32_t i = 0; i < k; ++i) part[i] = lo[i];
      while (d > 0) {
        int best = -1;
        for (uint32_t i = 0; i < k; ++i) {
          if (hi[i] != lo[i] + 1 || part[i] != lo[i]) continue;  /* no candidate, or taken */
          if (best < 0 || run[i][lo[i]] < run[best][lo[best]]) best = (int)i;
        }
        if (best < 0) {
          st = OR_ERR_INVALID_ARG;  /* cannot happen while sum lo < m < sum hi */
          break;
        }
        part[best] = lo[best] + 1;
        --d;
      }
      goto done;
    }
    const uint64_t mid = (lo[l] + hi[l]) / 2;
    const uint64_t t = run[l][mid];
    uint64_t sum_mul = 0, sum_muh = 0;
    for (uint32_t i = 0; i < k; ++i) {
      mul[i] = count_below(run[i], len[i], t, 0);
      muh[i] = count_below(run[i], len[i], t, 1);
      sum_mul += mul[i];
      sum_muh += muh[i];
    }
    if (sum_mul <= m && m <= sum_muh) {
      /* Last step, case 2: t is the threshold; its copies shared in run order. */
      uint64_t d = m - sum_mul;
      for (uint32_t i = 0; i < k; ++i) {
        const uint64_t take = muh[i] - mul[i] < d ? muh[i] - mul[i] : d;
        part[i] = mul[i] + take;
        d -= take;
      }
      goto done;
    }
    if (m < sum_mul) {          /* case 2: the threshold is below t */
      for (uint32_t i = 0; i < k; ++i) hi[i] = mul[i];
    } else {                    /* case 3: the threshold is above t */
      for (uint32_t i = 0; i < k; ++i) lo[i] = muh[i];
    }
  }
done:
  free(lo); free(hi); free(mul); free(muh);
  return st;
}

typedef struct {
  uint64_t key;
  uint64_t val;
  uint64_t pos;
} or_kv;

static int cmp_kv(const void* x, const void* y) {
  const or_kv* a = (const or_kv*)x;
  const or_kv* b = (const or_kv*)y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->pos != b->pos) return a->pos < b->pos ? -1 : 1;
  return 0;
}

/* Stable sort of n (key, value) pairs in place (the underlying sort of a
 * block: qsort with the position as the last key). */
static int stable_sort_kv(uint64_t* keys, uint64_t* vals, uint64_t n) {
  or_kv* r = (or_kv*)malloc(sizeof(or_kv) * (n ? (size_t)n : 1));
  if (!r) return OR_ERR_OOM;
  for (uint64_t q = 0; q < n; ++q) {
    r[q].key = keys[q];
    r[q].val = vals[q];
    r[q].pos = q;
  }
  qsort(r, (size_t)n, sizeof(or_kv), cmp_kv);
  for (uint64_t q = 0; q < n; ++q) {
    keys[q] = r[q].key;
    vals[q] = r[q].val;
  }
  free(r);
  return OR_OK;
}

/* The COPASS block sort (Appendix A, Fig. A): keys[0..n) with values, in
 * blocks of `block` elements (the last block may be shorter), sorted stably
 * by key keeping the block structure, with an auxiliary array of one block.
 *   1. every block is sorted on its own;
 *   2. for output block o = 0, 1, ...: the remaining runs (the sorted
 *      blocks, shortened from the front as elements leave them) are
 *      partitioned with m = the size of block o; the left partitions are
 *      copied to the auxiliary array, the right partitions shifted to the
 *      end of the array (run by run, last run first) so that block o is
 *      free, the auxiliary array copied into block o and sorted.
 * The runs stay in their original order, so equal keys keep it. */
int or_copass_sort(uint64_t* keys, uint64_t* vals, uint64_t n, uint64_t block) {
  if (block == 0) return OR_ERR_INVALID_ARG;
  if (n == 0) return OR_OK;
  const uint64_t nb = (n + block - 1) / block;
  uint64_t* run_off = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nb);
  uint64_t* run_len = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nb);
  uint64_t* part = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nb);
  const uint64_t** run = (const uint64_t**)malloc(sizeof(uint64_t*) * (size_t)nb);
  uint64_t* aux_k = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)block);
  uint64_t* aux_v = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)block);
  int st = (!run_off || !run_len || !part || !run || !aux_k || !aux_v) ? OR_ERR_OOM : OR_OK;
  for (uint64_t b = 0; b < nb && !st; ++b) {
    run_off[b] = b * block;
    run_len[b] = b * block + block <= n ? block : n - b * block;
    st = stable_sort_kv(keys + run_off[b], vals + run_off[b], run_len[b]);
  }
  for (uint64_t o = 0; o < nb && !st; ++o) {
    const uint64_t first = o * block;
    const uint64_t size = first + block <= n ? block : n - first;
    /* Every run, in its original order (emptied runs have length 0). */
    const uint32_t k = (uint32_t)nb;
    for (uint32_t i = 0; i < k; ++i) run[i] = keys + run_off[i];
    st = or_copass_partition(run, run_len, k, size, part);
    if (st) break;
    /* Left partitions to the auxiliary array, in run order. */
    uint64_t a = 0;
    for (uint32_t i = 0; i < k; ++i) {
      memcpy(aux_k + a, keys + run_off[i], sizeof(uint64_t) * (size_t)part[i]);
      memcpy(aux_v + a, vals + run_off[i], sizeof(uint64_t) * (size_t)part[i]);
      a += part[i];
    }
    /* Right partitions shifted to the end, last run first. */
    uint64_t end = n;
    for (uint32_t i = k; i-- > 0;) {
      const uint64_t src = run_off[i] + part[i], len = run_len[i] - part[i];
      end -= len;
      memmove(keys + end, keys + src, sizeof(uint64_t) * (size_t)len);
      memmove(vals + end, vals + src, sizeof(uint64_t) * (size_t)len);
      run_off[i] = end;
      run_len[i] = len;
    }
    /* The auxiliary array becomes block o, sorted. */
    memcpy(keys + first, aux_k, sizeof(uint64_t) * (size_t)size);
    memcpy(vals + first, aux_v, sizeof(uint64_t) * (size_t)size);
    st = stable_sort_kv(keys + first, vals + first, size);
  }
  free(run_off); free(run_len); free(part); free(run); free(aux_k); free(aux_v);
  return st;
}

/* Spike delivery through the index (Sec. 2.3): entry e of the spike array
 * names source src[e], the grp[e]-th of its connection groups (groups in
 * position order, i.e. by increasing delay) and a multiplicity mult[e];
 * every connection q of that group adds weight[q] * mult[e] to the input of
 * its target.  The group's connections are positions group_first[g] up to
 * the next group's first position, or up to row_ptr[src + 1] for the
 * source's last group.  Accumulated in double precision, entries in order;
 * abs_in[t] collects |weight * mult| and n_terms[t] the number of additions
 * (the bound of any fp32 summation order).  *bad counts the entries that name
 * no group (skipped). */
int or_deliver(uint32_t n_nodes, uint64_t n_syn, const uint64_t* row_ptr, const uint64_t* group_ptr,
               const uint64_t* group_first, const uint32_t* tgt, const float* weight, uint64_t n_spikes,
               const uint32_t* src, const uint32_t* grp, const float* mult, double* input, double* abs_in,
               uint64_t* n_terms, uint64_t* bad) {
  *bad = 0;
  for (uint32_t t = 0; t < n_nodes; ++t) {
    input[t] = 0.0;
    abs_in[t] = 0.0;
    n_terms[t] = 0;
  }
  for (uint64_t e = 0; e < n_spikes; ++e) {
    const uint32_t s = src[e];
    if (s >= n_nodes || (uint64_t)grp[e] >= group_ptr[s + 1] - group_ptr[s]) {
      *bad += 1;
      continue;
    }
    const uint64_t g = group_ptr[s] + grp[e];
    const uint64_t first = group_first[g];
    const uint64_t last = g + 1 < group_ptr[s + 1] ? group_first[g + 1] : row_ptr[s + 1];
    for (uint64_t q = first; q < last && q < n_syn; ++q) {
      const double x = (double)weight[q] * (double)mult[e];
      input[tgt[q]] += x;
      abs_in[tgt[q]] += x < 0 ? -x : x;
      n_terms[tgt[q]] += 1;
    }
  }
  return OR_OK;
}
