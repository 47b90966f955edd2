/*
 * snc_oracle_par.c -- the CPU oracle of snc_oracle.c run on several host
 * threads (OpenMP), for full-size checks and the multi-core CPU baseline.
 *
 * TEST INFRASTRUCTURE ONLY, like snc_oracle.c, which it includes whole: every
 * connection is still made by the same functions (gen_primary, emit_wd,
 * gen_total_number, the tables), so the arithmetic is the pinned
 * single-thread oracle's.  Only the order of the work changes:
 *   - the primary nodes of a per-primary rule (Sec. 2.1 numbering: targets of
 *     fixed_indegree and pairwise_bernoulli, sources of fixed_outdegree, the
 *     source rows of all_to_all) are generated in parallel, each into the
 *     range an exclusive scan of the per-primary counts gives it, so the
 *     output is the single-thread output position for position;
 *   - fixed_total_number draws its slots in parallel; with autapses or
 *     multapses forbidden each redraw round sorts its (pair, slot) claims
 *     (gen_total_number_par below states why the winners are the same);
 *   - the stable (source, delay) sort is a merge sort: chunks sorted in
 *     parallel by the same comparison (source, delay, generation position,
 *     a total order, so the result is unique), then merged pairwise.
 * tests/test_oracle_parallel.py pins it: equal to the single-thread oracle,
 * bit for bit, on every rule and flag pair, explicit arrays included.
 */
#include "snc_oracle.c"

#include <omp.h>

/* Connections of primary node b of fixed_indegree, fixed_outdegree (K
 * each) or pairwise_bernoulli (the count gen_primary draws: the COUNT word
 * through the table of the node's candidates, one left out when the node
 * itself is among the sources and autapses are off). */
static uint64_t count_primary(const or_net* net, uint32_t proj, const or_proj* pj, const or_tables* t,
                              uint32_t b) {
  if (pj->rule != OR_PAIRWISE_BERNOULLI) return pj->k;
  uint32_t node = tgt_node(pj, b);
  int64_t q = pj->allow_autapses ? -1 : position_of(pj, t, 0, node);
  int skip = q >= 0;
  uint32_t w[4];
  draw(net, proj, OR_TAG_COUNT, 0, b, 0, w);
  return table_value(t->b_base[skip], t->b_thr[skip], t->b_len[skip], w[0]);
}

/* ------------------------------------------------------------------------ */
/* fixed_total_number with autapses or multapses forbidden, on host threads. */
/* The rule of gen_total_number, round by round: a slot whose pair is not     */
/* allowed redraws; in round 0 the lowest slot drawing a pair takes it, in   */
/* round r >= 1 the lowest pending slot drawing a pair that no earlier round */
/* took.  Visiting slots in ascending order with a running set (the single- */
/* thread form) and sorting each round's (pair, slot) claims give the same   */
/* winners: both pick, per pair, the lowest claiming slot of the first round */
/* in which the pair is claimed.                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t key;
  uint64_t slot;
} or_claim;

static int cmp_claim(const void* x, const void* y) {
  const or_claim* a = (const or_claim*)x;
  const or_claim* b = (const or_claim*)y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;
  return 0;
}

/* Sorts c[0..n) by (key, slot) on host threads (chunks, then pairwise merges). */
static int sort_claims(or_claim* c, uint64_t n) {
  if (n < 2) return OR_OK;
  or_claim* tmp = (or_claim*)malloc(sizeof(or_claim) * (size_t)n);
  if (!tmp) return OR_ERR_OOM;
  int chunks = 1;
  while (chunks < 4 * omp_get_max_threads() && (uint64_t)chunks * 65536 < n) chunks <<= 1;
  const uint64_t per = (n + chunks - 1) / chunks;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < chunks; ++k) {
    const uint64_t lo = (uint64_t)k * per < n ? (uint64_t)k * per : n;
    const uint64_t hi = lo + per < n ? lo + per : n;
    qsort(c + lo, (size_t)(hi - lo), sizeof(or_claim), cmp_claim);
  }
  or_claim* from = c;
  or_claim* to = tmp;
  for (uint64_t width = per; width < n; width *= 2) {
    const uint64_t pairs = (n + 2 * width - 1) / (2 * width);
#pragma omp parallel for schedule(dynamic, 1)
    for (uint64_t k = 0; k < pairs; ++k) {
      const uint64_t lo = k * 2 * width;
      const uint64_t mid = lo + width < n ? lo + width : n;
      const uint64_t hi = mid + width < n ? mid + width : n;
      uint64_t i = lo, j = mid, o = lo;
      while (i < mid && j < hi) to[o++] = cmp_claim(&from[j], &from[i]) < 0 ? from[j++] : from[i++];
      while (i < mid) to[o++] = from[i++];
      while (j < hi) to[o++] = from[j++];
    }
    or_claim* x = from;
    from = to;
    to = x;
  }
  if (from != c) memcpy(c, from, sizeof(or_claim) * (size_t)n);
  free(tmp);
  return OR_OK;
}

static int key_in(const uint64_t* keys, uint64_t n, uint64_t k) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    if (keys[mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo < n && keys[lo] == k;
}

static int cmp_u64(const void* x, const void* y) {
  const uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
  return a < b ? -1 : (a > b ? 1 : 0);
}

static int gen_total_number_par(const or_net* net, uint32_t proj, const or_proj* pj, const or_tables* t,
                                or_sink* out) {
  const uint32_t Ns = pj->src_n, Nt = pj->tgt_n;
  const uint64_t N = pj->k;
  if (N == 0) return OR_OK;
  if (out->src && out->pos + N > out->cap) return OR_ERR_INVALID_ARG;
  const int dedup = !pj->allow_multapses;
  int st = OR_OK;
  uint32_t* ps = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint32_t* pt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  unsigned char* okv = (unsigned char*)malloc((size_t)N);
  uint64_t* pending = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
  or_claim* claims = dedup ? (or_claim*)malloc(sizeof(or_claim) * (size_t)N) : 0;
  uint64_t* taken = dedup ? (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N) : 0; /* sorted keys taken */
  uint64_t n_taken = 0;
  if (!ps || !pt || !okv || !pending || (dedup && (!claims || !taken))) st = OR_ERR_OOM;
  uint64_t n_pending = 0;
  for (uint32_t round = 0; !st; ++round) {
    if (round > OR_MAX_ROUND) {
      st = OR_ERR_TIMEOUT;
      break;
    }
    const uint64_t n_visit = round == 0 ? N : n_pending;
    if (round > 0 && n_pending == 0) break;
    /* Draw every visited slot's pair (round 0: WD word 1 and IDX word
     * i mod 4; later rounds: words 0 and 1 of the round's DEDUP draw). */
#pragma omp parallel for schedule(static)
    for (uint64_t q = 0; q < n_visit; ++q) {
      const uint64_t i = round == 0 ? q : pending[q];
      uint32_t w[4];
      if (round == 0) {
        uint32_t x[4];
        draw(net, proj, OR_TAG_WD, 0, OR_PRIMARY_NONE, i, w);
        draw(net, proj, OR_TAG_IDX, 0, OR_PRIMARY_NONE, i / 4, x);
        ps[i] = src_node(pj, rand_below(w[1], Ns));
        pt[i] = tgt_node(pj, rand_below(x[i % 4], Nt));
      } else {
        draw(net, proj, OR_TAG_DEDUP, round, OR_PRIMARY_NONE, i, w);
        ps[i] = src_node(pj, rand_below(w[0], Ns));
        pt[i] = tgt_node(pj, rand_below(w[1], Nt));
      }
      okv[i] = pj->allow_autapses || ps[i] != pt[i];
      if (okv[i] && dedup && key_in(taken, n_taken, ((uint64_t)ps[i] << 32) | pt[i])) okv[i] = 0;
    }
    if (dedup) {
      /* Among this round's allowed claims the lowest slot of each pair wins. */
      uint64_t nc = 0;
      for (uint64_t q = 0; q < n_visit; ++q) {
        const uint64_t i = round == 0 ? q : pending[q];
        if (okv[i]) {
          claims[nc].key = ((uint64_t)ps[i] << 32) | pt[i];
          claims[nc].slot = i;
          ++nc;
        }
      }
      st = sort_claims(claims, nc);
      if (st) break;
      uint64_t n_new = 0;
      for (uint64_t c = 0; c < nc; ++c) {
        if (c > 0 && claims[c].key == claims[c - 1].key) {
          okv[claims[c].slot] = 0;  /* a lower slot took the pair this round */
        } else {
          taken[n_taken + n_new++] = claims[c].key;
        }
      }
      n_taken += n_new;
      if (round > 0) qsort(taken, (size_t)n_taken, sizeof(uint64_t), cmp_u64);
    }
    /* The losers, ascending, are the next round's pending slots. */
    uint64_t still = 0;
    for (uint64_t q = 0; q < n_visit; ++q) {
      const uint64_t i = round == 0 ? q : pending[q];
      if (!okv[i]) pending[still++] = i;
    }
    n_pending = still;
  }
  if (!st) {
#pragma omp parallel for schedule(static) reduction(| : st)
    for (uint64_t i = 0; i < N; ++i) {
      or_sink one = {out->src ? out->src + out->pos + i : 0, out->tgt ? out->tgt + out->pos + i : 0,
                     out->delay ? out->delay + out->pos + i : 0, out->weight ? out->weight + out->pos + i : 0, 0,
                     1};
      st |= emit_wd(net, proj, pj, t, OR_PRIMARY_NONE, i, i, ps[i], pt[i], &one);
    }
    out->pos += N;
  }
  free(ps);
  free(pt);
  free(okv);
  free(pending);
  free(claims);
  free(taken);
  return st;
}

static uint64_t sel_size(const or_proj* pj) {
  if (pj->rule == OR_PAIRWISE_BERNOULLI || pj->rule == OR_ALL_TO_ALL) return (uint64_t)pj->src_n + 1;
  return pj->k + 1;
}

/* One projection appended to `out`: per-primary rules and all_to_all rows
 * in parallel, the rest as in snc_oracle.c. */
static int gen_projection_par(const or_net* net, uint32_t proj, const or_proj* pj, const or_tables* t,
                              or_sink* out) {
  const int rule = pj->rule;
  if (rule == OR_FIXED_TOTAL_NUMBER && pj->allow_multapses && pj->allow_autapses) {
    /* No redraws: slot i is connection i, its pair from its own draws. */
    const uint64_t N = pj->k;
    if (out->src && out->pos + N > out->cap) return OR_ERR_INVALID_ARG;
    int st = OR_OK;
#pragma omp parallel for schedule(static) reduction(| : st)
    for (uint64_t i = 0; i < N; ++i) {
      uint32_t w[4], x[4];
      draw(net, proj, OR_TAG_WD, 0, OR_PRIMARY_NONE, i, w);
      draw(net, proj, OR_TAG_IDX, 0, OR_PRIMARY_NONE, i / 4, x);
      const uint32_t s = src_node(pj, rand_below(w[1], pj->src_n));
      const uint32_t tg = tgt_node(pj, rand_below(x[i % 4], pj->tgt_n));
      or_sink one = {out->src ? out->src + out->pos + i : 0, out->tgt ? out->tgt + out->pos + i : 0,
                     out->delay ? out->delay + out->pos + i : 0, out->weight ? out->weight + out->pos + i : 0, 0, 1};
      st |= emit_wd(net, proj, pj, t, OR_PRIMARY_NONE, i, i, s, tg, &one);
    }
    out->pos += N;
    return st;
  }
  if (rule == OR_FIXED_TOTAL_NUMBER) return gen_total_number_par(net, proj, pj, t, out);
  if (rule != OR_FIXED_INDEGREE && rule != OR_FIXED_OUTDEGREE && rule != OR_PAIRWISE_BERNOULLI &&
      rule != OR_ALL_TO_ALL)
    return gen_projection(net, proj, pj, t, out);
  /* all_to_all is numbered source row by source row (i = a*Nt + b); its
   * rows are the units here, each row written by the loop of snc_oracle.c. */
  const int rows = rule == OR_ALL_TO_ALL;
  const uint32_t n_unit = rows ? pj->src_n : (rule == OR_FIXED_OUTDEGREE ? pj->src_n : pj->tgt_n);
  uint64_t* off = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n_unit + 1));
  if (!off) return OR_ERR_OOM;
  int st = OR_OK;
#pragma omp parallel for schedule(dynamic, 64)
  for (uint32_t u = 0; u < n_unit; ++u) {
    uint64_t c = 0;
    if (rows) {
      for (uint32_t b = 0; b < pj->tgt_n; ++b)
        if (pj->allow_autapses || src_node(pj, u) != tgt_node(pj, b)) ++c;
    } else {
      c = count_primary(net, proj, pj, t, u);
    }
    off[u + 1] = c;
  }
  off[0] = out->pos;
  for (uint32_t u = 0; u < n_unit; ++u) off[u + 1] += off[u];
  if (out->src && off[n_unit] > out->cap) {
    free(off);
    return OR_ERR_INVALID_ARG;
  }
  if (out->src) {
#pragma omp parallel reduction(| : st)
    {
      uint32_t* sel = rows ? 0 : (uint32_t*)malloc(sizeof(uint32_t) * (size_t)sel_size(pj));
      if (!rows && !sel) st |= OR_ERR_OOM;
#pragma omp for schedule(dynamic, 64)
      for (uint32_t u = 0; u < n_unit; ++u) {
        if (st) continue;
        const uint64_t o = off[u];
        or_sink part = {out->src + o, out->tgt + o, out->delay + o, out->weight + o, 0, off[u + 1] - o};
        if (rows) {
          for (uint32_t b = 0; b < pj->tgt_n && !st; ++b) {
            const uint32_t s = src_node(pj, u), tg = tgt_node(pj, b);
            if (!pj->allow_autapses && s == tg) continue;
            st |= emit_wd(net, proj, pj, t, b, u, (uint64_t)u * pj->tgt_n + b, s, tg, &part);
          }
        } else {
          st |= gen_primary(net, proj, pj, t, u, sel, &part);
        }
      }
      free(sel);
    }
  }
  out->pos = off[n_unit];
  free(off);
  return st;
}

/* or_generate on host threads: the same output, position for position. */
int or_generate_par(const or_net* net, const or_proj* projs, uint32_t* src, uint32_t* tgt, uint16_t* delay,
                    float* weight, uint64_t cap, uint64_t* n_out, uint64_t* per_proj, int threads) {
  if (threads > 0) omp_set_num_threads(threads);
  or_sink out = {src, tgt, delay, weight, 0, cap};
  for (uint32_t p = 0; p < net->n_proj; ++p) {
    int st = or_check_projection(net, &projs[p]);
    if (st) return st;
  }
  for (uint32_t p = 0; p < net->n_proj; ++p) {
    or_tables t;
    uint64_t before = out.pos;
    int st = make_tables(net, &projs[p], &t);
    if (!st) st = gen_projection_par(net, p, &projs[p], &t, &out);
    free_tables(&t);
    if (st) return st;
    if (per_proj) per_proj[p] = out.pos - before;
  }
  *n_out = out.pos;
  return OR_OK;
}

static void merge_runs(const or_rec* a, uint64_t na, const or_rec* b, uint64_t nb, or_rec* dst) {
  uint64_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) dst[k++] = cmp_rec(&b[j], &a[i]) < 0 ? b[j++] : a[i++];
  while (i < na) dst[k++] = a[i++];
  while (j < nb) dst[k++] = b[j++];
}

/* or_sort_index with the sort on host threads (same comparison, a total
 * order: the result is the single-thread result). */
int or_sort_index_par(uint32_t n_nodes, uint64_t n, uint32_t* src, uint32_t* tgt, uint16_t* delay, float* weight,
                      uint64_t* row_ptr, uint64_t* group_ptr, uint64_t* group_first, uint64_t* n_groups,
                      int threads) {
  if (threads > 0) omp_set_num_threads(threads);
  or_rec* r = (or_rec*)malloc(sizeof(or_rec) * (n ? (size_t)n : 1));
  or_rec* tmp = (or_rec*)malloc(sizeof(or_rec) * (n ? (size_t)n : 1));
  if (!r || !tmp) {
    free(r);
    free(tmp);
    return OR_ERR_OOM;
  }
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (uint64_t q = 0; q < n; ++q) {
    if (src[q] >= n_nodes || tgt[q] >= n_nodes) bad = 1;
    r[q].s = src[q];
    r[q].t = tgt[q];
    r[q].d = delay[q];
    r[q].w = weight[q];
    r[q].gen = q;
  }
  if (bad) {
    free(r);
    free(tmp);
    return OR_ERR_INVALID_ARG;
  }
  /* Chunks (a power of two of them) sorted in parallel, then merged pairwise. */
  int chunks = 1;
  while (chunks < 4 * omp_get_max_threads() && (uint64_t)chunks * 65536 < n) chunks <<= 1;
  const uint64_t per = (n + chunks - 1) / chunks;
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < chunks; ++c) {
    const uint64_t lo = (uint64_t)c * per < n ? (uint64_t)c * per : n;
    const uint64_t hi = lo + per < n ? lo + per : n;
    qsort(r + lo, (size_t)(hi - lo), sizeof(or_rec), cmp_rec);
  }
  or_rec* from = r;
  or_rec* to = tmp;
  for (uint64_t width = per; width < n; width *= 2) {
    const uint64_t pairs = (n + 2 * width - 1) / (2 * width);
#pragma omp parallel for schedule(dynamic, 1)
    for (uint64_t k = 0; k < pairs; ++k) {
      const uint64_t lo = k * 2 * width;
      const uint64_t mid = lo + width < n ? lo + width : n;
      const uint64_t hi = mid + width < n ? mid + width : n;
      merge_runs(from + lo, mid - lo, from + mid, hi - mid, to + lo);
    }
    or_rec* x = from;
    from = to;
    to = x;
  }
#pragma omp parallel for schedule(static)
  for (uint64_t q = 0; q < n; ++q) {
    src[q] = from[q].s;
    tgt[q] = from[q].t;
    delay[q] = from[q].d;
    weight[q] = from[q].w;
  }
  free(r);
  free(tmp);
  /* Index exactly as or_sort_index builds it (one pass, O(n)). */
  for (uint32_t i = 0; i <= n_nodes; ++i) row_ptr[i] = 0;
  for (uint64_t q = 0; q < n; ++q) row_ptr[src[q] + 1] += 1;
  for (uint32_t i = 0; i < n_nodes; ++i) row_ptr[i + 1] += row_ptr[i];
  uint64_t g = 0;
  for (uint32_t i = 0; i <= n_nodes; ++i) group_ptr[i] = 0;
  for (uint64_t q = 0; q < n; ++q) {
    int start = q == 0 || src[q] != src[q - 1] || delay[q] != delay[q - 1];
    if (start) {
      group_first[g++] = q;
      group_ptr[src[q] + 1] += 1;
    }
  }
  for (uint32_t i = 0; i < n_nodes; ++i) group_ptr[i + 1] += group_ptr[i];
  *n_groups = g;
  return OR_OK;
}

int or_max_threads(void) { return omp_get_max_threads(); }
