// arrays.cpp -- host-side checks and sizing of Connect calls with explicit
// node-id arrays and per-connection weight/delay arrays (Sec. 2.1).
#include "arrays.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace snc {

namespace {

snc_status refuse(snc_status st, std::string* why, const char* fmt, unsigned long long a = 0,
                  unsigned long long b = 0) {
  if (why) {
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, b);
    *why = buf;
  }
  return st;
}

// Node id at position i of a list given by ids or by its range.
inline uint32_t node_at(const uint32_t* ids, const snc_range& r, uint32_t i) {
  return ids ? ids[i] : r.first + i;
}

}  // namespace

snc_status delay_step_of(double d_ms, double dt_ms, uint32_t* step) {
  if (!std::isfinite(d_ms)) return SNC_ERR_INVALID_ARG;
  double q = std::floor(d_ms / dt_ms + 0.5);
  if (q < 1.0) q = 1.0;
  if (q > 65535.0) return SNC_ERR_UNSUPPORTED;
  *step = static_cast<uint32_t>(q);
  return SNC_OK;
}

snc_status check_connect_arrays(uint32_t n_nodes, double dt_ms, const snc_range& src, const snc_range& tgt,
                                const snc_conn_rule& rule, const ConnectArrays& a, ArrayPlan* plan,
                                std::string* why) {
  if (!plan) return refuse(SNC_ERR_INVALID_ARG, why, "null plan");
  *plan = ArrayPlan{};
  if (!(dt_ms > 0.0)) return refuse(SNC_ERR_INVALID_ARG, why, "dt must be > 0");
  const bool aut = rule.allow_autapses != 0, mult = rule.allow_multapses != 0;
  // The two node lists: ids below n_nodes (or the range inside the nodes),
  // distinct where the reading asks for it.
  for (int side = 0; side < 2; ++side) {
    const uint32_t* ids = side ? a.tgt_ids : a.src_ids;
    const snc_range& r = side ? tgt : src;
    if (!ids) {
      if (static_cast<uint64_t>(r.first) + r.n > n_nodes)
        return refuse(SNC_ERR_INVALID_ARG, why, "node range outside the created populations");
      continue;
    }
    std::vector<uint8_t> seen;
    const bool drawn_from = side ? rule.kind == SNC_FIXED_OUTDEGREE
                                 : (rule.kind == SNC_FIXED_INDEGREE || rule.kind == SNC_PAIRWISE_BERNOULLI);
    const bool distinct = !mult || (!aut && drawn_from);
    if (distinct) seen.assign(n_nodes, 0);
    for (uint32_t i = 0; i < r.n; ++i) {
      const uint32_t v = ids[i];
      if (v >= n_nodes)
        return refuse(SNC_ERR_INVALID_ARG, why, "node id %llu at or above the %llu created nodes", v, n_nodes);
      if (distinct) {
        if (seen[v]) return refuse(SNC_ERR_INVALID_ARG, why, "node id %llu listed twice", v);
        seen[v] = 1;
      }
    }
  }
  // Autapse pairs among all position pairs: sum over nodes of (times listed
  // as a source) x (times listed as a target).
  uint64_t eq = 0;
  if (!a.src_ids && !a.tgt_ids) {
    const uint64_t lo = std::max<uint64_t>(src.first, tgt.first);
    const uint64_t hi = std::min<uint64_t>(static_cast<uint64_t>(src.first) + src.n,
                                           static_cast<uint64_t>(tgt.first) + tgt.n);
    eq = hi > lo ? hi - lo : 0;
  } else {
    std::vector<uint32_t> as_source(n_nodes, 0);
    for (uint32_t i = 0; i < src.n; ++i) ++as_source[node_at(a.src_ids, src, i)];
    for (uint32_t j = 0; j < tgt.n; ++j) eq += as_source[node_at(a.tgt_ids, tgt, j)];
  }
  plan->equal_pairs = eq;
  // The rule's limits, as for ranges with the autapse pairs counted above.
  switch (rule.kind) {
    case SNC_ONE_TO_ONE: {
      if (src.n != tgt.n) return refuse(SNC_ERR_INVALID_ARG, why, "one_to_one: source and target sizes differ");
      plan->numbered = src.n;
      uint64_t same = 0;  // pairs i with equal nodes: for two ranges all or none
      if (!a.src_ids && !a.tgt_ids)
        same = src.first == tgt.first ? src.n : 0;
      else
        for (uint32_t i = 0; i < src.n; ++i) same += node_at(a.src_ids, src, i) == node_at(a.tgt_ids, tgt, i);
      plan->count = src.n - (aut ? 0 : same);
      break;
    }
    case SNC_ALL_TO_ALL:
      plan->numbered = static_cast<uint64_t>(src.n) * tgt.n;
      plan->count = plan->numbered - (aut ? 0 : eq);
      break;
    case SNC_FIXED_INDEGREE:
    case SNC_FIXED_OUTDEGREE: {
      const bool indeg = rule.kind == SNC_FIXED_INDEGREE;
      const uint64_t n_other = indeg ? src.n : tgt.n, n_primary = indeg ? tgt.n : src.n;
      if (rule.k > 0 && n_primary > 0) {
        if (rule.k > 0xFFFFFFFFull) return refuse(SNC_ERR_INVALID_ARG, why, "degree K above 2^32 - 1");
        // With autapses off a primary listed in the other list loses one candidate.
        const uint64_t least = (!aut && eq > 0) ? n_other - 1 : n_other;
        if (least == 0) return refuse(SNC_ERR_INVALID_ARG, why, "degree rule: no candidate nodes");
        if (!mult && rule.k > least)
          return refuse(SNC_ERR_INVALID_ARG, why, "degree K=%llu above the %llu candidates without multapses",
                        rule.k, least);
      }
      plan->numbered = plan->count = n_primary * rule.k;
      break;
    }
    case SNC_FIXED_TOTAL_NUMBER:
      if (rule.k > 0) {
        const uint64_t allowed = static_cast<uint64_t>(src.n) * tgt.n - (aut ? 0 : eq);
        if (allowed == 0) return refuse(SNC_ERR_INVALID_ARG, why, "fixed_total_number: no allowed pair");
        if (!mult && rule.k > allowed)
          return refuse(SNC_ERR_INVALID_ARG, why, "fixed_total_number: N=%llu above the %llu allowed pairs",
                        rule.k, allowed);
      }
      plan->numbered = plan->count = rule.k;
      break;
    case SNC_PAIRWISE_BERNOULLI:
      if (!(rule.p >= 0.0 && rule.p <= 1.0)) return refuse(SNC_ERR_INVALID_ARG, why, "pairwise_bernoulli: p outside [0, 1]");
      if (a.weights || a.delays_ms)
        return refuse(SNC_ERR_INVALID_ARG, why, "pairwise_bernoulli takes no per-connection arrays");
      break;
    default:
      return refuse(SNC_ERR_INVALID_ARG, why, "unknown rule %llu", static_cast<unsigned long long>(rule.kind));
  }
  // Per-connection arrays: one element per numbered connection; delays to steps.
  if (a.weights || a.delays_ms) {
    if (a.n_conn != plan->numbered)
      return refuse(SNC_ERR_INVALID_ARG, why, "%llu per-connection values for %llu numbered connections",
                    a.n_conn, plan->numbered);
    if (a.delays_ms) {
      plan->steps.resize(a.n_conn);
      for (uint64_t i = 0; i < a.n_conn; ++i) {
        uint32_t step = 1;
        const snc_status st = delay_step_of(static_cast<double>(a.delays_ms[i]), dt_ms, &step);
        if (st != SNC_OK)
          return refuse(st, why, st == SNC_ERR_UNSUPPORTED ? "delay %llu above 65535 steps"
                                                           : "delay %llu is not a finite number",
                        i);
        plan->steps[i] = static_cast<uint16_t>(step);
        if (step > plan->max_step) plan->max_step = step;
      }
    }
  }
  return SNC_OK;
}

}  // namespace snc
