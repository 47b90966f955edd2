// arrays.h -- explicit node-id arrays and per-connection weight/delay arrays
// of one Connect call (Sec. 2.1): the host-side checks and sizing.
//
// Sec. 2.1: when sources or targets are given as an array of node ids, the
// rule's index formulas give positions in the array; weights and delays may
// be given per connection by arrays as long as the number of connections.
// The reading this library takes (and its oracle restates):
//   - positions and draws are those of a range of the same length; the node
//     at position a is src_ids[a] (tgt_ids[b]); an autapse is a pair of
//     equal node ids;
//   - with multapses off both arrays hold distinct ids; with autapses off the
//     list a per-primary rule draws from (sources of fixed_indegree and
//     pairwise_bernoulli, targets of fixed_outdegree) holds distinct ids;
//   - element i of a per-connection array belongs to connection number i of
//     the rule (one_to_one i; all_to_all a * Nt + b; fixed_indegree b * K + j;
//     fixed_outdegree a * K + j; fixed_total_number the slot); pairwise_bernoulli
//     takes none (its count is drawn); a number whose pair is dropped as an
//     autapse stays unused;
//   - a delay in ms becomes floor(d / dt + 1/2) steps in double, at least one;
//     non-finite delays are INVALID_ARG, steps above 65535 UNSUPPORTED.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/snc.h"

namespace snc {

// The arrays of one Connect call (host memory, read during the call only);
// a null id array means the call's node range.
struct ConnectArrays {
  const uint32_t* src_ids = nullptr;  // src.n node ids
  const uint32_t* tgt_ids = nullptr;  // tgt.n node ids
  const float* weights = nullptr;     // n_conn weights, or null
  const float* delays_ms = nullptr;   // n_conn delays in ms, or null
  uint64_t n_conn = 0;                // length of weights / delays_ms
};

// What the checks establish about an accepted call.
struct ArrayPlan {
  uint64_t numbered = 0;        // connections the rule numbers (before autapse drops)
  uint64_t count = 0;           // connections made (pairwise_bernoulli: 0, drawn later)
  uint64_t equal_pairs = 0;     // position pairs (a, b) whose nodes coincide
  std::vector<uint16_t> steps;  // delay step of each numbered connection (delays given)
  uint32_t max_step = 0;        // largest of steps (0 without delays)
};

// Checks one Connect call with arrays against n_nodes created nodes and the
// time step dt_ms.  Returns SNC_OK and fills *plan, or the status of the
// first failed check (in the order of the list above: lists, rule limits,
// per-connection arrays) with its reason in *why.
snc_status check_connect_arrays(uint32_t n_nodes, double dt_ms, const snc_range& src, const snc_range& tgt,
                                const snc_conn_rule& rule, const ConnectArrays& arrays, ArrayPlan* plan,
                                std::string* why);

// Delay of d ms in steps of dt_ms (the conversion above); SNC_OK or the
// status of a non-finite or too long delay.
snc_status delay_step_of(double d_ms, double dt_ms, uint32_t* step);

}  // namespace snc
