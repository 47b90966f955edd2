// tables.cpp -- host construction of the inverse-CDF threshold tables that
// the kernels use to turn one 32-bit uniform into an integer:
//   value(u) = base + #{ i : thr[i] <= u },  thr[i] = floor(2^32 * F(base + i)).
// Entries equal to 0 fold into `base`; the table stops before the first entry
// equal to 2^32.  Evaluated in IEEE double in a fixed operation order, without
// contraction, so that the same inputs give the same table on any host.
#include <cmath>
#include <cstdint>
#include <vector>

#include "snc_internal.h"

namespace snc {

namespace {
constexpr uint32_t kMaxStep = 65535u;
constexpr size_t kMaxTable = 16384;
constexpr double kTwo32 = 4294967296.0;
constexpr double kSqrtHalf = 0.70710678118654752440;

// floor(2^32 * Phi(((k + 1/2) dt - mu) / sigma)) as an integer <= 2^32.
uint64_t delay_threshold(uint32_t k, double mu, double sigma, double dt) {
  const double x = ((static_cast<double>(k) + 0.5) * dt - mu) / sigma;
  const double phi = 0.5 * std::erfc(-x * kSqrtHalf);
  return static_cast<uint64_t>(std::floor(std::ldexp(phi, 32)));
}
}  // namespace

// Delay in time steps (Sec. 2.1): d / dt rounded to an integer, at least one
// step.  For d ~ N(mu, sigma), P(step <= k) = Phi(((k + 1/2) dt - mu) / sigma).
int delay_thresholds(double mu, double sigma, double dt, std::vector<uint32_t>& thr, uint32_t& base) {
  thr.clear();
  if (!(dt > 0.0) || !(sigma > 0.0) || !std::isfinite(mu) || !std::isfinite(sigma))
    return SNC_ERR_INVALID_ARG;
  uint32_t k = 1;
  uint64_t t = delay_threshold(k, mu, sigma, dt);
  while (t == 0) {
    if (++k > kMaxStep) return SNC_ERR_UNSUPPORTED;
    t = delay_threshold(k, mu, sigma, dt);
  }
  base = k;
  while (t < (1ull << 32)) {
    if (thr.size() >= kMaxTable) return SNC_ERR_UNSUPPORTED;
    thr.push_back(static_cast<uint32_t>(t));
    if (++k > kMaxStep) return SNC_ERR_UNSUPPORTED;
    t = delay_threshold(k, mu, sigma, dt);
  }
  return SNC_OK;
}

// Binomial(n, p) counts of the pairwise Bernoulli rule.  The pmf is walked
// outward from the mode m = floor((n + 1) p) by the ratio of consecutive
// terms, (n - k) / (k + 1) * p / (1 - p), each walk stopping before the first
// term below 1e-20 of the mode; the thresholds are the ascending partial sums
// over the total.
int binomial_thresholds(uint64_t n, double p, std::vector<uint32_t>& thr, uint64_t& base) {
  thr.clear();
  if (!(p >= 0.0) || !(p <= 1.0)) return SNC_ERR_INVALID_ARG;
  if (n == 0 || p == 0.0) {
    base = 0;
    return SNC_OK;
  }
  if (p == 1.0) {
    base = n;
    return SNC_OK;
  }
  const double ratio = p / (1.0 - p);
  uint64_t mode = static_cast<uint64_t>(std::floor((static_cast<double>(n) + 1.0) * p));
  if (mode > n) mode = n;
  const size_t walk_cap = 4 * kMaxTable;
  std::vector<double> above, below;
  double w = 1.0;
  for (uint64_t k = mode; k < n; ++k) {
    const double next = (w * (static_cast<double>(n - k) / static_cast<double>(k + 1))) * ratio;
    if (next < 1e-20) break;
    if (above.size() >= walk_cap) return SNC_ERR_UNSUPPORTED;
    above.push_back(next);
    w = next;
  }
  w = 1.0;
  for (uint64_t k = mode; k > 0; --k) {
    const double next = (w * (static_cast<double>(k) / static_cast<double>(n - k + 1))) / ratio;
    if (next < 1e-20) break;
    if (below.size() >= walk_cap) return SNC_ERR_UNSUPPORTED;
    below.push_back(next);
    w = next;
  }
  const uint64_t lo = mode - below.size();
  std::vector<double> pmf;
  pmf.reserve(below.size() + 1 + above.size());
  for (size_t i = below.size(); i-- > 0;) pmf.push_back(below[i]);
  pmf.push_back(1.0);
  for (double v : above) pmf.push_back(v);
  double total = 0.0;
  for (double v : pmf) total += v;
  double cum = 0.0;
  bool have_base = false;
  for (size_t i = 0; i < pmf.size(); ++i) {
    cum += pmf[i];
    const uint64_t t = static_cast<uint64_t>(std::floor(std::ldexp(cum / total, 32)));
    if (t >= (1ull << 32)) {
      if (!have_base) {
        base = lo + i;
        have_base = true;
      }
      break;
    }
    if (t == 0) continue;
    if (!have_base) {
      base = lo + i;
      have_base = true;
    }
    if (thr.size() >= kMaxTable) return SNC_ERR_UNSUPPORTED;
    thr.push_back(static_cast<uint32_t>(t));
  }
  if (!have_base) base = lo + pmf.size() - 1;
  return SNC_OK;
}

// guide[h] = #{ i : thr[i] <= h * 2^24 }, h = 0..256 (guide[256] = size).
void guide_table(const std::vector<uint32_t>& thr, uint16_t* guide) {
  size_t i = 0;
  for (int h = 0; h < 256; ++h) {
    const uint64_t floor_u = static_cast<uint64_t>(h) << 24;
    while (i < thr.size() && thr[i] <= floor_u) ++i;
    guide[h] = static_cast<uint16_t>(i);
  }
  guide[256] = static_cast<uint16_t>(thr.size());
}

}  // namespace snc
