// snc_device.cuh -- per-connection arithmetic shared by the generation
// kernels: the counter-based random stream, rand(N), the delay and count
// threshold tables and the weight transform.
//
// Random stream: Philox4x32-10 (Salmon et al., SC'11).  Key = (seed lo,
// seed hi ^ projection); counter = (slot lo, primary node, tag | round << 8,
// slot hi).  Every connection's draws are a pure function of those numbers,
// so a connection is reproducible independently of the launch shape.
#pragma once

#include <cstdint>

namespace snc {

enum : uint32_t { kTagWD = 0u, kTagIdx = 1u, kTagCount = 2u, kTagDedup = 3u };
constexpr uint32_t kPrimaryNone = 0xFFFFFFFFu;

struct Words {
  uint32_t x, y, z, w;
};

// Ten Philox4x32 rounds: the two products by the round multipliers, their
// high halves xor-ed with the other two counter words and the round key.
__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Words{c0, c1, c2, c3};
}

__device__ __forceinline__ Words draw(uint32_t k0, uint32_t k1, uint32_t tag, uint32_t round,
                                      uint32_t primary, uint64_t slot) {
  return philox(static_cast<uint32_t>(slot), primary, tag | (round << 8),
                static_cast<uint32_t>(slot >> 32), k0, k1);
}

// rand(N) of Sec. 2.1 by multiply-shift: floor(u * N / 2^32).
__device__ __forceinline__ uint32_t rand_below(uint32_t u, uint32_t n) { return __umulhi(u, n); }

// Endpoint in a range of n nodes, optionally leaving out local index `skip`
// (so that a connection can never join a node to itself).
__device__ __forceinline__ uint32_t endpoint(uint32_t u, uint32_t n, bool skip, uint32_t skip_local) {
  if (!skip) return rand_below(u, n);
  uint32_t r = rand_below(u, n - 1u);
  return r + (r >= skip_local ? 1u : 0u);
}

// Inverse-CDF lookup: value = base + #{i < len : thr[i] <= u}.  `guide` has
// 257 entries: guide[h] = #{i : thr[i] <= h << 24} (guide[256] = len), so the
// linear scan starts at the first threshold above the bucket floor.
__device__ __forceinline__ uint32_t table_lookup(const uint32_t* thr, const uint16_t* guide,
                                                 uint32_t len, uint32_t u) {
  uint32_t i = guide[u >> 24];
  while (i < len && thr[i] <= u) ++i;
  return i;
}

// Normal weight by the Box-Muller transform (cosine branch) of two 24-bit
// uniforms u1 in (0, 1] and u2 in [0, 1), in single precision.
__device__ __forceinline__ float normal_weight(float mean, float std, uint32_t w2, uint32_t w3) {
  const float u1 = static_cast<float>((w2 >> 8) + 1u) * 0x1p-24f;
  const float u2 = static_cast<float>(w3 >> 8) * 0x1p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  const float c = cospif(2.0f * u2);
  return fmaf(std, r * c, mean);
}

}  // namespace snc
