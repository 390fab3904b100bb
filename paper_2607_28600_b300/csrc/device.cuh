// Counter-based random streams (device side).
#pragma once

#include <cstdint>

#include "plan_dev.hpp"

namespace symft {

__device__ __forceinline__ uint32_t pick(uint4 v, uint32_t s) {
  return s == 0 ? v.x : (s == 1 ? v.y : (s == 2 ? v.z : v.w));
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) {
  return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0))
// with the key bumped by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The same block function with the round keys precomputed (launch-parameter
// operands instead of key additions in every round).
__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ K.k[2 * r], lo1, hi0 ^ c.w ^ K.k[2 * r + 1], lo0);
  }
  return c;
}

// Early exit under postselection (Sec. 6, detector postselection): whether a
// postselected detector of group q fires for request-local shot r.  Group q
// holds the postselected detectors that follow exactly q active measurements
// in circuit order, in annotation order; their values are the sign kernel's
// exogenous columns XOR the shot's active outcomes (bit j of m3bits), all of
// which are decided once active measurement q - 1 is.
__device__ __forceinline__ bool group_rejects(const DevPlan& p, const uint64_t* det_exo, uint64_t W, uint64_t r,
                                              uint32_t q, const uint32_t* m3bits) {
  const uint32_t e1 = __ldg(p.post_chk_off + q + 1);
  for (uint32_t e = __ldg(p.post_chk_off + q); e < e1; ++e) {
    const uint32_t d = __ldg(p.post_chk + e);
    uint32_t v = (uint32_t)((__ldg(det_exo + (uint64_t)d * W + (r >> 6)) >> (r & 63)) & 1ull);
    const uint32_t i = p.tgt_det0 + d;
    const uint32_t ce = __ldg(p.tgt_causal_off + i + 1);
    for (uint32_t c = __ldg(p.tgt_causal_off + i); c < ce; ++c) {
      const uint32_t j = __ldg(p.tgt_causal + c);
      v ^= (m3bits[j >> 5] >> (j & 31)) & 1u;
    }
    if (v) return true;
  }
  return false;
}

}  // namespace symft
