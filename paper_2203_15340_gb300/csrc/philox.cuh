// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), shared by
// the randomized inner chains and the warm-start network's initialization.
#pragma once

#include <stdint.h>

namespace ils {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-P network with
// multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 53-bit uniform in [0,1) from the top 27 bits of a and the top 26 bits of b.
__device__ __forceinline__ double to_uniform(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void step_uniforms(uint64_t seed, uint32_t chain, uint32_t k, uint64_t t,
                                              double* u0, double* u1) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), k, chain),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  *u0 = to_uniform(w.x, w.y);
  *u1 = to_uniform(w.z, w.w);
}

}  // namespace ils
