// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
// from its published definition: ten rounds, each multiplying words 0 and 2 by the Philox
// constants and mixing the high halves with words 1 and 3 and the key, with the key advanced
// by the Weyl increments between rounds.
#pragma once

#include <stdint.h>

namespace ugp {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = c.x * 0xD2511F53u, hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u, hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform on the 2^-24 grid in [0, 1): exact in float32.
__device__ __forceinline__ float u24(uint32_t x) { return float(x >> 8) * (1.0f / 16777216.0f); }

// Exponential variate of primitive k in the race that chooses the scattering primitive
// among those active at t_u: key (bits of u2, 0x2406C0DE), counter (k, 0, 0, 0),
// U = ((x0 >> 8) + 1) / 2^24 in (0, 1], E = -ln U.
__device__ __forceinline__ float race_exponential(float u2, int k) {
  const uint4 x = philox4x32_10(make_uint4(uint32_t(k), 0u, 0u, 0u), make_uint2(__float_as_uint(u2), 0x2406C0DEu));
  const float U = float((x.x >> 8) + 1u) * (1.0f / 16777216.0f);
  return -logf(U);
}

}  // namespace ugp
