// Counter-based noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC 2011), from its published
// definition.  Ten rounds of (hi0, lo0) = M0 c0, (hi1, lo1) = M1 c2,
// c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), the key bumped by the Weyl
// constants between rounds; uniforms (x + 0.5) 2^-32.
#pragma once
#include <math.h>
#include <stdint.h>

namespace specula {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
    if (r < 9) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
}

__device__ __forceinline__ double philox_uniform(uint32_t x) {
  return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

// Four standard normals from counter c (Box-Muller on the uniforms of words
// 0/1 and 2/3, in float64): (r0 cos 2 pi u1, r0 sin 2 pi u1, r1 cos 2 pi u3,
// r1 sin 2 pi u3), r = sqrt(-2 ln u).
__device__ __forceinline__ void philox_normals4(uint32_t c[4], uint64_t seed, double g[4]) {
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  double u[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) u[i] = philox_uniform(c[i]);
  const double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
  const double t0 = 2.0 * M_PI * u[1], t1 = 2.0 * M_PI * u[3];
  g[0] = r0 * cos(t0);
  g[1] = r0 * sin(t0);
  g[2] = r1 * cos(t1);
  g[3] = r1 * sin(t1);
}

}  // namespace specula
