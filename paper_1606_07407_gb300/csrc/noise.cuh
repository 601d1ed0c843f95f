// Noise of the synthetic black box: complex Gaussian samples from the Philox4x32-10
// counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC 2011) and the Box-Muller transform.
//
// Sample (set n, point x) of round i takes Philox4x32-10 of the counter (x, n, i, 0) under the
// key (seed mod 2^32, seed div 2^32).  Its first two words give u1 = (w0 + 1/2) / 2^32 in (0, 1)
// and u2 = w1 / 2^32, and the noise is sqrt(-2 ln u1) e^{2 pi i u2} sigma / sqrt(2), so that
// Re and Im are each N(0, sigma^2 / 2).
#pragma once

#include "sfft_internal.cuh"

namespace sfft {

// One Philox4x32 round: 64-bit products of c0 and c2 with the two multipliers, then
// c <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); ten rounds with the key
// advanced by the two increments between them.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   // round multipliers
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   // key increments
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Noise of sample (set n, point x) of round `round` (see above); sigma = 0 gives 0.
template <typename T>
__device__ __forceinline__ c2<T> black_box_noise(unsigned long long seed, int round, int n, int64_t x, double sigma);

template <>
__device__ __forceinline__ float2 black_box_noise<float>(unsigned long long seed, int round, int n, int64_t x,
                                                         double sigma) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)x, (uint32_t)n, (uint32_t)round, 0u), (uint32_t)seed,
                                (uint32_t)(seed >> 32));
  const float u1 = fmaf(__uint2float_rn(w.x), 0x1p-32f, 0x1p-33f);
  const float u2 = __uint2float_rn(w.y) * 0x1p-32f;
  const float r = sqrtf(-2.0f * logf(u1)) * (float)(sigma * 0.70710678118654752440);
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

template <>
__device__ __forceinline__ double2 black_box_noise<double>(unsigned long long seed, int round, int n, int64_t x,
                                                           double sigma) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)x, (uint32_t)n, (uint32_t)round, 0u), (uint32_t)seed,
                                (uint32_t)(seed >> 32));
  const double u1 = ((double)w.x + 0.5) * 0x1p-32;
  const double u2 = (double)w.y * 0x1p-32;
  const double r = sqrt(-2.0 * log(u1)) * (sigma * 0.70710678118654752440);
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(r * c, r * s);
}

}  // namespace sfft
