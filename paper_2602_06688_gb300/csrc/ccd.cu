// Detector noise of the CCD object (App. A, Tab. 4; App. B, Listing 2:
// photon_noise, readout_noise, readout_level, quantum_eff).  Pixel p of the
// noise-free detector image reads k + ron g, k ~ Poisson(lambda), lambda =
// det[p] scale (scale = photons per frame x quantum efficiency / pupil
// pixels), g a standard normal.  Draws: Philox4x32-10 with counter
// (p, frame, block, stream) and key (seed low, seed high).
//   lambda <= kLambdaSwitch: the multiplicative method (Knuth, TAOCP vol. 2,
//     3.4.1): k = the number of uniforms whose running float64 product stays
//     above exp(-lambda), at most kKmax; uniform j is word j mod 4 of block
//     j / 4 of stream 2;
//   lambda > kLambdaSwitch: k = max(0, floor(lambda + sqrt(lambda) g0 + 1/2)),
//     g0 the first Box-Muller normal of block 0 of stream 3;
//   the readout normal g is that block's second normal.
// The integer decision and the sum are float64; the result is rounded once
// to float32.  One thread per pixel; the loop of the multiplicative method
// is bounded by kKmax.
#include <math.h>

#include "internal.h"
#include "philox.cuh"

namespace specula {

constexpr double kLambdaSwitch = 30.0;
constexpr int kKmax = 1000;

__global__ void __launch_bounds__(256) k_ccd(const float *__restrict__ det, float *__restrict__ out,
                                             int n, double scale, double ron, uint32_t k0,
                                             uint32_t k1, uint32_t frame) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double lam = (double)det[p] * scale;
  uint32_t c[4] = {(uint32_t)p, frame, 0u, 3u};
  philox4x32_10(c, k0, k1);
  const double u0 = philox_uniform(c[0]), u1 = philox_uniform(c[1]);
  const double r = sqrt(__dmul_rn(-2.0, log(u0))), t = __dmul_rn(2.0 * M_PI, u1);
  const double g0 = r * cos(t), g1 = r * sin(t);
  int k = 0;
  if (lam > kLambdaSwitch) {
    // the float64 operations as written, one rounding each (no contraction)
    const double v = floor(__dadd_rn(__dadd_rn(lam, __dmul_rn(sqrt(lam), g0)), 0.5));
    k = v > 0.0 ? (v < 2147483647.0 ? (int)v : 2147483647) : 0;
  } else {
    const double L = exp(-lam);
    double prod = 1.0;
    uint32_t w[4];
    for (int j = 0; j <= kKmax; ++j) {
      if ((j & 3) == 0) {
        w[0] = (uint32_t)p;
        w[1] = frame;
        w[2] = (uint32_t)(j >> 2);
        w[3] = 2u;
        philox4x32_10(w, k0, k1);
      }
      prod *= philox_uniform(w[j & 3]);
      if (!(prod > L)) break;
      ++k;
    }
    k = k < kKmax ? k : kKmax;
  }
  out[p] = (float)__dadd_rn((double)k, __dmul_rn(ron, g1));
}

}  // namespace specula

using namespace specula;

extern "C" int specula_ccd(specula_ctx *ctx, int32_t n, const float *det_dev, double scale,
                           double ron, uint64_t seed, uint32_t frame, float *out_dev,
                           void *stream) {
  if (!ctx || !det_dev || !out_dev || n < 1) return SPECULA_EINVAL;
  if (!(scale >= 0.0) || !isfinite(scale) || !(ron >= 0.0) || !isfinite(ron))
    return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  SPECULA_LAUNCH(ctx, SPECULA_K_CCD, st,
                 k_ccd<<<(n + 255) / 256, 256, 0, st>>>(det_dev, out_dev, n, scale, ron,
                                                         (uint32_t)seed, (uint32_t)(seed >> 32),
                                                         frame));
  return SPECULA_OK;
}
