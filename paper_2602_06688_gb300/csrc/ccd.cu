// Detector noise of the CCD object (App. A, Tab. 4; App. B, Listing 2:
// photon_noise, readout_noise, readout_level, quantum_eff).  Pixel p of the
// noise-free detector image reads k + ron g, k ~ Poisson(lambda), lambda =
// det[p] scale (scale = photons per frame x quantum efficiency / pupil
// pixels), g a standard normal.  Draws: Philox4x32-10 with counter
// (p, frame, block, stream) and key (seed low, seed high); the uniform of a
// word x is (x + 1/2) 2^-32.
//   lambda <= kLambdaSwitch: the multiplicative method (Knuth, TAOCP vol. 2,
//     3.4.1): k = the number of uniforms whose running product stays above
//     exp(-lambda), at most kKmax; uniform j is word j mod 4 of block j / 4
//     of stream 2.  The uniforms, their product and the threshold are
//     float32 here (float64 is slow on this part): a count can differ by one
//     from the float64 statement of the method where the product ends within
//     a few float32 roundings of the threshold;
//   lambda > kLambdaSwitch: k = max(0, floor(lambda + sqrt(lambda) g0 + 1/2))
//     in float64 (the rounded normal approximation of the Poisson law);
//   (g0, g) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), the Box-Muller pair
//     of words 0 and 1 of block 0 of stream 3, in float32.
// k + ron g is summed in float64 and rounded once to float32.
#include <math.h>

#include "internal.h"
#include "philox.cuh"

namespace specula {

constexpr double kLambdaSwitch = 30.0;
constexpr int kKmax = 1000;

// The uniform (x + 1/2) 2^-32 rounded once to float32: (2x + 1) 2^-33 has at
// most 33 significant bits; the integer-to-float conversion rounds it once and
// the power-of-two scaling is exact.
__device__ __forceinline__ float uniform_f32(uint32_t x) {
  return __fmul_rn(__ull2float_rn(2ull * x + 1ull), 0x1p-33f);
}

// The Box-Muller pair of block 0 of stream 3.
__device__ __forceinline__ void box_muller(uint32_t p, uint32_t frame, uint32_t k0, uint32_t k1,
                                           float *g0, float *g1) {
  uint32_t c[4] = {p, frame, 0u, 3u};
  philox4x32_10(c, k0, k1);
  const float r = sqrtf(-2.0f * logf(uniform_f32(c[0])));
  float s, co;
  sincospif(2.0f * uniform_f32(c[1]), &s, &co);
  *g0 = r * co;
  *g1 = r * s;
}

__global__ void __launch_bounds__(256) k_ccd(const float *__restrict__ det, float *__restrict__ out,
                                             int n, double scale, double ron, uint32_t k0,
                                             uint32_t k1, uint32_t frame0,
                                             const uint32_t *__restrict__ frame_dev) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t frame = frame0 + (frame_dev ? *frame_dev : 0u);
  const double lam = (double)det[p] * scale;
  const bool normal_branch = lam > kLambdaSwitch;
  float g0 = 0.f, g1 = 0.f;
  if (normal_branch || ron > 0.0) box_muller((uint32_t)p, frame, k0, k1, &g0, &g1);
  int k = 0;
  if (normal_branch) {
    const double v = floor(lam + sqrt(lam) * (double)g0 + 0.5);
    k = v > 0.0 ? (v < 2147483647.0 ? (int)v : 2147483647) : 0;
  } else {
    const float L = expf(-(float)lam);
    float prod = 1.f;
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    for (int j = 0; j <= kKmax; ++j) {
      if ((j & 3) == 0) {
        uint32_t w[4] = {(uint32_t)p, frame, (uint32_t)(j >> 2), 2u};
        philox4x32_10(w, k0, k1);
        w0 = w[0];
        w1 = w[1];
        w2 = w[2];
        w3 = w[3];
      }
      const uint32_t x = (j & 3) == 0 ? w0 : ((j & 3) == 1 ? w1 : ((j & 3) == 2 ? w2 : w3));
      prod = prod * uniform_f32(x);
      if (!(prod > L)) break;
      ++k;
    }
    k = k < kKmax ? k : kKmax;
  }
  const double rd = ron > 0.0 ? ron * (double)g1 : 0.0;
  out[p] = (float)((double)k + rd);
}

// Area-weighted rebinning n_in -> n_out (detector sampling at a non-integer
// pixel ratio): out[J][I] = sum_j sum_i wy(J, j) wx(I, i) in[j][i] with
// w(I, i) = |[i, i + 1) n [I b, (I + 1) b)|, b = n_in / n_out.  In units of
// 1 / n_out the overlaps are integers (n_in, n_out <= 4096 keep them exact in
// float32); the sum is taken row by row in index order and scaled by
// 1 / n_out^2 at the end.  One thread per output pixel.
__global__ void k_rebin(const float *__restrict__ in, int n_in, int n_out, int n_batch,
                        float *__restrict__ out) {
  const size_t per = (size_t)n_out * n_out;
  const float inv = 1.0f / ((float)n_out * (float)n_out);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < per * n_batch;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / per;
    const int J = (int)((e % per) / n_out), I = (int)(e % n_out);
    const float *src = in + b * (size_t)n_in * n_in;
    const int j0 = (J * n_in) / n_out, j1 = ((J + 1) * n_in - 1) / n_out;
    const int i0 = (I * n_in) / n_out, i1 = ((I + 1) * n_in - 1) / n_out;
    float acc = 0.f;
    for (int j = j0; j <= j1; ++j) {
      const int wy = min((j + 1) * n_out, (J + 1) * n_in) - max(j * n_out, J * n_in);
      float row = 0.f;
      for (int i = i0; i <= i1; ++i) {
        const int wx = min((i + 1) * n_out, (I + 1) * n_in) - max(i * n_out, I * n_in);
        row = fmaf((float)wx, src[(size_t)j * n_in + i], row);
      }
      acc = fmaf((float)wy, row, acc);
    }
    out[e] = acc * inv;
  }
}

}  // namespace specula

using namespace specula;

extern "C" int specula_rebin(specula_ctx *ctx, const float *in_dev, int32_t n_in, int32_t n_out,
                             int32_t n_batch, float *out_dev, void *stream) {
  if (!ctx || n_in < 1 || n_out < 1 || n_in > 4096 || n_out > 4096 || n_batch < 0)
    return SPECULA_EINVAL;
  if (n_batch == 0) return SPECULA_OK;
  if (!in_dev || !out_dev) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)n_out * n_out * n_batch;
  const unsigned grid = (unsigned)(n < (size_t)152 * 8 * 256 ? (n + 255) / 256 : 152 * 8);
  SPECULA_LAUNCH(ctx, SPECULA_K_CCD, st,
                 k_rebin<<<grid, 256, 0, st>>>(in_dev, n_in, n_out, n_batch, out_dev));
  return SPECULA_OK;
}

extern "C" int specula_ccd(specula_ctx *ctx, int32_t n, const float *det_dev, double scale,
                           double ron, uint64_t seed, uint32_t frame, const uint32_t *frame_dev,
                           float *out_dev, void *stream) {
  if (!ctx || !det_dev || !out_dev || n < 1) return SPECULA_EINVAL;
  if (!(scale >= 0.0) || !isfinite(scale) || !(ron >= 0.0) || !isfinite(ron))
    return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  SPECULA_LAUNCH(ctx, SPECULA_K_CCD, st,
                 k_ccd<<<(n + 255) / 256, 256, 0, st>>>(det_dev, out_dev, n, scale, ron,
                                                         (uint32_t)seed, (uint32_t)(seed >> 32),
                                                         frame, frame_dev));
  return SPECULA_OK;
}
