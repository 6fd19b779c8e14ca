// Detector noise of the CCD object (App. A, Tab. 4; App. B, Listing 2:
// photon_noise, readout_noise, readout_level, quantum_eff).  Pixel p of the
// noise-free detector image reads k + ron g, k ~ Poisson(lambda), lambda =
// det[p] scale (scale = photons per frame x quantum efficiency / pupil
// pixels), g a standard normal.  Draws: Philox4x32-10 with counter
// (p, frame, block, stream) and key (seed low, seed high).  Every step is a
// chain of IEEE basic operations with one rounding each (no library function
// and no contraction), so the counts are reproducible bit for bit by any
// implementation of the same steps:
//   lambda <= kLambdaSwitch: the multiplicative method (Knuth, TAOCP vol. 2,
//     3.4.1): k = the number of float32 uniforms whose running float32
//     product stays above L, at most kKmax; uniform j is word j mod 4 of
//     block j / 4 of stream 2; L = exp(-lambda) as T(lambda / 64)^64 in
//     float32, T the degree-9 Taylor polynomial of exp(-x) by Horner's rule;
//   lambda > kLambdaSwitch: k = max(0, floor(lambda + sqrt(lambda) g0 + 1/2))
//     in float64, g0 the Irwin-Hall normal of blocks 0-2 of stream 3 (the sum
//     of their twelve uniforms minus 6);
//   g: the Irwin-Hall normal of blocks 3-5 of stream 3.
// k + ron g is summed in float64 and rounded once to float32.  float64 is
// slow on this part; the common multiplicative branch runs in float32 and no
// branch calls a transcendental function.
#include <math.h>

#include "internal.h"
#include "philox.cuh"

namespace specula {

constexpr double kLambdaSwitch = 30.0;
constexpr int kKmax = 1000;

// 1 / k!, k = 0 .. 9, rounded once to float32
__constant__ float c_inv_fact[10] = {
    (float)1.0, (float)1.0, (float)(1.0 / 2.0), (float)(1.0 / 6.0), (float)(1.0 / 24.0),
    (float)(1.0 / 120.0), (float)(1.0 / 720.0), (float)(1.0 / 5040.0), (float)(1.0 / 40320.0),
    (float)(1.0 / 362880.0)};

__device__ __forceinline__ float exp_neg_f32(double lam) {
  const float x = __fmul_rn((float)lam, 0.015625f);          // lambda / 64, exact
  float p = c_inv_fact[9];
#pragma unroll
  for (int k = 8; k >= 0; --k) p = __fadd_rn(__fmul_rn(p, -x), c_inv_fact[k]);
#pragma unroll
  for (int i = 0; i < 6; ++i) p = __fmul_rn(p, p);
  return p;
}

// Sum of the twelve uniforms of blocks b0 .. b0 + 2 of stream 3, minus 6.
// Every uniform (x + 1/2) 2^-32 is a multiple of 2^-33 below 1 and the sum
// stays below 16, so the float64 sum is exact whatever the order: it equals
// (S + 6) 2^-32 with S the integer sum of the words.
__device__ __forceinline__ double irwin_hall(uint32_t p, uint32_t frame, uint32_t b0,
                                             uint32_t k0, uint32_t k1) {
  unsigned long long S = 6ull;
#pragma unroll
  for (uint32_t b = 0; b < 3; ++b) {
    uint32_t c[4] = {p, frame, b0 + b, 3u};
    philox4x32_10(c, k0, k1);
#pragma unroll
    for (int i = 0; i < 4; ++i) S += c[i];
  }
  return __dsub_rn(__dmul_rn((double)S, 1.0 / 4294967296.0), 6.0);
}

// The uniform (x + 1/2) 2^-32 rounded once to float32: (2x + 1) 2^-33 has at
// most 33 significant bits; the integer-to-float conversion rounds it once and
// the power-of-two scaling is exact.
__device__ __forceinline__ float uniform_f32(uint32_t x) {
  return __fmul_rn(__ull2float_rn(2ull * x + 1ull), 0x1p-33f);
}

__global__ void __launch_bounds__(256) k_ccd(const float *__restrict__ det, float *__restrict__ out,
                                             int n, double scale, double ron, uint32_t k0,
                                             uint32_t k1, uint32_t frame0,
                                             const uint32_t *__restrict__ frame_dev) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t frame = frame0 + (frame_dev ? *frame_dev : 0u);
  const double lam = __dmul_rn((double)det[p], scale);
  int k = 0;
  if (lam > kLambdaSwitch) {
    const double g0 = irwin_hall((uint32_t)p, frame, 0u, k0, k1);
    const double v = floor(__dadd_rn(__dadd_rn(lam, __dmul_rn(sqrt(lam), g0)), 0.5));
    k = v > 0.0 ? (v < 2147483647.0 ? (int)v : 2147483647) : 0;
  } else {
    const float L = exp_neg_f32(lam);
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
      prod = __fmul_rn(prod, uniform_f32(x));
      if (!(prod > L)) break;
      ++k;
    }
    k = k < kKmax ? k : kKmax;
  }
  const double rd = ron > 0.0 ? __dmul_rn(ron, irwin_hall((uint32_t)p, frame, 3u, k0, k1)) : 0.0;
  out[p] = (float)__dadd_rn((double)k, rd);
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
