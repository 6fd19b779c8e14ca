// Closed adaptive-optics loop pieces (the SOUL example's DM, IirFilter
// integrator and delayed connection, App. B, Listing 2; Sect. 2.2 for the
// ":-1" delayed input): the modal mirror's shape, the residual phase with its
// statistics, and the integrator update.  Per step k of a loop:
//   residual = phi_atm(t_k) - B^T c_{k-1},   m = R (slopes(residual) - ref),
//   c_k = (1 - leak) c_{k-1} + gain m.
// Every sum runs in a fixed order (no float atomics), so a loop is
// bit-reproducible.
#include "internal.h"

namespace specula {

constexpr int kDmThreads = 256;
constexpr int kDmUnroll = 8;
constexpr int kLoopThreads = 256;

// phase[p] = sum over j = 0 .. n_modes-1, in order, of cmd[j] B[j][p]: one
// thread per pixel, the coefficients staged in shared memory, eight mode
// rows' loads in flight (consecutive threads read consecutive pixels).
__global__ void __launch_bounds__(kDmThreads) k_dm_shape(const float *__restrict__ B,
                                                         const float *__restrict__ cmd,
                                                         float *__restrict__ phase, int n_modes,
                                                         int n_pix2) {
  extern __shared__ float s_c[];
  for (int j = threadIdx.x; j < n_modes; j += blockDim.x) s_c[j] = cmd[j];
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix2) return;
  const float *b = B + p;
  float acc = 0.f;
  int j = 0;
  for (; j + kDmUnroll <= n_modes; j += kDmUnroll) {
    float v[kDmUnroll];
#pragma unroll
    for (int u = 0; u < kDmUnroll; ++u) v[u] = __ldg(b + (size_t)(j + u) * n_pix2);
#pragma unroll
    for (int u = 0; u < kDmUnroll; ++u) acc += s_c[j + u] * v[u];
  }
  for (; j < n_modes; ++j) acc += s_c[j] * __ldg(b + (size_t)j * n_pix2);
  phase[p] = acc;
}

// residual = atm - dm over the grid; per-CTA float64 partial sums over the
// pupil (weights amp): sum w, sum w r, sum w r^2, sum w cos(k r), sum w sin(k r)
// (k = lambda_wfs / lambda_sci), block-strided so the order is fixed.
__global__ void __launch_bounds__(kLoopThreads) k_loop_residual(
    const float *__restrict__ amp, const float *__restrict__ atm, const float *__restrict__ dm,
    float *__restrict__ resid, double *__restrict__ part, int n_pix2, float k) {
  __shared__ double s_p[5][kLoopThreads / 32];
  double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pix2; p += gridDim.x * blockDim.x) {
    const float r = atm[p] - dm[p];
    resid[p] = r;
    const double w = (double)amp[p];
    float sv, cv;
    sincosf(r * k, &sv, &cv);
    a[0] += w;
    a[1] += w * (double)r;
    a[2] += w * (double)r * (double)r;
    a[3] += w * (double)cv;
    a[4] += w * (double)sv;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double v = a[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_p[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int w = 0; w < kLoopThreads / 32; ++w) v += s_p[threadIdx.x][w];
    part[(size_t)blockIdx.x * 5 + threadIdx.x] = v;
  }
}

// stats[0] = sqrt(sum w r^2 / sum w - mean^2), stats[1] = |sum w e^{ikr}|^2 / (sum w)^2,
// the CTA partials summed in CTA order.
__global__ void k_loop_stats(const double *__restrict__ part, int n_part,
                             double *__restrict__ stats) {
  if (threadIdx.x != 0) return;
  double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < n_part; ++b)
    for (int q = 0; q < 5; ++q) a[q] += part[(size_t)b * 5 + q];
  if (!(a[0] > 0.0)) {
    stats[0] = 0.0;
    stats[1] = 0.0;
    return;
  }
  const double mean = a[1] / a[0];
  const double var = a[2] / a[0] - mean * mean;
  stats[0] = sqrt(var > 0.0 ? var : 0.0);
  stats[1] = (a[3] * a[3] + a[4] * a[4]) / (a[0] * a[0]);
}

__global__ void __launch_bounds__(256) k_loop_integrate(const float *__restrict__ m,
                                                        float *__restrict__ cmd, int n,
                                                        float keep, float gain) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) cmd[j] = keep * cmd[j] + gain * m[j];
}

int loop_alloc_workspace(specula_ctx *ctx) {
  if (cudaMalloc(&ctx->loop_part, (size_t)kLoopMaxBlocks * 5 * sizeof(double)) != cudaSuccess)
    return SPECULA_ENOMEM;
  return SPECULA_OK;
}

}  // namespace specula

using namespace specula;

extern "C" int specula_dm_shape(specula_ctx *ctx, int32_t n_modes, int32_t n_pix2,
                                const float *basis_dev, const float *cmd_dev, float *phase_dev,
                                void *stream) {
  if (!ctx || !basis_dev || !cmd_dev || !phase_dev) return SPECULA_EINVAL;
  if (n_modes < 1 || n_pix2 < 1) return SPECULA_EINVAL;
  if (n_modes > 12288) return SPECULA_EUNSUPPORTED;   // coefficients in 48 KB of shared memory
  cudaStream_t st = (cudaStream_t)stream;
  SPECULA_LAUNCH(ctx, SPECULA_K_LOOP, st,
                 k_dm_shape<<<(n_pix2 + kDmThreads - 1) / kDmThreads, kDmThreads,
                              n_modes * sizeof(float), st>>>(basis_dev, cmd_dev, phase_dev,
                                                             n_modes, n_pix2));
  return SPECULA_OK;
}

extern "C" int specula_loop_residual(specula_ctx *ctx, int32_t n_pix2, const float *amp_dev,
                                     const float *atm_dev, const float *dm_dev,
                                     double wfs_over_sci, float *resid_dev, double *stats_dev,
                                     void *stream) {
  if (!ctx || !amp_dev || !atm_dev || !dm_dev || !resid_dev || !stats_dev) return SPECULA_EINVAL;
  if (n_pix2 < 1 || !(wfs_over_sci > 0.0) || !isfinite(wfs_over_sci)) return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = (n_pix2 + kLoopThreads * 8 - 1) / (kLoopThreads * 8);
  blocks = blocks < 1 ? 1 : (blocks > kLoopMaxBlocks ? kLoopMaxBlocks : blocks);
  SPECULA_LAUNCH(ctx, SPECULA_K_LOOP, st,
                 k_loop_residual<<<blocks, kLoopThreads, 0, st>>>(
                     amp_dev, atm_dev, dm_dev, resid_dev, ctx->loop_part, n_pix2,
                     (float)wfs_over_sci));
  SPECULA_LAUNCH(ctx, SPECULA_K_LOOP, st,
                 k_loop_stats<<<1, 32, 0, st>>>(ctx->loop_part, blocks, stats_dev));
  return SPECULA_OK;
}

extern "C" int specula_loop_integrate(specula_ctx *ctx, int32_t n_modes, float gain, float leak,
                                      const float *modes_dev, float *cmd_dev, void *stream) {
  if (!ctx || !modes_dev || !cmd_dev || n_modes < 1) return SPECULA_EINVAL;
  if (!isfinite(gain) || !isfinite(leak) || leak < 0.f || leak > 1.f) return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  SPECULA_LAUNCH(ctx, SPECULA_K_LOOP, st,
                 k_loop_integrate<<<(n_modes + 255) / 256, 256, 0, st>>>(modes_dev, cmd_dev,
                                                                         n_modes, 1.f - leak,
                                                                         gain));
  return SPECULA_OK;
}
