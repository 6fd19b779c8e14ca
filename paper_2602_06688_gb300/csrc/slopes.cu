// Slope computers (PyrSlopec / ShSlopec, App. A, Tab. 4; Slopes, Tab. 3).
// Output per batch element: all x slopes, then all y slopes.  Every reduction
// runs in a fixed order (per-thread strided sums, then a fixed shuffle tree,
// then warps in index order), so results are bit-reproducible.
#include "internal.h"

namespace specula {

constexpr int kPyrThreads = 1024;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA per batch element.
// An index outside [0, n_sub^2) is recorded in the status word and read as
// subaperture 0 (never out of bounds).
__device__ __forceinline__ int checked_idx(const int32_t *idx, int k, int n_sub, int32_t *status) {
  int s = idx[k];
  if (s < 0 || s >= n_sub * n_sub) {
    atomicExch(status, SPECULA_EINVAL);
    s = 0;
  }
  return s;
}

__global__ void __launch_bounds__(kPyrThreads) k_pyr_slopes(
    const float *__restrict__ det, const int32_t *__restrict__ idx, const float *__restrict__ ref,
    int n_sub, int n_valid, float *__restrict__ out, int32_t *status) {
  __shared__ float s_w[kPyrThreads / 32];
  __shared__ float s_T;
  const int b = blockIdx.x;
  const int w2 = 2 * n_sub;
  const float *d = det + (size_t)b * w2 * w2;
  float part = 0.f;
#pragma unroll 4
  for (int k = threadIdx.x; k < n_valid; k += blockDim.x) {
    const int s = checked_idx(idx, k, n_sub, status);
    const int a = s / n_sub, c = s % n_sub;
    const float q1 = d[(n_sub + a) * w2 + n_sub + c], q2 = d[(n_sub + a) * w2 + c];
    const float q3 = d[a * w2 + c], q4 = d[a * w2 + n_sub + c];
    part += ((q1 + q2) + q3) + q4;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_w[i];
    s_T = t / (float)n_valid;
  }
  __syncthreads();
  const float T = s_T;
  float *o = out + (size_t)b * 2 * n_valid;
#pragma unroll 4
  for (int k = threadIdx.x; k < n_valid; k += blockDim.x) {
    const int s = checked_idx(idx, k, n_sub, status);
    const int a = s / n_sub, c = s % n_sub;
    const float q1 = d[(n_sub + a) * w2 + n_sub + c], q2 = d[(n_sub + a) * w2 + c];
    const float q3 = d[a * w2 + c], q4 = d[a * w2 + n_sub + c];
    float sx = ((q1 + q4) - (q2 + q3)) / T;
    float sy = ((q1 + q2) - (q3 + q4)) / T;
    if (ref) {
      sx -= ref[k];
      sy -= ref[n_valid + k];
    }
    o[k] = sx;
    o[n_valid + k] = sy;
  }
}

// One warp per (batch element, subaperture): centre of gravity of the spot.
__global__ void __launch_bounds__(256) k_sh_cog(const float *__restrict__ spots,
                                                const float *__restrict__ ref, int nf,
                                                int n_valid, int n_batch,
                                                float *__restrict__ out) {
  const long long task = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (task >= (long long)n_valid * n_batch) return;   // warp-uniform
  const int b = (int)(task / n_valid), k = (int)(task % n_valid);
  const float *sp = spots + (size_t)task * nf * nf;
  const float c = 0.5f * (float)(nf - 1);
  float si = 0.f, sx = 0.f, sy = 0.f;
  for (int e = lane; e < nf * nf; e += 32) {
    const float v = sp[e];
    const int y = e / nf, x = e - y * nf;
    si += v;
    sx += v * ((float)x - c);
    sy += v * ((float)y - c);
  }
  si = warp_sum(si);
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (lane == 0) {
    float gx = sx / si, gy = sy / si;
    if (ref) {
      gx -= ref[k];
      gy -= ref[n_valid + k];
    }
    out[(size_t)b * 2 * n_valid + k] = gx;
    out[(size_t)b * 2 * n_valid + n_valid + k] = gy;
  }
}

int slopes_pyr_run(specula_ctx *ctx, const int32_t *idx, int n_sub, int n_valid,
                   const float *det, const float *ref, int n_batch, float *out, cudaStream_t st) {
  SPECULA_LAUNCH(ctx, SPECULA_K_SLOPES, st,
                 k_pyr_slopes<<<n_batch, kPyrThreads, 0, st>>>(det, idx, ref, n_sub, n_valid, out,
                                                               ctx->status_dev));
  return SPECULA_OK;
}

}  // namespace specula

using namespace specula;

extern "C" int specula_slopes(specula_ctx *ctx, const specula_slopec_desc *d, const float *img_dev,
                              const float *ref_dev, int32_t n_batch, float *slopes_dev,
                              void *stream) {
  if (!ctx || !d || !img_dev || !slopes_dev || n_batch < 0) return SPECULA_EINVAL;
  if (d->n_valid < 1 || d->n_sub < 1) return SPECULA_EINVAL;
  if (n_batch == 0) return SPECULA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (d->kind == SPECULA_SLOPES_PYR) {
    if (!d->subap_idx_dev || d->n_valid > d->n_sub * d->n_sub) return SPECULA_EINVAL;
    return slopes_pyr_run(ctx, d->subap_idx_dev, d->n_sub, d->n_valid, img_dev, ref_dev, n_batch,
                          slopes_dev, st);
  } else if (d->kind == SPECULA_SLOPES_SH) {
    if (d->fft_n < 2) return SPECULA_EINVAL;
    const long long tasks = (long long)d->n_valid * n_batch;
    SPECULA_LAUNCH(ctx, SPECULA_K_SLOPES, st,
                   k_sh_cog<<<(unsigned)((tasks + 7) / 8), 256, 0, st>>>(
                       img_dev, ref_dev, d->fft_n, d->n_valid, n_batch, slopes_dev));
  } else {
    return SPECULA_EINVAL;
  }
  return SPECULA_OK;
}
