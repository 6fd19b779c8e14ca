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

// Non-finite guard: one status write per offending output, so the cost is
// nil when the slopes are finite.
__device__ __forceinline__ void guard_finite(float a, float b, int32_t *nf_status) {
  if (nf_status && !(isfinite(a) && isfinite(b))) atomicExch(nf_status, SPECULA_ENONFINITE);
}

// grid (ceil(n_valid / kPyrThreads), n_batch): every CTA forms the global
// normalisation T itself (the detector is small and L2-resident; the same
// fixed-order reduction in every CTA gives the same T bit for bit), then
// the slopes of its kPyrThreads subapertures from the four values each
// thread kept while summing T (its own subaperture is among those it
// sums: two dependent rounds of loads per frame, not four).  Index checks
// are branch-free (an out-of-range index reads subaperture 0 and is
// reported once per CTA), so the loads of several subapertures are in
// flight together.
__global__ void __launch_bounds__(kPyrThreads) k_pyr_slopes(
    const float *__restrict__ det, const int32_t *__restrict__ idx, const float *__restrict__ ref,
    int n_sub, int n_valid, float *__restrict__ out, int32_t *status, int32_t *nf_status) {
  __shared__ float s_w[kPyrThreads / 32];
  __shared__ float s_T;
  const int b = blockIdx.y;
  const int w2 = 2 * n_sub;
  const unsigned n2 = (unsigned)(n_sub * n_sub);
  const float *d = det + (size_t)b * w2 * w2;
  const int kown = blockIdx.x * kPyrThreads + threadIdx.x;   // this thread's output
  float r0 = 0.f, r1 = 0.f;
  if (ref && kown < n_valid) {
    r0 = ref[kown];
    r1 = ref[n_valid + kown];
  }
  float q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f;   // kown's four pupil-image values
  float part = 0.f;
  int bad = 0;
  for (int k0 = threadIdx.x; k0 < n_valid; k0 += 8 * kPyrThreads) {
    int sv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u * kPyrThreads;
      int s = k < n_valid ? __ldg(idx + k) : 0;
      bad |= (unsigned)s >= n2;
      sv[u] = (unsigned)s < n2 ? s : 0;
    }
    float q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int s = sv[u], a = s / n_sub, c = s - a * n_sub;
      const float v1 = d[(n_sub + a) * w2 + n_sub + c], v2 = d[(n_sub + a) * w2 + c];
      const float v3 = d[a * w2 + c], v4 = d[a * w2 + n_sub + c];
      q[u] = ((v1 + v2) + v3) + v4;
      if (k0 + u * kPyrThreads == kown) {
        q1 = v1;
        q2 = v2;
        q3 = v3;
        q4 = v4;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u * kPyrThreads < n_valid) part += q[u];
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = part;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < kPyrThreads / 32; ++i) t += s_w[i];
    s_T = t / (float)n_valid;
    if (bad) atomicExch(status, SPECULA_EINVAL);
  }
  __syncthreads();
  const float T = s_T;
  const int k = kown;
  if (k >= n_valid) return;
  float *o = out + (size_t)b * 2 * n_valid;
  float sx = ((q1 + q4) - (q2 + q3)) / T;
  float sy = ((q1 + q2) - (q3 + q4)) / T;
  if (ref) {
    sx -= r0;
    sy -= r1;
  }
  o[k] = sx;
  o[n_valid + k] = sy;
  guard_finite(sx, sy, nf_status);
}

// The same slopes from explicit detector indices of the four pupil images
// (map[q n_valid + k] for image q = Q1..Q4 of subaperture k; any padding and
// image separation): same grid, same fixed-order sums, the thread's own
// four values kept from the T pass.
__global__ void __launch_bounds__(kPyrThreads) k_pyr_slopes_maps(
    const float *__restrict__ det, const int32_t *__restrict__ map, const float *__restrict__ ref,
    int n_det2, int n_valid, float *__restrict__ out, int32_t *status, int32_t *nf_status) {
  __shared__ float s_w[kPyrThreads / 32];
  __shared__ float s_T;
  const int b = blockIdx.y;
  const float *d = det + (size_t)b * n_det2;
  const unsigned lim = (unsigned)n_det2;
  const int kown = blockIdx.x * kPyrThreads + threadIdx.x;   // this thread's output
  float r0 = 0.f, r1 = 0.f;
  if (ref && kown < n_valid) {
    r0 = ref[kown];
    r1 = ref[n_valid + kown];
  }
  float qo[4] = {0.f, 0.f, 0.f, 0.f};   // kown's four pupil-image values
  float part = 0.f;
  int bad = 0;
  for (int k0 = threadIdx.x; k0 < n_valid; k0 += 8 * kPyrThreads) {
    float q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u * kPyrThreads;
      int i[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int v = k < n_valid ? __ldg(map + (size_t)c * n_valid + k) : 0;
        bad |= (unsigned)v >= lim;
        i[c] = (unsigned)v < lim ? v : 0;
      }
      float v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = d[i[c]];
      q[u] = ((v[0] + v[1]) + v[2]) + v[3];
      if (k == kown) {
#pragma unroll
        for (int c = 0; c < 4; ++c) qo[c] = v[c];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u * kPyrThreads < n_valid) part += q[u];
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = part;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < kPyrThreads / 32; ++i) t += s_w[i];
    s_T = t / (float)n_valid;
    if (bad) atomicExch(status, SPECULA_EINVAL);
  }
  __syncthreads();
  const float T = s_T;
  const int k = kown;
  if (k >= n_valid) return;
  float *o = out + (size_t)b * 2 * n_valid;
  float sx = ((qo[0] + qo[3]) - (qo[1] + qo[2])) / T;
  float sy = ((qo[0] + qo[1]) - (qo[2] + qo[3])) / T;
  if (ref) {
    sx -= r0;
    sy -= r1;
  }
  o[k] = sx;
  o[n_valid + k] = sy;
  guard_finite(sx, sy, nf_status);
}

// One warp per (batch element, subaperture): centre of gravity of the spot.
__global__ void __launch_bounds__(256) k_sh_cog(const float *__restrict__ spots,
                                                const float *__restrict__ ref, int nf,
                                                int n_valid, int n_batch,
                                                float *__restrict__ out, int32_t *nf_status) {
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
    guard_finite(gx, gy, nf_status);
  }
}

int slopes_pyr_run(specula_ctx *ctx, const int32_t *idx, int n_sub, int n_valid,
                   const float *det, const float *ref, int n_batch, float *out, cudaStream_t st) {
  SPECULA_LAUNCH(ctx, SPECULA_K_SLOPES, st,
                 k_pyr_slopes<<<dim3((n_valid + kPyrThreads - 1) / kPyrThreads, n_batch),
                                kPyrThreads, 0, st>>>(det, idx, ref, n_sub, n_valid, out,
                                                      ctx->status_dev,
                                                      ctx->guard ? ctx->status_dev : nullptr));
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
  } else if (d->kind == SPECULA_SLOPES_PYR_MAPS) {
    if (!d->subap_idx_dev || d->n_sub < 1) return SPECULA_EINVAL;
    SPECULA_LAUNCH(ctx, SPECULA_K_SLOPES, st,
                   k_pyr_slopes_maps<<<dim3((d->n_valid + kPyrThreads - 1) / kPyrThreads, n_batch),
                                       kPyrThreads, 0, st>>>(
                       img_dev, d->subap_idx_dev, ref_dev, d->n_sub * d->n_sub, d->n_valid,
                       slopes_dev, ctx->status_dev, ctx->guard ? ctx->status_dev : nullptr));
  } else if (d->kind == SPECULA_SLOPES_SH) {
    if (d->fft_n < 2) return SPECULA_EINVAL;
    const long long tasks = (long long)d->n_valid * n_batch;
    SPECULA_LAUNCH(ctx, SPECULA_K_SLOPES, st,
                   k_sh_cog<<<(unsigned)((tasks + 7) / 8), 256, 0, st>>>(
                       img_dev, ref_dev, d->fft_n, d->n_valid, n_batch, slopes_dev,
                       ctx->guard ? ctx->status_dev : nullptr));
  } else {
    return SPECULA_EINVAL;
  }
  return SPECULA_OK;
}
