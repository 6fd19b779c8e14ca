// Frozen-flow layer extraction along a source direction (AtmoEvolution +
// AtmoPropagation, App. A, Tab. 4; parameters of App. B, Listing 2).
//
// phase[j][i] = (500 / lambda) sum_l bilinear_periodic(S_l, u_l(i), v_l(j)),
//   u = ((x_i * s) + ((h * theta_x) - (vx * t))) / pitch_l + side_l / 2,
//   x_i = (i - (n - 1) / 2) * pupil_pitch,  s = 1 - h / H.
// floor(u) and the fraction are decided in float64 with the operations above
// in that order, rounded individually (no contraction), so the integer sample
// indices agree exactly with any IEEE float64 evaluation of the same formula.
// The interpolation and the layer sum run in float32.
//
// A CTA covers a 32 x 8 pixel tile: it first evaluates the tile's 32 column
// and 8 row coordinates of every layer in float64 into shared memory (40
// evaluations per layer instead of 256), then each thread sums its pixel over
// the layers, four layers' gathers in flight at a time.  A warp reads 32
// consecutive columns of one screen row: coalesced.
#include <math.h>

#include "internal.h"

namespace specula {

constexpr int kMaxLayers = 64;
constexpr int kTileX = 32, kTileY = 8;

struct AtmoParams {
  const float *scr[kMaxLayers];
  int side[kMaxLayers];
  double pitch[kMaxLayers], h[kMaxLayers], vx[kMaxLayers], vy[kMaxLayers];
  int n_layers;
  int n_pix;
  double pupil_pitch;
  double theta_x, theta_y, H;
  float scale;   // 500 / lambda
};

__device__ __forceinline__ void coord(double idx, int n, double pupil_pitch, double s, double h,
                                      double theta, double v, double t, double pitch, int side,
                                      int *i0, float *fr) {
  const double x = __dmul_rn(__dsub_rn(idx, (double)(n - 1) / 2.0), pupil_pitch);
  const double off = __dsub_rn(__dmul_rn(h, theta), __dmul_rn(v, t));
  const double u = __dadd_rn(__ddiv_rn(__dadd_rn(__dmul_rn(x, s), off), pitch), (double)side / 2.0);
  const double u0 = floor(u);
  const double f = __dsub_rn(u, u0);
  long long k = (long long)u0 % side;
  if (k < 0) k += side;
  *i0 = (int)k;
  *fr = (float)f;
}

__global__ void __launch_bounds__(256) k_atmo_extract(const AtmoParams P, double t_host,
                                                      const double *__restrict__ t_dev,
                                                      float *__restrict__ phase) {
  __shared__ int s_ix[kMaxLayers][kTileX], s_iy[kMaxLayers][kTileY];
  __shared__ float s_fx[kMaxLayers][kTileX], s_fy[kMaxLayers][kTileY];
  const double t = t_dev ? *t_dev : t_host;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  constexpr int PER = kTileX + kTileY;
  for (int e = tid; e < P.n_layers * PER; e += nthr) {
    const int l = e / PER, r = e % PER;
    const double s = __dsub_rn(1.0, __ddiv_rn(P.h[l], P.H));
    if (r < kTileX) {
      coord((double)(x0 + r), P.n_pix, P.pupil_pitch, s, P.h[l], P.theta_x, P.vx[l], t,
            P.pitch[l], P.side[l], &s_ix[l][r], &s_fx[l][r]);
    } else {
      const int q = r - kTileX;
      coord((double)(y0 + q), P.n_pix, P.pupil_pitch, s, P.h[l], P.theta_y, P.vy[l], t,
            P.pitch[l], P.side[l], &s_iy[l][q], &s_fy[l][q]);
    }
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = x0 + tx, j = y0 + ty;
  float acc = 0.f;
#pragma unroll 4
  for (int l = 0; l < P.n_layers; ++l) {
    const float *S = P.scr[l];
    const int M = P.side[l];
    const int ix0 = s_ix[l][tx];
    const int ix1 = ix0 + 1 == M ? 0 : ix0 + 1;
    const float fx = s_fx[l][tx];
    const int iy0 = s_iy[l][ty];
    const int iy1 = iy0 + 1 == M ? 0 : iy0 + 1;
    const float fy = s_fy[l][ty];
    const float s00 = __ldg(S + (size_t)iy0 * M + ix0), s01 = __ldg(S + (size_t)iy0 * M + ix1);
    const float s10 = __ldg(S + (size_t)iy1 * M + ix0), s11 = __ldg(S + (size_t)iy1 * M + ix1);
    const float a = s00 + fx * (s01 - s00);
    const float b = s10 + fx * (s11 - s10);
    acc += a + fy * (b - a);
  }
  if (i < P.n_pix && j < P.n_pix) phase[(size_t)j * P.n_pix + i] = acc * P.scale;
}

}  // namespace specula

using namespace specula;

extern "C" int specula_atmo_extract(specula_ctx *ctx, int32_t n_layers,
                                    const specula_layer_desc *layers,
                                    const float *const *screens_dev,
                                    const specula_source_desc *src,
                                    const specula_pupil_desc *pupil, double t_s,
                                    const double *t_dev, float *phase_dev, void *stream) {
  if (!ctx || !layers || !screens_dev || !src || !pupil || !phase_dev) return SPECULA_EINVAL;
  if (n_layers < 1) return SPECULA_EINVAL;
  if (n_layers > kMaxLayers) return SPECULA_EUNSUPPORTED;
  if (pupil->n_pix < 1 || pupil->n_pix > 16384 || !(pupil->pitch_m > 0)) return SPECULA_EINVAL;
  if (!(src->wavelength_nm > 0) || !(src->height_m > 0)) return SPECULA_EINVAL;
  if (!t_dev && !isfinite(t_s)) return SPECULA_EINVAL;
  AtmoParams P;
  P.n_layers = n_layers;
  P.n_pix = pupil->n_pix;
  P.pupil_pitch = pupil->pitch_m;
  P.theta_x = src->theta_x_rad;
  P.theta_y = src->theta_y_rad;
  P.H = src->height_m;
  P.scale = (float)(500.0 / src->wavelength_nm);
  for (int l = 0; l < n_layers; ++l) {
    const specula_layer_desc &L = layers[l];
    if (!screens_dev[l] || L.side < 2 || !(L.pitch_m > 0) || !isfinite(L.height_m) ||
        L.height_m < 0 || !isfinite(L.vx_mps) || !isfinite(L.vy_mps))
      return SPECULA_EINVAL;
    if (isfinite(src->height_m) && L.height_m >= src->height_m) return SPECULA_EINVAL;
    P.scr[l] = screens_dev[l];
    P.side[l] = L.side;
    P.pitch[l] = L.pitch_m;
    P.h[l] = L.height_m;
    P.vx[l] = L.vx_mps;
    P.vy[l] = L.vy_mps;
  }
  dim3 grid((pupil->n_pix + kTileX - 1) / kTileX, (pupil->n_pix + kTileY - 1) / kTileY);
  dim3 block(32, 8);
  SPECULA_LAUNCH(ctx, SPECULA_K_ATMO, (cudaStream_t)stream,
                 k_atmo_extract<<<grid, block, 0, (cudaStream_t)stream>>>(P, t_s, t_dev, phase_dev));
  return SPECULA_OK;
}
