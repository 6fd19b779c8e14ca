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
// The coordinates are separable (u depends on the column only, v on the row
// only), so k_atmo_coords evaluates them once per frame, 2 n_pix per layer,
// into a context-owned table (float64 is slow on this part: evaluating them
// per tile would cost more than the gathers).  k_atmo_extract covers 32 x 8
// pixel tiles: it stages its tile's table entries in shared memory, then each
// thread sums its pixel over the layers, four layers' gathers in flight at a
// time.  A warp reads 32 consecutive columns of one screen row: coalesced.
#include <math.h>

#include <mutex>

#include "internal.h"

namespace specula {

constexpr int kMaxLayers = SPECULA_ATMO_MAX_LAYERS;
constexpr int kMaxPix = SPECULA_ATMO_MAX_PIX;
constexpr int kTileX = 32, kTileY = 8;

struct AtmoParams {
  const float *scr[kMaxLayers];
  int side[kMaxLayers];
  double pitch[kMaxLayers], h[kMaxLayers], vx[kMaxLayers], vy[kMaxLayers];
  double s[kMaxLayers];   // cone factor 1 - h / H, rounded as on the device
  int n_layers;
  int n_pix;
  double pupil_pitch;
  double theta_x, theta_y, H;
  float scale;   // 500 / lambda
};

// table layout: [layer][axis (0 = x, 1 = y)][pixel]
__global__ void __launch_bounds__(256) k_atmo_coords(const AtmoParams P, double t_host,
                                                     const double *__restrict__ t_dev,
                                                     int *__restrict__ tab_i,
                                                     float *__restrict__ tab_f) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_pix;
  if (e >= P.n_layers * 2 * n) return;
  const int l = e / (2 * n), r = e % (2 * n);
  const int axis = r / n, idx = r % n;
  const double t = t_dev ? *t_dev : t_host;
  const double s = P.s[l];
  const double theta = axis ? P.theta_y : P.theta_x;
  const double v = axis ? P.vy[l] : P.vx[l];
  const int side = P.side[l];
  const double x = __dmul_rn(__dsub_rn((double)idx, (double)(n - 1) / 2.0), P.pupil_pitch);
  const double off = __dsub_rn(__dmul_rn(P.h[l], theta), __dmul_rn(v, t));
  const double u =
      __dadd_rn(__ddiv_rn(__dadd_rn(__dmul_rn(x, s), off), P.pitch[l]), (double)side / 2.0);
  const double u0 = floor(u);
  const double f = __dsub_rn(u, u0);
  long long k = (long long)u0 % side;
  if (k < 0) k += side;
  const size_t o = ((size_t)l * 2 + axis) * kMaxPix + idx;
  tab_i[o] = (int)k;
  tab_f[o] = (float)f;
}

__global__ void __launch_bounds__(256) k_atmo_extract(const AtmoParams P,
                                                      const int *__restrict__ tab_i,
                                                      const float *__restrict__ tab_f,
                                                      float *__restrict__ phase) {
  __shared__ int s_ix[kMaxLayers][kTileX], s_iy[kMaxLayers][kTileY];
  __shared__ float s_fx[kMaxLayers][kTileX], s_fy[kMaxLayers][kTileY];
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  constexpr int PER = kTileX + kTileY;
  for (int e = tid; e < P.n_layers * PER; e += nthr) {
    const int l = e / PER, r = e % PER;
    if (r < kTileX) {
      const int i = min(x0 + r, P.n_pix - 1);
      s_ix[l][r] = tab_i[(size_t)(2 * l) * kMaxPix + i];
      s_fx[l][r] = tab_f[(size_t)(2 * l) * kMaxPix + i];
    } else {
      const int q = r - kTileX;
      const int j = min(y0 + q, P.n_pix - 1);
      s_iy[l][q] = tab_i[(size_t)(2 * l + 1) * kMaxPix + j];
      s_fy[l][q] = tab_f[(size_t)(2 * l + 1) * kMaxPix + j];
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

int atmo_alloc_tables(specula_ctx *ctx) {
  const size_t n = (size_t)kMaxLayers * 2 * kMaxPix;
  if (cudaMalloc(&ctx->atmo_tab_i, n * sizeof(int)) != cudaSuccess) return SPECULA_ENOMEM;
  if (cudaMalloc(&ctx->atmo_tab_f, n * sizeof(float)) != cudaSuccess) return SPECULA_ENOMEM;
  return SPECULA_OK;
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
  if (pupil->n_pix < 1 || !(pupil->pitch_m > 0)) return SPECULA_EINVAL;
  if (pupil->n_pix > kMaxPix) return SPECULA_EUNSUPPORTED;
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
    P.s[l] = 1.0 - L.height_m / src->height_m;   // one IEEE division, one subtraction
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nc = n_layers * 2 * pupil->n_pix;
  SPECULA_LAUNCH(ctx, SPECULA_K_ATMO, st,
                 k_atmo_coords<<<(nc + 255) / 256, 256, 0, st>>>(P, t_s, t_dev, ctx->atmo_tab_i,
                                                                 ctx->atmo_tab_f));
  dim3 grid((pupil->n_pix + kTileX - 1) / kTileX, (pupil->n_pix + kTileY - 1) / kTileY);
  dim3 block(32, 8);
  SPECULA_LAUNCH(ctx, SPECULA_K_ATMO, st,
                 k_atmo_extract<<<grid, block, 0, st>>>(P, ctx->atmo_tab_i, ctx->atmo_tab_f,
                                                        phase_dev));
  return SPECULA_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of specula_atmo_extract.
//
// Some callers cannot call cudaMalloc: a host that runs its own CUDA graphs
// and may only enqueue work, a real-time loop with a fixed memory budget
// that forbids allocations after start-up, or an embedding that hands out
// every byte of device memory itself.  specula_atmo_extract needs the
// coordinate table that specula_ctx_create allocates; this variant keeps the
// table in a fixed device array instead, so it needs no context and
// allocates nothing.
//
// The array holds [64 layers][2 axes][8192 pixels] int32 sample indices
// followed by the same number of float32 fractions: 8 MiB, which every GPU
// that loads this library keeps until the process exits.  Every call shares
// it: calls whose kernels overlap on the GPU (different streams, or
// different threads) race on it and must be ordered by the caller.  Each
// call overwrites every entry it reads, so nothing needs clearing.
//
// The array's device address is looked up once per device, with that device
// current, by the first call made on it (cudaGetSymbolAddress; in host code
// the array's name is only a host-side stand-in).  Make that first call
// before any stream capture on the device.  The address is cached per device
// number for the rest of the process, so a device reset (which recreates the
// primary context and may move the array) leaves it stale: the header tells
// callers not to use this entry point on a device after a reset.
namespace {

constexpr int kNoAllocEntries = SPECULA_ATMO_MAX_LAYERS * 2 * SPECULA_ATMO_MAX_PIX;
static __device__ __align__(256) int32_t g_atmo_noalloc_scratch[2 * kNoAllocEntries];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

int noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SPECULA_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_atmo_noalloc_scratch) != cudaSuccess || !p)
      return SPECULA_ECUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SPECULA_OK;
}

}  // namespace

extern "C" int specula_atmo_extract_noalloc(int32_t n_layers, const specula_layer_desc *layers,
                                            const float *const *screens_dev,
                                            const specula_source_desc *src,
                                            const specula_pupil_desc *pupil, double t_s,
                                            const double *t_dev, float *phase_dev,
                                            void *stream) {
  if (!layers || !screens_dev || !src || !pupil || !phase_dev) return SPECULA_EINVAL;
  if (n_layers < 1) return SPECULA_EINVAL;
  if (n_layers > kMaxLayers) return SPECULA_EUNSUPPORTED;   // beyond the fixed array
  if (pupil->n_pix < 1 || !(pupil->pitch_m > 0)) return SPECULA_EINVAL;
  if (pupil->n_pix > kMaxPix) return SPECULA_EUNSUPPORTED;  // beyond the fixed array
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
    P.s[l] = 1.0 - L.height_m / src->height_m;   // one IEEE division, one subtraction
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPECULA_ECUDA;
  void *base = nullptr;
  int s = noalloc_scratch(dev, &base);
  if (s) return s;
  int *tab_i = static_cast<int *>(base);
  float *tab_f = reinterpret_cast<float *>(tab_i + kNoAllocEntries);
  cudaStream_t st = (cudaStream_t)stream;
  const int nc = n_layers * 2 * pupil->n_pix;
  k_atmo_coords<<<(nc + 255) / 256, 256, 0, st>>>(P, t_s, t_dev, tab_i, tab_f);
  if (cudaGetLastError() != cudaSuccess) return SPECULA_ECUDA;
  dim3 grid((pupil->n_pix + kTileX - 1) / kTileX, (pupil->n_pix + kTileY - 1) / kTileY);
  k_atmo_extract<<<grid, dim3(32, 8), 0, st>>>(P, tab_i, tab_f, phase_dev);
  if (cudaGetLastError() != cudaSuccess) return SPECULA_ECUDA;
  return SPECULA_OK;
}
