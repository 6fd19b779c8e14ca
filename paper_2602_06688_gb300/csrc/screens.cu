// Von Karman phase screens by the FFT method with subharmonics (set-up call;
// AtmoEvolution, App. A, Tab. 4; Listing 2 `L0`, `Cn2`, `seed`).
//
//   Phi(f) = 0.023 r0^(-5/3) (|f|^2 + L0^-2)^(-11/6), Phi(0) = 0  [rad^2 m^2]
//   screen[y][x] = Re sum_k c_k sqrt(Phi(f_k)) df exp(2 pi i f_k . (x, y) pitch)
//                + subharmonics - their spatial mean
//
// Everything runs in float64 on the device (a set-up cost, not per frame):
// spectral weighting, a radix-2 Stockham FFT along rows in shared memory, a
// tiled transpose, the second row pass, and a final kernel that adds the
// separable subharmonic sum and rounds to float32 once.
#include <math.h>

#include <vector>

#include "internal.h"
#include "philox.cuh"

namespace specula {

// A[ky][kx] = noise[ky][kx] * sqrt(Phi(f)) * df
__global__ void k_psd_weight(const double2 *__restrict__ noise, double2 *__restrict__ A, int M,
                             double Md, double coef, double k0) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x, ky = blockIdx.y;
  if (kx >= M) return;
  const int sx = kx >= M / 2 ? kx - M : kx, sy = ky >= M / 2 ? ky - M : ky;
  const double fx = (double)sx / Md, fy = (double)sy / Md;
  const double f2 = fx * fx + fy * fy;
  double a = 0.0;
  if (f2 > 0.0) a = sqrt(coef * pow(f2 + k0, -11.0 / 6.0)) / Md;
  const double2 c = noise[(size_t)ky * M + kx];
  A[(size_t)ky * M + kx] = make_double2(c.x * a, c.y * a);
}

// In-place unnormalised inverse DFT of each row (exp(+2 pi i k n / M)),
// radix-2 Stockham in shared memory.  One CTA per row.
__global__ void k_fft_rows_f64(double2 *__restrict__ data, const double2 *__restrict__ tw, int M,
                               int logM) {
  extern __shared__ double2 sm[];
  double2 *a = sm, *b = sm + M;
  double2 *row = data + (size_t)blockIdx.x * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) a[i] = row[i];
  __syncthreads();
  // Stockham: stage with half-size Ls, stride; out[j*2Ls + k] etc.
  int L = 1;
  for (int s = 0; s < logM; ++s) {
    const int Ls = L;  // current sub-transform length
    L <<= 1;
    const int half = M / 2;
    for (int q = threadIdx.x; q < half; q += blockDim.x) {
      const int k = q % Ls;        // index within sub-transform
      const int j = q / Ls;        // which sub-transform pair
      const double2 u = a[j * Ls + k];
      const double2 v0 = a[j * Ls + k + half];
      // twiddle exp(+2 pi i k / L) = tw[k * (M / L)]
      const double2 w = tw[k * (M / L)];
      const double2 v = make_double2(v0.x * w.x - v0.y * w.y, v0.x * w.y + v0.y * w.x);
      b[j * L + k] = make_double2(u.x + v.x, u.y + v.y);
      b[j * L + k + Ls] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
    double2 *t = a; a = b; b = t;
  }
  for (int i = threadIdx.x; i < M; i += blockDim.x) row[i] = a[i];
}

__global__ void k_transpose_f64(const double2 *__restrict__ in, double2 *__restrict__ out, int M) {
  __shared__ double2 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    tile[r][threadIdx.x] = in[(size_t)(by + r) * M + bx + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    out[(size_t)(bx + r) * M + by + threadIdx.x] = tile[threadIdx.x][r];
}

// screen[y][x] = Re(T[x][y]) + sum_{p,a,b} Re(C[p][b][a] tx[p][a][x] tx[p][b][y]) - mean
__global__ void k_screen_final(const double2 *__restrict__ T, const double2 *__restrict__ tab,
                               const double2 *__restrict__ coef, double sub_mean, int M,
                               int levels, float *__restrict__ out) {
  __shared__ double2 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  // T is stored transposed: T[x][y]
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    tile[r][threadIdx.x] = T[(size_t)(bx + r) * M + by + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int y = by + r, x = bx + threadIdx.x;
    double v = tile[threadIdx.x][r].x;
    double sub = 0.0;
    for (int p = 0; p < levels; ++p)
      for (int bb = 0; bb < 3; ++bb)
        for (int aa = 0; aa < 3; ++aa) {
          if (aa == 1 && bb == 1) continue;
          const double2 ex = tab[((size_t)p * 3 + aa) * M + x];
          const double2 ey = tab[((size_t)p * 3 + bb) * M + y];
          const double2 e = make_double2(ex.x * ey.x - ex.y * ey.y, ex.x * ey.y + ex.y * ey.x);
          const double2 c = coef[(p * 3 + bb) * 3 + aa];
          sub += c.x * e.x - c.y * e.y;
        }
    out[(size_t)y * M + x] = (float)(v + (sub - sub_mean));
  }
}

// four standard normals for counter (pair index, sample, stream)
__device__ __forceinline__ void normals4(uint64_t pair, uint32_t sample, uint32_t stream,
                                         uint64_t seed, double g[4]) {
  uint32_t c[4] = {(uint32_t)pair, (uint32_t)(pair >> 32), sample, stream};
  philox_normals4(c, seed, g);
}

// n complex normals per sample: element 2i, 2i+1 from counter i
__global__ void k_rng_complex(uint64_t seed, int sample0, int stream_id, long long n,
                              double2 *__restrict__ out) {
  const long long pair = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (2 * pair >= n) return;
  double g[4];
  normals4((uint64_t)pair, (uint32_t)(sample0 + b), (uint32_t)stream_id, seed, g);
  out[(size_t)b * n + 2 * pair] = make_double2(g[0], g[1]);
  if (2 * pair + 1 < n) out[(size_t)b * n + 2 * pair + 1] = make_double2(g[2], g[3]);
}

// Philox screen noise (stream 0) times the spectral amplitude, per screen b
__global__ void k_noise_psd_batch(double2 *__restrict__ A, int M, double Md, double coef,
                                  double k0, uint64_t seed, int sample0) {
  const long long pair = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  const long long n = (long long)M * M;
  if (2 * pair >= n) return;
  double g[4];
  normals4((uint64_t)pair, (uint32_t)(sample0 + b), 0u, seed, g);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const long long e = 2 * pair + q;
    const int ky = (int)(e / M), kx = (int)(e % M);
    const int sx = kx >= M / 2 ? kx - M : kx, sy = ky >= M / 2 ? ky - M : ky;
    const double fx = (double)sx / Md, fy = (double)sy / Md;
    const double f2 = fx * fx + fy * fy;
    double a = 0.0;
    if (f2 > 0.0) a = sqrt(coef * pow(f2 + k0, -11.0 / 6.0)) / Md;
    A[(size_t)b * n + e] = make_double2(g[2 * q] * a, g[2 * q + 1] * a);
  }
}

__global__ void k_transpose_f64_batch(const double2 *__restrict__ in, double2 *__restrict__ out,
                                      int M) {
  __shared__ double2 tile[32][33];
  const size_t off = (size_t)blockIdx.z * M * M;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    tile[r][threadIdx.x] = in[off + (size_t)(by + r) * M + bx + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    out[off + (size_t)(bx + r) * M + by + threadIdx.x] = tile[threadIdx.x][r];
}

// per screen: subharmonic coefficients (Philox stream 1: 27 complex values,
// element (p * 3 + b) * 3 + a) times the amplitudes, and the spatial mean of
// the subharmonic sum (separable: sum Re(c mean(ex_a) mean(ey_b)))
__global__ void k_sub_coef_batch(const double *__restrict__ amp27, const double2 *__restrict__ tmean,
                                 uint64_t seed, int sample0, int n_screens,
                                 double2 *__restrict__ coef, double *__restrict__ sub_mean) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_screens) return;
  double2 c[28];
  for (int pr = 0; pr < 14; ++pr) {
    double g[4];
    normals4((uint64_t)pr, (uint32_t)(sample0 + b), 1u, seed, g);
    c[2 * pr] = make_double2(g[0], g[1]);
    c[2 * pr + 1] = make_double2(g[2], g[3]);
  }
  double mean = 0.0;
  for (int e = 0; e < 27; ++e) {
    const int p = e / 9, bb = (e / 3) % 3, a = e % 3;
    const double2 v = make_double2(c[e].x * amp27[e], c[e].y * amp27[e]);
    coef[(size_t)b * 27 + e] = v;
    const double2 mx = tmean[p * 3 + a], my = tmean[p * 3 + bb];
    const double2 m = make_double2(mx.x * my.x - mx.y * my.y, mx.x * my.y + mx.y * my.x);
    mean += v.x * m.x - v.y * m.y;
  }
  sub_mean[b] = mean;
}

__global__ void k_screen_final_batch(const double2 *__restrict__ T, const double2 *__restrict__ tab,
                                     const double2 *__restrict__ coef,
                                     const double *__restrict__ sub_mean, int M, int levels,
                                     float *__restrict__ out) {
  __shared__ double2 tile[32][33];
  const int b = blockIdx.z;
  const size_t off = (size_t)b * M * M;
  const double2 *cf = coef + (size_t)b * 27;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    tile[r][threadIdx.x] = T[off + (size_t)(bx + r) * M + by + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int y = by + r, x = bx + threadIdx.x;
    double sub = 0.0;
    for (int p = 0; p < levels; ++p)
      for (int bb = 0; bb < 3; ++bb)
        for (int aa = 0; aa < 3; ++aa) {
          if (aa == 1 && bb == 1) continue;
          const double2 ex = tab[((size_t)p * 3 + aa) * M + x];
          const double2 ey = tab[((size_t)p * 3 + bb) * M + y];
          const double2 e = make_double2(ex.x * ey.x - ex.y * ey.y, ex.x * ey.y + ex.y * ey.x);
          const double2 c = cf[(p * 3 + bb) * 3 + aa];
          sub += c.x * e.x - c.y * e.y;
        }
    out[off + (size_t)y * M + x] = (float)(tile[threadIdx.x][r].x + (sub - sub_mean[b]));
  }
}

// phase[b][j][i] = scale[b] * screen[b][j + o][i + o], o = (side - n) / 2
__global__ void k_random_phase(const float *__restrict__ scr, int side, int n,
                               const float *__restrict__ scale, float *__restrict__ phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, b = blockIdx.z;
  if (i >= n) return;
  const int o = (side - n) / 2;
  phase[((size_t)b * n + j) * n + i] =
      scale[b] * scr[((size_t)b * side + j + o) * side + i + o];
}

}  // namespace specula

using namespace specula;

static double psd_host(double fx, double fy, double r0, double L0) {
  const double f2 = fx * fx + fy * fy;
  if (!(f2 > 0)) return 0.0;
  const double k0 = isinf(L0) ? 0.0 : 1.0 / (L0 * L0);
  return 0.023 * pow(r0, -5.0 / 3.0) * pow(f2 + k0, -11.0 / 6.0);
}

extern "C" int specula_screen_generate(specula_ctx *ctx, int32_t side, double pitch_m,
                                       double r0_m, double L0_m, const double *noise_dev,
                                       const double *noise_sub_host, float *screen_dev,
                                       void *stream) {
  if (!ctx || !noise_dev || !noise_sub_host || !screen_dev) return SPECULA_EINVAL;
  if (side < 32 || side > 4096 || (side & (side - 1))) return SPECULA_EINVAL;
  if (!(pitch_m > 0) || !(r0_m > 0) || !(L0_m > 0)) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int M = side;
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  const double Md = (double)M * pitch_m;
  const double df = 1.0 / Md;
  const double coef = 0.023 * pow(r0_m, -5.0 / 3.0);
  const double k0 = isinf(L0_m) ? 0.0 : 1.0 / (L0_m * L0_m);
  const int levels = 3;

  // host tables: FFT twiddles exp(+2 pi i k / M); subharmonic exponentials and
  // coefficients; the spatial mean of the subharmonic sum
  std::vector<double2> tw(M / 2);
  for (int k = 0; k < M / 2; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)M;
    tw[k] = make_double2(cos(a), sin(a));
  }
  std::vector<double2> tab((size_t)levels * 3 * M), coefs(levels * 9);
  std::vector<double2> tmean(levels * 3);
  double sub_mean = 0.0;
  for (int p = 0; p < levels; ++p) {
    const double dfp = df / pow(3.0, p + 1);
    for (int a = 0; a < 3; ++a) {
      const double f = (a - 1) * dfp;
      double sr = 0, si = 0;
      for (int x = 0; x < M; ++x) {
        const double ang = 2.0 * M_PI * f * ((double)x * pitch_m);
        const double2 e = make_double2(cos(ang), sin(ang));
        tab[((size_t)p * 3 + a) * M + x] = e;
        sr += e.x;
        si += e.y;
      }
      tmean[p * 3 + a] = make_double2(sr / M, si / M);
    }
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        double2 c = make_double2(0, 0);
        if (!(a == 1 && b == 1)) {
          const double amp = sqrt(psd_host((a - 1) * dfp, (b - 1) * dfp, r0_m, L0_m)) * dfp;
          const double *n = noise_sub_host + 2 * ((p * 3 + b) * 3 + a);
          c = make_double2(n[0] * amp, n[1] * amp);
          const double2 mx = tmean[p * 3 + a], my = tmean[p * 3 + b];
          const double2 e = make_double2(mx.x * my.x - mx.y * my.y, mx.x * my.y + mx.y * my.x);
          sub_mean += c.x * e.x - c.y * e.y;
        }
        coefs[(p * 3 + b) * 3 + a] = c;
      }
  }

  DevBuf A, B, dtw, dtab, dcoef;
  int s;
  if ((s = A.alloc((size_t)M * M * sizeof(double2)))) return s;
  if ((s = B.alloc((size_t)M * M * sizeof(double2)))) return s;
  if ((s = dtw.upload(tw.data(), tw.size() * sizeof(double2)))) return s;
  if ((s = dtab.upload(tab.data(), tab.size() * sizeof(double2)))) return s;
  if ((s = dcoef.upload(coefs.data(), coefs.size() * sizeof(double2)))) return s;

  k_psd_weight<<<dim3((M + 255) / 256, M), 256, 0, st>>>((const double2 *)noise_dev,
                                                          A.as<double2>(), M, Md, coef, k0);
  SPECULA_CK_LAUNCH();
  const size_t sm = 2 * (size_t)M * sizeof(double2);
  if ((s = ensure_dynamic_smem((const void *)k_fft_rows_f64, sm))) return s;
  k_fft_rows_f64<<<M, 256, sm, st>>>(A.as<double2>(), dtw.as<double2>(), M, logM);
  SPECULA_CK_LAUNCH();
  k_transpose_f64<<<dim3(M / 32, M / 32), dim3(32, 8), 0, st>>>(A.as<double2>(), B.as<double2>(), M);
  SPECULA_CK_LAUNCH();
  k_fft_rows_f64<<<M, 256, sm, st>>>(B.as<double2>(), dtw.as<double2>(), M, logM);
  SPECULA_CK_LAUNCH();
  k_screen_final<<<dim3(M / 32, M / 32), dim3(32, 8), 0, st>>>(
      B.as<double2>(), dtab.as<double2>(), dcoef.as<double2>(), sub_mean, M, levels, screen_dev);
  SPECULA_CK_LAUNCH();
  // the temporaries are freed on return; wait for the kernels that use them
  SPECULA_CK(cudaStreamSynchronize(st));
  return SPECULA_OK;
}

extern "C" int specula_rng_complex(specula_ctx *ctx, uint64_t seed, int32_t sample0,
                                   int32_t n_samples, int32_t stream_id, int64_t n_per_sample,
                                   double *out_dev, void *stream) {
  if (!ctx || !out_dev || n_samples < 1 || n_per_sample < 1 || sample0 < 0 || stream_id < 0)
    return SPECULA_EINVAL;
  if (n_samples > 65535) return SPECULA_EUNSUPPORTED;
  const long long pairs = (n_per_sample + 1) / 2;
  dim3 grid((unsigned)((pairs + 255) / 256), n_samples);
  cudaStream_t st = (cudaStream_t)stream;
  SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                 k_rng_complex<<<grid, 256, 0, st>>>(seed, sample0, stream_id, n_per_sample,
                                                     (double2 *)out_dev));
  return SPECULA_OK;
}

extern "C" int specula_screen_generate_batch(specula_ctx *ctx, int32_t n_screens, int32_t side,
                                             double pitch_m, double r0_m, double L0_m,
                                             uint64_t seed, int32_t sample0, float *screens_dev,
                                             void *stream) {
  if (!ctx || !screens_dev || n_screens < 1 || sample0 < 0) return SPECULA_EINVAL;
  if (side < 32 || side > 4096 || (side & (side - 1))) return SPECULA_EINVAL;
  if (!(pitch_m > 0) || !(r0_m > 0) || !(L0_m > 0)) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int M = side;
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  const double Md = (double)M * pitch_m;
  const double df = 1.0 / Md;
  const double coef = 0.023 * pow(r0_m, -5.0 / 3.0);
  const double k0 = isinf(L0_m) ? 0.0 : 1.0 / (L0_m * L0_m);
  const int levels = 3;
  std::vector<double2> tw(M / 2);
  for (int k = 0; k < M / 2; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)M;
    tw[k] = make_double2(cos(a), sin(a));
  }
  std::vector<double2> tab((size_t)levels * 3 * M), tmean(levels * 3);
  std::vector<double> amp27(27, 0.0);
  for (int p = 0; p < levels; ++p) {
    const double dfp = df / pow(3.0, p + 1);
    for (int a = 0; a < 3; ++a) {
      const double f = (a - 1) * dfp;
      double sr = 0, si = 0;
      for (int x = 0; x < M; ++x) {
        const double ang = 2.0 * M_PI * f * ((double)x * pitch_m);
        const double2 e = make_double2(cos(ang), sin(ang));
        tab[((size_t)p * 3 + a) * M + x] = e;
        sr += e.x;
        si += e.y;
      }
      tmean[p * 3 + a] = make_double2(sr / M, si / M);
    }
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        if (!(a == 1 && b == 1))
          amp27[(p * 3 + b) * 3 + a] = sqrt(psd_host((a - 1) * dfp, (b - 1) * dfp, r0_m, L0_m)) * dfp;
  }
  DevBuf dtw, dtab, dtmean, damp;
  int s;
  if ((s = dtw.upload(tw.data(), tw.size() * sizeof(double2)))) return s;
  if ((s = dtab.upload(tab.data(), tab.size() * sizeof(double2)))) return s;
  if ((s = dtmean.upload(tmean.data(), tmean.size() * sizeof(double2)))) return s;
  if ((s = damp.upload(amp27.data(), amp27.size() * sizeof(double)))) return s;
  // screens per group: two complex float64 work arrays of at most 1 GiB in all
  const size_t per = (size_t)M * M * sizeof(double2);
  const int G = (int)std::max<size_t>(1, std::min<size_t>(n_screens, (1ull << 30) / (2 * per)));
  DevBuf A, B, cf, sm;
  if ((s = A.alloc(G * per)) || (s = B.alloc(G * per)) ||
      (s = cf.alloc((size_t)G * 27 * sizeof(double2))) || (s = sm.alloc((size_t)G * sizeof(double))))
    return s;
  const size_t smem = 2 * (size_t)M * sizeof(double2);
  if ((s = ensure_dynamic_smem((const void *)k_fft_rows_f64, smem))) return s;
  for (int g0 = 0; g0 < n_screens; g0 += G) {
    const int ng = std::min(G, n_screens - g0);
    const long long pairs = (long long)M * M / 2;
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_noise_psd_batch<<<dim3((unsigned)((pairs + 255) / 256), ng), 256, 0, st>>>(
                       A.as<double2>(), M, Md, coef, k0, seed, sample0 + g0));
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_fft_rows_f64<<<ng * M, 256, smem, st>>>(A.as<double2>(), dtw.as<double2>(), M,
                                                             logM));
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_transpose_f64_batch<<<dim3(M / 32, M / 32, ng), dim3(32, 8), 0, st>>>(
                       A.as<double2>(), B.as<double2>(), M));
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_fft_rows_f64<<<ng * M, 256, smem, st>>>(B.as<double2>(), dtw.as<double2>(), M,
                                                             logM));
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_sub_coef_batch<<<(ng + 63) / 64, 64, 0, st>>>(
                       damp.as<double>(), dtmean.as<double2>(), seed, sample0 + g0, ng,
                       cf.as<double2>(), sm.as<double>()));
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_screen_final_batch<<<dim3(M / 32, M / 32, ng), dim3(32, 8), 0, st>>>(
                       B.as<double2>(), dtab.as<double2>(), cf.as<double2>(), sm.as<double>(), M,
                       levels, screens_dev + (size_t)g0 * M * M));
  }
  SPECULA_CK(cudaStreamSynchronize(st));   // the work arrays are freed on return
  return SPECULA_OK;
}

extern "C" int specula_random_phase(specula_ctx *ctx, const float *screens_dev, int32_t n,
                                    int32_t side, int32_t n_pix, const float *scale_dev,
                                    float *phase_dev, void *stream) {
  if (!ctx || !screens_dev || !scale_dev || !phase_dev || n < 1 || n_pix < 1 || side < n_pix)
    return SPECULA_EINVAL;
  if (n > 65535) return SPECULA_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((n_pix + 127) / 128, n_pix, n);
  SPECULA_LAUNCH(ctx, SPECULA_K_ATMO, st,
                 k_random_phase<<<grid, 128, 0, st>>>(screens_dev, side, n_pix, scale_dev,
                                                      phase_dev));
  return SPECULA_OK;
}
