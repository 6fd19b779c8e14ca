// Infinite phase screens: the InfinitePhaseScreen data object (Tab. 3) and the
// AtmoInfiniteEvolution processing object (Tab. 4).  The paper names them
// without their construction; this is the conditional growth of Assemat,
// Wilson and Gendron (Optics Express 14, 988, 2006).  A screen grows one line
// (row or column) at a time, each new line Z drawn from its Gaussian
// distribution given the n_st lines behind it (X):
//
//   Z = A X + B b,  A = C_ZX C_XX^+,  B = (C_ZZ - A C_XZ)^(1/2),  b ~ N(0, I).
//
// Set-up (specula_infscreen_operators, float64 on the GPU):
//  * the von Karman phase covariance of the FFT screens' spectrum
//    (0.023 r0^-5/3 (f^2 + L0^-2)^-11/6) is, by its Hankel transform,
//      C(r) = 0.023 (2 pi / (2^(5/6) Gamma(11/6))) (L0/r0)^(5/3) x^nu K_nu(x),
//    x = 2 pi r / L0, nu = 5/6.  x^nu K_nu(x) is evaluated from the integral
//    K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the trapezoid rule
//    with step 1/16.  The integrand is analytic and even, so the rule
//    converges geometrically; with this step the discretisation error is far
//    below float64 rounding.  The sum stops once the terms are past their
//    peak and below 1e-18 of it.  Only (n_st + 1) side distances occur, so
//    one table of them feeds the three covariance blocks;
//  * C_XX = V diag(lambda) V^T by parallel Jacobi, A = C_ZX V diag(1/lambda)
//    V^T with eigenvalues at or below rcond lambda_max dropped;
//  * C_ZZ - A C_ZX^T = W diag(mu) W^T, B = W diag(sqrt(max(mu, 0))) W^T (the
//    symmetric square root).
// Per frame (specula_infscreen_lines): one CTA per (task, 16 output pixels);
// the stencil and the noise are staged in shared memory, each warp forms two
// output pixels' dot products (float32, lanes strided, then a butterfly sum)
// and writes them into the ring slot of the new line.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "internal.h"
#include "philox.cuh"

namespace specula {

constexpr int kInfMaxSide = 1024;
constexpr int kInfMaxStencil = 4;
constexpr int kInfRowsPerCta = 16;     // output pixels per CTA (two per warp)

// x^nu K_nu(x), x > 0, by the trapezoid rule on int_0^inf e^{-x cosh t} cosh(nu t) dt
__device__ double xnu_knu(double x, double nu) {
  const double h = 1.0 / 16.0;
  double sum = 0.5 * exp(-x);          // t = 0 (weight 1/2), cosh(0) = 1
  double peak = sum;
  for (int k = 1; k < 8192; ++k) {
    const double t = k * h;
    const double v = exp(-x * cosh(t)) * cosh(nu * t);
    sum += v;
    peak = fmax(peak, v);
    // past the peak (the integrand decreases once x sinh t > nu tanh(nu t))
    if (x * sinh(t) > nu && v < 1e-18 * peak) break;
  }
  return pow(x, nu) * (h * sum);
}

// T[d][q] = C(pitch sqrt(q^2 + d^2)), d = 0..n_st, q = 0..side-1
__global__ void k_vk_table(double *__restrict__ T, int side, int n_st, double pitch, double L0,
                           double scale, double c_zero) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (n_st + 1) * side) return;
  const int d = e / side, q = e % side;
  const double r = pitch * sqrt((double)q * q + (double)d * d);
  const double x = 2.0 * M_PI * r / L0;
  T[e] = scale * (x == 0.0 ? c_zero : xnu_knu(x, 5.0 / 6.0));
}

// C_XX[(d-1) side + p][(d'-1) side + p'] = T[|d - d'|][|p - p'|]   (m x m)
// C_ZX[p][(d-1) side + p']              = T[d][|p - p'|]          (side x m)
// C_ZZ[p][p']                           = T[0][|p - p'|]          (side x side)
__global__ void k_vk_blocks(const double *__restrict__ T, int side, int n_st,
                            double *__restrict__ Cxx, double *__restrict__ Czx,
                            double *__restrict__ Czz) {
  const int m = side * n_st;
  const size_t nxx = (size_t)m * m, nzx = (size_t)side * m, nzz = (size_t)side * side;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nxx + nzx + nzz;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < nxx) {
      const int i = (int)(e / m), j = (int)(e % m);
      const int d = i / side, p = i % side, d2 = j / side, p2 = j % side;
      Cxx[e] = T[(size_t)abs(d - d2) * side + abs(p - p2)];
    } else if (e < nxx + nzx) {
      const size_t f = e - nxx;
      const int p = (int)(f / m), j = (int)(f % m);
      const int d = j / side + 1, p2 = j % side;
      Czx[f] = T[(size_t)d * side + abs(p - p2)];
    } else {
      const size_t f = e - nxx - nzx;
      const int p = (int)(f / side), p2 = (int)(f % side);
      Czz[f] = T[abs(p - p2)];
    }
  }
}

// d[k] = f(lambda_k) from the diagonal of G: mode 0 1/lambda for lambda > rcond
// lambda_max (else 0); mode 1 sqrt(max(lambda, 0)).  One CTA, fixed order.
__global__ void k_eig_fn(const double *__restrict__ G, int n, int mode, double rcond,
                         double *__restrict__ d) {
  __shared__ double s_max;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, G[(size_t)k * n + k]);
    s_max = mx;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double l = G[(size_t)k * n + k];
    d[k] = mode == 0 ? ((l > rcond * s_max && l > 0.0) ? 1.0 / l : 0.0) : sqrt(fmax(l, 0.0));
  }
}

// S = (Czz - P + (Czz - P)^T) / 2 with P = A C_ZX^T (symmetrised)
__global__ void k_sym_diff(const double *__restrict__ Czz, const double *__restrict__ P, int n,
                           double *__restrict__ S) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const size_t i = e / n, j = e % n;
  S[e] = 0.5 * ((Czz[e] - P[e]) + (Czz[j * n + i] - P[j * n + i]));
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

struct InfTasks {
  specula_inf_line t[SPECULA_INF_MAX_TASKS];
};

__device__ __forceinline__ int ring_slot(int64_t line, int side) {
  const int64_t s = line % side;
  return (int)(s < 0 ? s + side : s);
}

// grid (ceil(side / kInfRowsPerCta), n_tasks), 256 threads
__global__ void __launch_bounds__(256) k_inf_lines(const __grid_constant__ InfTasks tasks,
                                                   int side, int n_st,
                                                   uint64_t seed,
                                                   const float *__restrict__ noise) {
  __shared__ float sx[kInfMaxSide * kInfMaxStencil];
  __shared__ float sb[kInfMaxSide];
  const specula_inf_line &T = tasks.t[blockIdx.y];
  const int m = side * n_st;
  float *scr = T.screen_dev;
  // stencil: line L - dir d at position p, X index (d - 1) side + p
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int d = k / side + 1, p = k % side;
    const int s = ring_slot(T.line - (int64_t)T.direction * d, side);
    sx[k] = T.axis == 0 ? scr[(size_t)s * side + p] : scr[(size_t)p * side + s];
  }
  if (noise) {
    for (int p = threadIdx.x; p < side; p += blockDim.x)
      sb[p] = noise[(size_t)blockIdx.y * side + p];
  } else {
    // Box-Muller in float32 (every CTA of the task needs all side values;
    // float64 transcendentals here cost more than the line's dot products)
    const uint64_t L = (uint64_t)T.line;
    for (int q = threadIdx.x; q < (side + 3) / 4; q += blockDim.x) {
      uint32_t c[4] = {(uint32_t)q, (uint32_t)L, (uint32_t)(L >> 32), (uint32_t)T.stream_id};
      philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
      float u[4], g[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) u[i] = ((float)c[i] + 0.5f) * 2.3283064365386963e-10f;  // 2^-32
      const float r0 = sqrtf(-2.0f * logf(u[0])), r1 = sqrtf(-2.0f * logf(u[2]));
      float s0, c0, s1, c1;
      sincospif(2.0f * u[1], &s0, &c0);
      sincospif(2.0f * u[3], &s1, &c1);
      g[0] = r0 * c0;
      g[1] = r0 * s0;
      g[2] = r1 * c1;
      g[3] = r1 * s1;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (4 * q + i < side) sb[4 * q + i] = g[i];
    }
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int snew = ring_slot(T.line, side);
  for (int r = warp; r < kInfRowsPerCta; r += 8) {
    const int i = blockIdx.x * kInfRowsPerCta + r;
    if (i >= side) break;
    const float *a = T.A_dev + (size_t)i * m;
    const float *b = T.B_dev + (size_t)i * side;
    float acc = 0.f, accb = 0.f;
    for (int k = lane; k < m; k += 32) acc = fmaf(a[k], sx[k], acc);
    for (int k = lane; k < side; k += 32) accb = fmaf(b[k], sb[k], accb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
      accb += __shfl_xor_sync(0xffffffffu, accb, o);
    }
    if (lane == 0) {
      const float v = fmaf(T.b_scale, accb, acc);
      if (T.axis == 0) scr[(size_t)snew * side + i] = v;
      else scr[(size_t)i * side + snew] = v;
    }
  }
}

}  // namespace specula

using namespace specula;

extern "C" int specula_infscreen_operators(specula_ctx *ctx, int32_t side, int32_t n_st,
                                           double pitch_m, double r0_m, double L0_m,
                                           double rcond, float *A_dev, float *B_dev,
                                           double *A64_dev, double *B64_dev, void *stream) {
  if (!ctx || !A_dev || !B_dev) return SPECULA_EINVAL;
  if (side < 2 || side > kInfMaxSide || n_st < 1 || n_st > kInfMaxStencil || n_st >= side)
    return SPECULA_EINVAL;
  if (!(pitch_m > 0) || !(r0_m > 0) || !(L0_m > 0) || !isfinite(pitch_m) || !isfinite(r0_m) ||
      !isfinite(L0_m) || !(rcond > 0) || !(rcond < 1))
    return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int m = side * n_st;
  DevBuf T, Cxx, Czx, Czz, V, D, W, A, P;
  int s;
  if ((s = T.alloc((size_t)(n_st + 1) * side * sizeof(double)))) return s;
  if ((s = Cxx.alloc((size_t)m * m * sizeof(double)))) return s;
  if ((s = Czx.alloc((size_t)side * m * sizeof(double)))) return s;
  if ((s = Czz.alloc((size_t)side * side * sizeof(double)))) return s;
  if ((s = V.alloc((size_t)m * m * sizeof(double)))) return s;
  if ((s = D.alloc((size_t)m * sizeof(double)))) return s;
  if ((s = W.alloc((size_t)m * m * sizeof(double)))) return s;
  if ((s = A.alloc((size_t)side * m * sizeof(double)))) return s;
  if ((s = P.alloc((size_t)side * side * sizeof(double)))) return s;
  const double nu = 5.0 / 6.0;
  const double scale = 0.023 * 2.0 * M_PI / (pow(2.0, nu) * tgamma(11.0 / 6.0)) *
                       pow(L0_m / r0_m, 5.0 / 3.0);
  const double c_zero = pow(2.0, nu - 1.0) * tgamma(nu);
  const int ne = (n_st + 1) * side;
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_vk_table<<<(ne + 127) / 128, 128, 0, st>>>(T.as<double>(), side, n_st, pitch_m,
                                                              L0_m, scale, c_zero));
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_vk_blocks<<<1216, 256, 0, st>>>(T.as<double>(), side, n_st, Cxx.as<double>(),
                                                   Czx.as<double>(), Czz.as<double>()));
  // A = C_ZX V diag(1/lambda) V^T
  if ((s = sym_eig_f64(ctx, st, Cxx.as<double>(), V.as<double>(), m))) return s;
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_eig_fn<<<1, 256, 0, st>>>(Cxx.as<double>(), m, 0, rcond, D.as<double>()));
  if ((s = gemm_f64(ctx, st, V.as<double>(), m, 1, V.as<double>(), 1, m, D.as<double>(),
                    W.as<double>(), m, m, m)))
    return s;
  if ((s = gemm_f64(ctx, st, Czx.as<double>(), m, 1, W.as<double>(), m, 1, nullptr,
                    A.as<double>(), side, m, m)))
    return s;
  // B = (C_ZZ - A C_ZX^T)^(1/2), reusing Cxx's storage for the side x side work
  if ((s = gemm_f64(ctx, st, A.as<double>(), m, 1, Czx.as<double>(), 1, m, nullptr,
                    P.as<double>(), side, side, m)))
    return s;
  double *S = Cxx.as<double>();
  double *Wz = V.as<double>();
  const size_t n2 = (size_t)side * side;
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_sym_diff<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(
                     Czz.as<double>(), P.as<double>(), side, S));
  if ((s = sym_eig_f64(ctx, st, S, Wz, side))) return s;
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_eig_fn<<<1, 256, 0, st>>>(S, side, 1, 0.0, D.as<double>()));
  // B = Wz diag(sqrt mu) Wz^T: the weights multiply one factor only, so form
  // Wz diag(sqrt mu) then multiply by Wz^T
  if ((s = gemm_f64(ctx, st, Wz, side, 1, Wz, 1, side, D.as<double>(), P.as<double>(), side,
                    side, side)))
    return s;
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_to_f32<<<256, 256, 0, st>>>(A.as<double>(), A_dev, (size_t)side * m));
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_to_f32<<<256, 256, 0, st>>>(P.as<double>(), B_dev, n2));
  if (A64_dev)
    SPECULA_CK(cudaMemcpyAsync(A64_dev, A.p, (size_t)side * m * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
  if (B64_dev)
    SPECULA_CK(cudaMemcpyAsync(B64_dev, P.p, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SPECULA_CK(cudaStreamSynchronize(st));   // the work arrays are freed on return
  return SPECULA_OK;
}

extern "C" int specula_infscreen_lines(specula_ctx *ctx, int32_t side, int32_t n_st,
                                       int32_t n_tasks, const specula_inf_line *tasks,
                                       uint64_t seed, const float *noise_dev, void *stream) {
  if (!ctx || !tasks) return SPECULA_EINVAL;
  if (side < 2 || side > kInfMaxSide || n_st < 1 || n_st > kInfMaxStencil || n_st >= side)
    return SPECULA_EINVAL;
  if (n_tasks < 0 || n_tasks > SPECULA_INF_MAX_TASKS) return SPECULA_EINVAL;
  if (n_tasks == 0) return SPECULA_OK;
  InfTasks P;
  for (int i = 0; i < n_tasks; ++i) {
    const specula_inf_line &t = tasks[i];
    if (!t.screen_dev || !t.A_dev || !t.B_dev || (t.axis != 0 && t.axis != 1) ||
        (t.direction != 1 && t.direction != -1) || !isfinite(t.b_scale))
      return SPECULA_EINVAL;
    for (int j = 0; j < i; ++j)
      if (tasks[j].screen_dev == t.screen_dev) return SPECULA_EINVAL;
    P.t[i] = t;
  }
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid((side + kInfRowsPerCta - 1) / kInfRowsPerCta, n_tasks);
  SPECULA_LAUNCH(ctx, SPECULA_K_INFSCREEN, st,
                 k_inf_lines<<<grid, 256, 0, st>>>(P, side, n_st, seed, noise_dev));
  return SPECULA_OK;
}

// ---- native ring planner --------------------------------------------------------

namespace specula {
// first / last fractional screen index of the pupil footprint along x
// (axis 1) or y (axis 0): the extraction's formula
// u = ((x s) + ((h theta) - (v t))) / pitch + side / 2 at the two pupil edges
static void inf_footprint(const specula_layer_desc &l, const specula_source_desc &src,
                          const specula_pupil_desc &pu, int side, double t, int axis,
                          double *first, double *last) {
  const double s = 1.0 - l.height_m / src.height_m;
  const double th = axis == 1 ? src.theta_x_rad : src.theta_y_rad;
  const double v = axis == 1 ? l.vx_mps : l.vy_mps;
  const double off = (l.height_m * th) - (v * t);
  const double x0 = (0 - (pu.n_pix - 1) / 2.0) * pu.pitch_m;
  const double x1 = ((pu.n_pix - 1) - (pu.n_pix - 1) / 2.0) * pu.pitch_m;
  const double u0 = ((x0 * s) + off) / l.pitch_m + side / 2.0;
  const double u1 = ((x1 * s) + off) / l.pitch_m + side / 2.0;
  *first = fmin(u0, u1);
  *last = fmax(u0, u1);
}

// at most this many lines per layer and axis in one plan (a larger jump in t
// is refused before any move is listed)
constexpr int64_t kInfMaxMovesPerAxis = (int64_t)1 << 20;

static int inf_plan(int32_t n_layers, const specula_layer_desc *layers,
                    const specula_source_desc *src, const specula_pupil_desc *pupil, int32_t side,
                    int32_t margin, double t, int64_t *lo, std::vector<specula_inf_move> *out) {
  if (n_layers < 0 || n_layers > SPECULA_INF_MAX_TASKS || (n_layers && (!layers || !lo)) ||
      !src || !pupil || side < 2 || side > kInfMaxSide || margin < 0 || margin > 64 ||
      !isfinite(t) || pupil->n_pix < 1 || !(pupil->pitch_m > 0))
    return SPECULA_EINVAL;
  for (int l = 0; l < n_layers; ++l) {
    if (!(layers[l].pitch_m > 0) || !isfinite(layers[l].vx_mps) || !isfinite(layers[l].vy_mps))
      return SPECULA_EINVAL;
    int64_t lo2[2] = {lo[2 * l], lo[2 * l + 1]};
    for (int axis = 1; axis >= 0; --axis) {   // columns first, then rows
      double a, b;
      inf_footprint(layers[l], *src, *pupil, side, t, axis, &a, &b);
      if (!isfinite(a) || !isfinite(b) || fabs(a) > 9e15 || fabs(b) > 9e15) return SPECULA_EINVAL;
      const int64_t first = (int64_t)floor(a) - margin, last = (int64_t)floor(b) + 1 + margin;
      if (last - first + 1 > side) return SPECULA_EUNSUPPORTED;   // ring too small
      int64_t w = lo2[axis];
      const int64_t need = w > first ? w - first : (last > w + side - 1 ? last - (w + side - 1) : 0);
      if (need > kInfMaxMovesPerAxis) return SPECULA_EUNSUPPORTED;
      while (w > first) {
        --w;
        out->push_back({l, axis, -1, w});
      }
      while (w + side - 1 < last) {
        out->push_back({l, axis, +1, w + side});
        ++w;
      }
      lo2[axis] = w;
    }
    lo[2 * l] = lo2[0];
    lo[2 * l + 1] = lo2[1];
  }
  return SPECULA_OK;
}
}  // namespace specula

extern "C" int specula_infscreen_plan(int32_t n_layers, const specula_layer_desc *layers,
                                      const specula_source_desc *source,
                                      const specula_pupil_desc *pupil, int32_t side,
                                      int32_t margin, double t, int64_t *lo, int32_t max_moves,
                                      specula_inf_move *moves, int32_t *n_moves) {
  if (!n_moves || max_moves < 0 || (max_moves && !moves)) return SPECULA_EINVAL;
  std::vector<int64_t> lo_try(lo ? lo : (int64_t *)nullptr,
                              lo ? lo + 2 * (size_t)(n_layers > 0 ? n_layers : 0) : nullptr);
  std::vector<specula_inf_move> mv;
  const int s = inf_plan(n_layers, layers, source, pupil, side, margin, t, lo_try.data(), &mv);
  if (s) return s;
  *n_moves = (int32_t)(mv.size() > 0x7fffffff ? 0x7fffffff : mv.size());
  if (mv.size() > (size_t)max_moves) return SPECULA_EUNSUPPORTED;
  for (size_t i = 0; i < mv.size(); ++i) moves[i] = mv[i];
  for (int i = 0; i < 2 * n_layers; ++i) lo[i] = lo_try[i];
  return SPECULA_OK;
}

extern "C" int specula_infscreen_advance(specula_ctx *ctx, int32_t n_layers,
                                         const specula_layer_desc *layers,
                                         const specula_source_desc *source,
                                         const specula_pupil_desc *pupil, int32_t side,
                                         int32_t n_st, int32_t margin, float *const *screens_dev,
                                         const float *const *A_dev, const float *const *B_dev,
                                         const float *b_scale, int64_t *lo, double t,
                                         uint64_t seed, int32_t *n_calls, void *stream) {
  if (!ctx || (n_layers && (!screens_dev || !A_dev || !B_dev || !b_scale))) return SPECULA_EINVAL;
  if (n_st < 1 || n_st > kInfMaxStencil || margin + n_st >= side) return SPECULA_EINVAL;
  std::vector<int64_t> lo_try(lo ? lo : (int64_t *)nullptr,
                              lo ? lo + 2 * (size_t)(n_layers > 0 ? n_layers : 0) : nullptr);
  std::vector<specula_inf_move> mv;
  int s = inf_plan(n_layers, layers, source, pupil, side, margin, t, lo_try.data(), &mv);
  if (s) return s;
  for (int l = 0; l < n_layers; ++l)
    if (!screens_dev[l] || !A_dev[l] || !B_dev[l] || !isfinite(b_scale[l])) return SPECULA_EINVAL;
  // per layer its moves in order; round k carries the k-th move of each layer
  std::vector<std::vector<specula_inf_move>> per(n_layers);
  for (const auto &m : mv) per[m.layer].push_back(m);
  size_t rounds = 0;
  for (const auto &p : per) rounds = p.size() > rounds ? p.size() : rounds;
  for (size_t k = 0; k < rounds; ++k) {
    specula_inf_line tasks[SPECULA_INF_MAX_TASKS];
    int n = 0;
    for (int l = 0; l < n_layers; ++l) {
      if (k >= per[l].size()) continue;
      const specula_inf_move &m = per[l][k];
      tasks[n++] = {screens_dev[l], A_dev[l], B_dev[l], b_scale[l], m.axis, m.direction,
                    2 * l + m.axis, m.line};
    }
    if ((s = specula_infscreen_lines(ctx, side, n_st, n, tasks, seed, nullptr, stream))) return s;
  }
  for (int i = 0; i < 2 * n_layers; ++i) lo[i] = lo_try[i];
  if (n_calls) *n_calls = (int32_t)rounds;
  return SPECULA_OK;
}
