// Modulated pyramid, shifted-mask form (a second discretisation of the
// modulation of ModulatedPyramid, App. A, Tab. 4).
//
// The tilt form tilts the field by s_m = r pad (cos t_m, sin t_m) frequency
// bins before each forward transform.  The shifted-mask form takes the
// forward transform once per frame and moves the mask instead:
//   F = DFT2(padded field),  O_m = IDFT2(M(u + s_mx, v + s_my) F),
//   I = sum over m of |O_m|^2 / n_mod,
// with the analytic mask exp(-2 pi i c (|u + s_x| + |v + s_y|) / N) at the
// shifted frequencies.  It equals the tilt form up to a phase that vanishes
// in |O_m|^2 wherever no shifted frequency leaves the centred range, and
// differs where the field's spectrum wraps.
//
// The mask stays separable, so the inverse transform splits like the
// two-pass tilt form: a row pass per distinct shift s_x (points m and
// n_mod - m share cos t_m: n_mod / 2 + 1 slots) applies the x factor and the
// inverse row transform to every row of F, and a column pass per point m
// applies the y factor and the inverse column transform, squares, scales by
// 1 / n_mod and bins.  Against the tilt form no forward transform is done per
// point: the column pass does one transform per column instead of two.
//
//   k_sm_fwd_rows   field rows (amp exp(i phi) times the centred-DFT input
//                   phase), pruned forward row transform -> frows [Np][N]
//   k_sm_fwd_cols   input phase along y, pruned forward column transform
//                   -> F [N][N] (row-major)
//   k_sm_rowfilt    per (slot, row): x factor, inverse row transform
//                   -> R [slot][N][N]
//   k_sm_colfilt_bin per (point, column tile): y factor, inverse column
//                   transform, |.|^2 / n_mod, b x b bins -> part [m][nd][nd]
// followed by the detector reduction of the tilt form (modulation order).
#include <math.h>

#include <algorithm>

#include "fft_regs.cuh"
#include "internal.h"
#include "pwfs_common.cuh"

namespace specula {

int pwfs_shifted_init_device() {
  return upload_codelet_twiddles() == cudaSuccess ? SPECULA_OK : SPECULA_ECUDA;
}

namespace {

__device__ __forceinline__ void sm_cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void sm_cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Exchange buffer per one-group vector (complex): both split orders.
template <int N1, int N2> struct SmCfg {
  using S = Split<N1, N2>;
  static constexpr int XBF = N2 * S::S1 > N1 * S::S2 ? N2 * S::S1 : N1 * S::S2;
  static constexpr int CS = imax3(S::N, N2 * S::S1, N1 * S::S2) | 1;
};

// ---- forward transform of the padded field, rows ----------------------------
// grid ceil(n_pix / VPC), block VPC G: row j of the pupil, lane n1 < N1 holds
// the padded row's entries n1 + N1 n2; only n2 in [N2/4, 3 N2/4) are non-zero.
template <int N1, int N2>
__global__ void __launch_bounds__(256) k_sm_fwd_rows(const float *__restrict__ amp,
                                                     const float *__restrict__ phase,
                                                     const float2 *__restrict__ pre,
                                                     const float2 *__restrict__ twA,
                                                     float2 *__restrict__ frows, int n_pix,
                                                     float phase_scale) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  extern __shared__ float2 sm_x[];
  const int vpc = blockDim.x / G;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  float2 *xb = sm_x + vec * SmCfg<N1, N2>::XBF;
  const int j = blockIdx.x * vpc + vec;
  const bool row_ok = j < n_pix;
  float2 r[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  if (row_ok && lane < N1) {
#pragma unroll
    for (int h = 0; h < QH; ++h) {
      const int i = lane + N1 * h;                      // pupil column
      float sv, cv;
      sincosf(phase[(size_t)j * n_pix + i] * phase_scale, &sv, &cv);
      const float a = amp[(size_t)j * n_pix + i];
      r[Q0 + h] = cmul(make_float2(a * cv, a * sv), __ldg(pre + i));
    }
  }
  RegDFT<N2, false>::run(r);
  __syncwarp();
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = cmulc(r[k2], __ldg(twA + k2 * N1 + lane));
  }
  __syncwarp();
  float2 r2[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) r2[n1] = lane < N2 ? xb[lane * S1 + n1] : make_float2(0.f, 0.f);
  RegDFT<N1, false>::run(r2);
  if (row_ok && lane < N2) {
    float2 *dst = frows + (size_t)j * N + lane;        // frequency N2 k1 + lane
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) dst[N2 * k1] = r2[k1];
  }
}

// ---- forward transform, columns ----------------------------------------------
// grid N / TC, block TC G (TC = 4): the tile's n_pix rows are staged with
// 16-byte copies; warp c transforms column col0 + c (input phase along y).
template <int N1, int N2>
__global__ void __launch_bounds__(256) k_sm_fwd_cols(const float2 *__restrict__ frows,
                                                     const float2 *__restrict__ pre,
                                                     const float2 *__restrict__ twA,
                                                     float2 *__restrict__ fspec, int n_pix) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  constexpr int CS = SmCfg<N1, N2>::CS;
  extern __shared__ __align__(16) float2 sm_c[];
  const int TC = blockDim.x / G;                       // even: 16-byte rows
  const int WS = TC + 2;                               // window row stride (16-byte multiple)
  const int col0 = blockIdx.x * TC;
  const int nch = TC / 2;
  for (int e = threadIdx.x; e < n_pix * nch; e += blockDim.x) {
    const int jj = e / nch, q = e - jj * nch;
    sm_cp_async16(sm_c + jj * WS + 2 * q, frows + (size_t)jj * N + col0 + 2 * q);
  }
  sm_cp_async_wait_all();
  __syncthreads();
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  float2 r[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  if (lane < N1) {
#pragma unroll
    for (int h = 0; h < QH; ++h) {
      const int jj = lane + N1 * h;
      r[Q0 + h] = cmul(sm_c[jj * WS + vec], __ldg(pre + jj));
    }
  }
  __syncthreads();                                     // the window is reused below
  float2 *xb = sm_c + vec * CS;
  RegDFT<N2, false>::run(r);
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = cmulc(r[k2], __ldg(twA + k2 * N1 + lane));
  }
  __syncwarp();
  float2 r2[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) r2[n1] = lane < N2 ? xb[lane * S1 + n1] : make_float2(0.f, 0.f);
  RegDFT<N1, false>::run(r2);
  // through shared memory to whole rows of the tile: 16-byte stores of
  // consecutive columns instead of one 8-byte store per spectrum row
  __syncthreads();
  float2 *tile = sm_c;                                 // [N][TC]
  if (lane < N2) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) tile[(N2 * k1 + lane) * TC + vec] = r2[k1];   // row N2 k1 + lane
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * nch; e += blockDim.x) {
    const int v = e / nch, q = e - v * nch;
    *reinterpret_cast<float4 *>(fspec + (size_t)v * N + col0 + 2 * q) =
        *reinterpret_cast<const float4 *>(tile + v * TC + 2 * q);
  }
}

// ---- row pass: x factor of the slot's shifted mask, inverse row transform -----
// grid (ceil(N / VPC), slots), block VPC G.  Lane k2 < N2 loads frequencies
// N2 k1 + k2 of row v: the order the inverse transform's first step takes.
template <int N1, int N2>
__global__ void __launch_bounds__(256) k_sm_rowfilt(const float2 *__restrict__ fspec,
                                                    const float2 *__restrict__ mxs,
                                                    const float2 *__restrict__ twB,
                                                    float2 *__restrict__ rows, int slot0) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S2 = S::S2;
  extern __shared__ float2 sm_r[];
  const int vpc = blockDim.x / G;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  float2 *xb = sm_r + vec * SmCfg<N1, N2>::XBF;
  const int v = blockIdx.x * vpc + vec;
  const int it = blockIdx.y;
  const bool ok = v < N;
  const float2 *mk = mxs + (size_t)(slot0 + it) * N;
  float2 r2[N1];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) r2[k1] = make_float2(0.f, 0.f);
  if (ok && lane < N2) {
    const float2 *src = fspec + (size_t)v * N + lane;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) r2[k1] = cmul(src[N2 * k1], __ldg(mk + N2 * k1 + lane));
  }
  RegDFT<N1, true>::run(r2);
  if (lane < N2) {
#pragma unroll
    for (int k2 = 0; k2 < N1; ++k2) xb[k2 * S2 + lane] = cmul(r2[k2], __ldg(twB + k2 * N2 + lane));
  }
  __syncwarp();
  float2 r3[N2];
#pragma unroll
  for (int n1 = 0; n1 < N2; ++n1) r3[n1] = lane < N1 ? xb[lane * S2 + n1] : make_float2(0.f, 0.f);
  RegDFT<N2, true>::run(r3);
  if (ok && lane < N1) {
    float2 *dst = rows + ((size_t)it * N + v) * N + lane;   // x = N1 k1 + lane
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1) dst[N1 * k1] = r3[k1];
  }
}

// ---- column pass: y factor, inverse column transform, |.|^2, bins -------------
// grid (N / TC, 2 slots), block TC G; y = 2 p + w is point m = c (w = 0) or
// m = n_mod - c (w = 1, when distinct) of slot p = slot0 + blockIdx.y / 2.
// The tile (all N rows) is staged as a row-major window of W = TC rounded up
// to even columns from an even start column (16-byte cp.async.cg copies; the
// spare column of an odd TC may read the first entry of the next row, and
// the row buffer carries padding after its last row).
template <int N1, int N2, int MAXT = 256>
__global__ void __launch_bounds__(MAXT, MAXT <= 160 ? 4 : 3) k_sm_colfilt_bin(
    const float2 *__restrict__ rows, const float2 *__restrict__ mys,
    const float2 *__restrict__ twB, float *__restrict__ part, int bsz, float scale, int n_mod,
    int slot0) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S2 = S::S2;
  constexpr int CS = SmCfg<N1, N2>::CS;
  extern __shared__ __align__(16) float2 sm_k[];
  const int TC = blockDim.x / G;
  const int it = blockIdx.y >> 1;
  const int cslot = slot0 + it;
  const int m = (blockIdx.y & 1) ? n_mod - cslot : cslot;
  if ((blockIdx.y & 1) && (cslot == 0 || 2 * cslot == n_mod)) return;   // no second point
  const int col0 = blockIdx.x * TC;
  const int col0e = col0 & ~1, sh = col0 - col0e;
  const int W = (TC + 1) & ~1, nch = W / 2;
  {
    const float2 *src = rows + (size_t)it * N * N + col0e;
    for (int e = threadIdx.x; e < N * nch; e += blockDim.x) {
      const int jj = e / nch, q = e - jj * nch;
      sm_cp_async16(sm_k + jj * W + 2 * q, src + (size_t)jj * N + 2 * q);
    }
  }
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  sm_cp_async_wait_all();
  __syncthreads();
  float2 r2[N1];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) r2[k1] = make_float2(0.f, 0.f);
  if (lane < N2) {
    const float2 *mk = mys + (size_t)m * N + lane;
    const float2 *w = sm_k + sh + vec + lane * W;       // row N2 k1 + lane
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) r2[k1] = cmul(w[N2 * k1 * W], __ldg(mk + N2 * k1));
  }
  __syncthreads();                                     // the window is reused below
  float2 *col = sm_k + vec * CS;
  RegDFT<N1, true>::run(r2);
  if (lane < N2) {
#pragma unroll
    for (int k2 = 0; k2 < N1; ++k2) col[k2 * S2 + lane] = cmul(r2[k2], __ldg(twB + k2 * N2 + lane));
  }
  __syncwarp();
  float2 r3[N2];
#pragma unroll
  for (int n1 = 0; n1 < N2; ++n1) r3[n1] = lane < N1 ? col[lane * S2 + n1] : make_float2(0.f, 0.f);
  RegDFT<N2, true>::run(r3);
  __syncwarp();
  float *colI = reinterpret_cast<float *>(col);        // intensity, y = N1 k1 + lane
  if (lane < N1) {
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1)
      colI[N1 * k1 + lane] = (r3[k1].x * r3[k1].x + r3[k1].y * r3[k1].y) * scale;
  }
  __syncthreads();
  const int nd = N / bsz, nbx = TC / bsz;
  float *dst = part + (size_t)m * nd * nd;
  const float *s_I = reinterpret_cast<const float *>(sm_k);
  for (int q = threadIdx.x; q < nd * nbx; q += blockDim.x) {
    const int yb = q / nbx, xb = q - yb * nbx;
    float acc = 0.f;
    for (int rr = 0; rr < bsz; ++rr)
      for (int cc = 0; cc < bsz; ++cc) acc += s_I[(size_t)(xb * bsz + cc) * 2 * CS + yb * bsz + rr];
    dst[(size_t)yb * nd + col0 / bsz + xb] = acc;
  }
}

constexpr int kSmFwdColsTC = 4;   // columns per CTA of the forward column pass (even)
constexpr size_t kSmRowsL2Budget = 48u << 20;   // row-pass output kept under this per launch

template <int N1, int N2>
int sm_prepare(PwfsPlan *p) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G;
  const int Np = p->n_pix, bsz = Np / p->n_sub;
  if (2 * Np != N || Np != N1 * (N2 / 2)) return SPECULA_EUNSUPPORTED;   // pad 2: pruned halves
  if (p->fq != 1) return SPECULA_EUNSUPPORTED;                          // whole bins
  // column tile: TC = k bsz with TC G <= 256 (every bin in one CTA)
  int k = 0;
  for (int d = 1; d <= 2 * p->n_sub; ++d)
    if ((2 * p->n_sub) % d == 0 && d * bsz * G <= 256) k = d;
  if (k == 0 || N % (k * bsz) != 0 || N % kSmFwdColsTC != 0) return SPECULA_EUNSUPPORTED;
  const int tc = k * bsz;
  p->sm_blockK = tc * G;
  p->sm_smemK = std::max((size_t)N * ((tc + 1) & ~1), (size_t)tc * SmCfg<N1, N2>::CS) *
                sizeof(float2);
  p->sm_smemR = (size_t)(256 / G) * SmCfg<N1, N2>::XBF * sizeof(float2);
  p->sm_smemC = std::max(std::max((size_t)Np * (kSmFwdColsTC + 2), (size_t)N * kSmFwdColsTC),
                         (size_t)kSmFwdColsTC * SmCfg<N1, N2>::CS) * sizeof(float2);
  if (p->sm_smemK > 227 * 1024 || p->sm_smemC > 227 * 1024 || p->sm_smemR > 227 * 1024)
    return SPECULA_EUNSUPPORTED;
  int s;
  if ((s = ensure_dynamic_smem((const void *)k_sm_fwd_rows<N1, N2>, p->sm_smemR)) ||
      (s = ensure_dynamic_smem((const void *)k_sm_fwd_cols<N1, N2>, p->sm_smemC)) ||
      (s = ensure_dynamic_smem((const void *)k_sm_rowfilt<N1, N2>, p->sm_smemR)) ||
      (s = ensure_dynamic_smem((const void *)k_sm_colfilt_bin<N1, N2>, p->sm_smemK)) ||
      (s = ensure_dynamic_smem((const void *)k_sm_colfilt_bin<N1, N2, 160>, p->sm_smemK)))
    return s;
  // tables: input phase over the pupil, shifted mask factors per slot (x)
  // and per point (y), each with its 1 / N of the inverse normalisation
  const int off = (N - Np) / 2, nc = p->nc;
  std::vector<float2> pre(Np), mx((size_t)nc * N), my((size_t)p->n_mod * N);
  for (int i = 0; i < Np; ++i) {
    // exp(i pi (N-1) n / N) with (N-1) n reduced modulo 2N first
    const long long a = ((long long)(N - 1) * (off + i)) % (2LL * N);
    const double ang = M_PI * (double)a / (double)N;
    pre[i] = make_float2((float)cos(ang), (float)sin(ang));
  }
  const double c = p->pup_dist / 2.0, pad = (double)N / Np;
  auto axis = [&](double shift, float2 *t) {
    for (int q = 0; q < N; ++q) {
      const double u = (double)q - (N - 1) / 2.0;
      const double ang = -2.0 * M_PI * c * fabs(u + shift) / N;
      t[q] = make_float2((float)(cos(ang) / N), (float)(sin(ang) / N));
    }
  };
  for (int m = 0; m < p->n_mod; ++m) {
    const double th = 2.0 * M_PI * m / p->n_mod;
    if (m < nc) axis(p->mod_amp * pad * cos(th), mx.data() + (size_t)m * N);
    axis(p->mod_amp * pad * sin(th), my.data() + (size_t)m * N);
  }
  if ((s = p->sm_pre.upload(pre.data(), pre.size() * sizeof(float2))) ||
      (s = p->sm_mx.upload(mx.data(), mx.size() * sizeof(float2))) ||
      (s = p->sm_my.upload(my.data(), my.size() * sizeof(float2))))
    return s;
  p->sm_chunk = (int)std::max<size_t>(1, std::min<size_t>(nc, kSmRowsL2Budget / ((size_t)N * N * 8)));
  if ((s = p->sm_frows.alloc((size_t)Np * N * sizeof(float2))) ||
      (s = p->sm_fspec.alloc((size_t)N * N * sizeof(float2))) ||
      (s = p->sm_rows.alloc(((size_t)p->sm_chunk * N * N + 2) * sizeof(float2))) ||
      (s = p->sm_part.alloc((size_t)p->n_mod * (2 * p->n_sub) * (2 * p->n_sub) * sizeof(float))))
    return s;
  return SPECULA_OK;
}

template <int N1, int N2>
int sm_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase, int n_batch,
           float *det, cudaStream_t st) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G;
  const int Np = p->n_pix, bsz = Np / p->n_sub, nd = N / bsz, nc = p->nc;
  const int vpc = 256 / G, tc = p->sm_blockK / G;
  const float scale = 1.0f / (float)p->n_mod;
  for (int b = 0; b < n_batch; ++b) {
    SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_SM_FWD, st,
                   k_sm_fwd_rows<N1, N2><<<(Np + vpc - 1) / vpc, 256, p->sm_smemR, st>>>(
                       amp, phase + (size_t)b * Np * Np, p->sm_pre.as<float2>(),
                       p->twA.as<float2>(), p->sm_frows.as<float2>(), Np, p->run_phase_scale));
    SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_SM_FWD, st,
                   k_sm_fwd_cols<N1, N2><<<N / kSmFwdColsTC, kSmFwdColsTC * G, p->sm_smemC, st>>>(
                       p->sm_frows.as<float2>(), p->sm_pre.as<float2>(), p->twA.as<float2>(),
                       p->sm_fspec.as<float2>(), Np));
    for (int j0 = 0; j0 < nc; j0 += p->sm_chunk) {
      const int nj = std::min(p->sm_chunk, nc - j0);
      SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_SM_ROWS, st,
                     k_sm_rowfilt<N1, N2><<<dim3((N + vpc - 1) / vpc, nj), 256, p->sm_smemR, st>>>(
                         p->sm_fspec.as<float2>(), p->sm_mx.as<float2>(), p->twB.as<float2>(),
                         p->sm_rows.as<float2>(), j0));
      const dim3 gK(N / tc, 2 * nj);
      if (G == 32 && p->sm_blockK <= 160)
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_SM_COLS, st,
                       k_sm_colfilt_bin<N1, N2, 160><<<gK, p->sm_blockK, p->sm_smemK, st>>>(
                           p->sm_rows.as<float2>(), p->sm_my.as<float2>(), p->twB.as<float2>(),
                           p->sm_part.as<float>(), bsz, scale, p->n_mod, j0));
      else
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_SM_COLS, st,
                       k_sm_colfilt_bin<N1, N2><<<gK, p->sm_blockK, p->sm_smemK, st>>>(
                           p->sm_rows.as<float2>(), p->sm_my.as<float2>(), p->twB.as<float2>(),
                           p->sm_part.as<float>(), bsz, scale, p->n_mod, j0));
    }
    int s = pwfs_bin_reduce(ctx, p->sm_part.as<float>(), det + (size_t)b * nd * nd, nd * nd,
                            p->n_mod, p->run_alpha, p->run_beta, st);
    if (s) return s;
  }
  return SPECULA_OK;
}

}  // namespace

int pwfs_shifted_prepare(PwfsPlan *p) {
  switch (p->N) {
    case 64: return sm_prepare<8, 8>(p);
    case 128: return sm_prepare<8, 16>(p);
    case 240: return sm_prepare<15, 16>(p);
    case 320: return sm_prepare<20, 16>(p);
    case 960: return sm_prepare<30, 32>(p);
    default: return SPECULA_EUNSUPPORTED;
  }
}

int pwfs_shifted_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                     int n_batch, float *det, cudaStream_t st) {
  switch (p->N) {
    case 64: return sm_run<8, 8>(ctx, p, amp, phase, n_batch, det, st);
    case 128: return sm_run<8, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 240: return sm_run<15, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 320: return sm_run<20, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 960: return sm_run<30, 32>(ctx, p, amp, phase, n_batch, det, st);
    default: return SPECULA_EUNSUPPORTED;
  }
}

}  // namespace specula
