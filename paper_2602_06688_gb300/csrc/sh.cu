// Shack-Hartmann spots (SH / Lenslet / SubapData, App. A, Tabs. 3-4; the
// per-subaperture FFT workload of Sect. 6, Tab. 2).
//
// For each valid subaperture, its SP x SP block of E = amp exp(i phase) is
// centred in an NF x NF zero grid and imaged with the centred DFT:
//   spot = |DFT2(pad(E) . p_x p_y)|^2 / NF^2,  p(n) = exp(i pi (NF-1) n / NF)
// (the centred transform's output phase disappears in |.|^2).
//
// One warp per (batch element, subaperture): lanes r < SP transform the SP
// non-zero rows in registers (NF-point DFT, half the inputs zero), the row
// spectra are transposed through shared memory, lanes k < NF transform the
// columns and write the spot column-interleaved (coalesced across lanes).
#include <math.h>

#include "fft_regs.cuh"
#include "internal.h"

namespace specula {

int sh_init_device() {
  return upload_codelet_twiddles() == cudaSuccess ? SPECULA_OK : SPECULA_ECUDA;
}

constexpr int kShWarps = 8;

template <int NF, int SP>
__global__ void __launch_bounds__(kShWarps * 32) k_sh_spots(
    const float *__restrict__ amp, const float *__restrict__ phase,
    const int32_t *__restrict__ valid, const float2 *__restrict__ pre, int n_pix, int n_sub,
    int n_valid, int n_batch, float phase_scale, float *__restrict__ spots) {
  constexpr int OFF = (NF - SP) / 2;
  constexpr int XS = SP | 1;
  __shared__ float2 s_x[kShWarps][NF * XS];
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long task = (long long)blockIdx.x * kShWarps + w;
  const bool ok = task < (long long)n_valid * n_batch;
  const int bidx = ok ? (int)(task / n_valid) : 0;
  const int sidx = ok ? (int)(task % n_valid) : 0;
  const int idx = ok ? valid[sidx] : 0;
  const int a = idx / n_sub, bcol = idx % n_sub;
  float2 *xs = s_x[w];

  // rows: lane r < SP holds padded row OFF + r
  float2 v[NF];
#pragma unroll
  for (int n = 0; n < NF; ++n) v[n] = make_float2(0.f, 0.f);
  if (ok && lane < SP) {
    const size_t rowbase = (size_t)(a * SP + lane) * n_pix + (size_t)bcol * SP;
    const float *ph = phase + (size_t)bidx * n_pix * n_pix + rowbase;
    const float *am = amp + rowbase;
    const float2 py = pre[OFF + lane];
#pragma unroll
    for (int c = 0; c < SP; ++c) {
      float sv, cv;
      sincosf(ph[c] * phase_scale, &sv, &cv);
      const float A = am[c];
      v[OFF + c] = cmul(cmul(make_float2(A * cv, A * sv), pre[OFF + c]), py);
    }
  }
  RegDFT<NF, false>::run(v);
  __syncwarp();
  if (lane < SP) {
#pragma unroll
    for (int k = 0; k < NF; ++k) xs[k * XS + lane] = v[k];
  }
  __syncwarp();
  // columns: lane k < NF (spots wider than a warp: columns lane, lane + 32, ...)
  constexpr float inv = 1.0f / (float)(NF * NF);
#pragma unroll 1
  for (int k = lane; k < (NF > 32 ? NF : 32); k += 32) {
#pragma unroll
    for (int n = 0; n < NF; ++n) v[n] = make_float2(0.f, 0.f);
    if (k < NF) {
#pragma unroll
      for (int r = 0; r < SP; ++r) v[OFF + r] = xs[k * XS + r];
    }
    RegDFT<NF, false>::run(v);
    if (ok && k < NF) {
      float *dst = spots + (size_t)task * NF * NF + k;
#pragma unroll
      for (int q = 0; q < NF; ++q) dst[q * NF] = (v[q].x * v[q].x + v[q].y * v[q].y) * inv;
    }
  }
}

ShPlan *sh_plan_find(specula_ctx *ctx, const specula_pupil_desc *pupil, const specula_sh_desc *sh) {
  for (auto &p : ctx->sh)
    if (p->n_pix == pupil->n_pix && p->n_sub == sh->n_sub && p->sub_pix == sh->sub_pix &&
        p->fft_n == sh->fft_n && p->obsc == pupil->obsc_frac)
      return p.get();
  return nullptr;
}

int sh_plan_build(specula_ctx *ctx, const specula_pupil_desc *pupil, const specula_sh_desc *sh,
                  ShPlan **out) {
  std::unique_ptr<ShPlan> p(new ShPlan());
  p->n_pix = pupil->n_pix;
  p->n_sub = sh->n_sub;
  p->sub_pix = sh->sub_pix;
  p->fft_n = sh->fft_n;
  p->obsc = pupil->obsc_frac;
  std::vector<int32_t> idx((size_t)sh->n_sub * sh->n_sub);
  int32_t nv = 0;
  host_valid_subaps(pupil->n_pix, pupil->obsc_frac, sh->n_sub, idx.data(), &nv);
  p->n_valid = nv;
  const int NF = sh->fft_n;
  std::vector<float2> pre(NF);
  for (int n = 0; n < NF; ++n) {
    long long r = ((long long)(NF - 1) * n) % (2 * NF);
    const double ang = M_PI * (double)r / (double)NF;
    pre[n] = make_float2((float)cos(ang), (float)sin(ang));
  }
  int s;
  if ((s = p->valid.upload(idx.data(), (size_t)(nv > 0 ? nv : 1) * sizeof(int32_t)))) return s;
  if ((s = p->pre.upload(pre.data(), pre.size() * sizeof(float2)))) return s;
  *out = p.get();
  ctx->sh.push_back(std::move(p));
  return SPECULA_OK;
}

int sh_run(specula_ctx *ctx, ShPlan *p, const float *amp, const float *phase, int n_batch,
           float *spots, cudaStream_t st, float phase_scale) {
  // the imaged block of the valid list: spots are compact over it
  const int lo = p->sub_lo, nv = (p->sub_hi < 0 ? p->n_valid : p->sub_hi) - lo;
  const int32_t *valid = p->valid.as<int32_t>() + lo;
  const long long tasks = (long long)nv * n_batch;
  if (tasks == 0) return SPECULA_OK;
  const unsigned grid = (unsigned)((tasks + kShWarps - 1) / kShWarps);
  if (p->fft_n == 24 && p->sub_pix == 12)
    SPECULA_LAUNCH(ctx, SPECULA_K_SH, st,
                   k_sh_spots<24, 12><<<grid, kShWarps * 32, 0, st>>>(
                       amp, phase, valid, p->pre.as<float2>(), p->n_pix, p->n_sub, nv, n_batch,
                       phase_scale, spots));
  else if (p->fft_n == 16 && p->sub_pix == 8)
    SPECULA_LAUNCH(ctx, SPECULA_K_SH, st,
                   k_sh_spots<16, 8><<<grid, kShWarps * 32, 0, st>>>(
                       amp, phase, valid, p->pre.as<float2>(), p->n_pix, p->n_sub, nv, n_batch,
                       phase_scale, spots));
  else if (p->fft_n == 56 && p->sub_pix == 8)   // Tab. 2's SCAO SH spots (56 = 8 x 7)
    SPECULA_LAUNCH(ctx, SPECULA_K_SH, st,
                   k_sh_spots<56, 8><<<grid, kShWarps * 32, 0, st>>>(
                       amp, phase, valid, p->pre.as<float2>(), p->n_pix, p->n_sub, nv, n_batch,
                       phase_scale, spots));
  else if (p->fft_n == 68 && p->sub_pix == 4)   // Tab. 2's ERIS spots (68 = 4 x 17)
    SPECULA_LAUNCH(ctx, SPECULA_K_SH, st,
                   k_sh_spots<68, 4><<<grid, kShWarps * 32, 0, st>>>(
                       amp, phase, valid, p->pre.as<float2>(), p->n_pix, p->n_sub, nv, n_batch,
                       phase_scale, spots));
  else
    return SPECULA_EUNSUPPORTED;
  return SPECULA_OK;
}

// Polychromatic spots: accumulate weight r^2 (W S W^T) of one wavelength's
// spots S (pixel lambda_i / (NF d), 1 / r detector pixels, r = lambda_ref /
// lambda_i) onto the reference detector lattice.  W[o][j] is the overlap of
// detector pixel o, [o - NF/2 - 1/2, o - NF/2 + 1/2), with spot pixel j,
// [(j - NF/2 - 1/2) / r, (j - NF/2 + 1/2) / r), in detector pixels; r^2 turns
// a spot pixel's value into the flux density over its area.  One CTA per
// spot; out = (first ? 0 : out) + weight r^2 W S W^T, in the caller's order.
template <int NF>
__global__ void __launch_bounds__(256) k_sh_poly_acc(const float *__restrict__ spots, int n_spots,
                                                     float r, float wr2, int first,
                                                     float *__restrict__ out) {
  __shared__ float s_S[NF * NF], s_T[NF * NF], s_W[NF * NF];
  const int sp = blockIdx.x;
  if (sp >= n_spots) return;
  const float *S = spots + (size_t)sp * NF * NF;
  for (int e = threadIdx.x; e < NF * NF; e += blockDim.x) {
    s_S[e] = S[e];
    const int o = e / NF, j = e - o * NF;
    const float alo = (float)(o - NF / 2) - 0.5f, ahi = alo + 1.0f;
    const float blo = ((float)(j - NF / 2) - 0.5f) / r, bhi = ((float)(j - NF / 2) + 0.5f) / r;
    s_W[e] = fmaxf(0.f, fminf(ahi, bhi) - fmaxf(alo, blo));
  }
  __syncthreads();
  // T[o][jx] = sum_jy W[o][jy] S[jy][jx]
  for (int e = threadIdx.x; e < NF * NF; e += blockDim.x) {
    const int o = e / NF, jx = e - o * NF;
    float v = 0.f;
#pragma unroll 8
    for (int jy = 0; jy < NF; ++jy) v += s_W[o * NF + jy] * s_S[jy * NF + jx];
    s_T[e] = v;
  }
  __syncthreads();
  // D[oy][ox] = sum_jx T[oy][jx] W[ox][jx]
  float *D = out + (size_t)sp * NF * NF;
  for (int e = threadIdx.x; e < NF * NF; e += blockDim.x) {
    const int oy = e / NF, ox = e - oy * NF;
    float v = 0.f;
#pragma unroll 8
    for (int jx = 0; jx < NF; ++jx) v += s_T[oy * NF + jx] * s_W[ox * NF + jx];
    D[e] = first ? wr2 * v : D[e] + wr2 * v;
  }
}

int sh_poly_acc(specula_ctx *ctx, int fft_n, const float *spots, int n_spots, double ratio,
                double weight, bool first, float *out, cudaStream_t st) {
  if (n_spots == 0) return SPECULA_OK;
  const float r = (float)ratio, wr2 = (float)(weight * ratio * ratio);
  if (fft_n == 24)
    SPECULA_LAUNCH(ctx, SPECULA_K_SH, st,
                   k_sh_poly_acc<24><<<n_spots, 256, 0, st>>>(spots, n_spots, r, wr2,
                                                              first ? 1 : 0, out));
  else if (fft_n == 16)
    SPECULA_LAUNCH(ctx, SPECULA_K_SH, st,
                   k_sh_poly_acc<16><<<n_spots, 256, 0, st>>>(spots, n_spots, r, wr2,
                                                              first ? 1 : 0, out));
  else
    return SPECULA_EUNSUPPORTED;
  return SPECULA_OK;
}

}  // namespace specula
