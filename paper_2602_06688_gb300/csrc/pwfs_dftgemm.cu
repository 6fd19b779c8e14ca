// Modulated pyramid image with the two separable filters as dense DFT-as-GEMM
// contractions on the tensor cores (ModulatedPyramid + CCD binning, App. A,
// Tab. 4; the FFT workload column of Sect. 6, Tab. 2 for small padded grids).
//
// The separable form of pwfs.cu filters every pupil row with
//     K = IDFT_N . diag(mask / N) . DFT_N[:, pupil columns]      (N x n_pix)
// and then every column with the same K (the mask is the same per axis).  K
// only depends on (output - input - pupil offset) mod N, so the host builds
// it in float64 from one circulant kernel row
//     h[d] = sum_k mask[k] exp(2 pi i k d / N).
// Each filter is then one real GEMM on tcgen05 (gemm.cu): the complex
// product in its real embedding,
//     [Re Y | Im Y] = [Re U | Im U] . [[Re K, -Im K], [Im K, Re K]]^T,
// with three-term split precision along K to reach float32-level error:
//     A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,   x_lo = x - x_hi,
// in bf16 (SPECULA_PWFS_FORM_DFTGEMM_BF16) or tf32 (..._TF32) operands, FP32
// accumulation.  Per batch element:
//   field E (pwfs.cu)      -> pack rows: U[c][j][:] = E[j][:] gx[c][:], split
//   GEMM 1 (rows)          -> R[c][j][x]            (nc x n_pix rows)
//   pack columns           -> V[m][x][:] = R[c(m)][:][x] gy[m][:], split
//                             (a 32 x 32 tiled transpose)
//   GEMM 2 (columns)       -> Y[m][x][y]            (n_mod x N rows)
//   bins                   -> part[m] = the b x b bins of |Y[m]|^2 / n_mod, then
//                             det = the sum over m in order (as the FFT forms)
// The inverse row transform's output phase depends on x only and vanishes in
// |.|^2, as in the FFT forms.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <complex>
#include <cstring>
#include <vector>

#include "internal.h"

namespace specula {

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// hi and lo parts of x in the operand type
template <typename T> struct SplitOp;
template <> struct SplitOp<__nv_bfloat16> {
  static __device__ __forceinline__ void run(float x, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    *hi = h;
    *lo = __float2bfloat16_rn(x - __bfloat162float(h));
  }
};
template <> struct SplitOp<float> {
  static __device__ __forceinline__ void run(float x, float *hi, float *lo) {
    const float h = tf32_rna(x);
    *hi = h;
    *lo = tf32_rna(x - h);
  }
};

// A row of the split operand: [re hi | im hi | re hi | im hi | re lo | im lo],
// n_pix entries each (the order that meets [B_hi | B_lo | B_hi] along K).
template <typename T>
__device__ __forceinline__ void put_split(T *row, int n_pix, int i, float re, float im) {
  T rh, rl, ih, il;
  SplitOp<T>::run(re, &rh, &rl);
  SplitOp<T>::run(im, &ih, &il);
  row[i] = rh;
  row[n_pix + i] = ih;
  row[2 * n_pix + i] = rh;
  row[3 * n_pix + i] = ih;
  row[4 * n_pix + i] = rl;
  row[5 * n_pix + i] = il;
}

// Rows of GEMM 1: slot c (representative point m = c), pupil row j.
// grid (ceil(n_pix / 128), n_pix, nc); block 128.
template <typename T>
__global__ void k_dg_pack_rows(const float2 *__restrict__ field, const float2 *__restrict__ gx,
                               T *__restrict__ A, int n_pix) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pix) return;
  const int j = blockIdx.y, c = blockIdx.z;
  const float2 e = field[(size_t)j * n_pix + i], g = gx[(size_t)c * n_pix + i];
  const float re = e.x * g.x - e.y * g.y, im = e.x * g.y + e.y * g.x;
  put_split(A + ((size_t)c * n_pix + j) * 6 * n_pix, n_pix, i, re, im);
}

// Rows of GEMM 2: point m, column x; the inputs are R[c(m)][j][x] over the
// pupil rows j times gy[m][j].  32 x 32 tiles of (j, x) through shared memory:
// coalesced reads along x, coalesced writes along j.
// grid (ceil(N / 32), ceil(n_pix / 32), n_mod); block (32, 8).
template <typename T>
__global__ void k_dg_pack_cols(const float *__restrict__ R, const float2 *__restrict__ gy,
                               T *__restrict__ A, int n_pix, int N, int n_mod) {
  __shared__ float2 tile[32][33];
  const int x0 = blockIdx.x * 32, j0 = blockIdx.y * 32, m = blockIdx.z;
  const int c = m <= n_mod - m ? m : n_mod - m;   // the slot sharing cos(theta_m)
  const int tx = threadIdx.x;
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int j = j0 + ty, x = x0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (j < n_pix && x < N) {
      const float *row = R + ((size_t)c * n_pix + j) * 2 * N;
      v = make_float2(row[x], row[N + x]);
    }
    tile[ty][tx] = v;
  }
  __syncthreads();
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int x = x0 + ty, j = j0 + tx;
    if (x < N && j < n_pix) {
      const float2 v = tile[tx][ty], g = gy[(size_t)m * n_pix + j];
      const float re = v.x * g.x - v.y * g.y, im = v.x * g.y + v.y * g.x;
      put_split(A + ((size_t)m * N + x) * 6 * n_pix, n_pix, j, re, im);
    }
  }
}

// Per-point bins: part[m][yb][xb] = sum_{x, y in the bin} |Y[m][x][y]|^2 scale,
// summed in the order x, y; the detector is then the sum over m in order
// (k_bin_reduce of pwfs.cu).  grid (ceil(nd^2 / 128), n_mod); block 128;
// yb fastest, so a warp reads consecutive runs of y.
__global__ void k_dg_bins(const float *__restrict__ Y, float *__restrict__ part, int N, int bsz,
                          float scale) {
  const int nd = N / bsz;
  const int q = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  if (q >= nd * nd) return;
  const int yb = q % nd, xb = q / nd;
  float v = 0.f;
  for (int xx = 0; xx < bsz; ++xx) {
    const float *row = Y + ((size_t)m * N + xb * bsz + xx) * 2 * N + yb * bsz;
    for (int yy = 0; yy < bsz; ++yy) {
      const float re = row[yy], im = row[N + yy];
      v += (re * re + im * im) * scale;
    }
  }
  part[(size_t)m * nd * nd + (size_t)yb * nd + xb] = v;
}

// ---- host --------------------------------------------------------------------

static size_t round128(size_t n) { return (n + 127) / 128 * 128; }

int pwfs_dftgemm_prepare(PwfsPlan *p, int form) {
  const bool tf32 = form == SPECULA_PWFS_FORM_DFTGEMM_TF32;
  const int Np = p->n_pix, N = p->N, off = (N - Np) / 2;
  // GEMM shapes: 2N outputs (multiple of 128), K = 6 n_pix (multiple of the
  // operand's 128-byte row: 64 bf16 or 32 tf32); dense operators are meant
  // for small padded grids
  if (N > 512 || (2 * N) % 128 || (6 * Np) % (tf32 ? 32 : 64)) return SPECULA_EUNSUPPORTED;
  if (p->fq != 1) return SPECULA_EUNSUPPORTED;   // whole bins
  // circulant kernel row h[d] = sum_k mask[k] exp(2 pi i k d / N), float64
  std::vector<std::complex<double>> mk(N), h(N);
  for (int k = 0; k < N; ++k) {
    long long a = 2LL * k - N + 1;
    if (a < 0) a = -a;
    const double ang = -M_PI * (double)p->pup_dist * (double)a / (2.0 * N);
    mk[k] = std::complex<double>(cos(ang), sin(ang)) / (double)N;
  }
  for (int d = 0; d < N; ++d) {
    std::complex<double> acc = 0.0;
    for (int k = 0; k < N; ++k) {
      const long long r = ((long long)k * d) % N;
      const double ang = 2.0 * M_PI * (double)r / (double)N;
      acc += mk[k] * std::complex<double>(cos(ang), sin(ang));
    }
    h[d] = acc;
  }
  // B rows: o < N: [Re K, -Im K]; N + o: [Im K, Re K]; then [hi | lo | hi]
  const int K2 = 6 * Np;
  std::vector<float> Bf((size_t)2 * N * K2);
  auto split = [&](double v, float *hi, float *lo) {
    if (tf32) {
      auto rna = [](float f) {
        uint32_t u;
        memcpy(&u, &f, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        float r;
        memcpy(&r, &u, 4);
        return r;
      };
      const float x = (float)v;
      *hi = rna(x);
      *lo = rna(x - *hi);
    } else {
      const float x = (float)v;
      const __nv_bfloat16 hb = __float2bfloat16_rn(x);
      *hi = __bfloat162float(hb);
      *lo = __bfloat162float(__float2bfloat16_rn(x - *hi));
    }
  };
  for (int o = 0; o < N; ++o)
    for (int i = 0; i < Np; ++i) {
      const std::complex<double> kv = h[(((o - i - off) % N) + N) % N];
      const double vals[2][2] = {{kv.real(), -kv.imag()}, {kv.imag(), kv.real()}};
      for (int half = 0; half < 2; ++half) {
        float *row = Bf.data() + (size_t)(half * N + o) * K2;
        for (int part = 0; part < 2; ++part) {
          float hi, lo;
          split(vals[half][part], &hi, &lo);
          row[part * Np + i] = hi;                // B_hi
          row[2 * Np + part * Np + i] = lo;       // B_lo
          row[4 * Np + part * Np + i] = hi;       // B_hi
        }
      }
    }
  int s;
  if (tf32) {
    if ((s = p->dg_B.upload(Bf.data(), Bf.size() * sizeof(float)))) return s;
  } else {
    std::vector<__nv_bfloat16> Bb(Bf.size());
    for (size_t e = 0; e < Bf.size(); ++e) Bb[e] = __float2bfloat16_rn(Bf[e]);   // exact
    if ((s = p->dg_B.upload(Bb.data(), Bb.size() * sizeof(__nv_bfloat16)))) return s;
  }
  const size_t es = tf32 ? 4 : 2;
  p->dg_M1 = (int)round128((size_t)p->nc * Np);
  p->dg_M2 = (int)round128((size_t)p->n_mod * N);
  if ((s = p->dg_A1.alloc((size_t)p->dg_M1 * K2 * es))) return s;
  if ((s = p->dg_A2.alloc((size_t)p->dg_M2 * K2 * es))) return s;
  if ((s = p->dg_C1.alloc((size_t)p->dg_M1 * 2 * N * sizeof(float)))) return s;
  if ((s = p->dg_C2.alloc((size_t)p->dg_M2 * 2 * N * sizeof(float)))) return s;
  if ((s = p->dg_work.alloc((size_t)2 * p->dg_M1 * 2 * N * sizeof(float)))) return s;
  // the padding rows past nc n_pix and n_mod N stay zero
  SPECULA_CK(cudaMemset(p->dg_A1.p, 0, p->dg_A1.bytes));
  SPECULA_CK(cudaMemset(p->dg_A2.p, 0, p->dg_A2.bytes));
  if (p->field.bytes < (size_t)Np * Np * sizeof(float2)) {
    if ((s = p->field.alloc((size_t)Np * Np * sizeof(float2)))) return s;
    p->nbw = 1;
  }
  p->dg_form = form;
  return SPECULA_OK;
}

template <typename T>
static int dg_run_t(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                    int n_batch, float *det, cudaStream_t st) {
  constexpr bool tf32 = sizeof(T) == 4;
  const int Np = p->n_pix, N = p->N, K2 = 6 * Np;
  const int bsz = Np / p->n_sub, nd = N / bsz;
  const float scale = 1.0f / (float)p->n_mod;
  T *A1 = p->dg_A1.as<T>(), *A2 = p->dg_A2.as<T>();
  int s;
  for (int b = 0; b < n_batch; ++b) {
    if ((s = pwfs_field_launch(ctx, p, amp, phase, b, 1, st))) return s;
    const float2 *field = p->field.as<float2>() + (size_t)(b % p->nbw) * Np * Np;
    SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_DFTGEMM, st,
                   k_dg_pack_rows<T><<<dim3((Np + 127) / 128, Np, p->nc), 128, 0, st>>>(
                       field, p->gx.as<float2>(), A1, Np));
    if (tf32)
      s = gemm_tf32_tn(ctx, reinterpret_cast<const float *>(A1), p->dg_B.as<float>(), p->dg_M1,
                       2 * N, K2, p->dg_C1.as<float>(), 2, p->dg_work.as<float>(), st);
    else
      s = gemm_bf16_tn(ctx, A1, p->dg_B.p, p->dg_M1, 2 * N, K2, p->dg_C1.as<float>(), 2,
                       p->dg_work.as<float>(), st);
    if (s) return s;
    SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_DFTGEMM, st,
                   k_dg_pack_cols<T><<<dim3((N + 31) / 32, (Np + 31) / 32, p->n_mod), dim3(32, 8),
                                       0, st>>>(p->dg_C1.as<float>(), p->gy.as<float2>(), A2, Np,
                                                N, p->n_mod));
    if (tf32)
      s = gemm_tf32_tn(ctx, reinterpret_cast<const float *>(A2), p->dg_B.as<float>(), p->dg_M2,
                       2 * N, K2, p->dg_C2.as<float>(), 1, nullptr, st);
    else
      s = gemm_bf16_tn(ctx, A2, p->dg_B.p, p->dg_M2, 2 * N, K2, p->dg_C2.as<float>(), 1,
                       nullptr, st);
    if (s) return s;
    SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_DFTGEMM, st,
                   k_dg_bins<<<dim3((nd * nd + 127) / 128, p->n_mod), 128, 0, st>>>(
                       p->dg_C2.as<float>(),
                       p->part.as<float>() + (size_t)(b % p->nbw) * p->n_mod * nd * nd, N, bsz,
                       scale));
    if ((s = pwfs_bin_reduce_range(ctx, p, det, nd * nd, b, 1, st))) return s;
  }
  return SPECULA_OK;
}

int pwfs_dftgemm_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                     int n_batch, float *det, cudaStream_t st) {
  if (p->slot_hi >= 0) return SPECULA_EUNSUPPORTED;   // slot ranges: the two-pass forms
  if (p->dg_form == SPECULA_PWFS_FORM_DFTGEMM_TF32)
    return dg_run_t<float>(ctx, p, amp, phase, n_batch, det, st);
  return dg_run_t<__nv_bfloat16>(ctx, p, amp, phase, n_batch, det, st);
}

}  // namespace specula
