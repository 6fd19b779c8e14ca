// Modal reconstructor: modes[b] = R slopes[b] (Modalrec / Recmat, App. A,
// Tabs. 3-4; Listing 2 `recmat_object`).
//
// At batch 1 the product is bound by reading R once from HBM (4 bytes per
// element in float32, 2 in bfloat16).  One warp owns one row of R and streams
// it with 16-byte loads that bypass L1 allocation; the slope vectors stay in
// L1 through read-only loads.  NB slope vectors share each row load.  The
// per-lane partial sums run in a fixed order and are combined by a fixed
// shuffle tree: bit-reproducible.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"

namespace specula {

constexpr int kReconWarps = 8;

__device__ __forceinline__ float4 ld_stream(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

__device__ __forceinline__ float warp_sum_r(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32, vectorised (n_slopes % 4 == 0, 16-byte aligned rows).
template <int NB>
__global__ void __launch_bounds__(kReconWarps * 32) k_mvm_f32(
    const float *__restrict__ R, const float *__restrict__ s, float *__restrict__ m, int n_modes,
    int n_slopes, int n_batch, int b0) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n_modes) return;
  const float4 *r4 = reinterpret_cast<const float4 *>(R + (size_t)row * n_slopes);
  const int n4 = n_slopes / 4;
  float acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) acc[q] = 0.f;
  // UL independent 16-byte row loads in flight per lane
  constexpr int UL = NB == 1 ? 8 : 4;
  for (int j0 = lane; j0 < n4; j0 += UL * 32) {
    float4 a[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u)
      a[u] = (j0 + 32 * u < n4) ? ld_stream(r4 + j0 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int j = j0 + 32 * u;
      if (j < n4) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          if (b0 + q < n_batch) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(s + (size_t)(b0 + q) * n_slopes) + j);
            acc[q] += a[u].x * x.x + a[u].y * x.y + a[u].z * x.z + a[u].w * x.w;
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const float v = warp_sum_r(acc[q]);
    if (lane == 0 && b0 + q < n_batch) m[(size_t)(b0 + q) * n_modes + row] = v;
  }
}

// FP32, one slope vector, one row per CTA of kSplitWarps warps: warp w streams
// the w-th contiguous segment of the row (UL 16-byte loads in flight per
// lane), then the warps' sums are added in warp order.  Four streams per row
// keep more bytes in flight per row than one warp does.
constexpr int kSplitWarps = 4;
__global__ void __launch_bounds__(kSplitWarps * 32) k_mvm_f32_split(
    const float *__restrict__ R, const float *__restrict__ s, float *__restrict__ m, int n_modes,
    int n_slopes) {
  __shared__ float s_w[kSplitWarps];
  const int row = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float4 *r4 = reinterpret_cast<const float4 *>(R + (size_t)row * n_slopes);
  const float4 *s4 = reinterpret_cast<const float4 *>(s);
  const int n4 = n_slopes / 4;
  const int seg = (n4 + kSplitWarps - 1) / kSplitWarps;
  const int lo = warp * seg, hi = min(n4, lo + seg);
  constexpr int UL = 4;
  float acc = 0.f;
  for (int j0 = lo + lane; j0 < hi; j0 += UL * 32) {
    float4 a[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u)
      a[u] = (j0 + 32 * u < hi) ? ld_stream(r4 + j0 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int j = j0 + 32 * u;
      if (j < hi) {
        const float4 x = __ldg(s4 + j);
        acc += a[u].x * x.x + a[u].y * x.y + a[u].z * x.z + a[u].w * x.w;
      }
    }
  }
  acc = warp_sum_r(acc);
  if (lane == 0) s_w[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kSplitWarps; ++w) v += s_w[w];
    m[row] = v;
  }
}

// FP32, scalar fallback for unaligned sizes.
__global__ void __launch_bounds__(kReconWarps * 32) k_mvm_f32_scalar(
    const float *__restrict__ R, const float *__restrict__ s, float *__restrict__ m, int n_modes,
    int n_slopes, int n_batch) {
  const int row = blockIdx.x * kReconWarps + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n_modes) return;
  for (int b = 0; b < n_batch; ++b) {
    float acc = 0.f;
    for (int j = lane; j < n_slopes; j += 32)
      acc += R[(size_t)row * n_slopes + j] * s[(size_t)b * n_slopes + j];
    acc = warp_sum_r(acc);
    if (lane == 0) m[(size_t)b * n_modes + row] = acc;
  }
}

// BF16 (SPLIT = false) or BF16 hi + lo (SPLIT = true); n_slopes % 8 == 0.
template <int NB, bool SPLIT>
__global__ void __launch_bounds__(kReconWarps * 32) k_mvm_bf16(
    const uint16_t *__restrict__ Rh, const uint16_t *__restrict__ Rl, const float *__restrict__ s,
    float *__restrict__ m, int n_modes, int n_slopes, int n_batch, int b0) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n_modes) return;
  const uint4 *h8 = reinterpret_cast<const uint4 *>(Rh + (size_t)row * n_slopes);
  const uint4 *l8 = SPLIT ? reinterpret_cast<const uint4 *>(Rl + (size_t)row * n_slopes) : nullptr;
  const int n8 = n_slopes / 8;
  float acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) acc[q] = 0.f;
  // UL independent 16-byte loads (per operand) in flight per lane, issued
  // before any use
  constexpr int UL = NB == 1 ? (SPLIT ? 4 : 8) : 2;
  for (int j0 = lane; j0 < n8; j0 += UL * 32) {
    uint4 hv[UL], lv[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const bool ok = j0 + 32 * u < n8;
      hv[u] = ok ? ld_stream_u4(h8 + j0 + 32 * u) : make_uint4(0u, 0u, 0u, 0u);
      if (SPLIT) lv[u] = ok ? ld_stream_u4(l8 + j0 + 32 * u) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int j = j0 + 32 * u;
      if (j >= n8) break;
      float r[8] = {bf_lo(hv[u].x), bf_hi(hv[u].x), bf_lo(hv[u].y), bf_hi(hv[u].y),
                    bf_lo(hv[u].z), bf_hi(hv[u].z), bf_lo(hv[u].w), bf_hi(hv[u].w)};
      if (SPLIT) {
        r[0] += bf_lo(lv[u].x); r[1] += bf_hi(lv[u].x); r[2] += bf_lo(lv[u].y); r[3] += bf_hi(lv[u].y);
        r[4] += bf_lo(lv[u].z); r[5] += bf_hi(lv[u].z); r[6] += bf_lo(lv[u].w); r[7] += bf_hi(lv[u].w);
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (b0 + q < n_batch) {
          const float4 *sv = reinterpret_cast<const float4 *>(s + (size_t)(b0 + q) * n_slopes) + 2 * j;
          const float4 x0 = __ldg(sv), x1 = __ldg(sv + 1);
          acc[q] += r[0] * x0.x + r[1] * x0.y + r[2] * x0.z + r[3] * x0.w +
                    r[4] * x1.x + r[5] * x1.y + r[6] * x1.z + r[7] * x1.w;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const float v = warp_sum_r(acc[q]);
    if (lane == 0 && b0 + q < n_batch) m[(size_t)(b0 + q) * n_modes + row] = v;
  }
}

__global__ void k_convert_bf16(const float *__restrict__ R, uint16_t *__restrict__ hi,
                               uint16_t *__restrict__ lo, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = R[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = __bfloat16_as_ushort(h);
    if (lo) lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
  }
}

// Batched bf16 products on the tensor cores: the slopes are split into
// bf16 halves x = xh + xl and the modes come from one multi-term GEMM,
// m = xh Rh^T + xh Rl^T + xl Rh^T (BF16X2: float32-level error, the dropped
// xl Rl^T term is 2^-16 of the others) or xh Rh^T + xl Rh^T (BF16: the
// matrix's own rounding only), float32 accumulation.
constexpr int kGemmBatch = 32;

// K slices of the batched product: enough to fill the SMs, and at most
// kMaxKb K blocks of 64 per accumulator: the tensor cores' float32
// accumulation loses precision over long runs (relative error 6.8e-5 in one
// 40k-long accumulation of 4000 x 13344 x 3 products, 1.1e-5 in slices of 70
// blocks); the slices are summed in float32 on the CUDA cores
static int recon_splits(const specula_recon_desc *rec, int nb, int sms) {
  constexpr int kMaxKb = 128;
  const bool split = rec->precision == SPECULA_PREC_BF16X2;
  const int tiles = ((nb + 127) / 128) * ((rec->n_modes + 255) / 256);
  const int kb = (split ? 3 : 2) * ((rec->n_slopes + 63) / 64);
  return std::max(std::min(16, (kb + kMaxKb - 1) / kMaxKb),
                  std::max(1, std::min(16, (sms + tiles / 2) / std::max(tiles, 1))));
}

// workspace bytes of a batch of nb: the slopes' two bf16 halves (256-byte
// aligned) and the split-K partials
static size_t recon_ws_bytes(const specula_recon_desc *rec, int nb, int sms, size_t *xb_out) {
  const int splits = recon_splits(rec, nb, sms);
  const size_t xb = ((size_t)nb * rec->n_slopes * 2 + 255) / 256 * 256;
  if (xb_out) *xb_out = xb;
  return 2 * xb + (splits > 1 ? (size_t)splits * nb * rec->n_modes * 4 : 0);
}

static int recon_sms(int *sms) {
  int dev = 0;
  SPECULA_CK(cudaGetDevice(&dev));
  SPECULA_CK(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  return SPECULA_OK;
}

static int recon_gemm(specula_ctx *ctx, const specula_recon_desc *rec, const float *X, int nb,
                      float *modes, cudaStream_t st) {
  const bool split = rec->precision == SPECULA_PREC_BF16X2;
  const int K = rec->n_slopes, N = rec->n_modes;
  int sms = 0, s = recon_sms(&sms);
  if (s) return s;
  const int splits = recon_splits(rec, nb, sms);
  const size_t nx = (size_t)nb * K;
  size_t xb = 0;
  const size_t need = recon_ws_bytes(rec, nb, sms, &xb);
  if (ctx->recon_ws.bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SPECULA_CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SPECULA_EUNSUPPORTED;   // grow before capture
    SPECULA_CK(cudaStreamSynchronize(st));
    if ((s = ctx->recon_ws.alloc(need))) return s;
  }
  uint8_t *w = static_cast<uint8_t *>(ctx->recon_ws.p);
  uint16_t *xh = reinterpret_cast<uint16_t *>(w), *xl = reinterpret_cast<uint16_t *>(w + xb);
  float *part = reinterpret_cast<float *>(w + 2 * xb);
  SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st,
                 k_convert_bf16<<<(unsigned)std::min<size_t>((nx + 255) / 256, 4096), 256, 0,
                                  st>>>(X, xh, xl, nx));
  const void *A3[3] = {xh, xh, xl}, *B3[3] = {rec->R_dev, rec->R_lo_dev, rec->R_dev};
  const void *A2[2] = {xh, xl}, *B2[2] = {rec->R_dev, rec->R_dev};
  return split ? gemm_bf16_terms(ctx, 3, A3, B3, nb, N, K, modes, splits, part, st)
               : gemm_bf16_terms(ctx, 2, A2, B2, nb, N, K, modes, splits, part, st);
}

}  // namespace specula

using namespace specula;

extern "C" int specula_recon(specula_ctx *ctx, const specula_recon_desc *rec,
                             const float *slopes_dev, int32_t n_batch, float *modes_dev,
                             void *stream) {
  if (!ctx || !rec || !slopes_dev || !modes_dev || n_batch < 0) return SPECULA_EINVAL;
  if (rec->n_modes < 1 || rec->n_slopes < 1 || !rec->R_dev) return SPECULA_EINVAL;
  if (n_batch == 0) return SPECULA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned grid = (rec->n_modes + kReconWarps - 1) / kReconWarps;
  const int blk = kReconWarps * 32;
  // one slope vector: one warp per CTA, so the rows spread over the SMs
  // within one row of each other (8-row CTAs leave some SMs a third more)
  const unsigned grid1 = (unsigned)rec->n_modes;
  const int blk1 = 32;
  const bool al16 = ((uintptr_t)rec->R_dev % 16 == 0) && ((uintptr_t)slopes_dev % 16 == 0);
  constexpr int NB = 4;
  switch (rec->precision) {
    case SPECULA_PREC_FP32:
      if (rec->n_slopes % 4 == 0 && al16) {
        for (int b0 = 0; b0 < n_batch; b0 += NB) {
          if (n_batch == 1)
            SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st,
                           k_mvm_f32_split<<<grid1, kSplitWarps * 32, 0, st>>>(
                               (const float *)rec->R_dev, slopes_dev, modes_dev, rec->n_modes,
                               rec->n_slopes));
          else if (n_batch - b0 == 1)
            SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_f32<1><<<grid1, blk1, 0, st>>>((const float *)rec->R_dev, slopes_dev, modes_dev,
                                               rec->n_modes, rec->n_slopes, n_batch, b0));
          else
            SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_f32<NB><<<grid, blk, 0, st>>>((const float *)rec->R_dev, slopes_dev, modes_dev,
                                                rec->n_modes, rec->n_slopes, n_batch, b0));
        }
      } else {
        SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_f32_scalar<<<grid, blk, 0, st>>>((const float *)rec->R_dev, slopes_dev, modes_dev,
                                               rec->n_modes, rec->n_slopes, n_batch));
      }
      return SPECULA_OK;
    case SPECULA_PREC_BF16:
    case SPECULA_PREC_BF16X2: {
      const bool split = rec->precision == SPECULA_PREC_BF16X2;
      if (split && !rec->R_lo_dev) return SPECULA_EINVAL;
      if (rec->n_slopes % 8 != 0 || !al16 || (split && (uintptr_t)rec->R_lo_dev % 16))
        return SPECULA_EUNSUPPORTED;
      if (n_batch >= kGemmBatch) return recon_gemm(ctx, rec, slopes_dev, n_batch, modes_dev, st);
      for (int b0 = 0; b0 < n_batch; b0 += NB) {
        const bool one = n_batch - b0 == 1;
        const uint16_t *h = (const uint16_t *)rec->R_dev, *l = (const uint16_t *)rec->R_lo_dev;
        if (split) {
          if (one) SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_bf16<1, true><<<grid1, blk1, 0, st>>>(h, l, slopes_dev, modes_dev, rec->n_modes, rec->n_slopes, n_batch, b0));
          else SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_bf16<NB, true><<<grid, blk, 0, st>>>(h, l, slopes_dev, modes_dev, rec->n_modes, rec->n_slopes, n_batch, b0));
        } else {
          if (one) SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_bf16<1, false><<<grid1, blk1, 0, st>>>(h, l, slopes_dev, modes_dev, rec->n_modes, rec->n_slopes, n_batch, b0));
          else SPECULA_LAUNCH(ctx, SPECULA_K_RECON, st, k_mvm_bf16<NB, false><<<grid, blk, 0, st>>>(h, l, slopes_dev, modes_dev, rec->n_modes, rec->n_slopes, n_batch, b0));
        }
      }
      return SPECULA_OK;
    }
    default:
      return SPECULA_EINVAL;
  }
}

extern "C" int specula_recon_reserve(specula_ctx *ctx, const specula_recon_desc *rec,
                                     int32_t max_batch) {
  if (!ctx || !rec || max_batch < 0 || rec->n_modes < 1 || rec->n_slopes < 1) return SPECULA_EINVAL;
  if (rec->precision != SPECULA_PREC_BF16 && rec->precision != SPECULA_PREC_BF16X2)
    return SPECULA_OK;   // the float32 products use no workspace
  if (max_batch < kGemmBatch) return SPECULA_OK;
  SPECULA_CK(cudaSetDevice(ctx->device));
  int sms = 0, s = recon_sms(&sms);
  if (s) return s;
  size_t need = 0;
  for (int nb = kGemmBatch; nb <= max_batch; ++nb)
    need = std::max(need, recon_ws_bytes(rec, nb, sms, nullptr));
  if (ctx->recon_ws.bytes >= need) return SPECULA_OK;
  SPECULA_CK(cudaDeviceSynchronize());   // calls in flight may use the old workspace
  return ctx->recon_ws.alloc(need);
}

extern "C" int specula_recon_convert(specula_ctx *ctx, int32_t n_modes, int32_t n_slopes,
                                     const float *R_dev, int32_t precision, void *hi_dev,
                                     void *lo_dev, void *stream) {
  if (!ctx || !R_dev || !hi_dev || n_modes < 1 || n_slopes < 1) return SPECULA_EINVAL;
  if (precision != SPECULA_PREC_BF16 && precision != SPECULA_PREC_BF16X2) return SPECULA_EINVAL;
  if (precision == SPECULA_PREC_BF16X2 && !lo_dev) return SPECULA_EINVAL;
  const size_t n = (size_t)n_modes * n_slopes;
  k_convert_bf16<<<1216, 256, 0, (cudaStream_t)stream>>>(
      R_dev, (uint16_t *)hi_dev, precision == SPECULA_PREC_BF16X2 ? (uint16_t *)lo_dev : nullptr, n);
  SPECULA_CK_LAUNCH();
  return SPECULA_OK;
}
