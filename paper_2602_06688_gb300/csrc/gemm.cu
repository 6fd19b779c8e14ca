// BF16 and TF32 GEMMs on the 5th-generation tensor cores (tcgen05), FP32
// accumulate:
//     C[M][N] = A[M][K] . B[N][K]^T        (both operands K-major, row-major)
// The dense contractions of the learned reconstructor (its forward layers,
// their gradients), batched reconstructor MVMs and the DFT-as-GEMM pyramid
// variant run here.  The TF32 kernel reads float32 storage (the tensor cores
// use its upper 19 bits).
//
// One CTA per 128 x 128 output tile and K slice (split-K for small grids):
//   warp 0, one thread : TMA loads of A and B tiles (128 bytes of K: 64 bf16
//                        or 32 tf32, 128-byte swizzle) into a 4-stage
//                        shared-memory ring
//   warp 1             : allocates 128 tensor-memory columns; one thread
//                        issues 4 tcgen05.mma (K = 16 each) per stage and
//                        commits each stage back to the producer
//   warps 4-7          : drain the 128 x 128 FP32 accumulator (tcgen05.ld,
//                        one row per thread) to global memory
// Split-K partials go to a caller workspace and are summed in split order by
// k_split_reduce (no atomics: bit-reproducible).  Every wait is bounded:
// on timeout the CTA records SPECULA_ETIMEOUT in the context status word,
// waits for its own copies, frees its tensor memory and returns.
#include <cuda.h>

#include <mutex>

#include "internal.h"
#include "tc_gemm.cuh"

namespace specula {

constexpr int GBM = 128, GBN = 128, GBK = 64, GSTAGES = 4;   // GBK: bf16 elements
constexpr uint32_t G_A_BYTES = GBM * GBK * 2, G_B_BYTES = GBN * GBK * 2;
// K elements per 128-byte row of a stage: 64 bf16 (TF32 = false) or 32 tf32
template <bool TF32> constexpr int gbk() { return TF32 ? 32 : 64; }
constexpr size_t G_SMEM = 1024 + GSTAGES * (G_A_BYTES + G_B_BYTES) + 256;

__device__ __forceinline__ bool wait_noabort(uint64_t *bar, uint32_t parity) {
  return tc::mbar_wait(bar, parity, nullptr);
}

template <bool TF32>
__global__ void __launch_bounds__(256, 1) k_gemm_tn(const __grid_constant__ CUtensorMap ta,
                                                         const __grid_constant__ CUtensorMap tb,
                                                         float *__restrict__ out, int M, int N,
                                                         int kb_per_split, int kb_total,
                                                         int32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = base;
  uint8_t *sB = base + GSTAGES * G_A_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + GSTAGES * G_B_BYTES);
  uint64_t *empty = full + GSTAGES;
  uint64_t *done = empty + GSTAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * GBN, m0 = blockIdx.y * GBM, split = blockIdx.z;
  const int kb0 = split * kb_per_split;
  const int nk = min(kb_per_split, kb_total - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      tc::mbar_init(full + s, 1);
      tc::mbar_init(empty + s, 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, GBN);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % GSTAGES;
        if (i >= GSTAGES && !tc::mbar_wait(empty + s, ((i / GSTAGES) & 1) ^ 1, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        tc::mbar_arrive_expect_tx(full + s, G_A_BYTES + G_B_BYTES);
        tc::tma_load_2d(sA + s * G_A_BYTES, &ta, full + s, (kb0 + i) * gbk<TF32>(), m0);
        tc::tma_load_2d(sB + s * G_B_BYTES, &tb, full + s, (kb0 + i) * gbk<TF32>(), n0);
        ++issued;
      }
      // every issued copy lands before the CTA may leave
      for (int s = 0; s < GSTAGES && s < issued; ++s) {
        const int last = s + ((issued - 1 - s) / GSTAGES) * GSTAGES;
        wait_noabort(full + s, (last / GSTAGES) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc =
          TF32 ? tc::idesc_tf32_f32(GBM, GBN) : tc::idesc_bf16_f32(GBM, GBN);
      for (int i = 0; i < nk; ++i) {
        const int s = i % GSTAGES;
        if (!tc::mbar_wait(full + s, (i / GSTAGES) & 1, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after();
        const uint64_t ad = tc::desc_sw128(tc::smem_u32(sA + s * G_A_BYTES));
        const uint64_t bd = tc::desc_sw128(tc::smem_u32(sB + s * G_B_BYTES));
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {   // +32 bytes of K per step (16 bf16 or 8 tf32)
          if constexpr (TF32)
            tc::mma_tf32(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i | kk) ? 1u : 0u);
          else
            tc::mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i | kk) ? 1u : 0u);
        }
        tc::mma_commit(empty + s);
      }
      tc::mma_commit(done);   // arrives when every issued MMA has finished
    }
  } else if (warp >= 4) {
    bool go = wait_noabort(done, 0);
    if (!go) *abort_flag = 1;
    go = __all_sync(0xffffffffu, go && !*abort_flag);
    if (go) {
      tc::fence_after();
      const int wl = warp - 4;   // tensor-memory lanes 32 wl .. 32 wl + 31
      const int row = m0 + wl * 32 + lane;
      float *dst = out + ((size_t)split * M + row) * N + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < GBN; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(wl * 32) << 16) + (uint32_t)c0, v);
        float4 *d4 = reinterpret_cast<float4 *>(dst + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, GBN);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(status, SPECULA_ETIMEOUT);
}

__global__ void k_split_reduce(const float *__restrict__ part, int splits, size_t n,
                               float *__restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int s = 0; s < splits; ++s) v += part[(size_t)s * n + e];
    out[e] = v;
  }
}

// ---- host --------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// rows x K row-major (bf16, or float32 read as tf32), box of 128 bytes of K
// x box_rows, 128-byte swizzle
static int make_map(CUtensorMap *m, const void *ptr, int rows, int K, int box_rows,
                    bool tf32 = false) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return SPECULA_ECUDA;
  const int es_bytes = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * es_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es_bytes), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_TFLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void *>(ptr), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SPECULA_OK : SPECULA_ECUDA;
}

int gemm_check(const void *A, const void *B, int M, int N, int K, bool tf32) {
  if (!A || !B || M < 1 || N < 1 || K < 1) return SPECULA_EINVAL;
  if (M % GBM || N % GBN || K % (tf32 ? gbk<true>() : gbk<false>())) return SPECULA_EUNSUPPORTED;
  if ((uintptr_t)A % 16 || (uintptr_t)B % 16) return SPECULA_EINVAL;
  return SPECULA_OK;
}

// splits that keep every K slice non-empty
int gemm_splits(int K, int want, bool tf32) {
  const int kb = K / (tf32 ? gbk<true>() : gbk<false>());
  int s = std::max(1, std::min(want, kb));
  const int per = (kb + s - 1) / s;
  return (kb + per - 1) / per;
}

template <bool TF32>
static int gemm_tn(specula_ctx *ctx, const void *A, const void *B, int M, int N, int K, float *C,
                   int splits, float *work, cudaStream_t st) {
  int s = gemm_check(A, B, M, N, K, TF32);
  if (s) return s;
  static bool attr_done[64] = {};
  int dev = 0;
  SPECULA_CK(cudaGetDevice(&dev));
  if (dev < 64 && !attr_done[dev]) {
    SPECULA_CK(cudaFuncSetAttribute(k_gemm_tn<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)G_SMEM));
    attr_done[dev] = true;
  }
  CUtensorMap ta, tb;
  if ((s = make_map(&ta, A, M, K, GBM, TF32))) return s;
  if ((s = make_map(&tb, B, N, K, GBN, TF32))) return s;
  const int kb = K / gbk<TF32>();
  splits = gemm_splits(K, splits, TF32);
  const int per = (kb + splits - 1) / splits;
  if (splits > 1 && !work) return SPECULA_EINVAL;
  float *dst = splits > 1 ? work : C;
  dim3 grid(N / GBN, M / GBM, splits);
  SPECULA_LAUNCH(ctx, SPECULA_K_GEMM, st,
                 k_gemm_tn<TF32><<<grid, 256, G_SMEM, st>>>(ta, tb, dst, M, N, per, kb,
                                                           ctx->status_dev));
  if (splits > 1) {
    const size_t n = (size_t)M * N;
    SPECULA_LAUNCH(ctx, SPECULA_K_GEMM, st,
                   k_split_reduce<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0,
                                    st>>>(work, splits, n, C));
  }
  return SPECULA_OK;
}

int gemm_bf16_tn(specula_ctx *ctx, const void *A, const void *B, int M, int N, int K, float *C,
                 int splits, float *work, cudaStream_t st) {
  return gemm_tn<false>(ctx, A, B, M, N, K, C, splits, work, st);
}

int gemm_tf32_tn(specula_ctx *ctx, const float *A, const float *B, int M, int N, int K, float *C,
                 int splits, float *work, cudaStream_t st) {
  return gemm_tn<true>(ctx, A, B, M, N, K, C, splits, work, st);
}

}  // namespace specula

using namespace specula;

extern "C" int specula_gemm_bf16(specula_ctx *ctx, const void *A_dev, const void *B_dev,
                                 int32_t M, int32_t N, int32_t K, float *C_dev, int32_t splits,
                                 float *work_dev, void *stream) {
  if (!ctx || !C_dev || splits < 1) return SPECULA_EINVAL;
  return gemm_bf16_tn(ctx, A_dev, B_dev, M, N, K, C_dev, splits, work_dev,
                      (cudaStream_t)stream);
}

extern "C" int specula_gemm_tf32(specula_ctx *ctx, const float *A_dev, const float *B_dev,
                                 int32_t M, int32_t N, int32_t K, float *C_dev, int32_t splits,
                                 float *work_dev, void *stream) {
  if (!ctx || !C_dev || splits < 1) return SPECULA_EINVAL;
  return gemm_tf32_tn(ctx, A_dev, B_dev, M, N, K, C_dev, splits, work_dev,
                      (cudaStream_t)stream);
}
