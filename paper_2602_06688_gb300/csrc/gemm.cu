// BF16 and TF32 GEMMs on the 5th-generation tensor cores (tcgen05), FP32
// accumulate:
//     C[M][N] = A[M][K] . B[N][K]^T        (both operands K-major, row-major)
// The dense contractions of the learned reconstructor (its forward layers,
// their gradients), batched reconstructor MVMs and the DFT-as-GEMM pyramid
// variant run here.  The TF32 kernel reads float32 storage (the tensor cores
// use its upper 19 bits).
//
// Persistent kernel, one CTA per SM, looping over (128 x BN output tile, K
// slice) work items, BN = 256 (128 where N is a multiple of 128 but not of
// 256); M and N need not be tile multiples (TMA fills rows beyond the
// operands with zeros, the epilogue masks its stores).  K is a sum of up to
// three terms C = sum_t A_t B_t^T over the same K extent (split-precision
// products such as hi.hi + hi.lo + lo.hi run as one accumulation); a K
// that is not a multiple of the stage depth is zero-filled the same way.
//   warp 0, one thread : TMA loads of A and B tiles (128 bytes of K: 64 bf16
//                        or 32 tf32, 128-byte swizzle) into a shared-memory
//                        ring (4 stages at BN = 256, 6 at BN = 128)
//   warp 1             : allocates 2 BN tensor-memory columns (two
//                        accumulators); one thread issues 4 tcgen05.mma
//                        (K = 16 bf16 or 8 tf32 each) per stage, commits each
//                        stage back to the producer and each finished tile
//                        to the epilogue
//   warps 4-7          : drain a finished accumulator (tcgen05.ld, one row
//                        per thread) to global memory while the next tile
//                        accumulates in the other one
// Split-K partials go to a caller workspace and are summed in split order by
// k_split_reduce (no atomics: bit-reproducible).  Every wait is bounded:
// on timeout the CTA records SPECULA_ETIMEOUT in the context status word,
// waits for its own copies and MMAs, frees its tensor memory and returns.
#include <cuda.h>

#include <string.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "tc_gemm.cuh"

namespace specula {

constexpr int GBM = 128;
constexpr int kMaxTerms = 3;
constexpr uint32_t G_A_BYTES = GBM * 128;   // 128 rows x 128 bytes of K
// K elements per 128-byte row of a stage: 64 bf16 (TF32 = false) or 32 tf32
template <bool TF32> constexpr int gbk() { return TF32 ? 32 : 64; }
template <int BN> struct GCfg {
  static constexpr int STAGES = BN == 256 ? 4 : 6;
  static constexpr uint32_t B_BYTES = BN * 128;
  static constexpr uint32_t TMEM_COLS = 2 * BN;
  static constexpr size_t SMEM = 1024 + STAGES * (G_A_BYTES + B_BYTES) + 256;
};

// the operand maps of every term (kernel parameter space)
struct GemmMaps {
  CUtensorMap a[kMaxTerms];
  CUtensorMap b[kMaxTerms];
};

struct GemmShape {
  int M, N;
  int tiles_m, tiles_n;
  int n_items;              // tiles_m x tiles_n x splits
  int splits;
  int kb_term;              // K blocks per term
  int kb_total;             // kb_term x terms
  int kb_per_split;
  int vec4;                 // N % 4 == 0 and a 16-byte aligned output
};

__device__ __forceinline__ bool wait_noabort(uint64_t *bar, uint32_t parity) {
  return tc::mbar_wait(bar, parity, nullptr);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// work item -> (m0, n0, split).  Tiles are taken in bands of kBand tile
// columns, row by row within a band: the CTAs running together (one per
// SM) then read a block of about 19 x 8 tiles, whose A rows and B columns
// (70 MB at K = 8192) stay in L2, instead of every row of A per wave.
constexpr int kBand = 8;
__device__ __forceinline__ void gemm_item(const GemmShape &g, int w, int BN, int &m0, int &n0,
                                          int &split) {
  const int tiles = g.tiles_m * g.tiles_n;
  split = w / tiles;
  const int t = w - split * tiles;
  const int band = t / (kBand * g.tiles_m);
  const int nb0 = band * kBand;
  const int gw = min(kBand, g.tiles_n - nb0);
  const int r = t - band * kBand * g.tiles_m;
  const int tm = r / gw;
  m0 = tm * GBM;
  n0 = (nb0 + (r - tm * gw)) * BN;
}

template <bool TF32, int BN>
__global__ void __launch_bounds__(256, 1) k_gemm_tn(const __grid_constant__ GemmMaps maps,
                                                    const GemmShape g, float *__restrict__ out,
                                                    int32_t *status) {
  using C = GCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = base;
  uint8_t *sB = base + C::STAGES * G_A_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + C::STAGES * C::B_BYTES);
  uint64_t *empty = full + C::STAGES;
  uint64_t *acc_full = empty + C::STAGES;   // [2]
  uint64_t *acc_empty = acc_full + 2;       // [2]
  uint64_t *done = acc_empty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      tc::mbar_init(full + s, 1);
      tc::mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(acc_full + b, 1);
      tc::mbar_init(acc_empty + b, 4);   // one arrival per epilogue warp
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;   // stage fills issued (ring position)
      bool ok = true;
      for (int w = blockIdx.x; w < g.n_items && ok; w += gridDim.x) {
        int m0, n0, split;
        gemm_item(g, w, BN, m0, n0, split);
        const int kb0 = split * g.kb_per_split;
        const int nk = min(g.kb_per_split, g.kb_total - kb0);
        for (int i = 0; i < nk; ++i, ++it) {
          const uint32_t s = it % C::STAGES;
          if (it >= (uint32_t)C::STAGES &&
              !tc::mbar_wait(empty + s, ((it / C::STAGES) & 1) ^ 1, abort_flag)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          const int gk = kb0 + i, term = gk / g.kb_term;
          const int kx = (gk - term * g.kb_term) * gbk<TF32>();
          tc::mbar_arrive_expect_tx(full + s, G_A_BYTES + C::B_BYTES);
          tc::tma_load_2d(sA + s * G_A_BYTES, &maps.a[term], full + s, kx, m0);
          tc::tma_load_2d(sB + s * C::B_BYTES, &maps.b[term], full + s, kx, n0);
        }
      }
      // every issued copy lands before the CTA may leave
      for (uint32_t s = 0; s < (uint32_t)C::STAGES && s < it; ++s) {
        const uint32_t last = s + ((it - 1 - s) / C::STAGES) * C::STAGES;
        wait_noabort(full + s, (last / C::STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc =
          TF32 ? tc::idesc_tf32_f32(GBM, BN) : tc::idesc_bf16_f32(GBM, BN);
      uint32_t it = 0;
      int j = 0;   // tiles of this CTA so far
      bool ok = true;
      for (int w = blockIdx.x; w < g.n_items && ok; w += gridDim.x, ++j) {
        int m0, n0, split;
        gemm_item(g, w, BN, m0, n0, split);
        const int nk = min(g.kb_per_split, g.kb_total - split * g.kb_per_split);
        const int buf = j & 1;
        // the epilogue has drained this accumulator's previous tile
        if (j >= 2 && !tc::mbar_wait(acc_empty + buf, ((j >> 1) - 1) & 1, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int i = 0; i < nk; ++i, ++it) {
          const uint32_t s = it % C::STAGES;
          if (!tc::mbar_wait(full + s, (it / C::STAGES) & 1, abort_flag)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc::fence_after();
          const uint64_t ad = tc::desc_sw128(tc::smem_u32(sA + s * G_A_BYTES));
          const uint64_t bd = tc::desc_sw128(tc::smem_u32(sB + s * C::B_BYTES));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // +32 bytes of K per step (16 bf16 or 8 tf32)
            if constexpr (TF32)
              tc::mma_tf32(d, ad + 2 * kk, bd + 2 * kk, idesc, (i | kk) ? 1u : 0u);
            else
              tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, (i | kk) ? 1u : 0u);
          }
          tc::mma_commit(empty + s);
        }
        if (ok) tc::mma_commit(acc_full + buf);
      }
      tc::mma_commit(done);      // arrives once every MMA issued has finished
      wait_noabort(done, 0);     // before the tensor memory is freed
    }
  } else if (warp >= 4) {
    const int wl = warp - 4;   // tensor-memory lanes 32 wl .. 32 wl + 31
    int j = 0;
    for (int w = blockIdx.x; w < g.n_items; w += gridDim.x, ++j) {
      int m0, n0, split;
      gemm_item(g, w, BN, m0, n0, split);
      const int buf = j & 1;
      bool go = tc::mbar_wait(acc_full + buf, (j >> 1) & 1, abort_flag);
      go = __all_sync(0xffffffffu, go);
      if (!go) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after();
      const int row = m0 + wl * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(wl * 32) << 16) + (uint32_t)(buf * BN + c0), v);
        const int col = n0 + c0;
        if (row < g.M && col < g.N) {
          float *dst = out + ((size_t)split * g.M + row) * g.N + col;
          if (g.vec4 && col + 32 <= g.N) {
            float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
            for (int q = 0; q < 8; ++q)
              d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (col + q < g.N) dst[q] = v[q];
          }
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + buf);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
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
  if (K % (tf32 ? 4 : 8)) return SPECULA_EUNSUPPORTED;   // rows of a multiple of 16 bytes (TMA)
  if ((uintptr_t)A % 16 || (uintptr_t)B % 16) return SPECULA_EINVAL;
  return SPECULA_OK;
}

// splits that keep every K slice of kb blocks non-empty
static int splits_for(int kb, int want) {
  int s = std::max(1, std::min(want, kb));
  const int per = (kb + s - 1) / s;
  return (kb + per - 1) / per;
}

int gemm_splits(int K, int want, bool tf32) {
  const int k = tf32 ? gbk<true>() : gbk<false>();
  return splits_for((K + k - 1) / k, want);
}

// output tile width: 128 where N is a multiple of 128 but not of 256 (no
// zero columns computed), else 256
static int gemm_bn(int N) { return (N % 128 == 0 && N % 256 != 0) ? 128 : 256; }

static int sm_count() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 64) return 0;
  if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev))
    return 0;
  return sms[dev];
}

template <bool TF32, int BN>
static int gemm_launch(specula_ctx *ctx, int n_terms, const void *const *A, const void *const *B,
                       int M, int N, int K, float *C, int splits, float *work,
                       cudaStream_t st) {
  using Cfg = GCfg<BN>;
  static bool attr_done[64] = {};
  int dev = 0;
  SPECULA_CK(cudaGetDevice(&dev));
  if (dev < 64 && !attr_done[dev]) {
    SPECULA_CK(cudaFuncSetAttribute(k_gemm_tn<TF32, BN>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Cfg::SMEM));
    attr_done[dev] = true;
  }
  const int sms = sm_count();
  if (sms < 1) return SPECULA_ECUDA;
  GemmMaps maps;
  memset(&maps, 0, sizeof(maps));
  int s;
  for (int t = 0; t < n_terms; ++t) {
    if ((s = make_map(&maps.a[t], A[t], M, K, GBM, TF32))) return s;
    if ((s = make_map(&maps.b[t], B[t], N, K, BN, TF32))) return s;
  }
  GemmShape g;
  g.M = M;
  g.N = N;
  g.kb_term = (K + gbk<TF32>() - 1) / gbk<TF32>();
  g.kb_total = g.kb_term * n_terms;
  g.splits = splits_for(g.kb_total, splits);
  g.kb_per_split = (g.kb_total + g.splits - 1) / g.splits;
  g.tiles_m = (M + GBM - 1) / GBM;
  g.tiles_n = (N + BN - 1) / BN;
  g.n_items = g.tiles_m * g.tiles_n * g.splits;
  if (g.splits > 1 && !work) return SPECULA_EINVAL;
  float *dst = g.splits > 1 ? work : C;
  g.vec4 = (N % 4 == 0) && ((uintptr_t)dst % 16 == 0);
  const int grid = std::min(g.n_items, sms);
  SPECULA_LAUNCH(ctx, SPECULA_K_GEMM, st,
                 k_gemm_tn<TF32, BN><<<grid, 256, Cfg::SMEM, st>>>(maps, g, dst,
                                                                   ctx->status_dev));
  if (g.splits > 1) {
    const size_t n = (size_t)M * N;
    SPECULA_LAUNCH(ctx, SPECULA_K_GEMM, st,
                   k_split_reduce<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0,
                                    st>>>(work, g.splits, n, C));
  }
  return SPECULA_OK;
}

template <bool TF32>
static int gemm_terms(specula_ctx *ctx, int n_terms, const void *const *A, const void *const *B,
                      int M, int N, int K, float *C, int splits, float *work, cudaStream_t st) {
  if (!ctx || !C || n_terms < 1 || n_terms > kMaxTerms || splits < 1) return SPECULA_EINVAL;
  for (int t = 0; t < n_terms; ++t) {
    const int s = gemm_check(A[t], B[t], M, N, K, TF32);
    if (s) return s;
  }
  if (gemm_bn(N) == 128)
    return gemm_launch<TF32, 128>(ctx, n_terms, A, B, M, N, K, C, splits, work, st);
  return gemm_launch<TF32, 256>(ctx, n_terms, A, B, M, N, K, C, splits, work, st);
}

int gemm_bf16_tn(specula_ctx *ctx, const void *A, const void *B, int M, int N, int K, float *C,
                 int splits, float *work, cudaStream_t st) {
  return gemm_terms<false>(ctx, 1, &A, &B, M, N, K, C, splits, work, st);
}

int gemm_bf16_terms(specula_ctx *ctx, int n_terms, const void *const *A, const void *const *B,
                    int M, int N, int K, float *C, int splits, float *work, cudaStream_t st) {
  return gemm_terms<false>(ctx, n_terms, A, B, M, N, K, C, splits, work, st);
}

int gemm_tf32_tn(specula_ctx *ctx, const float *A, const float *B, int M, int N, int K, float *C,
                 int splits, float *work, cudaStream_t st) {
  const void *a = A, *b = B;
  return gemm_terms<true>(ctx, 1, &a, &b, M, N, K, C, splits, work, st);
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
