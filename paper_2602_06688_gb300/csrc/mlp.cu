// Learned nonlinear reconstructor: a 3-layer perceptron (slopes -> modes)
// with GELU, trained by the project's own forward/backward kernels and Adam.
// Not in the paper (its reconstructor is the linear Modalrec): a nonlinear
// alternative trained on simulated pairs, with BF16 weights, FP32
// accumulation and batch 256 (the 8 m and 39 m learned workloads).
//
// Layout.  Widths are padded to multiples of 128 (zero pads stay zero: their
// inputs and output gradients are zero) and the batch to a multiple of 128,
// so every contraction is one tensor-core GEMM  C = A . B^T  with both
// operands K-major bf16 (specula_gemm_bf16):
//   forward   Z_l = H_{l-1} W_l^T          A = H_{l-1} [B][in],  B = W_l [out][in]
//   dW_l      dW_l = dZ_l^T H_{l-1}        A = dZ_l^T [out][B],  B = H_{l-1}^T [in][B]
//   dH_{l-1}  dH = dZ_l W_l                A = dZ_l [B][out],    B = W_l^T [in][out]
// The element-wise kernels that produce H, dZ and the bf16 weights also
// write their transposed copies (32 x 32 shared-memory tiles), so no GEMM
// needs an MN-major operand.  FP32 master weights and Adam moments; bf16
// copies refreshed after every update.  Reductions (bias gradients, loss)
// run in a fixed order: bit-reproducible.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace specula {

constexpr int TT = 32;   // transpose tile

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * (float)M_SQRT1_2));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float inv_sqrt_2pi = 0.5f * (float)M_2_SQRTPI * (float)M_SQRT1_2;   // 1/sqrt(2 pi)
  return 0.5f * (1.0f + erff(z * (float)M_SQRT1_2)) + z * expf(-0.5f * z * z) * inv_sqrt_2pi;
}

// Tiled writer of a bf16 matrix and its transpose.  Block (32, 8), grid
// (C/32, R/32); the value function is evaluated once per element.
template <class F>
__device__ __forceinline__ void tile_bf16_pair(int R, int C, __nv_bfloat16 *out,
                                               __nv_bfloat16 *outT, F value) {
  __shared__ __nv_bfloat16 tile[TT][TT + 2];
  const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
  for (int dr = threadIdx.y; dr < TT; dr += blockDim.y) {
    const int r = r0 + dr, c = c0 + threadIdx.x;
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (r < R && c < C) {
      v = __float2bfloat16_rn(value(r, c));
      out[(size_t)r * C + c] = v;
    }
    tile[dr][threadIdx.x] = v;
  }
  __syncthreads();
  for (int dc = threadIdx.y; dc < TT; dc += blockDim.y) {
    const int c = c0 + dc, r = r0 + threadIdx.x;
    if (r < R && c < C) outT[(size_t)c * R + r] = tile[threadIdx.x][dc];
  }
}

// X [B][n_in] float -> Xb [Bp][in_pad] and XbT [in_pad][Bp] (zero pads)
__global__ void k_pack_input(const float *__restrict__ X, int B, int n_in, int Bp, int in_pad,
                             __nv_bfloat16 *Xb, __nv_bfloat16 *XbT) {
  tile_bf16_pair(Bp, in_pad, Xb, XbT, [&](int r, int c) {
    return (r < B && c < n_in) ? X[(size_t)r * n_in + c] : 0.f;
  });
}

// Z += bias (in place); H = gelu(Z) and its transpose in bf16
__global__ void k_bias_gelu(float *__restrict__ Z, const float *__restrict__ bias, int R, int C,
                            __nv_bfloat16 *H, __nv_bfloat16 *HT) {
  tile_bf16_pair(R, C, H, HT, [&](int r, int c) {
    const float z = Z[(size_t)r * C + c] + bias[c];
    Z[(size_t)r * C + c] = z;
    return gelu_f(z);
  });
}

// dA (in place) <- dA * gelu'(Z); bf16 dZ and its transpose
__global__ void k_gelu_back(float *__restrict__ dA, const float *__restrict__ Z, int R, int C,
                            __nv_bfloat16 *dZb, __nv_bfloat16 *dZbT) {
  tile_bf16_pair(R, C, dZb, dZbT, [&](int r, int c) {
    const size_t e = (size_t)r * C + c;
    const float d = dA[e] * gelu_grad_f(Z[e]);
    dA[e] = d;
    return d;
  });
}

// dY = scale (Y - T) on the B x n_out block, zero on pads; squared residual
// sums per tile row into part (one float per (tile, row) pair)
__global__ void k_loss_grad(const float *__restrict__ Y, const float *__restrict__ T, int B,
                            int n_out, int Bp, int out_pad, float scale, float *__restrict__ dYf,
                            __nv_bfloat16 *dYb, __nv_bfloat16 *dYbT, float *__restrict__ part) {
  __shared__ float s_sq[8][TT];
  float sq = 0.f;
  tile_bf16_pair(Bp, out_pad, dYb, dYbT, [&](int r, int c) {
    float d = 0.f;
    if (r < B && c < n_out) d = Y[(size_t)r * out_pad + c] - T[(size_t)r * n_out + c];
    sq += d * d;
    const float g = scale * d;
    dYf[(size_t)r * out_pad + c] = g;
    return g;
  });
  s_sq[threadIdx.y][threadIdx.x] = sq;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float s = 0.f;
    for (int y = 0; y < 8; ++y)
      for (int x = 0; x < TT; ++x) s += s_sq[y][x];
    part[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_loss_final(const float *__restrict__ part, int n, float inv_count,
                             float *__restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = s * inv_count;
  }
}

__global__ void k_add_bias(float *__restrict__ Y, const float *__restrict__ bias, int R, int C) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < (size_t)R * C) Y[e] += bias[e % C];
}

__global__ void k_unpack_out(const float *__restrict__ Y, int B, int n_out, int out_pad,
                             float *__restrict__ out) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < (size_t)B * n_out) out[e] = Y[(e / n_out) * out_pad + e % n_out];
}

// db[c] = sum over r < R of D[r][c], rows in order
__global__ void k_colsum(const float *__restrict__ D, int R, int C, float *__restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += D[(size_t)r * C + c];
  db[c] = s;
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, size_t n, float lr_t, float b1, float b2,
                       float eps) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps);
  }
}

__global__ void k_cast_w(const float *__restrict__ W, int R, int C, __nv_bfloat16 *Wb,
                         __nv_bfloat16 *WbT) {
  tile_bf16_pair(R, C, Wb, WbT, [&](int r, int c) { return W[(size_t)r * C + c]; });
}

// column mean and standard deviation of X [R][C] (float64 sums, rows in order)
__global__ void k_col_stats(const float *__restrict__ X, int R, int C, float *__restrict__ mean,
                            float *__restrict__ stdv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double s = 0.0, s2 = 0.0;
  for (int r = 0; r < R; ++r) {
    const double v = X[(size_t)r * C + c];
    s += v;
    s2 += v * v;
  }
  const double m = s / R;
  const double var = s2 / R - m * m;
  mean[c] = (float)m;
  stdv[c] = (float)sqrt(var > 0.0 ? var : 0.0);
}

// out[r][c] = (X[r][c] - shift[c]) * mul[c]
__global__ void k_affine_cols(const float *__restrict__ X, size_t n, int C,
                              const float *__restrict__ shift, const float *__restrict__ mul,
                              float *__restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    out[e] = (X[e] - shift[c]) * mul[c];
  }
}

}  // namespace specula

using namespace specula;

extern "C" int specula_col_stats(specula_ctx *ctx, const float *X_dev, int32_t rows,
                                 int32_t cols, float *mean_dev, float *std_dev, void *stream) {
  if (!ctx || !X_dev || !mean_dev || !std_dev || rows < 1 || cols < 1) return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_col_stats<<<(cols + 127) / 128, 128, 0, st>>>(X_dev, rows, cols, mean_dev,
                                                                 std_dev));
  return SPECULA_OK;
}

extern "C" int specula_affine_cols(specula_ctx *ctx, const float *X_dev, int64_t rows,
                                   int32_t cols, const float *shift_dev, const float *mul_dev,
                                   float *out_dev, void *stream) {
  if (!ctx || !X_dev || !shift_dev || !mul_dev || !out_dev || rows < 1 || cols < 1)
    return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)rows * cols;
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_affine_cols<<<(unsigned)std::min<size_t>((n + 255) / 256, 8192), 256, 0, st>>>(
                     X_dev, n, cols, shift_dev, mul_dev, out_dev));
  return SPECULA_OK;
}

struct specula_mlp {
  specula_ctx *ctx = nullptr;
  int device = 0;  // copied from ctx so destroy never dereferences it
  int n[4];        // true widths: n_in, h1, h2, n_out
  int np[4];       // padded widths
  int bmax;        // padded batch capacity
  int t = 0;       // Adam steps taken
  int last_b = 0;  // batch of the last forward
  DevBuf W[3], b[3], mW[3], vW[3], mb[3], vb[3], Wb[3], WbT[3], gW[3], gb[3];
  DevBuf Xb, XbT, Z[2], H[2], HT[2], Y, dYf, dYb, dYbT, dA[2], dZb[2], dZbT[2];
  DevBuf work, part, loss;
  DevBuf Hi[2];    // inference activations, [kInferMax][np] float32
  size_t work_floats = 0;
};

static inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---- inference for a few vectors (specula_mlp_infer) ---------------------------
// A batch of a few slope vectors leaves the tensor-core GEMMs (128-row tiles)
// mostly padding, and the time goes to reading the bf16 weights.  Each layer
// is instead one warp per output row streaming that row (16-byte loads, 8 in
// flight per lane) against every input vector in float32, then bias and
// GELU: the weights are read once, activations stay float32.
constexpr int kInferMax = 4;

__device__ __forceinline__ uint4 ld_stream_w(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// out[b][o] = act(sum_k W[o][k] x[b][k] + bias[o]), o < n_out, b < nb;
// W bf16 [.][ldw]; x float [nb][ldx] with k < K read; grid n_out, block 32.
template <int NB, bool GELU>
__global__ void __launch_bounds__(32) k_mlp_gemv(const __nv_bfloat16 *__restrict__ W, int ldw,
                                                 const float *__restrict__ x, int ldx, int K,
                                                 int nb, const float *__restrict__ bias,
                                                 float *__restrict__ out, int ldo) {
  const int o = blockIdx.x, lane = threadIdx.x;
  const uint4 *w8 = reinterpret_cast<const uint4 *>(W + (size_t)o * ldw);
  const int k8 = K / 8;
  float acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) acc[q] = 0.f;
  constexpr int UL = 8;
  for (int j0 = lane; j0 < k8; j0 += UL * 32) {
    uint4 wv[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u)
      wv[u] = j0 + 32 * u < k8 ? ld_stream_w(w8 + j0 + 32 * u) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int j = j0 + 32 * u;
      if (j >= k8) break;
      const float r[8] = {bf16_lo(wv[u].x), bf16_hi(wv[u].x), bf16_lo(wv[u].y), bf16_hi(wv[u].y),
                          bf16_lo(wv[u].z), bf16_hi(wv[u].z), bf16_lo(wv[u].w), bf16_hi(wv[u].w)};
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q < nb) {
          const float *xv = x + (size_t)q * ldx + 8 * j;
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[q] += r[e] * __ldg(xv + e);
        }
      }
    }
  }
  // the K % 8 tail
  for (int k = 8 * k8 + lane; k < K; k += 32) {
    const float wk = __bfloat162float(W[(size_t)o * ldw + k]);
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q < nb) acc[q] += wk * __ldg(x + (size_t)q * ldx + k);
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    float v = acc[q];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (lane == 0 && q < nb) {
      v += bias[o];
      out[(size_t)q * ldo + o] = GELU ? gelu_f(v) : v;
    }
  }
}

static int mlp_splits(int M, int N, int K) {
  const int tiles = (M / 128) * (N / 128);
  int want = std::max(1, (2 * 152 + tiles / 2) / std::max(tiles, 1));
  return gemm_splits(K, want);
}

static int mlp_gemm(specula_mlp *p, const void *A, const void *B, int M, int N, int K, float *C,
                    cudaStream_t st) {
  const int s = mlp_splits(M, N, K);
  if ((size_t)s * M * N > p->work_floats && s > 1) return SPECULA_EINVAL;
  return gemm_bf16_tn(p->ctx, A, B, M, N, K, C, s, p->work.as<float>(), st);
}

static int cast_layer(specula_mlp *p, int l, cudaStream_t st) {
  const int R = p->np[l + 1], C = p->np[l];
  dim3 g((C + TT - 1) / TT, (R + TT - 1) / TT);
  SPECULA_LAUNCH(p->ctx, SPECULA_K_MLP, st,
                 k_cast_w<<<g, dim3(TT, 8), 0, st>>>(p->W[l].as<float>(), R, C,
                                                    p->Wb[l].as<__nv_bfloat16>(),
                                                    p->WbT[l].as<__nv_bfloat16>()));
  return SPECULA_OK;
}

extern "C" int specula_mlp_create(specula_ctx *ctx, int32_t n_in, int32_t n_h1, int32_t n_h2,
                                  int32_t n_out, int32_t batch_max, specula_mlp **out) {
  if (!ctx || !out || n_in < 1 || n_out < 1 || batch_max < 1) return SPECULA_EINVAL;
  if (n_h1 < 128 || n_h2 < 128 || n_h1 % 128 || n_h2 % 128) return SPECULA_EUNSUPPORTED;
  if (n_in > 65536 || n_out > 65536 || batch_max > 65536) return SPECULA_EUNSUPPORTED;
  *out = nullptr;
  SPECULA_CK(cudaSetDevice(ctx->device));
  std::unique_ptr<specula_mlp> p(new specula_mlp());
  p->ctx = ctx;
  p->device = ctx->device;
  p->n[0] = n_in; p->n[1] = n_h1; p->n[2] = n_h2; p->n[3] = n_out;
  p->np[0] = round_up(n_in, 128); p->np[1] = n_h1; p->np[2] = n_h2; p->np[3] = round_up(n_out, 128);
  p->bmax = round_up(batch_max, 128);
  const int Bp = p->bmax;
  int s;
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)p->np[l + 1] * p->np[l], nb = p->np[l + 1];
    if ((s = p->W[l].alloc(nw * 4)) || (s = p->mW[l].alloc(nw * 4)) || (s = p->vW[l].alloc(nw * 4)) ||
        (s = p->gW[l].alloc(nw * 4)) || (s = p->Wb[l].alloc(nw * 2)) || (s = p->WbT[l].alloc(nw * 2)) ||
        (s = p->b[l].alloc(nb * 4)) || (s = p->mb[l].alloc(nb * 4)) || (s = p->vb[l].alloc(nb * 4)) ||
        (s = p->gb[l].alloc(nb * 4)))
      return s;
    SPECULA_CK(cudaMemset(p->W[l].p, 0, nw * 4));
    SPECULA_CK(cudaMemset(p->mW[l].p, 0, nw * 4));
    SPECULA_CK(cudaMemset(p->vW[l].p, 0, nw * 4));
    SPECULA_CK(cudaMemset(p->gW[l].p, 0, nw * 4));
    SPECULA_CK(cudaMemset(p->b[l].p, 0, nb * 4));
    SPECULA_CK(cudaMemset(p->mb[l].p, 0, nb * 4));
    SPECULA_CK(cudaMemset(p->vb[l].p, 0, nb * 4));
    SPECULA_CK(cudaMemset(p->gb[l].p, 0, nb * 4));
  }
  const int in = p->np[0], h1 = p->np[1], h2 = p->np[2], o = p->np[3];
  if ((s = p->Xb.alloc((size_t)Bp * in * 2)) || (s = p->XbT.alloc((size_t)Bp * in * 2)) ||
      (s = p->Z[0].alloc((size_t)Bp * h1 * 4)) || (s = p->Z[1].alloc((size_t)Bp * h2 * 4)) ||
      (s = p->H[0].alloc((size_t)Bp * h1 * 2)) || (s = p->H[1].alloc((size_t)Bp * h2 * 2)) ||
      (s = p->HT[0].alloc((size_t)Bp * h1 * 2)) || (s = p->HT[1].alloc((size_t)Bp * h2 * 2)) ||
      (s = p->Y.alloc((size_t)Bp * o * 4)) || (s = p->dYf.alloc((size_t)Bp * o * 4)) ||
      (s = p->dYb.alloc((size_t)Bp * o * 2)) || (s = p->dYbT.alloc((size_t)Bp * o * 2)) ||
      (s = p->dA[0].alloc((size_t)Bp * h1 * 4)) || (s = p->dA[1].alloc((size_t)Bp * h2 * 4)) ||
      (s = p->dZb[0].alloc((size_t)Bp * h1 * 2)) || (s = p->dZb[1].alloc((size_t)Bp * h2 * 2)) ||
      (s = p->dZbT[0].alloc((size_t)Bp * h1 * 2)) || (s = p->dZbT[1].alloc((size_t)Bp * h2 * 2)))
    return s;
  // split-K workspace: the largest of the eight GEMMs of a step, for every
  // padded batch up to the capacity
  size_t wf = 1;
  for (int b = 128; b <= Bp; b += 128) {
    const int shapes[8][3] = {{b, h1, in}, {b, h2, h1}, {b, o, h2}, {o, h2, b},
                              {b, h2, o},  {h2, h1, b}, {b, h1, h2}, {h1, in, b}};
    for (auto &sh : shapes)
      wf = std::max(wf, (size_t)mlp_splits(sh[0], sh[1], sh[2]) * sh[0] * sh[1]);
  }
  p->work_floats = wf;
  if ((s = p->work.alloc(wf * 4))) return s;
  if ((s = p->Hi[0].alloc((size_t)kInferMax * h1 * 4)) ||
      (s = p->Hi[1].alloc((size_t)kInferMax * h2 * 4)))
    return s;
  const int tiles = ((o + TT - 1) / TT) * ((Bp + TT - 1) / TT);
  if ((s = p->part.alloc((size_t)tiles * 4)) || (s = p->loss.alloc(4))) return s;
  for (int l = 0; l < 3; ++l)
    if ((s = cast_layer(p.get(), l, 0))) return s;
  SPECULA_CK(cudaDeviceSynchronize());
  *out = p.release();
  return SPECULA_OK;
}

extern "C" int specula_mlp_destroy(specula_mlp *mlp) {
  if (!mlp) return SPECULA_EINVAL;
  cudaSetDevice(mlp->device);
  cudaDeviceSynchronize();
  delete mlp;
  return SPECULA_OK;
}

extern "C" int specula_mlp_set_layer(specula_mlp *p, int32_t layer, const float *W_host,
                                     const float *b_host) {
  if (!p || layer < 0 || layer > 2 || !W_host || !b_host) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(p->ctx->device));
  const int R = p->n[layer + 1], C = p->n[layer], RP = p->np[layer + 1], CP = p->np[layer];
  std::vector<float> w((size_t)RP * CP, 0.f), b(RP, 0.f);
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < C; ++c) w[(size_t)r * CP + c] = W_host[(size_t)r * C + c];
  for (int r = 0; r < R; ++r) b[r] = b_host[r];
  SPECULA_CK(cudaMemcpy(p->W[layer].p, w.data(), w.size() * 4, cudaMemcpyHostToDevice));
  SPECULA_CK(cudaMemcpy(p->b[layer].p, b.data(), b.size() * 4, cudaMemcpyHostToDevice));
  for (DevBuf *z : {&p->mW[layer], &p->vW[layer]}) SPECULA_CK(cudaMemset(z->p, 0, z->bytes));
  for (DevBuf *z : {&p->mb[layer], &p->vb[layer]}) SPECULA_CK(cudaMemset(z->p, 0, z->bytes));
  p->t = 0;
  int s = cast_layer(p, layer, 0);
  if (s) return s;
  SPECULA_CK(cudaDeviceSynchronize());
  return SPECULA_OK;
}

static int copy_out(specula_mlp *p, int layer, const DevBuf &W, const DevBuf &b, float *W_host,
                    float *b_host) {
  SPECULA_CK(cudaSetDevice(p->ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());
  const int R = p->n[layer + 1], C = p->n[layer], CP = p->np[layer];
  std::vector<float> w(W.bytes / 4), bb(b.bytes / 4);
  SPECULA_CK(cudaMemcpy(w.data(), W.p, W.bytes, cudaMemcpyDeviceToHost));
  SPECULA_CK(cudaMemcpy(bb.data(), b.p, b.bytes, cudaMemcpyDeviceToHost));
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < C; ++c) W_host[(size_t)r * C + c] = w[(size_t)r * CP + c];
  for (int r = 0; r < R; ++r) b_host[r] = bb[r];
  return SPECULA_OK;
}

extern "C" int specula_mlp_get_layer(specula_mlp *p, int32_t layer, float *W_host,
                                     float *b_host) {
  if (!p || layer < 0 || layer > 2 || !W_host || !b_host) return SPECULA_EINVAL;
  return copy_out(p, layer, p->W[layer], p->b[layer], W_host, b_host);
}

extern "C" int specula_mlp_get_grad(specula_mlp *p, int32_t layer, float *dW_host,
                                    float *db_host) {
  if (!p || layer < 0 || layer > 2 || !dW_host || !db_host) return SPECULA_EINVAL;
  return copy_out(p, layer, p->gW[layer], p->gb[layer], dW_host, db_host);
}

extern "C" int specula_mlp_forward(specula_mlp *p, const float *X_dev, int32_t batch,
                                   float *Y_dev, void *stream) {
  if (!p || !X_dev || batch < 1) return SPECULA_EINVAL;
  const int Bp = round_up(batch, 128);
  if (Bp > p->bmax) return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  specula_ctx *ctx = p->ctx;
  const int in = p->np[0], h1 = p->np[1], h2 = p->np[2], o = p->np[3];
  const dim3 tb(TT, 8);
  int s;
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_pack_input<<<dim3(in / TT, Bp / TT), tb, 0, st>>>(
                     X_dev, batch, p->n[0], Bp, in, p->Xb.as<__nv_bfloat16>(),
                     p->XbT.as<__nv_bfloat16>()));
  const void *Hin = p->Xb.p;
  for (int l = 0; l < 2; ++l) {
    const int K = p->np[l], N = p->np[l + 1];
    if ((s = mlp_gemm(p, Hin, p->Wb[l].p, Bp, N, K, p->Z[l].as<float>(), st))) return s;
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                   k_bias_gelu<<<dim3(N / TT, Bp / TT), tb, 0, st>>>(
                       p->Z[l].as<float>(), p->b[l].as<float>(), Bp, N,
                       p->H[l].as<__nv_bfloat16>(), p->HT[l].as<__nv_bfloat16>()));
    Hin = p->H[l].p;
  }
  if ((s = mlp_gemm(p, Hin, p->Wb[2].p, Bp, o, h2, p->Y.as<float>(), st))) return s;
  const size_t ny = (size_t)Bp * o;
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_add_bias<<<(unsigned)((ny + 255) / 256), 256, 0, st>>>(
                     p->Y.as<float>(), p->b[2].as<float>(), Bp, o));
  if (Y_dev) {
    const size_t n = (size_t)batch * p->n[3];
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                   k_unpack_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                       p->Y.as<float>(), batch, p->n[3], o, Y_dev));
  }
  p->last_b = batch;
  (void)h1;
  return SPECULA_OK;
}

extern "C" int specula_mlp_infer(specula_mlp *p, const float *X_dev, int32_t batch,
                                 float *Y_dev, void *stream) {
  if (!p || !X_dev || !Y_dev || batch < 1) return SPECULA_EINVAL;
  if (batch > kInferMax) return specula_mlp_forward(p, X_dev, batch, Y_dev, stream);
  cudaStream_t st = (cudaStream_t)stream;
  specula_ctx *ctx = p->ctx;
  const __nv_bfloat16 *W0 = p->Wb[0].as<__nv_bfloat16>(), *W1 = p->Wb[1].as<__nv_bfloat16>(),
                      *W2 = p->Wb[2].as<__nv_bfloat16>();
  float *H0 = p->Hi[0].as<float>(), *H1 = p->Hi[1].as<float>();
  const int h1 = p->n[1], h2 = p->n[2];
#define SPECULA_GEMV(NB)                                                                      \
  do {                                                                                        \
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,                                                    \
                   (k_mlp_gemv<NB, true><<<h1, 32, 0, st>>>(W0, p->np[0], X_dev, p->n[0],     \
                                                            p->n[0], batch,                   \
                                                            p->b[0].as<float>(), H0, h1)));   \
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,                                                    \
                   (k_mlp_gemv<NB, true><<<h2, 32, 0, st>>>(W1, p->np[1], H0, h1, h1, batch,  \
                                                            p->b[1].as<float>(), H1, h2)));   \
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,                                                    \
                   (k_mlp_gemv<NB, false><<<p->n[3], 32, 0, st>>>(W2, p->np[2], H1, h2, h2,   \
                                                                  batch, p->b[2].as<float>(), \
                                                                  Y_dev, p->n[3])));          \
  } while (0)
  if (batch == 1)
    SPECULA_GEMV(1);
  else
    SPECULA_GEMV(kInferMax);
#undef SPECULA_GEMV
  return SPECULA_OK;
}

extern "C" int specula_mlp_backward(specula_mlp *p, const float *T_dev, int32_t batch,
                                    float *loss_dev, void *stream) {
  if (!p || !T_dev || batch < 1 || batch != p->last_b) return SPECULA_EINVAL;
  const int Bp = round_up(batch, 128);
  cudaStream_t st = (cudaStream_t)stream;
  specula_ctx *ctx = p->ctx;
  const int in = p->np[0], h1 = p->np[1], h2 = p->np[2], o = p->np[3];
  const dim3 tb(TT, 8);
  const float scale = 2.0f / ((float)batch * (float)p->n[3]);
  const dim3 gl(o / TT, Bp / TT);
  int s;
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_loss_grad<<<gl, tb, 0, st>>>(p->Y.as<float>(), T_dev, batch, p->n[3], Bp, o,
                                                scale, p->dYf.as<float>(),
                                                p->dYb.as<__nv_bfloat16>(),
                                                p->dYbT.as<__nv_bfloat16>(), p->part.as<float>()));
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_loss_final<<<1, 32, 0, st>>>(p->part.as<float>(), (int)(gl.x * gl.y),
                                                1.0f / ((float)batch * (float)p->n[3]),
                                                loss_dev ? loss_dev : p->loss.as<float>()));
  SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                 k_colsum<<<(o + 255) / 256, 256, 0, st>>>(p->dYf.as<float>(), batch, o,
                                                           p->gb[2].as<float>()));
  // layer 3: dW3 = dY^T H2, dH2 = dY W3
  if ((s = mlp_gemm(p, p->dYbT.p, p->HT[1].p, o, h2, Bp, p->gW[2].as<float>(), st))) return s;
  if ((s = mlp_gemm(p, p->dYb.p, p->WbT[2].p, Bp, h2, o, p->dA[1].as<float>(), st))) return s;
  for (int l = 1; l >= 0; --l) {
    const int N = p->np[l + 1], K = p->np[l];
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                   k_gelu_back<<<dim3(N / TT, Bp / TT), tb, 0, st>>>(
                       p->dA[l].as<float>(), p->Z[l].as<float>(), Bp, N,
                       p->dZb[l].as<__nv_bfloat16>(), p->dZbT[l].as<__nv_bfloat16>()));
    SPECULA_LAUNCH(ctx, SPECULA_K_MLP, st,
                   k_colsum<<<(N + 255) / 256, 256, 0, st>>>(p->dA[l].as<float>(), batch, N,
                                                             p->gb[l].as<float>()));
    const void *HinT = l == 1 ? p->HT[0].p : p->XbT.p;
    if ((s = mlp_gemm(p, p->dZbT[l].p, HinT, N, K, Bp, p->gW[l].as<float>(), st))) return s;
    if (l == 1)
      if ((s = mlp_gemm(p, p->dZb[1].p, p->WbT[1].p, Bp, h1, h2, p->dA[0].as<float>(), st)))
        return s;
  }
  (void)in;
  return SPECULA_OK;
}

extern "C" int specula_mlp_adam(specula_mlp *p, float lr, float b1, float b2, float eps,
                                void *stream) {
  if (!p || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps > 0))
    return SPECULA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  p->t += 1;
  const double lr_t = lr * sqrt(1.0 - pow((double)b2, p->t)) / (1.0 - pow((double)b1, p->t));
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)p->np[l + 1] * p->np[l], nb = p->np[l + 1];
    SPECULA_LAUNCH(p->ctx, SPECULA_K_MLP, st,
                   k_adam<<<(unsigned)std::min<size_t>((nw + 255) / 256, 4096), 256, 0, st>>>(
                       p->W[l].as<float>(), p->mW[l].as<float>(), p->vW[l].as<float>(),
                       p->gW[l].as<float>(), nw, (float)lr_t, b1, b2, eps));
    SPECULA_LAUNCH(p->ctx, SPECULA_K_MLP, st,
                   k_adam<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
                       p->b[l].as<float>(), p->mb[l].as<float>(), p->vb[l].as<float>(),
                       p->gb[l].as<float>(), nb, (float)lr_t, b1, b2, eps));
    int s = cast_layer(p, l, st);
    if (s) return s;
  }
  return SPECULA_OK;
}
