// Arithmetic peak probe.  The roof of the FFT stage is the FP32 CUDA-core
// rate, which the GPU's data sheet gives only as SMs x 128 lanes x 2 x clock;
// this kernel measures the fused multiply-add rate directly, in float32 and in
// float64 (the set-up path's Jacobi and covariance work runs in float64).
// Each thread keeps 8 independent a = a x + y chains (x slightly above 1, so
// the values stay finite), unrolled so that loop control is a small share of
// the issue slots, and writes their sum so nothing is optimised away.
#include "internal.h"

namespace specula {

template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(int n_iter, T *__restrict__ sink) {
  T a[8];
  const T x = (T)1.0000001, y = (T)-1e-7;
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i);
#pragma unroll 4
  for (int k = 0; k < n_iter; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], x, y);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace specula

using namespace specula;

extern "C" int specula_fma_probe(specula_ctx *ctx, int32_t bits, int32_t n_ctas, int32_t n_iter,
                                 void *sink_dev, void *stream) {
  if (!ctx || !sink_dev || (bits != 32 && bits != 64) || n_ctas < 1 || n_ctas > 65535 ||
      n_iter < 1 || n_iter > (1 << 24))
    return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (bits == 32)
    SPECULA_LAUNCH(ctx, SPECULA_K_PEAK, st,
                   k_fma_probe<float><<<n_ctas, 256, 0, st>>>(n_iter, (float *)sink_dev));
  else
    SPECULA_LAUNCH(ctx, SPECULA_K_PEAK, st,
                   k_fma_probe<double><<<n_ctas, 256, 0, st>>>(n_iter, (double *)sink_dev));
  return SPECULA_OK;
}
