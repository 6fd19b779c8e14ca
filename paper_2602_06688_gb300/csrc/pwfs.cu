// Modulated pyramid wavefront sensor image (ModulatedPyramid + CCD binning,
// App. A, Tab. 4; parameters of App. B, Listing 2).
//
// Per modulation point m the sensor computes, on the N x N padded grid
// (N = 2 n_pix), I_m = |IDFT2( M . DFT2( pad(E . tilt_m) ) )|^2 with centred
// transforms.  The centred forward transform is an unshifted FFT between an
// input phase p(n) = exp(i pi (N-1) n / N) and an output phase; the output
// phase cancels against the input phase of the centred inverse, whose own
// output phase disappears in |.|^2.  So the GPU evaluates
//     I_m = |IFFT2( M . FFT2( pad(E . tilt_m . p_x p_y) ) )|^2 / N^4,
// with tilt_m . p folded into per-axis tables gx[m][i], gy[m][j] and the
// 1/N^2 folded into the per-axis mask tables.
//
// Pipeline, one chunk of K (batch element, modulation point) items at a time
// so that the intermediates stay L2-resident:
//   F  k_field          E = amp exp(i phase) once per batch element
//   A  k_rows_fwd       E . gx . gy, row FFT of the n_pix non-zero rows
//                       (input half zero: pruned)              -> rows ws
//   B  k_cols           per column tile (staged with cp.async): column FFT
//                       (pruned) -> mask -> inverse column FFT  -> cols ws
//   C  k_rows_inv_part  per (bin strip, item): row inverse FFT -> |.|^2 /
//                       n_mod -> b x b bins              -> part[b][m] ws
//   D  k_bin_reduce     once a batch element's n_mod items are done: the
//                       detector = sum over m in order (no atomics:
//                       bit-reproducible)
//
// Each N-point transform is a two-level split N = N1 x N2 evaluated by one
// group of G lanes: step 1, lane n1 < N1 holds x[n1 + N1 n2] (n2 < N2) and
// does an N2-point register DFT, multiplies by W_N^{n1 k2}; the values are
// exchanged through shared memory; step 2, lane k2 < N2 does an N1-point
// register DFT and holds X[N2 k1 + k2].  With N2 % 4 == 0 the non-zero half
// of a zero-padded input (indices N/4 .. 3N/4) is exactly registers
// N2/4 .. 3N2/4 of every lane, so zero inputs are never loaded.  The
// inter-step twiddles are read through the read-only cache: lane n1 reads
// table[k2][n1], so a warp's reads are consecutive for each k2.
#include <math.h>

#include <algorithm>

#include "fft_regs.cuh"
#include "internal.h"
#include "pwfs_common.cuh"

namespace specula {

int pwfs_init_device() {
  return upload_codelet_twiddles() == cudaSuccess ? SPECULA_OK : SPECULA_ECUDA;
}

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// a read-only load that does not allocate in L1 (data read once per CTA)
__device__ __forceinline__ float2 ld_stream2(const float2 *p) {
  float2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// The N1-point middle stage of a wide split (N2 > 32): lane k2 = lane + 32 t
// (t < NT2) takes column k2 of the exchange xa (xa[k2 S1 + n1]), applies the
// forward N1-point DFT, the mask factor of frequency N2 k1 + k2, the inverse
// N1-point DFT and the twiddle of the swapped split, and writes
// xo[k1 S2 + k2]; xo and xa do not overlap.
template <int N1, int N2>
__device__ __forceinline__ void wide_mid(const float2 *xa, float2 *xo,
                                         const float2 *__restrict__ mask,
                                         const float2 *__restrict__ twB, int lane) {
  using S = Split<N1, N2>;
#pragma unroll 1
  for (int t = 0; t < S::NT2; ++t) {
    const int k2 = lane + 32 * t;
    float2 r2[N1];
    if (k2 < N2) {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xa[k2 * S::S1 + n1];
    } else {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) r2[n1] = make_float2(0.f, 0.f);
    }
    RegDFT<N1, false>::run(r2);
    if (k2 < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) r2[k1] = cmul(r2[k1], __ldg(mask + N2 * k1 + k2));
    }
    RegDFT<N1, true>::run(r2);
    if (k2 < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) xo[k1 * S::S2 + k2] = cmul(r2[k1], __ldg(twB + k1 * N2 + k2));
    }
  }
}

// --------------------------------------------------------------------------
// F: field of the batch elements b0 .. b0 + gridDim.y - 1 into slots b % nbw.
__global__ void __launch_bounds__(256) k_field(const float *__restrict__ amp,
                                               const float *__restrict__ phase,
                                               float2 *__restrict__ field, int npix2, int b0,
                                               int nbw, float phase_scale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npix2) return;
  const int b = b0 + blockIdx.y;
  float sv, cv;
  sincosf(phase[(size_t)b * npix2 + e] * phase_scale, &sv, &cv);
  const float a = amp[e];
  field[(size_t)(b % nbw) * npix2 + e] = make_float2(a * cv, a * sv);
}

// --------------------------------------------------------------------------
// A: E . gx . gy and the row FFT of the non-zero rows.
// grid (ceil(n_pix / VPC), ceil(n_items / ka)); block VPC * G threads.
template <int N1, int N2>
__global__ void __launch_bounds__(256, 2) k_rows_fwd(
    const float2 *__restrict__ field, const float2 *__restrict__ gx,
    const float2 *__restrict__ gy, const float2 *__restrict__ twA, float2 *__restrict__ rows_out,
    int n_pix, int n_mod, int nbw, int item0, int n_items, int ka) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  extern __shared__ float2 smem[];
  const int vpc = blockDim.x / G;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  float2 *xb = smem + vec * S::XB;
  const int j = blockIdx.x * vpc + vec;
  const bool row_ok = j < n_pix;
  const bool in_lane = row_ok && lane < N1;

  float2 e[QH];
  int cur_b = -1;
  const int it_begin = blockIdx.y * ka;
  for (int q = 0; q < ka; ++q) {
    const int it = it_begin + q;
    if (it >= n_items) break;
    const int gi = item0 + it;
    const int b = gi / n_mod, m = gi - b * n_mod;
    if (b != cur_b) {
      cur_b = b;
      const float2 *src = field + ((size_t)(b % nbw) * n_pix + (row_ok ? j : 0)) * n_pix + lane;
#pragma unroll
      for (int h = 0; h < QH; ++h) e[h] = in_lane ? src[N1 * h] : make_float2(0.f, 0.f);
    }
    float2 r[N2];
    const float2 gyv = row_ok ? gy[(size_t)m * n_pix + j] : make_float2(0.f, 0.f);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
    if (in_lane) {
      const float2 *g = gx + (size_t)m * n_pix + lane;
#pragma unroll
      for (int h = 0; h < QH; ++h) r[Q0 + h] = cmul(cmul(e[h], __ldg(g + N1 * h)), gyv);
    }
    RegDFT<N2, false>::run(r);
    __syncwarp();
    if (lane < N1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2)
        xb[k2 * S1 + lane] = cmulc(r[k2], __ldg(twA + k2 * N1 + lane));
    }
    __syncwarp();
    if (lane < N2) {
      float2 r2[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xb[lane * S1 + n1];
      RegDFT<N1, false>::run(r2);
      if (row_ok) {
        float2 *dst = rows_out + ((size_t)it * n_pix + j) * N + lane;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) dst[N2 * k1] = r2[k1];
      }
    }
  }
}

// --------------------------------------------------------------------------
// B: per tile of TC columns: column FFT (rows n_pix non-zero) -> pyramid
// mask -> inverse column FFT, in a column-major shared tile whose column
// stride CS = 2 (mod 16) complex keeps the row-wise staging conflict-free.
// grid (N / TC, n_items); block TC * G threads.
template <int N1, int N2, int TC>
struct ColsCfg {
  using S = Split<N1, N2>;
  static constexpr int CS = round_cs(imax3(S::N, N2 * S::S1, N1 * S::S2));
  static constexpr size_t smem = (size_t)(TC * CS) * sizeof(float2);
};

template <int N1, int N2, int TC>
__global__ void __launch_bounds__(256, 3) k_cols(
    const float2 *__restrict__ rows_in, float2 *__restrict__ cols_out,
    const float2 *__restrict__ twA, const float2 *__restrict__ twB,
    const float2 *__restrict__ mask, int n_pix) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1, S2 = S::S2;
  constexpr int CS = ColsCfg<N1, N2, TC>::CS;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  extern __shared__ float2 smem[];
  float2 *s_tile = smem;
  const int it = blockIdx.y;
  const int col0 = blockIdx.x * TC;
  constexpr int off = N / 4;
  // all staging loads in flight at once (asynchronous copies into the tile)
  const float2 *src = rows_in + (size_t)it * n_pix * N + col0;
  for (int e = threadIdx.x; e < n_pix * TC; e += blockDim.x) {
    const int c = e % TC, jj = e / TC;
    cp_async8(s_tile + c * CS + off + jj, src + (size_t)jj * N + c);
  }
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  const float2 mk = __ldg(mask + col0 + vec);
  cp_async_wait_all();
  __syncthreads();

  float2 *col = s_tile + vec * CS;

  // forward, standard split; non-zero input rows are registers Q0..Q0+QH-1
  float2 r[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  if (lane < N1) {
#pragma unroll
    for (int h = 0; h < QH; ++h) r[Q0 + h] = col[lane + N1 * (Q0 + h)];
  }
  RegDFT<N2, false>::run(r);
  __syncwarp();
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2)
      col[k2 * S1 + lane] = cmulc(r[k2], __ldg(twA + k2 * N1 + lane));
  }
  __syncwarp();
  float2 r2[N1];
  if (lane < N2) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = col[lane * S1 + n1];
  } else {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = make_float2(0.f, 0.f);
  }
  RegDFT<N1, false>::run(r2);
  // lane k2 holds F[v = N2 k1 + k2] of column k = col0 + vec
  if (lane < N2) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      r2[k1] = cmul(r2[k1], cmul(__ldg(mask + N2 * k1 + lane), mk));
  }
  // inverse, swapped split: lane n1' = k2 (< N2), registers n2' = k1 (< N1)
  RegDFT<N1, true>::run(r2);
  __syncwarp();
  if (lane < N2) {
#pragma unroll
    for (int k2 = 0; k2 < N1; ++k2)
      col[k2 * S2 + lane] = cmul(r2[k2], __ldg(twB + k2 * N2 + lane));
  }
  __syncwarp();
  float2 r3[N2];
  if (lane < N1) {
#pragma unroll
    for (int n1 = 0; n1 < N2; ++n1) r3[n1] = col[lane * S2 + n1];
  } else {
#pragma unroll
    for (int n1 = 0; n1 < N2; ++n1) r3[n1] = make_float2(0.f, 0.f);
  }
  RegDFT<N2, true>::run(r3);
  __syncwarp();
  if (lane < N1) {
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1) col[N1 * k1 + lane] = r3[k1];   // y = N1 k1' + k2'
  }
  __syncthreads();
  float2 *dst = cols_out + (size_t)it * N * N + col0;
  for (int e = threadIdx.x; e < N * TC; e += blockDim.x) {
    const int c = e % TC, y = e / TC;
    dst[(size_t)y * N + c] = s_tile[c * CS + y];
  }
}

// --------------------------------------------------------------------------
// C: per (bin strip, item): row inverse FFTs, |.|^2 scaled by 1/n_mod, and
// the b x b bins of the strip into part[b % nbw][m].  Each warp's intensity
// row reuses its own exchange buffer.  grid (N / bsz, n_items);
// block round32(bsz G).
template <int N1, int N2>
__global__ void __launch_bounds__(256, 2) k_rows_inv_part(
    const float2 *__restrict__ cols_in, const float2 *__restrict__ twA, float *__restrict__ part,
    int bsz, float scale, int n_mod, int nbw, int item0) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  const bool act = vec < bsz;
  const int it = blockIdx.y;
  const int y = blockIdx.x * bsz + (act ? vec : 0);
  float2 *xb = smem + vec * S::XB;
  float2 r[N2];
  if (act && lane < N1) {
    const float2 *src = cols_in + ((size_t)it * N + y) * N + lane;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = src[N1 * n2];
  } else {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  }
  RegDFT<N2, true>::run(r);
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = cmul(r[k2], __ldg(twA + k2 * N1 + lane));
  }
  __syncwarp();
  float2 r2[N1];
  if (lane < N2) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xb[lane * S1 + n1];
  }
  __syncwarp();
  float *s_row = reinterpret_cast<float *>(xb);   // this warp's intensity row
  if (act && lane < N2) {
    RegDFT<N1, true>::run(r2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      s_row[N2 * k1 + lane] = (r2[k1].x * r2[k1].x + r2[k1].y * r2[k1].y) * scale;
  }
  __syncthreads();
  const int nd = N / bsz;
  const int gi = item0 + it;
  const int b = gi / n_mod, m = gi - b * n_mod;
  float *dst = part + (((size_t)(b % nbw) * n_mod + m) * nd + blockIdx.x) * nd;
  const float *s_I = reinterpret_cast<const float *>(smem);
  constexpr int RS = 2 * S::XB;   // row stride of the intensity rows (floats)
  for (int q = threadIdx.x; q < nd; q += blockDim.x) {
    float v = 0.f;
    for (int rr = 0; rr < bsz; ++rr)
      for (int xx = 0; xx < bsz; ++xx) v += s_I[rr * RS + q * bsz + xx];
    dst[q] = v;
  }
}

// --------------------------------------------------------------------------
// Two-pass form.  The pyramid mask is separable, M(u, v) = Mx(u) My(v), and
// so is the centred 2D transform, hence
//     IDFT2(M . DFT2(P)) = (IDFT_y My DFT_y) (IDFT_x Mx DFT_x) P :
// the x filter acts on each row alone and the y filter on each column alone.
// Pass R filters the n_pix non-zero rows of every item (forward row FFT of
// the pruned input, x mask, inverse row FFT); pass K filters every column
// (forward FFT of its n_pix non-zero entries, y mask, inverse FFT), squares,
// scales by 1/n_mod and bins, so the N x N intermediate of the three-pass
// form is never written.  Between the two, a slot's filtered rows are held
// column-major ([slot][x][row]): pass R transposes its rows on the way out,
// and pass K reads each column as one contiguous run, coalesced, straight
// into registers.  The inverse row transform's output phase depends
// on x only and vanishes in |.|^2.

template <int N1, int N2> struct RowFiltCfg {
  using S = Split<N1, N2>;
  static constexpr int XBF =
      S::WIDE ? S::XW : (N2 * S::S1 > N1 * S::S2 ? N2 * S::S1 : N1 * S::S2);
  static_assert(S::N <= XBF, "a row fits its vector's exchange buffer");
};

// Points m and n_mod - m share cos(theta), hence the x factor of the tilt;
// their y factors are constant along a row and commute with the row filter.
// So the row filter runs once per distinct cosine ("slot" c = 0 .. nc-1,
// representative m = c) without the y factor, and the column pass applies
// each item's own y factor gy[m][row] to its input.
// R: grid (ceil(n_pix / VPC), ceil(n_slots / ka)); block VPC * G threads;
// writes rows_out[slot][x][row].
// GEN: any padding (the pupil at padded offset `off`, each lane loading the
// registers whose padded index falls in the pupil); otherwise the pad-2
// layout, where the pupil is exactly registers N2/4 .. 3 N2/4 of every lane.
// One-warp transforms (G = 32) run four warps per CTA, five CTAs per SM at
// 96 registers (four rows per CTA: the transposed output goes out as whole
// 32-byte sectors), and reload the field row for every slot (caching it
// across slots needs 32 more registers: spills at that bound); smaller
// transforms run 256 threads, two CTAs per SM, with the cached row; wide
// splits run 128-thread CTAs (bounded for up to 256 threads, one CTA per SM,
// so that their 50-point transforms keep their registers).
template <int N1, int N2> struct RowFiltLaunch {
  using S = Split<N1, N2>;
  static constexpr int threads = S::WIDE ? 256 : (S::G == 32 ? 128 : 256);
  static constexpr int min_blocks = S::WIDE ? 1 : (S::G == 32 ? 5 : 2);
  static constexpr bool reload = S::G == 32;
};
template <int N1, int N2, bool GEN = false>
__global__ void __launch_bounds__(RowFiltLaunch<N1, N2>::threads,
                                  RowFiltLaunch<N1, N2>::min_blocks) k_rowfilt(
    const float2 *__restrict__ field, const float2 *__restrict__ gx,
    const float2 *__restrict__ twA, const float2 *__restrict__ twB,
    const float2 *__restrict__ mask, float2 *__restrict__ rows_out, int n_pix, int nc, int nbw,
    int slot0, int n_slots, int ka, int off, int s0) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1, S2 = S::S2;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  extern __shared__ float2 smem[];
  const int vpc = blockDim.x / G;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  constexpr int XBF = RowFiltCfg<N1, N2>::XBF;
  float2 *xb = smem + vec * XBF;
  // where vector v's output row sits in its buffer: 4 v complex in, as far
  // as the buffer's slack allows, and even, so that with an even XBF two
  // adjacent columns of a row are one aligned 16-byte load
  auto row_tile_off = [](int v) { return min(4 * v, (XBF - N) & ~1); };
  const int j = blockIdx.x * vpc + vec;
  const bool row_ok = j < n_pix;
  const bool in_lane = row_ok && lane < N1;
  float2 e[GEN ? 1 : QH];
  int cur_b = -1;
  const int it_begin = blockIdx.y * ka;
  for (int q = 0; q < ka; ++q) {
    const int it = it_begin + q;
    if (it >= n_slots) break;
    const int gi = slot0 + it;
    const int b = gi / nc, c = s0 + (gi - b * nc);   // nc slots per element from s0
    if (!GEN && (RowFiltLaunch<N1, N2>::reload || b != cur_b)) {
      cur_b = b;
      const float2 *src = field + ((size_t)(b % nbw) * n_pix + (row_ok ? j : 0)) * n_pix + lane;
#pragma unroll
      for (int h = 0; h < (GEN ? 1 : QH); ++h) e[h] = in_lane ? src[N1 * h] : make_float2(0.f, 0.f);
    }
    // forward row transform, pruned input (standard split)
    float2 r[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
    if (in_lane) {
      if constexpr (GEN) {
        const float2 *src = field + ((size_t)(b % nbw) * n_pix + j) * n_pix;
        const float2 *g = gx + (size_t)c * n_pix;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
          const int i = lane + N1 * n2 - off;                // pupil column
          if (i >= 0 && i < n_pix) r[n2] = cmul(src[i], __ldg(g + i));
        }
      } else {
        const float2 *g = gx + (size_t)c * n_pix + lane;
#pragma unroll
        for (int h = 0; h < QH; ++h) r[Q0 + h] = cmul(e[h], __ldg(g + N1 * h));
      }
    }
    RegDFT<N2, false>::run(r);
    __syncwarp();
    if (lane < N1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = cmulc(r[k2], __ldg(twA + k2 * N1 + lane));
    }
    __syncwarp();
    float2 *x3 = xb;   // input of the last stage
    if constexpr (S::WIDE) {
      x3 = xb + N2 * S1;
      wide_mid<N1, N2>(xb, x3, mask, twB, lane);
    } else {
      float2 r2[N1];
      if (lane < N2) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xb[lane * S1 + n1];
      } else {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) r2[n1] = make_float2(0.f, 0.f);
      }
      RegDFT<N1, false>::run(r2);
      // x mask, then the inverse row transform (swapped split)
      if (lane < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) r2[k1] = cmul(r2[k1], __ldg(mask + N2 * k1 + lane));
      }
      RegDFT<N1, true>::run(r2);
      __syncwarp();
      if (lane < N2) {
#pragma unroll
        for (int k2 = 0; k2 < N1; ++k2)
          xb[k2 * S2 + lane] = cmul(r2[k2], __ldg(twB + k2 * N2 + lane));
      }
    }
    __syncwarp();
    float2 r3[N2];
    if (lane < N1) {
#pragma unroll
      for (int n1 = 0; n1 < N2; ++n1) r3[n1] = x3[lane * S2 + n1];
    } else {
#pragma unroll
      for (int n1 = 0; n1 < N2; ++n1) r3[n1] = make_float2(0.f, 0.f);
    }
    RegDFT<N2, true>::run(r3);
    // The slot's block is column-major (rows_out[it][x][row]), so that the
    // column pass loads a column coalesced.  Each vector puts its row in
    // its own exchange buffer (T_v, offset a few complex per vector against
    // bank conflicts), and the CTA writes one run of vpc rows per column x,
    // as 16-byte row pairs where the rows allow.
    __syncwarp();   // this vector's last-stage loads are done
    if (lane < N1) {
#pragma unroll
      for (int k1 = 0; k1 < N2; ++k1) xb[N1 * k1 + lane + row_tile_off(vec)] = r3[k1];   // x = N1 k1 + lane
    }
    __syncthreads();
    {
      const int j0 = blockIdx.x * vpc;
      float2 *dst = rows_out + ((size_t)it * N) * n_pix + j0;
      if ((vpc & 1) == 0 && (n_pix & 1) == 0) {
        const int hp = vpc / 2, h = threadIdx.x % hp;   // rows 2h and 2h + 1
        if (j0 + 2 * h < n_pix) {                       // n_pix even: both rows exist
          const float2 *ta = smem + (2 * h) * XBF + row_tile_off(2 * h);
          const float2 *tb = smem + (2 * h + 1) * XBF + row_tile_off(2 * h + 1);
          if constexpr (XBF % 2 == 0) {
            // columns x and x + 1 of both rows: two 16-byte loads, two stores
            for (int x = 2 * (threadIdx.x / hp); x < N; x += 4 * G) {
              const float4 a = *reinterpret_cast<const float4 *>(ta + x);
              const float4 c = *reinterpret_cast<const float4 *>(tb + x);
              *reinterpret_cast<float4 *>(dst + (size_t)x * n_pix + 2 * h) =
                  make_float4(a.x, a.y, c.x, c.y);
              *reinterpret_cast<float4 *>(dst + (size_t)(x + 1) * n_pix + 2 * h) =
                  make_float4(a.z, a.w, c.z, c.w);
            }
          } else {
            for (int x = threadIdx.x / hp; x < N; x += 2 * G) {
              const float2 a = ta[x], c = tb[x];
              *reinterpret_cast<float4 *>(dst + (size_t)x * n_pix + 2 * h) =
                  make_float4(a.x, a.y, c.x, c.y);
            }
          }
        }
      } else {
        const int v = threadIdx.x % vpc;
        if (j0 + v < n_pix) {
          const float2 *tv = smem + v * XBF + row_tile_off(v);
          for (int x = threadIdx.x / vpc; x < N; x += G) dst[(size_t)x * n_pix + v] = tv[x];
        }
      }
    }
    if (q + 1 < ka && it + 1 < n_slots) __syncthreads();   // the buffers are the next slot's
  }
}

// K: per tile of TC = blockDim.x / G columns (a multiple of the bin side),
// read from rows_in[slot][x][row]: the item's y tilt, column filter,
// |.|^2 / n_mod, b x b bins ->
// part[b % nbw][m][ybin][xbin].  grid (N / TC, 2 n_slots): y = 2 p + w is
// item m = c (w = 0) or m = n_mod - c (w = 1, when distinct) of slot p.
// Column stride CS (complex) of the exchange buffers: at least the exchange
// buffer of a column, odd.
template <int N1, int N2> struct ColFiltCfg {
  using S = Split<N1, N2>;
  static constexpr int base = S::WIDE ? S::XW : imax3(S::N, N2 * S::S1, N1 * S::S2);
  static int stride(int) { return base | 1; }
};

// One-warp columns in tiles of at most 160 threads (five columns for the
// 39 m pupil's bin side 5) take the variant bounded at 160 threads x 4 CTAs
// per SM, the occupancy that 80 registers per thread gave them already:
// 96 registers per thread, so the twiddle loads can be issued earlier.
template <int N1, int N2, int MAXT = 256, bool GEN = false>
__global__ void __launch_bounds__(MAXT, Split<N1, N2>::WIDE
                                              ? 1
                                              : (MAXT <= 160 ? 4 : (MAXT <= 256 ? 3 : 2)))
    k_colfilt_bin(
    const float2 *__restrict__ rows_in, const float2 *__restrict__ gy,
    const float2 *__restrict__ twA, const float2 *__restrict__ twB,
    const float2 *__restrict__ mask, float *__restrict__ part, int n_pix, int fp, int fq,
    float scale, int n_mod, int nc, int nbw, int slot0, int CS, int off, int s0) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, G = S::G, S1 = S::S1, S2 = S::S2;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  extern __shared__ __align__(16) float2 smem_k[];
  float2 *s_tile = smem_k;
  const int TC = blockDim.x / G;
  const int it = blockIdx.y >> 1;              // slot within the chunk
  const int gs = slot0 + it;
  const int b = gs / nc, cslot = s0 + (gs - b * nc);   // nc slots per element from s0
  const int m = (blockIdx.y & 1) ? n_mod - cslot : cslot;
  if ((blockIdx.y & 1) && (cslot == 0 || 2 * cslot == n_mod)) return;   // no second item
  const int col0 = blockIdx.x * TC;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  // wide splits stage the item's y factors in shared memory (5% off their
  // column pass; at 960 the factors come through L1 as fast)
  float2 *s_gy = nullptr;
  if constexpr (S::WIDE) {
    s_gy = s_tile + ((TC * CS + 1) & ~1);   // 16-byte aligned
    const float2 *g = gy + (size_t)m * n_pix;
    if ((n_pix & 1) == 0) {
      for (int i = threadIdx.x; 2 * i < n_pix; i += blockDim.x) cp_async16(s_gy + 2 * i, g + 2 * i);
    } else {
      for (int i = threadIdx.x; i < n_pix; i += blockDim.x) cp_async8(s_gy + i, g + i);
    }
    cp_async_wait_all();
    __syncthreads();
  }
  // this vector's column x = col0 + vec: n_pix contiguous rows of the
  // slot's column-major block, loaded coalesced straight into registers and
  // past L1 (which keeps the twiddle, mask and tilt tables)
  const float2 *cx = rows_in + ((size_t)it * N + col0 + vec) * n_pix;
  float2 r[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  if (lane < N1) {
    if constexpr (GEN) {
      const float2 *g = gy + (size_t)m * n_pix;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int row = lane + N1 * n2 - off;                // pupil row
        if (row >= 0 && row < n_pix) {
          if constexpr (S::WIDE)
            r[n2] = cmul(ld_stream2(cx + row), s_gy[row]);
          else
            r[n2] = cmul(ld_stream2(cx + row), __ldg(g + row));
        }
      }
    } else {
      const float2 *g = gy + (size_t)m * n_pix + lane;   // pupil row lane + N1 h
      const float2 *w = cx + lane;
      float2 e[QH];
#pragma unroll
      for (int h = 0; h < QH; ++h) e[h] = ld_stream2(w + N1 * h);
#pragma unroll
      for (int h = 0; h < QH; ++h) r[Q0 + h] = cmul(e[h], __ldg(g + N1 * h));
    }
  }
  float2 *col = s_tile + vec * CS;   // this vector's exchange buffer
  RegDFT<N2, false>::run(r);
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) col[k2 * S1 + lane] = cmulc(r[k2], __ldg(twA + k2 * N1 + lane));
  }
  __syncwarp();
  float2 *x3 = col;   // input of the last stage
  if constexpr (S::WIDE) {
    x3 = col + N2 * S1;
    wide_mid<N1, N2>(col, x3, mask, twB, lane);
  } else {
    float2 r2[N1];
    if (lane < N2) {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) r2[n1] = col[lane * S1 + n1];
    } else {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) r2[n1] = make_float2(0.f, 0.f);
    }
    RegDFT<N1, false>::run(r2);
    if (lane < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) r2[k1] = cmul(r2[k1], __ldg(mask + N2 * k1 + lane));
    }
    RegDFT<N1, true>::run(r2);
    __syncwarp();
    if (lane < N2) {
#pragma unroll
      for (int k2 = 0; k2 < N1; ++k2)
        col[k2 * S2 + lane] = cmul(r2[k2], __ldg(twB + k2 * N2 + lane));
    }
  }
  __syncwarp();
  float2 r3[N2];
  if (lane < N1) {
#pragma unroll
    for (int n1 = 0; n1 < N2; ++n1) r3[n1] = x3[lane * S2 + n1];
  } else {
#pragma unroll
    for (int n1 = 0; n1 < N2; ++n1) r3[n1] = make_float2(0.f, 0.f);
  }
  RegDFT<N2, true>::run(r3);
  __syncwarp();
  float *colI = reinterpret_cast<float *>(col);   // this column's intensity, y = N1 k1 + lane
  if (lane < N1) {
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1)
      colI[N1 * k1 + lane] = (r3[k1].x * r3[k1].x + r3[k1].y * r3[k1].y) * scale;
  }
  __syncthreads();
  float *dst = part + ((size_t)(b % nbw) * n_mod + m) * (N * fq / fp) * (N * fq / fp);
  const float *s_I = reinterpret_cast<const float *>(smem_k);
  if (fq != 1) {
    // fractional detector pixels of fp / fq grid pixels (area-weighted
    // rebinning): output pixel o covers [o fp, (o + 1) fp) and grid pixel i
    // covers [i fq, (i + 1) fq) in units of 1 / fq; the weight is their
    // overlap, an integer, and the sum is divided by fq^2 once.  The tile's
    // TC = k fp columns hold exactly its k fq output columns.
    const int nd = N * fq / fp, nxo = TC / fp * fq, xo0 = col0 / fp * fq;
    const float inv = 1.0f / (float)(fq * fq);
    for (int q = threadIdx.x; q < nd * nxo; q += blockDim.x) {
      const int yo = q / nxo, X = xo0 + (q - yo * nxo);
      const int px0 = X * fp / fq, px1 = ((X + 1) * fp + fq - 1) / fq;
      const int py0 = yo * fp / fq, py1 = ((yo + 1) * fp + fq - 1) / fq;
      float v = 0.f;
      for (int py = py0; py < py1; ++py) {
        const int wy = min((py + 1) * fq, (yo + 1) * fp) - max(py * fq, yo * fp);
        for (int px = px0; px < px1; ++px) {
          const int wx = min((px + 1) * fq, (X + 1) * fp) - max(px * fq, X * fp);
          v += (float)(wx * wy) * s_I[(size_t)(px - col0) * 2 * CS + py];
        }
      }
      dst[(size_t)yo * nd + X] = v * inv;
    }
    return;
  }
  const int bsz = fp, nd = N / bsz, nbx = TC / bsz;
  if (bsz == 5 && nbx == 1) {
    // the 39 m pupil's 5 x 5 bins, one bin column per tile: unrolled sums
    for (int yb = threadIdx.x; yb < nd; yb += blockDim.x) {
      const float *c0 = s_I + yb * 5;
      float v = 0.f;
#pragma unroll
      for (int rr = 0; rr < 5; ++rr)
#pragma unroll
        for (int cc = 0; cc < 5; ++cc) v += c0[cc * 2 * CS + rr];
      dst[(size_t)yb * nd + col0 / 5] = v;
    }
    return;
  }
  for (int q = threadIdx.x; q < nd * nbx; q += blockDim.x) {
    const int yb = q / nbx, xb = q - yb * nbx;
    float v = 0.f;
    for (int rr = 0; rr < bsz; ++rr)
      for (int cc = 0; cc < bsz; ++cc) v += s_I[(size_t)(xb * bsz + cc) * 2 * CS + yb * bsz + rr];
    dst[(size_t)yb * nd + col0 / bsz + xb] = v;
  }
}

// --------------------------------------------------------------------------
// D: det[b] = sum over m = 0 .. n_mod-1 of part[b % nbw][m], in order.
// grid (ceil(nd^2 / 256), number of batch elements from b0).
__global__ void __launch_bounds__(256) k_bin_reduce(const float *__restrict__ part,
                                                    float *__restrict__ det, int nd2, int n_mod,
                                                    int nbw, int b0, float alpha, float beta) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= nd2) return;
  const int b = b0 + blockIdx.y;
  const float *src = part + (size_t)(b % nbw) * n_mod * nd2 + pix;
  // sixteen loads in flight, then the adds in order m = 0, 1, ...
  float v = 0.f;
  int m = 0;
  for (; m + 16 <= n_mod; m += 16) {
    float x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = src[(size_t)(m + u) * nd2];
#pragma unroll
    for (int u = 0; u < 16; ++u) v += x[u];
  }
  for (; m < n_mod; ++m) v += src[(size_t)m * nd2];
  // det = alpha v (beta = 0) or beta det + alpha v (accumulating images)
  float *d = det + (size_t)b * nd2 + pix;
  *d = beta == 0.f ? alpha * v : beta * *d + alpha * v;
}

// --------------------------------------------------------------------------
// host side

constexpr int kColsTile = 8;

template <int N1, int N2>
static int configure(PwfsPlan *p) {
  using S = Split<N1, N2>;
  {
    const int nd = p->pad * p->n_sub;
    int a = S::N, b = nd;
    while (b) {
      const int t = a % b;
      a = b;
      b = t;
    }
    p->fp = S::N / a;
    p->fq = nd / a;
  }
  int s;
  if constexpr (S::WIDE) {
    // wide splits: the two-pass form only
    p->blockA = p->blockB = p->blockC = 0;
    p->smemA = p->smemB = p->smemC = 0;
  } else {
    const int bsz = p->fq == 1 ? p->fp : 0;   // whole bins only below the two-pass form
    p->blockA = 256;
    const int vpcA = 256 / S::G;
    p->smemA = (size_t)(vpcA * S::XB) * sizeof(float2);
    p->blockB = kColsTile * S::G;
    p->smemB = ColsCfg<N1, N2, kColsTile>::smem;
    const int thrC = ((bsz * S::G + 31) / 32) * 32;
    if (thrC > 256) return SPECULA_EUNSUPPORTED;   // bin side too large for one CTA strip
    p->blockC = bsz ? thrC : 0;                     // 0: no three-pass form (fractional bins)
    const int nvecC = thrC / S::G;
    p->smemC = (size_t)(nvecC * S::XB) * sizeof(float2);
    if (p->smemA > 227 * 1024 || p->smemB > 227 * 1024 || p->smemC > 227 * 1024)
      return SPECULA_EUNSUPPORTED;
    if ((s = ensure_dynamic_smem((const void *)k_rows_fwd<N1, N2>, p->smemA)) ||
        (s = ensure_dynamic_smem((const void *)k_cols<N1, N2, kColsTile>, p->smemB)) ||
        (s = ensure_dynamic_smem((const void *)k_rows_inv_part<N1, N2>, p->smemC)))
      return s;
  }
  // two-pass form: column tiles of TC = k fp grid columns (k fq detector
  // columns, so every detector pixel lies in one CTA), k the largest divisor
  // of pad n_sub / fq with TC G <= 256 threads (352 where a detector pixel
  // is a fraction of grid pixels: the SOUL example's 11-column tiles)
  // (wide splits: 128-thread CTAs, two per SM within the register budget of
  // their 50-point transforms, so one CTA's barriers do not idle the SM)
  p->two_ok = false;
  p->blockR = S::WIDE ? 128 : RowFiltLaunch<N1, N2>::threads;
  p->smemR = (size_t)(p->blockR / S::G) * RowFiltCfg<N1, N2>::XBF * sizeof(float2);
  const int ndq = p->pad * p->n_sub / p->fq;
  const int maxt = S::WIDE ? 128 : (p->fq == 1 ? 256 : 352);
  int k = 0;
  for (int d = 1; d <= ndq; ++d)
    if (ndq % d == 0 && d * p->fp * S::G <= maxt) k = d;
  if (k > 0 && p->smemR <= 227 * 1024) {
    const int tc = k * p->fp;
    p->blockK = tc * S::G;
    p->csK = ColFiltCfg<N1, N2>::stride(tc);
    // the tile's exchange buffers (wide splits: and the item's n_pix y
    // factors, after a 16-byte boundary)
    p->smemK = ((size_t)tc * p->csK + (S::WIDE ? 1 + p->n_pix : 0)) * sizeof(float2);
    if (p->smemK <= 227 * 1024 && S::N % tc == 0) {
      if constexpr (S::WIDE) {
        // general-offset loads only (N2 % 4 != 0 or pad != 2), tiles of up to 128 threads
        if ((s = ensure_dynamic_smem((const void *)k_rowfilt<N1, N2, true>, p->smemR)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2, 256, true>, p->smemK)))
          return s;
      } else {
        if ((s = ensure_dynamic_smem((const void *)k_rowfilt<N1, N2>, p->smemR)) ||
            (s = ensure_dynamic_smem((const void *)k_rowfilt<N1, N2, true>, p->smemR)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2>, p->smemK)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2, 160>, p->smemK)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2, 256, true>, p->smemK)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2, 160, true>, p->smemK)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2, 352>, p->smemK)) ||
            (s = ensure_dynamic_smem((const void *)k_colfilt_bin<N1, N2, 352, true>, p->smemK)))
          return s;
      }
      p->two_ok = true;
    }
  }
  return SPECULA_OK;
}

// Two-pass form, one chunk of `chunk` row-filter slots (batch element,
// distinct cosine) at a time; each slot feeds one or two column items.
template <int N1, int N2>
static int run_split2(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                      int n_batch, float *det, cudaStream_t st) {
  using S = Split<N1, N2>;
  const int Np = p->n_pix;
  const int nd = p->pad * p->n_sub;   // detector side
  // the imaged cosine slots [s0, s0 + nc) of every batch element
  const int s0 = p->slot_lo;
  const int nc = (p->slot_hi < 0 ? p->nc : p->slot_hi) - s0;
  const int total = n_batch * nc;
  const int vpc = p->blockR / S::G;
  const int tc = p->blockK / S::G;
  const float scale = 1.0f / (float)p->n_mod;
  int field_done = -1, det_done = -1;
  for (int j0 = 0; j0 < total; j0 += p->chunk) {
    const int nj = std::min(p->chunk, total - j0);
    const int b0 = j0 / nc, b1 = (j0 + nj - 1) / nc;
    const int fb = std::max(b0, field_done + 1);
    if (fb <= b1) {
      dim3 gF((Np * Np + 255) / 256, b1 - fb + 1);
      SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_FIELD, st,
                     k_field<<<gF, 256, 0, st>>>(amp, phase, p->field.as<float2>(), Np * Np, fb,
                                                 p->nbw, p->run_phase_scale));
      field_done = b1;
    }
    dim3 gR((Np + vpc - 1) / vpc, (nj + p->ka - 1) / p->ka);
    const int off = (S::N - Np) / 2;                // the pupil's padded offset
    const bool gen = p->pad != 2 || N2 % 4 != 0;   // general-offset loads
#define SPECULA_ROWFILT(GEN_)                                                                  \
  SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_ROWFILT, st,                                              \
                 k_rowfilt<N1, N2, GEN_><<<gR, p->blockR, p->smemR, st>>>(                     \
                     p->field.as<float2>(), p->gx.as<float2>(), p->twA.as<float2>(),           \
                     p->twB.as<float2>(), p->mask.as<float2>(), p->rows.as<float2>(), Np, nc,  \
                     p->nbw, j0, nj, p->ka, off, s0))
#define SPECULA_COLFILT(MAXT_, GEN_)                                                           \
  SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_COLFILT, st,                                              \
                 k_colfilt_bin<N1, N2, MAXT_, GEN_><<<gK, p->blockK, p->smemK, st>>>(          \
                     p->rows.as<float2>(), p->gy.as<float2>(), p->twA.as<float2>(),            \
                     p->twB.as<float2>(), p->mask.as<float2>(), p->part.as<float>(), Np, p->fp, \
                     p->fq, scale, p->n_mod, nc, p->nbw, j0, p->csK, off, s0))
    dim3 gK(S::N / tc, 2 * nj);
    const bool k160 = S::G == 32 && p->blockK <= 160;
    if constexpr (S::WIDE) {
      SPECULA_ROWFILT(true);   // the plan refuses pad 2 for N2 % 4 != 0; wide tiles <= 128
      SPECULA_COLFILT(256, true);
    } else {
      if (gen)
        SPECULA_ROWFILT(true);
      else
        SPECULA_ROWFILT(false);
      if (p->blockK > 256 && gen)     // tiles of fractional detector pixels
        SPECULA_COLFILT(352, true);
      else if (p->blockK > 256)
        SPECULA_COLFILT(352, false);
      else if (k160 && gen)
        SPECULA_COLFILT(160, true);
      else if (k160)
        SPECULA_COLFILT(160, false);
      else if (gen)
        SPECULA_COLFILT(256, true);
      else
        SPECULA_COLFILT(256, false);
    }
#undef SPECULA_ROWFILT
#undef SPECULA_COLFILT
    const int complete = (j0 + nj) / nc - 1;
    if (complete > det_done) {
      dim3 gD((nd * nd + 255) / 256, complete - det_done);
      SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_BIN, st,
                     k_bin_reduce<<<gD, 256, 0, st>>>(p->part.as<float>(), det, nd * nd,
                                                      p->n_mod, p->nbw, det_done + 1,
                                                      p->run_alpha, p->run_beta));
      det_done = complete;
    }
  }
  return SPECULA_OK;
}

template <int N1, int N2>
static int run_split(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                     int n_batch, float *det, cudaStream_t st) {
  if (p->passes == 2) return run_split2<N1, N2>(ctx, p, amp, phase, n_batch, det, st);
  using S = Split<N1, N2>;
  if constexpr (S::WIDE) {
    return SPECULA_EUNSUPPORTED;   // the three-pass kernels hold N2 <= 32
  } else {
    const int Np = p->n_pix;
    const int bsz = Np / p->n_sub;
    const int nd = S::N / bsz;
    const int total = n_batch * p->n_mod;
    const int vpcA = p->blockA / S::G;
    const float scale = 1.0f / (float)p->n_mod;
    int field_done = -1;   // highest batch element whose field is in its slot
    int det_done = -1;     // highest batch element whose detector is written
    for (int i0 = 0; i0 < total; i0 += p->chunk) {
      const int ni = std::min(p->chunk, total - i0);
      const int b0 = i0 / p->n_mod, b1 = (i0 + ni - 1) / p->n_mod;
      const int fb = std::max(b0, field_done + 1);
      if (fb <= b1) {
        dim3 gF((Np * Np + 255) / 256, b1 - fb + 1);
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_FIELD, st,
                       k_field<<<gF, 256, 0, st>>>(amp, phase, p->field.as<float2>(), Np * Np, fb,
                                                   p->nbw, p->run_phase_scale));
        field_done = b1;
      }
      dim3 gA((Np + vpcA - 1) / vpcA, (ni + p->ka - 1) / p->ka);
      {
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_ROWS_FWD, st,
                       k_rows_fwd<N1, N2><<<gA, p->blockA, p->smemA, st>>>(
                           p->field.as<float2>(), p->gx.as<float2>(), p->gy.as<float2>(),
                           p->twA.as<float2>(), p->rows.as<float2>(), Np, p->n_mod, p->nbw, i0,
                           ni, p->ka));
        dim3 gB(S::N / kColsTile, ni);
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_COLS, st,
                       k_cols<N1, N2, kColsTile><<<gB, p->blockB, p->smemB, st>>>(
                           p->rows.as<float2>(), p->cols.as<float2>(), p->twA.as<float2>(),
                           p->twB.as<float2>(), p->mask.as<float2>(), Np));
        dim3 gC(S::N / bsz, ni);
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_ROWS_INV, st,
                       k_rows_inv_part<N1, N2><<<gC, p->blockC, p->smemC, st>>>(
                           p->cols.as<float2>(), p->twA.as<float2>(), p->part.as<float>(), bsz,
                           scale, p->n_mod, p->nbw, i0));
      }
      // batch elements whose last modulation point is in this chunk
      const int complete = (i0 + ni) / p->n_mod - 1;
      if (complete > det_done) {
        dim3 gD((nd * nd + 255) / 256, complete - det_done);
        SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_BIN, st,
                       k_bin_reduce<<<gD, 256, 0, st>>>(p->part.as<float>(), det, nd * nd,
                                                        p->n_mod, p->nbw, det_done + 1,
                                                        p->run_alpha, p->run_beta));
        det_done = complete;
      }
    }
    return SPECULA_OK;
  }
}

bool pwfs_split_for(int N, int *N1, int *N2) {
  switch (N) {
    case 64: *N1 = 8; *N2 = 8; return true;
    case 128: *N1 = 8; *N2 = 16; return true;
    case 240: *N1 = 15; *N2 = 16; return true;
    case 320: *N1 = 20; *N2 = 16; return true;
    case 660: *N1 = 30; *N2 = 22; return true;   // 22 = 2 x 11, prime-factor form
    case 960: *N1 = 30; *N2 = 32; return true;
    case 1600: *N1 = 32; *N2 = 50; return true;   // wide: 50 = 2 x 25 in two lane strides
    default: return false;
  }
}

int pwfs_set_tiles(PwfsPlan *p, int chunk, int ka, int passes) {
  if (passes < 2 || passes > 4) return SPECULA_EINVAL;
  if (passes == 2 && !p->two_ok) return SPECULA_EUNSUPPORTED;
  if (passes == 3 && (p->pad != 2 || !p->blockC)) return SPECULA_EUNSUPPORTED;   // pad-2, whole bins
  if (passes == 4 && !p->pair_ok) return SPECULA_EUNSUPPORTED;
  const int nd = p->pad * p->n_sub;   // detector side
  // batch elements one chunk can touch: chunk items (three-pass) or chunk
  // row-filter slots, nc per batch element (two-pass); the paired form runs
  // whole batch elements, chunk / nc (at least one) per launch
  const int per_b = passes == 3 ? p->n_mod : p->nc;
  if (passes == 4) chunk = std::max(1, chunk / p->nc) * p->nc;
  const int nbw = passes == 4 ? chunk / p->nc : (chunk + per_b - 1) / per_b + 1;
  const size_t need_field = (size_t)nbw * p->n_pix * p->n_pix * sizeof(float2);
  // two complex of padding: the paired form's column staging window may
  // read one entry past the last row
  const size_t need_rows = ((size_t)chunk * p->n_pix * p->N + 2) * sizeof(float2);
  const size_t need_cols = passes == 3 ? (size_t)chunk * p->N * p->N * sizeof(float2) : 0;
  const size_t need_part = (size_t)nbw * p->n_mod * nd * nd * sizeof(float);
  int s;
  if (need_rows > p->rows.bytes || need_cols > p->cols.bytes || need_field > p->field.bytes ||
      need_part > p->part.bytes) {
    cudaDeviceSynchronize();   // the old workspace may still be in use
    if ((s = p->field.alloc(std::max(need_field, p->field.bytes)))) return s;
    if ((s = p->rows.alloc(std::max(need_rows, p->rows.bytes)))) return s;
    if (need_cols > p->cols.bytes && (s = p->cols.alloc(need_cols))) return s;
    if ((s = p->part.alloc(std::max(need_part, p->part.bytes)))) return s;
    // items outside an imaged slot range are never written: they read as 0
    SPECULA_CK(cudaMemset(p->part.p, 0, p->part.bytes));
  }
  p->chunk = chunk;
  p->ka = ka;
  p->nbw = nbw;
  p->passes = passes;
  return SPECULA_OK;
}

int pwfs_bin_reduce(specula_ctx *ctx, const float *part, float *det, int nd2, int n_mod,
                    float alpha, float beta, cudaStream_t st) {
  SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_BIN, st,
                 k_bin_reduce<<<dim3((nd2 + 255) / 256, 1), 256, 0, st>>>(part, det, nd2, n_mod,
                                                                          1, 0, alpha, beta));
  return SPECULA_OK;
}

int pwfs_field_launch(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                      int fb, int nb, cudaStream_t st) {
  const int Np = p->n_pix;
  dim3 gF((Np * Np + 255) / 256, nb);
  SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_FIELD, st,
                 k_field<<<gF, 256, 0, st>>>(amp, phase, p->field.as<float2>(), Np * Np, fb, p->nbw,
                                             p->run_phase_scale));
  return SPECULA_OK;
}

int pwfs_bin_reduce_range(specula_ctx *ctx, PwfsPlan *p, float *det, int nd2, int b0, int nb,
                          cudaStream_t st) {
  dim3 gD((nd2 + 255) / 256, nb);
  SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_BIN, st,
                 k_bin_reduce<<<gD, 256, 0, st>>>(p->part.as<float>(), det, nd2, p->n_mod, p->nbw,
                                                  b0, p->run_alpha, p->run_beta));
  return SPECULA_OK;
}

int pwfs_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase, int n_batch,
             float *det, cudaStream_t st) {
  if (p->slot_hi >= 0 && (p->form != SPECULA_PWFS_FORM_TILT || p->passes == 3))
    return SPECULA_EUNSUPPORTED;   // slot ranges: the two-pass tilt forms only
  if (p->form == SPECULA_PWFS_FORM_SHIFTED)
    return pwfs_shifted_run(ctx, p, amp, phase, n_batch, det, st);
  if (p->form == SPECULA_PWFS_FORM_DFTGEMM_BF16 || p->form == SPECULA_PWFS_FORM_DFTGEMM_TF32)
    return pwfs_dftgemm_run(ctx, p, amp, phase, n_batch, det, st);
  if (p->passes == 4) return pwfs_pair_run(ctx, p, amp, phase, n_batch, det, st);
  switch (p->N) {
    case 64: return run_split<8, 8>(ctx, p, amp, phase, n_batch, det, st);
    case 128: return run_split<8, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 240: return run_split<15, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 320: return run_split<20, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 660: return run_split<30, 22>(ctx, p, amp, phase, n_batch, det, st);
    case 960: return run_split<30, 32>(ctx, p, amp, phase, n_batch, det, st);
    case 1600: return run_split<32, 50>(ctx, p, amp, phase, n_batch, det, st);
    default: return SPECULA_EUNSUPPORTED;
  }
}

// Time each candidate tiling on the caller's buffers (set-up call: may
// reallocate the workspace and synchronises) and keep the fastest.
int pwfs_autotune(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                  int n_batch, float *det, cudaStream_t st, int reps, size_t max_ws_bytes,
                  int *best_chunk, int *best_ka, int *best_passes) {
  static const int kChunks[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
  const size_t per_item = ((size_t)p->n_pix * p->N + (size_t)p->N * p->N) * sizeof(float2);
  const int total = n_batch * p->n_mod;
  float best = 1e30f;
  int bc = p->chunk, bk = p->ka, bp = p->passes;
  cudaEvent_t e0, e1;
  SPECULA_CK(cudaEventCreate(&e0));
  SPECULA_CK(cudaEventCreate(&e1));
  int status = SPECULA_OK;
  for (int passes = 2; passes <= 4; ++passes) {
    if (passes == 2 && !p->two_ok) continue;
    if (passes == 3 && p->pad != 2) continue;
    if (passes == 4 && !p->pair_ok) continue;
    const size_t item = passes != 3 ? (size_t)p->n_pix * p->N * sizeof(float2) : per_item;
    for (int c : kChunks) {
      if (passes == 4) {
        // whole batch elements: nc, 2 nc, 4 nc, ... slots
        if (c != 1 && (c & (c - 1))) continue;
        if (c > std::max(n_batch, 1) && c != 1) break;
        if ((size_t)c * p->nc * item > max_ws_bytes && c != 1) break;
      } else {
        if (c > std::max(total, 1) && c != 1) break;
        if ((size_t)c * item > max_ws_bytes && c != 1) break;
      }
      // ka sets the row pass's grid depth (slots per warp): values that fill
      // whole waves of CTAs can win (the ELT frame: ka 5, 300 CTAs on 304
      // slots), so the search goes to 8
      for (int ka = 1; ka <= (passes == 4 ? 1 : 8); ++ka) {
        if (ka > c) break;
        if ((status = pwfs_set_tiles(p, passes == 4 ? c * p->nc : c, ka, passes))) goto done;
        if ((status = pwfs_run(ctx, p, amp, phase, n_batch, det, st))) goto done;   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
          if ((status = pwfs_run(ctx, p, amp, phase, n_batch, det, st))) goto done;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { status = SPECULA_ECUDA; goto done; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bc = p->chunk; bk = ka; bp = passes; }
      }
    }
  }
  status = pwfs_set_tiles(p, bc, bk, bp);
  *best_chunk = bc;
  *best_ka = bk;
  *best_passes = bp;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

static int configure_for(PwfsPlan *p) {
  switch (p->N) {
    case 64: return configure<8, 8>(p);
    case 128: return configure<8, 16>(p);
    case 240: return configure<15, 16>(p);
    case 320: return configure<20, 16>(p);
    case 660: return configure<30, 22>(p);
    case 960: return configure<30, 32>(p);
    case 1600: return configure<32, 50>(p);
    default: return SPECULA_EUNSUPPORTED;
  }
}

PwfsPlan *pwfs_plan_find(specula_ctx *ctx, const specula_pupil_desc *pupil,
                         const specula_pwfs_desc *d) {
  for (auto &p : ctx->pwfs)
    if (p->n_pix == pupil->n_pix && p->pad == d->pad && p->n_mod == d->n_mod &&
        p->n_sub == d->n_sub && p->pup_dist == d->pup_dist_px && p->mod_amp == d->mod_amp)
      return p.get();
  return nullptr;
}

// exp(i * pi * num / den) with num reduced exactly modulo 2 den
static inline void exp_ipi(long long num, long long den, double *c, double *s) {
  long long r = num % (2 * den);
  if (r < 0) r += 2 * den;
  const double a = M_PI * (double)r / (double)den;
  *c = cos(a);
  *s = sin(a);
}

void pwfs_host_tables(int Np, int N, int N1, int N2, int n_mod, double mod_amp, int pup_dist,
                      PwfsTablesHost *t) {
  const int off = (N - Np) / 2;
  // modulation tilt x centred-DFT input phase, per axis, float64 -> float32
  std::vector<float2> gx((size_t)n_mod * Np), gy((size_t)n_mod * Np);
  for (int m = 0; m < n_mod; ++m) {
    const double th = 2.0 * M_PI * m / n_mod;
    const double ct = cos(th), sn = sin(th);
    for (int i = 0; i < Np; ++i) {
      const double x = (double)i - (Np - 1) / 2.0;
      double pc, ps;
      exp_ipi((long long)(N - 1) * (off + i), N, &pc, &ps);
      const double ax = 2.0 * M_PI * mod_amp * x * ct / Np;
      const double ay = 2.0 * M_PI * mod_amp * x * sn / Np;
      const double cx = cos(ax), sx = sin(ax), cy = cos(ay), sy = sin(ay);
      gx[(size_t)m * Np + i] = make_float2((float)(cx * pc - sx * ps), (float)(cx * ps + sx * pc));
      gy[(size_t)m * Np + i] = make_float2((float)(cy * pc - sy * ps), (float)(cy * ps + sy * pc));
    }
  }
  // pyramid mask per axis: exp(-2 pi i c |u| / N) / N, c = pup_dist / 2,
  // u = k - (N-1)/2: angle = -pi pup_dist |2k - N + 1| / (2N)
  std::vector<float2> mk(N);
  for (int k = 0; k < N; ++k) {
    long long a = 2LL * k - N + 1;
    if (a < 0) a = -a;
    double c, sn;
    exp_ipi(-(long long)pup_dist * a, 2LL * N, &c, &sn);
    mk[k] = make_float2((float)(c / N), (float)(sn / N));
  }
  // inter-step twiddles (cos, sin)(2 pi (a b mod N) / N)
  std::vector<float2> ta(N), tb(N);
  for (int a = 0; a < N2; ++a)
    for (int b = 0; b < N1; ++b) {
      double c, sn;
      exp_ipi(2LL * ((long long)a * b % N), N, &c, &sn);
      ta[a * N1 + b] = make_float2((float)c, (float)sn);
    }
  for (int a = 0; a < N1; ++a)
    for (int b = 0; b < N2; ++b) {
      double c, sn;
      exp_ipi(2LL * ((long long)a * b % N), N, &c, &sn);
      tb[a * N2 + b] = make_float2((float)c, (float)sn);
    }
  t->gx = std::move(gx);
  t->gy = std::move(gy);
  t->mask = std::move(mk);
  t->twA = std::move(ta);
  t->twB = std::move(tb);
}

int pwfs_plan_build(specula_ctx *ctx, const specula_pupil_desc *pupil,
                    const specula_pwfs_desc *d, PwfsPlan **out) {
  const int Np = pupil->n_pix, N = d->pad * Np;
  int N1, N2;
  if (!pwfs_split_for(N, &N1, &N2)) return SPECULA_EUNSUPPORTED;
  if (N2 % 4 && d->pad == 2) return SPECULA_EUNSUPPORTED;   // pruned pad-2 loads need N2 % 4 == 0
  std::unique_ptr<PwfsPlan> p(new PwfsPlan());
  p->n_pix = Np; p->pad = d->pad; p->n_mod = d->n_mod; p->n_sub = d->n_sub;
  p->pup_dist = d->pup_dist_px; p->mod_amp = d->mod_amp;
  p->N = N; p->N1 = N1; p->N2 = N2;
  // distinct cosines of the modulation angles 2 pi m / n_mod: m and n_mod - m
  p->nc = d->n_mod / 2 + 1;
  int s = configure_for(p.get());
  if (!s) s = pwfs_pair_configure(p.get());
  if (s) return s;
  PwfsTablesHost T;
  pwfs_host_tables(Np, N, N1, N2, d->n_mod, d->mod_amp, d->pup_dist_px, &T);
  if ((s = pwfs_pair_tables(p.get(), T))) return s;
  const std::vector<float2> &gx = T.gx, &gy = T.gy, &mk = T.mask, &ta = T.twA, &tb = T.twB;
  if ((s = p->gx.upload(gx.data(), gx.size() * sizeof(float2)))) return s;
  if ((s = p->gy.upload(gy.data(), gy.size() * sizeof(float2)))) return s;
  if ((s = p->mask.upload(mk.data(), mk.size() * sizeof(float2)))) return s;
  if ((s = p->twA.upload(ta.data(), ta.size() * sizeof(float2)))) return s;
  if ((s = p->twB.upload(tb.data(), tb.size() * sizeof(float2)))) return s;

  // chunk: keep the two intermediates of a chunk near 48 MB (L2-resident)
  const size_t per_item = ((size_t)Np * N + (size_t)N * N) * sizeof(float2);
  int chunk = (int)std::max<size_t>(1, (48u << 20) / per_item);
  chunk = std::min(chunk, 64);
  if ((s = pwfs_set_tiles(p.get(), chunk, 1, p->two_ok ? 2 : 3))) return s;
  *out = p.get();
  ctx->pwfs.push_back(std::move(p));
  return SPECULA_OK;
}

}  // namespace specula
