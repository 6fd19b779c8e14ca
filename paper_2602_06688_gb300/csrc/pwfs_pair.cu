// Modulated pyramid image, separable two-pass form with packed-pair
// arithmetic (ModulatedPyramid + CCD binning, App. A, Tab. 4; the FFT
// workload of Sect. 6, Tab. 2).
//
// The same filter chain as the two-pass form in pwfs.cu, per modulation
// point m on the N x N padded grid (N = 2 n_pix):
//     I_m = |IDFT_y My DFT_y . IDFT_x Mx DFT_x (pad(E . tilt_m . pre))|^2 / n_mod,
// binned b x b, with the row filter shared by the points m and n_mod - m
// (same cos theta_m, hence the same x factor of the tilt).  What differs is
// the evaluation: every thread carries two transforms at once in packed
// float32 pairs (fft_pair.cuh), which halves the instructions per transform
// of these issue-bound kernels.
//   row filter (P1): a warp filters two pupil rows of one cosine slot;
//   column filter (P2): a warp filters one column for the two items of a
//     pair unit (the points m and n_mod - m of one slot, which share the
//     staged rows and differ only in the y factor of their tilt; the points
//     with no partner, m = 0 and m = n_mod / 2, are paired with each other,
//     and a last unpaired point with itself, writing one result).
// Both evaluate one N = N1 x N2 transform per warp as in pwfs.cu: lane n1
// holds the N2-point DFT along n2, the values cross lanes through shared
// memory, lane k2 holds the N1-point DFT along n1.  The forward transform's
// input is the pupil's half of the padded line, so the first stage is the
// padded-input DFT of fft_pair.cuh (two N2/2-point DFTs); its quarter-turn
// output phase is folded into the inter-step twiddle table twA2.
#include <math.h>

#include <algorithm>

#include "fft_pair.cuh"
#include "internal.h"
#include "pwfs_common.cuh"

namespace specula {

int pwfs_pair_init_device() {
  return upload_pair_twiddles() == cudaSuccess ? SPECULA_OK : SPECULA_ECUDA;
}

__device__ __forceinline__ void pair_cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void pair_cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int N1, int N2> struct PairCfg {
  static constexpr int N = N1 * N2;
  static constexpr int S1 = N1 | 1;   // exchange strides (odd: conflict-free 16-byte accesses)
  static constexpr int S2 = N2 | 1;
  static constexpr int XB = N2 * S1 > N1 * S2 ? N2 * S1 : N1 * S2;   // C2 per warp
  static_assert(N1 <= 32 && N2 <= 32 && N2 % 4 == 0, "one warp per transform, pruned input");
  static_assert(2 * XB >= N, "a warp's exchange buffer must hold its N intensity pairs");
};

// Both halves of the forward split: the N2-point padded-input DFT of lane
// n1's pupil values z (times twA2, which carries the quarter-turn phase),
// the exchange, the N1-point DFT, the mask, the inverse N1-point DFT, the
// exchange with twB2, and the inverse N2-point DFT: out[k1] is the filtered
// value at position N1 k1 + lane of the line.  xb: this warp's buffer.
template <int N1, int N2>
__device__ __forceinline__ void pair_line_filter(C2 (&z)[N2 / 2], C2 (&out)[N2], C2 *xb,
                                                 int lane, const float4 *__restrict__ twA2,
                                                 const float4 *__restrict__ twB2,
                                                 const float4 *__restrict__ mask2) {
  using P = PairCfg<N1, N2>;
  constexpr int S1 = P::S1, S2 = P::S2;
  {
    C2 X[N2];
    pair_dft_padded<N2>(z, X);
    if (lane < N1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = c2_mul(X[k2], __ldg(twA2 + k2 * N1 + lane));
    }
  }
  __syncwarp();
  C2 r2[N1];
  if (lane < N2) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xb[lane * S1 + n1];
  } else {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = C2{0ull, 0ull};
  }
  __syncwarp();
  PairDFT<N1, false>::run(r2);
  if (lane < N2) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) r2[k1] = c2_mul(r2[k1], __ldg(mask2 + N2 * k1 + lane));
  }
  PairDFT<N1, true>::run(r2);
  if (lane < N2) {
#pragma unroll
    for (int k = 0; k < N1; ++k) xb[k * S2 + lane] = c2_mul(r2[k], __ldg(twB2 + k * N2 + lane));
  }
  __syncwarp();
  if (lane < N1) {
#pragma unroll
    for (int n1 = 0; n1 < N2; ++n1) out[n1] = xb[lane * S2 + n1];
  } else {
#pragma unroll
    for (int n1 = 0; n1 < N2; ++n1) out[n1] = C2{0ull, 0ull};
  }
  __syncwarp();
  PairDFT<N2, true>::run(out);
}

// P1: row filter.  grid (ceil(n_pix / (2 VPC)), n_slots); block VPC warps;
// warp v of CTA x filters the rows j = 2 (x VPC + v) and j + 1 of slot it
// (batch element b = (slot0 + it) / nc, cosine slot c = s0 + (slot0 + it) % nc).
template <int N1, int N2>
__global__ void __launch_bounds__(128, 3) k_rowfilt_pair(
    const float2 *__restrict__ field, const float4 *__restrict__ gx2,
    const float4 *__restrict__ twA2, const float4 *__restrict__ twB2,
    const float4 *__restrict__ mask2, float2 *__restrict__ rows_out, int n_pix, int nc, int nbw,
    int slot0, int s0) {
  using P = PairCfg<N1, N2>;
  constexpr int N = P::N, QH = N2 / 2;
  extern __shared__ __align__(16) C2 smem_p1[];
  const int vec = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C2 *xb = smem_p1 + vec * P::XB;
  const int j = 2 * (blockIdx.x * (blockDim.x >> 5) + vec);
  const bool ok0 = j < n_pix, ok1 = j + 1 < n_pix;
  const int it = blockIdx.y;
  const int gi = slot0 + it;
  const int b = gi / nc, c = s0 + (gi - b * nc);
  C2 z[QH];
  if (ok0 && lane < N1) {
    const float2 *ea = field + ((size_t)(b % nbw) * n_pix + j) * n_pix + lane;
    const float2 *eb = ok1 ? ea + n_pix : ea;
    const float4 *g = gx2 + (size_t)c * n_pix + lane;
#pragma unroll
    for (int h = 0; h < QH; ++h) {
      const float2 a = __ldg(ea + N1 * h), bb = __ldg(eb + N1 * h);
      z[h] = c2_mul(C2{f2_pack(a.x, bb.x), f2_pack(a.y, bb.y)}, __ldg(g + N1 * h));
    }
  } else {
#pragma unroll
    for (int h = 0; h < QH; ++h) z[h] = C2{0ull, 0ull};
  }
  C2 out[N2];
  pair_line_filter<N1, N2>(z, out, xb, lane, twA2, twB2, mask2);
  if (ok0 && lane < N1) {
    float2 *da = rows_out + ((size_t)it * n_pix + j) * N + lane;
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1) {
      const float2 re = f2_unpack(out[k1].r), im = f2_unpack(out[k1].i);
      da[N1 * k1] = make_float2(re.x, im.x);
      if (ok1) da[N + N1 * k1] = make_float2(re.y, im.y);
    }
  }
}

// P2: column filter, |.|^2 / n_mod and b x b bins of a pair unit.
// grid (N / TC, n_units x batch elements in the chunk); block TC warps, one
// column each; TC a multiple of the bin side.  unit u = (slot a, point a,
// slot b, point b or -1): slots relative to s0; gyp[u][row] = the two
// points' y factors as (re_a, re_b, im_a, im_b).
template <int N1, int N2>
__global__ void __launch_bounds__(160, 2) k_colfilt_pair(
    const float2 *__restrict__ rows_in, const float4 *__restrict__ gyp,
    const int4 *__restrict__ units, int n_units, const float4 *__restrict__ twA2,
    const float4 *__restrict__ twB2, const float4 *__restrict__ mask2, float *__restrict__ part,
    int n_pix, int bsz, float scale, int n_mod, int nc, int nbw, int b0) {
  using P = PairCfg<N1, N2>;
  constexpr int N = P::N, QH = N2 / 2;
  extern __shared__ __align__(16) C2 smem_p2[];
  const int TC = blockDim.x >> 5;
  const int vec = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bl = blockIdx.y / n_units, u = blockIdx.y - bl * n_units;
  const int4 U = __ldg(units + u);
  const int b = b0 + bl;
  const int itA = bl * nc + U.x, itB = bl * nc + U.z;
  const bool same = itA == itB;
  const int col0 = blockIdx.x * TC;
  // Stage the rows of the unit's slot(s): a row-major window of W complex
  // from the even column col0e, 16-byte cp.async.cg copies (the row buffer
  // carries two complex of padding after its last row for the odd-TC spare
  // column).  Thread t copies 16-byte chunk t % nch of rows t / nch + k R.
  const int col0e = col0 & ~1, sh = col0 - col0e;
  const int W = (TC + 1) & ~1, nch = W >> 1;
  float2 *tA = reinterpret_cast<float2 *>(smem_p2);
  float2 *tB = same ? tA : tA + (size_t)n_pix * W;
  {
    const int R = blockDim.x / nch;
    const int t = threadIdx.x;
    if (t < R * nch) {
      const int q = t % nch, r0 = t / nch;
      const float2 *srcA = rows_in + (size_t)itA * n_pix * N + col0e + 2 * q;
      for (int r = r0; r < n_pix; r += R)
        pair_cp_async16(tA + r * W + 2 * q, srcA + (size_t)r * N);
      if (!same) {
        const float2 *srcB = rows_in + (size_t)itB * n_pix * N + col0e + 2 * q;
        for (int r = r0; r < n_pix; r += R)
          pair_cp_async16(tB + r * W + 2 * q, srcB + (size_t)r * N);
      }
    }
  }
  pair_cp_async_wait_all();
  __syncthreads();
  C2 z[QH];
  if (lane < N1) {
    const float4 *g = gyp + (size_t)u * n_pix + lane;   // pupil row lane + N1 h
    const float2 *wa = tA + sh + vec + lane * W;
    if (same) {
#pragma unroll
      for (int h = 0; h < QH; ++h) {
        const float2 x = wa[N1 * h * W];
        z[h] = c2_mul(C2{f2_pack(x.x, x.x), f2_pack(x.y, x.y)}, __ldg(g + N1 * h));
      }
    } else {
      const float2 *wb = tB + sh + vec + lane * W;
#pragma unroll
      for (int h = 0; h < QH; ++h) {
        const float2 xa = wa[N1 * h * W], xv = wb[N1 * h * W];
        z[h] = c2_mul(C2{f2_pack(xa.x, xv.x), f2_pack(xa.y, xv.y)}, __ldg(g + N1 * h));
      }
    }
  } else {
#pragma unroll
    for (int h = 0; h < QH; ++h) z[h] = C2{0ull, 0ull};
  }
  __syncthreads();   // the window becomes the warps' exchange buffers
  C2 *xb = smem_p2 + vec * P::XB;
  C2 out[N2];
  pair_line_filter<N1, N2>(z, out, xb, lane, twA2, twB2, mask2);
  // this column's intensity pairs, y = N1 k1 + lane
  f2x *colI = reinterpret_cast<f2x *>(xb);
  if (lane < N1) {
    const f2x s = f2_pack(scale, scale);
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1) colI[N1 * k1 + lane] = c2_norm(out[k1], s);
  }
  __syncthreads();
  const int nd = N / bsz, nbx = TC / bsz;
  const size_t plane = (size_t)nd * nd;
  float *dA = part + ((size_t)(b % nbw) * n_mod + U.y) * plane;
  float *dB = U.w >= 0 ? part + ((size_t)(b % nbw) * n_mod + U.w) * plane : nullptr;
  const f2x *s_I = reinterpret_cast<const f2x *>(smem_p2);
  for (int q = threadIdx.x; q < nd * nbx; q += blockDim.x) {
    const int yb = q / nbx, xq = q - yb * nbx;
    f2x v = 0ull;
    for (int cc = 0; cc < bsz; ++cc) {
      const f2x *colp = s_I + (size_t)(xq * bsz + cc) * (2 * P::XB) + yb * bsz;
      for (int rr = 0; rr < bsz; ++rr) v = f2_add(v, colp[rr]);
    }
    const float2 vv = f2_unpack(v);
    const size_t o = (size_t)yb * nd + col0 / bsz + xq;
    dA[o] = vv.x;
    if (dB) dB[o] = vv.y;
  }
}

// P2w: the column filter with two warps per column (one pair unit, one
// column), for N1 = 2 B1 with B1 odd (prime-factor split 2 x B1) and
// N2 = 2 H2.  Each warp holds about half of the pair's values at every
// stage, so the kernel runs with about half the registers of P2 and twice
// the warps per SM.  Warp h (0 or 1) of the pair:
//   stage 1 (lane n1 < N1): the outputs X'[2k' + h] of the padded-input
//     N2-point DFT, one H2-point DFT of z W_N2^{j h} (fft_pair.cuh), times
//     twA2, to row k2 of the pair's buffer;
//   stage 2 (lane k2 < N2): the B1-point DFT of the half a = h of the
//     prime-factor map n1 = (B1 a + 2 b) mod N1; the two halves cross
//     through the slots each warp has read (warp 0 keeps the outputs
//     kb < K0 = (B1 + 1) / 2, warp 1 the rest); the 2-point DFT, the mask
//     and the inverse 2-point DFT on the warp's kb (the forward output pair
//     of kb is the inverse's input pair of b' = V kb mod B1, V = 2^-1 mod
//     B1); the halves cross again (warp h keeps na = h) for the inverse
//     B1-point DFT, outputs n' = (B1 na + 2 V nb) mod N1, times twB2;
//   stage 4 (lane n' < N1): the inverse H2-point DFT of the inputs k2 = 2 j
//     + h (E for h = 0, O W_N2^-q for h = 1); the halves cross (warp 0
//     keeps q < H2 / 2) and x[q] = E + O', x[q + H2] = E - O';
//   then |x|^2 / n_mod into the pair's buffer and the CTA's bins.
// Named barrier 1 + pair (64 threads) orders the crossings of a pair.
// (constant ids, so the kernel reserves only the barriers it uses)
__device__ __forceinline__ void pair_bar(int id) {
  switch (id) {
    case 1: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 3: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    case 4: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    case 5: asm volatile("bar.sync 5, 64;" ::: "memory"); break;
    case 6: asm volatile("bar.sync 6, 64;" ::: "memory"); break;
    case 7: asm volatile("bar.sync 7, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 8, 64;" ::: "memory"); break;
  }
}

template <int N1, int N2, int H>
__device__ __forceinline__ void colpair2_body(C2 (&z)[N2 / 2], C2 *xb, f2x *colI, int lane,
                                              int bar, const float4 *__restrict__ twA2,
                                              const float4 *__restrict__ twB2,
                                              const float4 *__restrict__ mask2, float scale) {
  constexpr int B1 = N1 / 2, H2 = N2 / 2, S1 = N1 | 1, S2 = N2 | 1;
  constexpr int K0 = (B1 + 1) / 2;                 // kb < K0: warp 0's share
  constexpr int V = inverse_mod(2 % B1, B1);       // 2^-1 mod B1
  static_assert(N1 == 2 * B1 && B1 % 2 == 1 && H2 % 2 == 0, "split 2 x odd, even halves");
  // ---- stage 1: X'[2k' + H]
  if (lane < N1) {
    if (H == 1) {
#pragma unroll
      for (int j = 1; j < H2; ++j) z[j] = c2_tw<N2, false>(z[j], j);
    }
    PairDFT<H2, false>::run(z);
#pragma unroll
    for (int kk = 0; kk < H2; ++kk) {
      const int k2 = 2 * kk + H;
      xb[k2 * S1 + lane] = c2_mul(z[kk], __ldg(twA2 + k2 * N1 + lane));
    }
  }
  pair_bar(bar);
  // ---- stage 2: half a = H of the prime-factor map, lane k2
  C2 y[B1];
  C2 *row = xb + lane * S1;
  if (lane < N2) {
#pragma unroll
    for (int b = 0; b < B1; ++b) y[b] = row[(B1 * H + 2 * b) % N1];
    PairDFT<B1, false>::run(y);
    // cross: warp 0 hands over kb >= K0 (to even slots 0, 2, ...), warp 1
    // kb < K0 (to odd slots 1, 3, ...): the slots each warp has read
    if (H == 0) {
#pragma unroll
      for (int kb = K0; kb < B1; ++kb) row[2 * (kb - K0)] = y[kb];
    } else {
#pragma unroll
      for (int kb = 0; kb < K0; ++kb) row[2 * kb + 1] = y[kb];
    }
  }
  pair_bar(bar);
  constexpr int KLO = H == 0 ? 0 : K0, KHI = H == 0 ? K0 : B1, KN = KHI - KLO;
  C2 u0[KN], u1[KN];   // the warp's kb: halves a = 0 and a = 1
  if (lane < N2) {
#pragma unroll
    for (int i = 0; i < KN; ++i) {
      const int kb = KLO + i;
      if (H == 0) {
        u0[i] = y[kb];
        u1[i] = row[2 * kb + 1];
      } else {
        u0[i] = row[2 * (kb - K0)];
        u1[i] = y[kb];
      }
    }
#pragma unroll
    for (int i = 0; i < KN; ++i) {
      const int kb = KLO + i;
      const int k0 = (2 * V * kb) % N1, k1 = (B1 + 2 * V * kb) % N1;   // ka = 0, 1
      C2 x0 = c2_add(u0[i], u1[i]), x1 = c2_sub(u0[i], u1[i]);
      x0 = c2_mul(x0, __ldg(mask2 + N2 * k0 + lane));
      x1 = c2_mul(x1, __ldg(mask2 + N2 * k1 + lane));
      u0[i] = c2_add(x0, x1);   // na = 0 at b' = V kb mod B1
      u1[i] = c2_sub(x0, x1);   // na = 1
    }
    // cross again: warp h keeps na = h; slots 16.. of the row are unused by
    // the first crossing (it used slots 0 .. 2 K0 - 1)
    if (H == 0) {
#pragma unroll
      for (int i = 0; i < KN; ++i) row[2 * K0 + i] = u1[i];
    } else {
#pragma unroll
      for (int i = 0; i < KN; ++i) row[2 * K0 + K0 + i] = u0[i];
    }
  }
  pair_bar(bar);
  C2 w[B1];
  if (lane < N2) {
#pragma unroll
    for (int kb = 0; kb < B1; ++kb) {
      const int bp = (V * kb) % B1;
      C2 v;
      if (H == 0)
        v = kb < K0 ? u0[kb] : row[2 * K0 + K0 + (kb - K0)];
      else
        v = kb < K0 ? row[2 * K0 + kb] : u1[kb - K0];
      w[bp] = v;
    }
    PairDFT<B1, true>::run(w);
  }
  pair_bar(bar);   // every read of the rows is done before the column layout
  if (lane < N2) {
#pragma unroll
    for (int nb = 0; nb < B1; ++nb) {
      const int np = (B1 * H + 2 * V * nb) % N1;
      xb[np * S2 + lane] = c2_mul(w[nb], __ldg(twB2 + np * N2 + lane));
    }
  }
  pair_bar(bar);
  // ---- stage 4: inverse over k2 = 2 j + H, lane n'
  C2 e[H2];
  C2 *col = xb + lane * S2;
  if (lane < N1) {
#pragma unroll
    for (int j = 0; j < H2; ++j) e[j] = col[2 * j + H];
    PairDFT<H2, true>::run(e);
    if (H == 1) {
#pragma unroll
      for (int q = 1; q < H2; ++q) e[q] = c2_tw<N2, true>(e[q], q);
    }
    // cross: warp 0 hands over E[q], q >= H2/2 (even slots), warp 1 O'[q],
    // q < H2/2 (odd slots): the slots each warp has read
    if (H == 0) {
#pragma unroll
      for (int q = H2 / 2; q < H2; ++q) col[2 * q] = e[q];
    } else {
#pragma unroll
      for (int q = 0; q < H2 / 2; ++q) col[2 * q + 1] = e[q];
    }
  }
  pair_bar(bar);
  f2x iv[H2];
  if (lane < N1) {
    const f2x sc = f2_pack(scale, scale);
#pragma unroll
    for (int i = 0; i < H2 / 2; ++i) {
      const int q = H * (H2 / 2) + i;
      const C2 E = H == 0 ? e[q] : col[2 * q];
      const C2 O = H == 0 ? col[2 * q + 1] : e[q];
      iv[2 * i] = c2_norm(c2_add(E, O), sc);
      iv[2 * i + 1] = c2_norm(c2_sub(E, O), sc);
    }
  }
  pair_bar(bar);   // the crossing's reads are done before the intensities
  if (lane < N1) {
#pragma unroll
    for (int i = 0; i < H2 / 2; ++i) {
      const int q = H * (H2 / 2) + i;
      colI[N1 * q + lane] = iv[2 * i];
      colI[N1 * (q + H2) + lane] = iv[2 * i + 1];
    }
  }
}

template <int N1, int N2>
__global__ void __launch_bounds__(320, 2) k_colfilt_pair2(
    const float2 *__restrict__ rows_in, const float4 *__restrict__ gyp,
    const int4 *__restrict__ units, int n_units, const float4 *__restrict__ twA2,
    const float4 *__restrict__ twB2, const float4 *__restrict__ mask2, float *__restrict__ part,
    int n_pix, int bsz, float scale, int n_mod, int nc, int nbw, int b0) {
  using P = PairCfg<N1, N2>;
  constexpr int N = P::N, QH = N2 / 2;
  extern __shared__ __align__(16) C2 smem_p3[];
  const int TC = blockDim.x >> 6;                  // columns: two warps each
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vec = warp >> 1, h = warp & 1;
  const int bl = blockIdx.y / n_units, u = blockIdx.y - bl * n_units;
  const int4 U = __ldg(units + u);
  const int b = b0 + bl;
  const int itA = bl * nc + U.x, itB = bl * nc + U.z;
  const bool same = itA == itB;
  const int col0 = blockIdx.x * TC;
  const int col0e = col0 & ~1, sh = col0 - col0e;
  const int W = (TC + 1) & ~1, nch = W >> 1;
  float2 *tA = reinterpret_cast<float2 *>(smem_p3);
  float2 *tB = same ? tA : tA + (size_t)n_pix * W;
  {
    const int R = blockDim.x / nch;
    const int t = threadIdx.x;
    if (t < R * nch) {
      const int q = t % nch, r0 = t / nch;
      const float2 *srcA = rows_in + (size_t)itA * n_pix * N + col0e + 2 * q;
      for (int r = r0; r < n_pix; r += R)
        pair_cp_async16(tA + r * W + 2 * q, srcA + (size_t)r * N);
      if (!same) {
        const float2 *srcB = rows_in + (size_t)itB * n_pix * N + col0e + 2 * q;
        for (int r = r0; r < n_pix; r += R)
          pair_cp_async16(tB + r * W + 2 * q, srcB + (size_t)r * N);
      }
    }
  }
  pair_cp_async_wait_all();
  __syncthreads();
  C2 z[QH];
  if (lane < N1) {
    const float4 *g = gyp + (size_t)u * n_pix + lane;   // pupil row lane + N1 j
    const float2 *wa = tA + sh + vec + lane * W;
    const float2 *wb = tB + sh + vec + lane * W;
#pragma unroll
    for (int j = 0; j < QH; ++j) {
      const float2 xa = wa[N1 * j * W], xv = wb[N1 * j * W];
      z[j] = c2_mul(C2{f2_pack(xa.x, xv.x), f2_pack(xa.y, xv.y)}, __ldg(g + N1 * j));
    }
  }
  __syncthreads();   // the window becomes the pairs' buffers
  C2 *xb = smem_p3 + vec * P::XB;
  f2x *colI = reinterpret_cast<f2x *>(xb);
  if (h == 0)
    colpair2_body<N1, N2, 0>(z, xb, colI, lane, 1 + vec, twA2, twB2, mask2, scale);
  else
    colpair2_body<N1, N2, 1>(z, xb, colI, lane, 1 + vec, twA2, twB2, mask2, scale);
  __syncthreads();
  const int nd = N / bsz, nbx = TC / bsz;
  const size_t plane = (size_t)nd * nd;
  float *dA = part + ((size_t)(b % nbw) * n_mod + U.y) * plane;
  float *dB = U.w >= 0 ? part + ((size_t)(b % nbw) * n_mod + U.w) * plane : nullptr;
  const f2x *s_I = reinterpret_cast<const f2x *>(smem_p3);
  for (int q = threadIdx.x; q < nd * nbx; q += blockDim.x) {
    const int yb = q / nbx, xq = q - yb * nbx;
    f2x v = 0ull;
    for (int cc = 0; cc < bsz; ++cc) {
      const f2x *colp = s_I + (size_t)(xq * bsz + cc) * (2 * P::XB) + yb * bsz;
      for (int rr = 0; rr < bsz; ++rr) v = f2_add(v, colp[rr]);
    }
    const float2 vv = f2_unpack(v);
    const size_t o = (size_t)yb * nd + col0 / bsz + xq;
    dA[o] = vv.x;
    if (dB) dB[o] = vv.y;
  }
}

// --------------------------------------------------------------------------
// host side


static float4 bcast(float2 w) { return make_float4(w.x, w.x, w.y, w.y); }

constexpr int kPairRowWarps = 4;

template <int N1, int N2>
static int pair_configure_t(PwfsPlan *p) {
  using P = PairCfg<N1, N2>;
  const int bsz = p->n_pix / p->n_sub;
  p->pair_ok = false;
  if (p->pad != 2 || p->pup_dist != p->n_pix || p->fq != 1) return SPECULA_OK;   // pad-2 quadrants
  // column tile: TC = k bsz columns, the largest k dividing the detector
  // side with TC <= 5 warps (two CTAs per SM by shared memory)
  int k = 0;
  for (int d = 1; d <= p->pad * p->n_sub; ++d)
    if ((p->pad * p->n_sub) % d == 0 && d * bsz <= 5) k = d;
  if (k == 0) return SPECULA_OK;
  const int tc = k * bsz;
  if (P::N % tc) return SPECULA_OK;
  const size_t win = 2 * (size_t)p->n_pix * ((tc + 1) & ~1) * sizeof(float2);
  const size_t xch = (size_t)tc * P::XB * sizeof(C2);
  // two warps per column where the N1-point stage splits as 2 x odd
  constexpr bool two = N1 % 2 == 0 && (N1 / 2) % 2 == 1;
  p->pair_blockK = tc * 32 * (two ? 2 : 1);
  p->pair_smemK = std::max(win, xch);
  p->pair_blockR = kPairRowWarps * 32;
  p->pair_smemR = (size_t)kPairRowWarps * P::XB * sizeof(C2);
  if (p->pair_smemK > 227 * 1024 || p->pair_smemR > 227 * 1024) return SPECULA_OK;
  int s;
  if ((s = ensure_dynamic_smem((const void *)k_rowfilt_pair<N1, N2>, p->pair_smemR)) ||
      (s = ensure_dynamic_smem((const void *)k_colfilt_pair<N1, N2>, p->pair_smemK)))
    return s;
  if constexpr (two) {
    if ((s = ensure_dynamic_smem((const void *)k_colfilt_pair2<N1, N2>, p->pair_smemK))) return s;
  }
  p->pair_ok = true;
  return SPECULA_OK;
}

int pwfs_pair_configure(PwfsPlan *p) {
  switch (p->N) {
    case 320: return pair_configure_t<20, 16>(p);
    case 960: return pair_configure_t<30, 32>(p);
    default: p->pair_ok = false; return SPECULA_OK;
  }
}

// Tables shared by every slot range: the inter-step twiddles as broadcast
// pairs (twA2 with the padded-input DFT's phase (-i)^k2 folded in, exact
// quarter turns of the float32 table), the mask and the x factors of the tilt.
int pwfs_pair_tables(PwfsPlan *p, const PwfsTablesHost &T) {
  if (!p->pair_ok) return SPECULA_OK;
  const int N = p->N, N1 = p->N1, N2 = p->N2;
  std::vector<float4> ta((size_t)N), tb((size_t)N), mk((size_t)N), gx(T.gx.size());
  for (int k2 = 0; k2 < N2; ++k2)
    for (int n1 = 0; n1 < N1; ++n1) {
      const float2 w = T.twA[(size_t)k2 * N1 + n1];
      float2 f = make_float2(w.x, -w.y);   // exp(-2 pi i n1 k2 / N)
      for (int r = 0; r < (k2 & 3); ++r) f = make_float2(f.y, -f.x);   // times -i
      ta[(size_t)k2 * N1 + n1] = bcast(f);
    }
  for (size_t e = 0; e < (size_t)N; ++e) {
    tb[e] = bcast(T.twB[e]);
    mk[e] = bcast(T.mask[e]);
  }
  for (size_t e = 0; e < gx.size(); ++e) gx[e] = bcast(T.gx[e]);
  int s;
  if ((s = p->twA2.upload(ta.data(), ta.size() * sizeof(float4)))) return s;
  if ((s = p->twB2.upload(tb.data(), tb.size() * sizeof(float4)))) return s;
  if ((s = p->mask2.upload(mk.data(), mk.size() * sizeof(float4)))) return s;
  if ((s = p->gx2.upload(gx.data(), gx.size() * sizeof(float4)))) return s;
  p->gy_host = T.gy;
  p->pair_units_for = -1;
  return SPECULA_OK;
}

// Pair units of the imaged slots [s0, s0 + nc) of one batch element, and
// their y factors.
static int pair_units(PwfsPlan *p, int s0, int nc) {
  const int key = s0 * 65536 + nc;
  if (p->pair_units_for == key) return SPECULA_OK;
  std::vector<int4> units;
  std::vector<int> singles;   // (relative slot, point) of points with no partner
  for (int c = s0; c < s0 + nc; ++c) {
    const int m2 = p->n_mod - c;
    if (c == 0 || m2 == c)
      singles.push_back(c - s0);
    else
      units.push_back(make_int4(c - s0, c, c - s0, m2));
  }
  for (size_t i = 0; i + 1 < singles.size(); i += 2) {
    const int ra = singles[i], rb = singles[i + 1];
    units.push_back(make_int4(ra, ra + s0, rb, rb + s0));
  }
  if (singles.size() % 2) {
    const int r = singles.back();
    units.push_back(make_int4(r, r + s0, r, -1));
  }
  const int Np = p->n_pix;
  std::vector<float4> gyp(units.size() * (size_t)Np);
  for (size_t u = 0; u < units.size(); ++u) {
    const int ma = units[u].y, mb = units[u].w >= 0 ? units[u].w : units[u].y;
    for (int i = 0; i < Np; ++i) {
      const float2 a = p->gy_host[(size_t)ma * Np + i], bq = p->gy_host[(size_t)mb * Np + i];
      gyp[u * Np + i] = make_float4(a.x, bq.x, a.y, bq.y);
    }
  }
  int s;
  if ((s = p->pair_units.upload(units.data(), units.size() * sizeof(int4)))) return s;
  if ((s = p->gyp.upload(gyp.data(), gyp.size() * sizeof(float4)))) return s;
  p->n_pair_units = (int)units.size();
  p->pair_units_for = key;
  return SPECULA_OK;
}

int pwfs_field_launch(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                      int fb, int nb, cudaStream_t st);

template <int N1, int N2>
static int pair_run_t(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                      int n_batch, float *det, cudaStream_t st) {
  using P = PairCfg<N1, N2>;
  const int Np = p->n_pix;
  const int bsz = Np / p->n_sub;
  const int nd = P::N / bsz;
  const int s0 = p->slot_lo;
  const int nc = (p->slot_hi < 0 ? p->nc : p->slot_hi) - s0;
  int s = pair_units(p, s0, nc);
  if (s) return s;
  // whole batch elements per chunk
  const int per = std::max(1, p->chunk / nc);
  constexpr bool two = N1 % 2 == 0 && (N1 / 2) % 2 == 1;
  const int tc = p->pair_blockK / (two ? 64 : 32);
  const int vpc = p->pair_blockR / 32;
  const float scale = 1.0f / (float)p->n_mod;
  for (int b0 = 0; b0 < n_batch; b0 += per) {
    const int nb = std::min(per, n_batch - b0);
    if ((s = pwfs_field_launch(ctx, p, amp, phase, b0, nb, st))) return s;
    dim3 gR((Np + 2 * vpc - 1) / (2 * vpc), nb * nc);
    SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_ROWFILT, st,
                   k_rowfilt_pair<N1, N2><<<gR, p->pair_blockR, p->pair_smemR, st>>>(
                       p->field.as<float2>(), p->gx2.as<float4>(), p->twA2.as<float4>(),
                       p->twB2.as<float4>(), p->mask2.as<float4>(), p->rows.as<float2>(), Np, nc,
                       p->nbw, b0 * nc, s0));
    dim3 gK(P::N / tc, nb * p->n_pair_units);
    if constexpr (two) {
      SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_COLFILT, st,
                     k_colfilt_pair2<N1, N2><<<gK, p->pair_blockK, p->pair_smemK, st>>>(
                         p->rows.as<float2>(), p->gyp.as<float4>(), p->pair_units.as<int4>(),
                         p->n_pair_units, p->twA2.as<float4>(), p->twB2.as<float4>(),
                         p->mask2.as<float4>(), p->part.as<float>(), Np, bsz, scale, p->n_mod,
                         nc, p->nbw, b0));
    } else {
      SPECULA_LAUNCH(ctx, SPECULA_K_PWFS_COLFILT, st,
                     k_colfilt_pair<N1, N2><<<gK, p->pair_blockK, p->pair_smemK, st>>>(
                         p->rows.as<float2>(), p->gyp.as<float4>(), p->pair_units.as<int4>(),
                         p->n_pair_units, p->twA2.as<float4>(), p->twB2.as<float4>(),
                         p->mask2.as<float4>(), p->part.as<float>(), Np, bsz, scale, p->n_mod,
                         nc, p->nbw, b0));
    }
    if ((s = pwfs_bin_reduce_range(ctx, p, det, nd * nd, b0, nb, st))) return s;
  }
  return SPECULA_OK;
}

int pwfs_pair_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                  int n_batch, float *det, cudaStream_t st) {
  if (!p->pair_ok) return SPECULA_EUNSUPPORTED;
  switch (p->N) {
    case 320: return pair_run_t<20, 16>(ctx, p, amp, phase, n_batch, det, st);
    case 960: return pair_run_t<30, 32>(ctx, p, amp, phase, n_batch, det, st);
    default: return SPECULA_EUNSUPPORTED;
  }
}

}  // namespace specula
