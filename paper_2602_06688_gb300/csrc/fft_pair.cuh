// Packed-pair DFT codelets: two independent complex transforms per thread.
//
// The pyramid's FFT stages (App. A, Tab. 4 ModulatedPyramid; FFT workloads
// of Sect. 6, Tab. 2) are issue-bound on sm_103a when each thread evaluates
// one transform with scalar float32 instructions.  Blackwell's packed
// float32 instructions (add/sub/mul/fma .f32x2) do two float32 operations
// per lane and issue slot.  Holding two transforms "a" and "b" in split
// form, C2 = { re = (re_a, re_b), im = (im_a, im_b) }, makes every complex
// operation of a butterfly two packed instructions that serve both
// transforms, so the instruction count per transform halves while the
// arithmetic (and its rounding) stays that of the scalar codelets.
//
// Twiddle and mask multipliers that both transforms share are stored as
// float4 (re, re, im, im): one 16-byte load gives both broadcast pairs.
//
// The ops without a rounding suffix may be contracted into fused
// multiply-adds by ptxas, as scalar float32 code is under --fmad=true.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "fft_regs.cuh"

namespace specula {

typedef unsigned long long f2x;   // (lane 0, lane 1) float32 pair

__device__ __forceinline__ f2x f2_pack(float a, float b) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float2 f2_unpack(f2x v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x d;
  asm("add.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
  f2x d;
  asm("sub.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x d;
  asm("mul.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {   // a b + c
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct C2 {
  f2x r, i;
};

__device__ __forceinline__ C2 c2_add(C2 a, C2 b) { return {f2_add(a.r, b.r), f2_add(a.i, b.i)}; }
__device__ __forceinline__ C2 c2_sub(C2 a, C2 b) { return {f2_sub(a.r, b.r), f2_sub(a.i, b.i)}; }
// b + s e and b - s e with s = -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ C2 c2_addmi(C2 b, C2 e) {
  return INV ? C2{f2_sub(b.r, e.i), f2_add(b.i, e.r)} : C2{f2_add(b.r, e.i), f2_sub(b.i, e.r)};
}
template <bool INV> __device__ __forceinline__ C2 c2_submi(C2 b, C2 e) {
  return INV ? C2{f2_add(b.r, e.i), f2_sub(b.i, e.r)} : C2{f2_sub(b.r, e.i), f2_add(b.i, e.r)};
}
// x times the shared multiplier w = (wr, wi), given as the pairs (wr, wr), (wi, wi)
__device__ __forceinline__ C2 c2_mul(C2 x, f2x wr, f2x wi) {
  return {f2_sub(f2_mul(x.r, wr), f2_mul(x.i, wi)), f2_fma(x.r, wi, f2_mul(x.i, wr))};
}
__device__ __forceinline__ C2 c2_mul(C2 x, float4 w) {   // w = (re, re, im, im)
  return c2_mul(x, f2_pack(w.x, w.y), f2_pack(w.z, w.w));
}
// x times conj(w)
__device__ __forceinline__ C2 c2_mulc(C2 x, f2x wr, f2x wi) {
  return {f2_fma(x.r, wr, f2_mul(x.i, wi)), f2_sub(f2_mul(x.i, wr), f2_mul(x.r, wi))};
}
// |x|^2 of both transforms, times s
__device__ __forceinline__ f2x c2_norm(C2 x, f2x s) {
  return f2_mul(f2_fma(x.r, x.r, f2_mul(x.i, x.i)), s);
}

// ---- codelet twiddles as broadcast pairs --------------------------------------
// (cos, cos, sin, sin)(2 pi j / n) for the sizes of kCodeletSizes, per TU.
static __constant__ float4 c_pair_tw[kCodeletTotal];

static inline cudaError_t upload_pair_twiddles() {
  float4 h[kCodeletTotal];
  for (int s = 0; s < kNumCodeletSizes; ++s) {
    const int n = kCodeletSizes[s];
    const int off = codelet_offset(n);
    for (int j = 0; j < n; ++j) {
      const double a = 2.0 * M_PI * (double)j / (double)n;
      const float c = (float)cos(a), sn = (float)sin(a);
      h[off + j] = make_float4(c, c, sn, sn);
    }
  }
  return cudaMemcpyToSymbol(c_pair_tw, h, sizeof(h));
}

template <int N> __device__ __forceinline__ float4 pair_tw(int j) {
  static_assert(codelet_offset(N) >= 0, "codelet size not tabulated");
  return c_pair_tw[codelet_offset(N) + j];
}

// W_N^J (exp(-2 pi i J / N) forward, exp(+...) inverse) applied to x
template <int N, bool INV> __device__ __forceinline__ C2 c2_tw(C2 x, int j) {
  j = j % N;
  if (j == 0) return x;
  if (4 * j == N) return INV ? C2{f2_sub(0ull, x.i), x.r} : C2{x.i, f2_sub(0ull, x.r)};
  if (2 * j == N) return C2{f2_sub(0ull, x.r), f2_sub(0ull, x.i)};
  if (4 * j == 3 * N) return INV ? C2{x.i, f2_sub(0ull, x.r)} : C2{f2_sub(0ull, x.i), x.r};
  const float4 w = pair_tw<N>(j);
  const f2x c = f2_pack(w.x, w.y), s = f2_pack(w.z, w.w);
  return INV ? c2_mul(x, c, s) : c2_mulc(x, c, s);
}

// ---- base butterflies ----------------------------------------------------------
template <bool INV> __device__ __forceinline__ void c2_bfly2(C2 &a, C2 &b) {
  const C2 t = a;
  a = c2_add(t, b);
  b = c2_sub(t, b);
}

template <bool INV> __device__ __forceinline__ void c2_bfly3(C2 &x0, C2 &x1, C2 &x2) {
  const float4 w = pair_tw<3>(1);   // cos 2pi/3 = -1/2, sin 2pi/3
  const f2x wc = f2_pack(w.x, w.y), ws = f2_pack(w.z, w.w);
  const C2 t1 = c2_add(x1, x2);
  const C2 t2 = {f2_fma(wc, t1.r, x0.r), f2_fma(wc, t1.i, x0.i)};
  const C2 d = c2_sub(x1, x2);
  const C2 t3 = {f2_mul(ws, d.r), f2_mul(ws, d.i)};
  x0 = c2_add(x0, t1);
  x1 = c2_addmi<INV>(t2, t3);
  x2 = c2_submi<INV>(t2, t3);
}

template <bool INV> __device__ __forceinline__ void c2_bfly4(C2 &x0, C2 &x1, C2 &x2, C2 &x3) {
  const C2 a = c2_add(x0, x2), b = c2_sub(x0, x2);
  const C2 c = c2_add(x1, x3), e = c2_sub(x1, x3);
  x0 = c2_add(a, c);
  x2 = c2_sub(a, c);
  x1 = c2_addmi<INV>(b, e);
  x3 = c2_submi<INV>(b, e);
}

template <bool INV>
__device__ __forceinline__ void c2_bfly5(C2 &x0, C2 &x1, C2 &x2, C2 &x3, C2 &x4) {
  const float4 w1 = pair_tw<5>(1), w2 = pair_tw<5>(2);
  const f2x c1 = f2_pack(w1.x, w1.y), s1 = f2_pack(w1.z, w1.w);
  const f2x c2 = f2_pack(w2.x, w2.y), s2 = f2_pack(w2.z, w2.w);
  const C2 a1 = c2_add(x1, x4), b1 = c2_sub(x1, x4);
  const C2 a2 = c2_add(x2, x3), b2 = c2_sub(x2, x3);
  const C2 p1 = {f2_fma(c1, a1.r, f2_fma(c2, a2.r, x0.r)), f2_fma(c1, a1.i, f2_fma(c2, a2.i, x0.i))};
  const C2 p2 = {f2_fma(c2, a1.r, f2_fma(c1, a2.r, x0.r)), f2_fma(c2, a1.i, f2_fma(c1, a2.i, x0.i))};
  const C2 q1 = {f2_fma(s1, b1.r, f2_mul(s2, b2.r)), f2_fma(s1, b1.i, f2_mul(s2, b2.i))};
  const C2 q2 = {f2_sub(f2_mul(s2, b1.r), f2_mul(s1, b2.r)),
                 f2_sub(f2_mul(s2, b1.i), f2_mul(s1, b2.i))};
  x0 = c2_add(x0, c2_add(a1, a2));
  x1 = c2_addmi<INV>(p1, q1);
  x4 = c2_submi<INV>(p1, q1);
  x2 = c2_addmi<INV>(p2, q2);
  x3 = c2_submi<INV>(p2, q2);
}

// ---- in-register DFT of both transforms: X[k] = sum_n x[n] W_N^{nk} ------------
template <int N, bool INV, int A = pfa_factor<N>::value> struct PairDFT {
  // Prime-factor (Good-Thomas) form, as RegDFT: no inner twiddles.
  static __device__ __forceinline__ void run(C2 (&x)[N]) {
    constexpr int B = N / A;
    constexpr int U = inverse_mod(B % A, A), V = inverse_mod(A % B, B);
    C2 y[A][B];
#pragma unroll
    for (int a = 0; a < A; ++a) {
#pragma unroll
      for (int b = 0; b < B; ++b) y[a][b] = x[(a * B + b * A) % N];
      PairDFT<B, INV>::run(y[a]);
    }
#pragma unroll
    for (int kb = 0; kb < B; ++kb) {
      C2 z[A];
#pragma unroll
      for (int a = 0; a < A; ++a) z[a] = y[a][kb];
      PairDFT<A, INV>::run(z);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) x[(ka * B * U + kb * A * V) % N] = z[ka];
    }
  }
};

template <int N, bool INV> struct PairDFT<N, INV, 0> {
  // Cooley-Tukey N = P Q: n = n1 + P n2, k = Q k1 + k2.
  static __device__ __forceinline__ void run(C2 (&x)[N]) {
    constexpr int P = first_factor<N>::value;
    constexpr int Q = N / P;
    static_assert(P * Q == N && P > 1, "unsupported codelet size");
    C2 y[P][Q];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) y[n1][n2] = x[n1 + P * n2];
      PairDFT<Q, INV>::run(y[n1]);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) y[n1][k2] = c2_tw<N, INV>(y[n1][k2], n1 * k2);
    }
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      C2 z[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) z[n1] = y[n1][k2];
      PairDFT<P, INV>::run(z);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) x[Q * k1 + k2] = z[k1];
    }
  }
};

template <bool INV> struct PairDFT<1, INV, 0> {
  static __device__ __forceinline__ void run(C2 (&)[1]) {}
};
template <bool INV> struct PairDFT<2, INV, 0> {
  static __device__ __forceinline__ void run(C2 (&x)[2]) { c2_bfly2<INV>(x[0], x[1]); }
};
template <bool INV> struct PairDFT<3, INV, 0> {
  static __device__ __forceinline__ void run(C2 (&x)[3]) { c2_bfly3<INV>(x[0], x[1], x[2]); }
};
template <bool INV> struct PairDFT<4, INV, 0> {
  static __device__ __forceinline__ void run(C2 (&x)[4]) {
    c2_bfly4<INV>(x[0], x[1], x[2], x[3]);
  }
};
template <bool INV> struct PairDFT<5, INV, 0> {
  static __device__ __forceinline__ void run(C2 (&x)[5]) {
    c2_bfly5<INV>(x[0], x[1], x[2], x[3], x[4]);
  }
};

// ---- forward DFT of a zero-padded input ----------------------------------------
// x[n] is non-zero only for N/4 <= n < 3N/4 (a 2x padded pupil).  With
// h = n - N/4,  X[k] = W_N^{(N/4) k} X'[k] and
//     X'[2k' + e] = sum_{h < N/2} (x[N/4 + h] W_N^{h e}) W_{N/2}^{h k'}:
// two N/2-point DFTs, of the input and of the input times W_N^h.  This
// returns X' (in natural order); the caller folds the quarter-turn phase
// W_N^{(N/4) k} = (-i)^k into its next twiddle table.  In: z[h] = x[N/4 + h].
template <int N> __device__ __forceinline__ void pair_dft_padded(C2 (&z)[N / 2], C2 (&X)[N]) {
  constexpr int H = N / 2;
  C2 o[H];
  o[0] = z[0];
#pragma unroll
  for (int h = 1; h < H; ++h) o[h] = c2_tw<N, false>(z[h], h);
  PairDFT<H, false>::run(z);
  PairDFT<H, false>::run(o);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    X[2 * k] = z[k];
    X[2 * k + 1] = o[k];
  }
}

}  // namespace specula
