// In-register mixed-radix DFT codelets (FP32 complex) for sm_103a.
//
// The pyramid and Shack-Hartmann sensors are FFT pipelines (App. A, Tab. 4:
// ModulatedPyramid, SH; workload sizes in Sect. 6, Tab. 2).  Every transform
// here is composed of small DFTs that one thread evaluates on values held in
// its registers; all indices are compile-time constants after unrolling, so
// permutations are free register renames and twiddles are constant-bank
// operands.
//
// Twiddle values W_n^j = exp(-2 pi i j / n) come from a table computed on the
// host in float64 from cos/sin and rounded once to float32 (see
// upload_codelet_twiddles).  Multiples of a quarter turn are applied exactly.
//
// Each translation unit that includes this header gets its own constant
// table and must call upload_codelet_twiddles() once per device.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace specula {

// ---- small complex helpers ------------------------------------------------
// A complex value (re, im) sits in a register pair, so complex additions and
// real scalings are single packed float32 instructions (add/mul/fma .f32x2 on
// sm_100+), rounded as the two scalar operations would be.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
// b + s e and b - s e with s = -i (forward) or +i (inverse): mixed signs per
// component, so two scalar additions each
template <bool INV> __device__ __forceinline__ float2 cadd_mi(float2 b, float2 e) {
  return INV ? make_float2(b.x - e.y, b.y + e.x) : make_float2(b.x + e.y, b.y - e.x);
}
template <bool INV> __device__ __forceinline__ float2 csub_mi(float2 b, float2 e) {
  return INV ? make_float2(b.x + e.y, b.y - e.x) : make_float2(b.x - e.y, b.y + e.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---- codelet twiddle table -------------------------------------------------
// Sizes for which W_n^j is tabulated; offsets are compile-time.
constexpr int kCodeletSizes[] = {3, 5, 6, 8, 10, 12, 15, 16, 20, 24, 30, 32, 40, 48, 60, 64, 25};
constexpr int kNumCodeletSizes = sizeof(kCodeletSizes) / sizeof(int);
constexpr int codelet_offset(int n, int i = 0, int acc = 0) {
  return i >= kNumCodeletSizes ? -1
         : (kCodeletSizes[i] == n ? acc : codelet_offset(n, i + 1, acc + kCodeletSizes[i]));
}
constexpr int codelet_total(int i = 0) {
  return i >= kNumCodeletSizes ? 0 : kCodeletSizes[i] + codelet_total(i + 1);
}
constexpr int kCodeletTotal = codelet_total();

// (cos, sin) of 2 pi j / n, per TU
static __constant__ float2 c_codelet_tw[kCodeletTotal];
// the base butterflies' real constants as broadcast pairs (c, c):
// [0] cos 2pi/3, [1] sin 2pi/3, [2] cos 2pi/5, [3] cos 4pi/5, [4] sin 2pi/5,
// [5] sin 4pi/5, [6] -sin 2pi/5
constexpr int kBflyPairs = 7;
static __constant__ float2 c_bfly_pairs[kBflyPairs];
// odd primes with a direct butterfly; for prime P (H = (P - 1) / 2) the
// block at prime_off(P) holds cos 2pi m/P, then sin 2pi m/P, then
// -sin 2pi m/P, m = 1 .. H, as broadcast pairs
constexpr int kPrimes[] = {7, 11, 13, 17};
constexpr int kNumPrimes = sizeof(kPrimes) / sizeof(int);
constexpr int prime_off(int P, int i = 0, int acc = 0) {
  return i >= kNumPrimes ? -1
         : (kPrimes[i] == P ? acc : prime_off(P, i + 1, acc + 3 * (kPrimes[i] - 1) / 2));
}
constexpr int prime_total(int i = 0) {
  return i >= kNumPrimes ? 0 : 3 * (kPrimes[i] - 1) / 2 + prime_total(i + 1);
}
constexpr int kPrimePairs = prime_total();
static __constant__ float2 c_prime_pairs[kPrimePairs];

static inline cudaError_t upload_codelet_twiddles() {
  float2 h[kCodeletTotal];
  for (int s = 0; s < kNumCodeletSizes; ++s) {
    int n = kCodeletSizes[s];
    int off = codelet_offset(n);
    for (int j = 0; j < n; ++j) {
      double a = 2.0 * M_PI * (double)j / (double)n;
      h[off + j] = make_float2((float)cos(a), (float)sin(a));
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_codelet_tw, h, sizeof(h));
  if (e != cudaSuccess) return e;
  const float v[kBflyPairs] = {(float)cos(2.0 * M_PI / 3.0), (float)sin(2.0 * M_PI / 3.0),
                               (float)cos(2.0 * M_PI / 5.0), (float)cos(4.0 * M_PI / 5.0),
                               (float)sin(2.0 * M_PI / 5.0), (float)sin(4.0 * M_PI / 5.0),
                               -(float)sin(2.0 * M_PI / 5.0)};
  float2 hp[kBflyPairs];
  for (int i = 0; i < kBflyPairs; ++i) hp[i] = make_float2(v[i], v[i]);
  e = cudaMemcpyToSymbol(c_bfly_pairs, hp, sizeof(hp));
  if (e != cudaSuccess) return e;
  float2 pp[kPrimePairs];
  for (int i = 0; i < kNumPrimes; ++i) {
    const int P = kPrimes[i], H = (P - 1) / 2, o = prime_off(P);
    for (int m = 1; m <= H; ++m) {
      const float c = (float)cos(2.0 * M_PI * m / P), sn = (float)sin(2.0 * M_PI * m / P);
      pp[o + m - 1] = make_float2(c, c);
      pp[o + H + m - 1] = make_float2(sn, sn);
      pp[o + 2 * H + m - 1] = make_float2(-sn, -sn);
    }
  }
  return cudaMemcpyToSymbol(c_prime_pairs, pp, sizeof(pp));
}

// W_N^J for the forward (exp(-2 pi i J/N)) or inverse (exp(+...)) sign.
template <int N, bool INV>
__device__ __forceinline__ float2 apply_tw(float2 a, int j) {
  j = j % N;
  if (j == 0) return a;
  if (4 * j == N) return mul_mi<INV>(a);
  if (2 * j == N) return make_float2(-a.x, -a.y);
  if (4 * j == 3 * N) return mul_mi<!INV>(a);
  static_assert(codelet_offset(N) >= 0, "codelet size not tabulated");
  float2 w = c_codelet_tw[codelet_offset(N) + j];
  return INV ? cmul(a, w) : cmulc(a, w);
}

// ---- base butterflies --------------------------------------------------------
template <bool INV> __device__ __forceinline__ void bfly2(float2 &a, float2 &b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV> __device__ __forceinline__ void bfly3(float2 &x0, float2 &x1, float2 &x2) {
  // x0 + c (x1 + x2) +- s (x1 - x2) rotated, c = cos(2pi/3) = -1/2, s = sin(2pi/3)
  const float2 t1 = cadd(x1, x2);
  const float2 t2 = __ffma2_rn(c_bfly_pairs[0], t1, x0);
  const float2 t3 = __fmul2_rn(c_bfly_pairs[1], csub(x1, x2));
  x0 = cadd(x0, t1);
  x1 = cadd_mi<INV>(t2, t3);
  x2 = csub_mi<INV>(t2, t3);
}

template <bool INV> __device__ __forceinline__ void bfly4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  const float2 a = cadd(x0, x2), b = csub(x0, x2);
  const float2 c = cadd(x1, x3), e = csub(x1, x3);
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd_mi<INV>(b, e);
  x3 = csub_mi<INV>(b, e);
}

template <bool INV>
__device__ __forceinline__ void bfly5(float2 &x0, float2 &x1, float2 &x2, float2 &x3, float2 &x4) {
  // (cos, sin) of 2pi/5 and 4pi/5 as broadcast pairs
  const float2 c1 = c_bfly_pairs[2], c2 = c_bfly_pairs[3];
  const float2 s1 = c_bfly_pairs[4], s2 = c_bfly_pairs[5], ns1 = c_bfly_pairs[6];
  const float2 a1 = cadd(x1, x4), b1 = csub(x1, x4);
  const float2 a2 = cadd(x2, x3), b2 = csub(x2, x3);
  const float2 p1 = __ffma2_rn(c1, a1, __ffma2_rn(c2, a2, x0));
  const float2 p2 = __ffma2_rn(c2, a1, __ffma2_rn(c1, a2, x0));
  const float2 q1 = __ffma2_rn(s1, b1, __fmul2_rn(s2, b2));
  const float2 q2 = __ffma2_rn(s2, b1, __fmul2_rn(ns1, b2));
  x0 = cadd(x0, cadd(a1, a2));
  x1 = cadd_mi<INV>(p1, q1);
  x4 = csub_mi<INV>(p1, q1);
  x2 = cadd_mi<INV>(p2, q2);
  x3 = csub_mi<INV>(p2, q2);
}

// P-point DFT for an odd prime P from the symmetric pairs a_j = x_j +
// x_{P-j}, b_j = x_j - x_{P-j} (j = 1 .. H, H = (P - 1) / 2): X_k = x_0 +
// sum_j a_j cos(2 pi jk/P) -+ i sum_j b_j sin(2 pi jk/P), X_{P-k} the other
// sign, k = 1 .. H; jk mod P folded onto 1 .. H with the sine's sign.
template <int P, bool INV> __device__ __forceinline__ void bfly_prime(float2 (&x)[P]) {
  constexpr int H = (P - 1) / 2, O = prime_off(P);
  static_assert(O >= 0, "prime not tabulated");
  float2 a[H + 1], b[H + 1];
#pragma unroll
  for (int j = 1; j <= H; ++j) {
    a[j] = cadd(x[j], x[P - j]);
    b[j] = csub(x[j], x[P - j]);
  }
  float2 y[P];
  float2 sa = a[1];
#pragma unroll
  for (int j = 2; j <= H; ++j) sa = cadd(sa, a[j]);
  y[0] = cadd(x[0], sa);
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    float2 p = x[0], q = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      const int m = (j * k) % P;
      const int f = m <= H ? m : P - m;                      // cos(2 pi m/P) = cos(2 pi f/P)
      const int si = m <= H ? O + H + f - 1 : O + 2 * H + f - 1;   // +-sin(2 pi f/P)
      p = __ffma2_rn(c_prime_pairs[O + f - 1], a[j], p);
      q = j == 1 ? __fmul2_rn(c_prime_pairs[si], b[j]) : __ffma2_rn(c_prime_pairs[si], b[j], q);
    }
    y[k] = cadd_mi<INV>(p, q);
    y[P - k] = csub_mi<INV>(p, q);
  }
#pragma unroll
  for (int k = 0; k < P; ++k) x[k] = y[k];
}

// ---- generic in-register DFT: X[k] = sum_n x[n] W_N^{nk}, natural order ----
template <int N> struct first_factor {
  static constexpr int value = (N % 4 == 0 && N != 8) ? 4 : (N % 2 == 0 ? 2 : (N % 3 == 0 ? 3 : (N % 5 == 0 ? 5 : N)));
};

// Coprime split N = A B for the prime-factor (Good-Thomas) form: A is the
// power of 2 in N, else the power of 3, when that is a proper factor; 0 if
// N has no such split (prime powers).
constexpr int prime_power_part(int n, int p) { return n % p == 0 ? p * prime_power_part(n / p, p) : 1; }
constexpr int inverse_mod(int a, int m, int x = 1) {
  return x >= m ? 1 : ((a * x) % m == 1 ? x : inverse_mod(a, m, x + 1));
}
template <int N> struct pfa_factor {
  static constexpr int p2 = prime_power_part(N, 2), p3 = prime_power_part(N, 3);
  static constexpr int value = (p2 > 1 && p2 < N) ? p2 : ((p3 > 1 && p3 < N) ? p3 : 0);
};

template <int N, bool INV, int A = pfa_factor<N>::value> struct RegDFT {
  // Prime-factor form, no twiddles: with N = A B, gcd(A, B) = 1, the input
  // index n = (a B + b A) mod N and the output index
  // k = (ka B (B^-1 mod A) + kb A (A^-1 mod B)) mod N make W_N^{nk} factor
  // into W_A^{a ka} W_B^{b kb}: a B-point DFT along b for every a, then an
  // A-point DFT along a for every kb.
  static __device__ __forceinline__ void run(float2 (&x)[N]) {
    constexpr int B = N / A;
    constexpr int U = inverse_mod(B % A, A), V = inverse_mod(A % B, B);
    float2 y[A][B];
#pragma unroll
    for (int a = 0; a < A; ++a) {
#pragma unroll
      for (int b = 0; b < B; ++b) y[a][b] = x[(a * B + b * A) % N];
      RegDFT<B, INV>::run(y[a]);
    }
#pragma unroll
    for (int kb = 0; kb < B; ++kb) {
      float2 z[A];
#pragma unroll
      for (int a = 0; a < A; ++a) z[a] = y[a][kb];
      RegDFT<A, INV>::run(z);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) x[(ka * B * U + kb * A * V) % N] = z[ka];
    }
  }
};

template <int N, bool INV> struct RegDFT<N, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[N]) {
    constexpr int P = first_factor<N>::value;
    constexpr int Q = N / P;
    static_assert(P * Q == N && P > 1, "unsupported codelet size");
    // n = n1 + P n2, k = Q k1 + k2:
    //   Y[n1][k2] = W_N^{n1 k2} sum_{n2} x[n1 + P n2] W_Q^{n2 k2}
    //   X[Q k1 + k2] = sum_{n1} Y[n1][k2] W_P^{n1 k1}
    float2 y[P][Q];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) y[n1][n2] = x[n1 + P * n2];
      RegDFT<Q, INV>::run(y[n1]);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) y[n1][k2] = apply_tw<N, INV>(y[n1][k2], n1 * k2);
    }
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      float2 z[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) z[n1] = y[n1][k2];
      RegDFT<P, INV>::run(z);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) x[Q * k1 + k2] = z[k1];
    }
  }
};

template <bool INV> struct RegDFT<1, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};
template <bool INV> struct RegDFT<2, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[2]) { bfly2<INV>(x[0], x[1]); }
};
template <bool INV> struct RegDFT<3, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[3]) { bfly3<INV>(x[0], x[1], x[2]); }
};
template <bool INV> struct RegDFT<4, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[4]) { bfly4<INV>(x[0], x[1], x[2], x[3]); }
};
template <bool INV> struct RegDFT<7, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[7]) { bfly_prime<7, INV>(x); }
};
template <bool INV> struct RegDFT<11, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[11]) { bfly_prime<11, INV>(x); }
};
template <bool INV> struct RegDFT<13, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[13]) { bfly_prime<13, INV>(x); }
};
template <bool INV> struct RegDFT<17, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[17]) { bfly_prime<17, INV>(x); }
};
template <bool INV> struct RegDFT<5, INV, 0> {
  static __device__ __forceinline__ void run(float2 (&x)[5]) { bfly5<INV>(x[0], x[1], x[2], x[3], x[4]); }
};

}  // namespace specula
