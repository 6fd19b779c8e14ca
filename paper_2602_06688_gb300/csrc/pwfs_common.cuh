// Two-level split N = N1 x N2 of the pyramid's FFT side, shared by the
// single-sensor passes and the multi-sensor persistent kernel, and the host
// tables both build (modulation tilt x centred-DFT input phase, pyramid mask,
// inter-step twiddles; App. A, Tab. 4 ModulatedPyramid).
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace specula {

template <int N1_, int N2_> struct Split {
  static constexpr int N1 = N1_, N2 = N2_, N = N1_ * N2_;
  static constexpr int MX = N1_ > N2_ ? N1_ : N2_;
  static constexpr int G = MX <= 8 ? 8 : (MX <= 16 ? 16 : 32);  // lanes per vector
  static constexpr int S1 = N1_ | 1;   // exchange stride, standard split (odd: no conflicts)
  static constexpr int S2 = N2_ | 1;   // exchange stride, swapped split
  static constexpr int XB = N2_ * S1;  // exchange buffer per vector (complex)
  // the pruned pad-2 loads take the pupil as rows N2/4 .. 3 N2/4 of the
  // strided input and need N2 % 4 == 0; other splits (660 = 30 x 22) run the
  // general-offset loads only (the plan refuses pad 2 for them)
  // Wide splits (N2 > 32, the two-pass kernels only): the N1-point stage
  // runs on lanes k2 = lane + 32 t, t < NT2, and writes a second buffer of
  // N1 S2 complex after the first, so that no lane overwrites exchange
  // values another lane has yet to read.
  static constexpr bool WIDE = N2_ > 32;
  static constexpr int NT2 = (N2_ + 31) / 32;
  static constexpr int XW = N2_ * S1 + N1_ * S2;   // both buffers of a wide split
  static_assert(N1_ <= 32 && N2_ <= 64, "N1 lanes per warp; N2 in at most two lane strides");
  static_assert(2 * XB >= N, "a vector's exchange buffer must hold N floats");
};

constexpr int round_cs(int base) { return base + ((2 - base % 16) + 16) % 16; }
constexpr int imax3(int a, int b, int c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }

// Host tables of one pyramid geometry, float64 rounded once to float32:
// gx, gy [n_mod][Np] (tilt of modulation point m times the centred-DFT input
// phase, per axis), mask [N] (per-axis mask factor over N), twA [N2][N1],
// twB [N1][N2] (inter-step twiddles).
struct PwfsTablesHost {
  std::vector<float2> gx, gy, mask, twA, twB;
};
void pwfs_host_tables(int Np, int N, int N1, int N2, int n_mod, double mod_amp, int pup_dist,
                      PwfsTablesHost *t);
bool pwfs_split_for(int N, int *N1, int *N2);

}  // namespace specula
