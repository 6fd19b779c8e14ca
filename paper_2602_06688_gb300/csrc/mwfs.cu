// A multi-sensor frame in one persistent launch: every wavefront sensor of a
// system (Shack-Hartmann and modulated pyramids of different sizes, each with
// its own guide star), their slopes and the reconstructor product, as the
// paper's multi-sensor simulations chain them (Sect. 6, Tab. 2; App. A,
// Tab. 4: AtmoPropagation per source, SH / ModulatedPyramid, ShSlopec /
// PyrSlopec, Modalrec on the concatenated slopes).
//
// The frame is a fixed list of tasks, built once on the host in an order in
// which every task comes after the tasks it depends on.  Each CTA takes the
// next task from a global ticket counter, waits (bounded) until the counter
// of its dependency reaches the required value, runs the task and bumps the
// counter of its own kind.  A CTA only ever waits for tasks with smaller
// tickets, which CTAs already running hold and which never wait for later
// ones, so the queue always drains.  Task kinds:
//
//   COORDS  (sensor, entries)    float64 extraction coordinates (the same
//                                operations, in the same order, as
//                                specula_atmo_extract)
//   FIELD   (pyramid, rows)      phase of the rows by bilinear extraction,
//                                E = amp exp(i phase)
//   SH      (sensor, subaps)     per valid subaperture: phase of its pixels,
//                                E . pre-phase, 2D DFT in registers, |.|^2,
//                                centre of gravity -> slopes (no spot written)
//   ROWS / COLS / RINV           the three FFT passes of the pyramid, as the
//                                single-sensor kernels compute them
//   BIN     (pyramid, pixels)    detector = sum over modulation points, in
//                                order
//   SLOPES  (pyramid)            quadrant slopes, global-mean normalisation
//   MVM     (sensor, modes)      modes_part[sensor] = R[:, sensor's slopes] s
//   FINAL   (modes)              modes = sum over sensors of modes_part, in
//                                sensor order
//
// Interleaving the HBM-bound MVM tasks of finished sensors with the ALU-bound
// FFT tasks of the others keeps both the memory system and the FP32 pipes
// busy in the same launch.  No float atomics: every sum runs in a fixed
// order, so frames are bit-reproducible for a given grid.  The last CTA to
// leave resets the counters for the next launch; a wait that exceeds the
// time limit records SPECULA_ETIMEOUT in the context status word and makes
// every CTA leave.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "fft_regs.cuh"
#include "internal.h"
#include "pwfs_common.cuh"

namespace specula {

int mwfs_init_device() {
  return upload_codelet_twiddles() == cudaSuccess ? SPECULA_OK : SPECULA_ECUDA;
}

constexpr int kMwThreads = 256;
constexpr int kMwWarps = kMwThreads / 32;
constexpr int kMwMaxSensors = 16;
constexpr int kMwMaxLayers = 64;
constexpr int kMwShSubPerTask = 16;
constexpr int kMwCoordsPerTask = kMwThreads;
constexpr int kMwBinPerTask = 1024;
constexpr int kMwMvmRows = 32;
constexpr int kMwFinalRows = 1024;
constexpr unsigned long long kMwWaitNs = 2000000000ull;      // default wait limit
constexpr long long kMwWaitMaxNs = 10000000000ll;            // largest settable limit

enum : int {
  MT_COORDS = 0, MT_FIELD, MT_SH, MT_ROWS, MT_COLS, MT_RINV, MT_BIN, MT_SLOPES, MT_MVM, MT_FINAL
};

struct MwTask {
  int type, sensor, a, b;
  int wait_ctr, wait_val, done_ctr, pad;
};

struct MwLayer {
  const float *scr;
  int side;
  double pitch, h, vx, vy;
};

struct MwSensor {
  int kind, n_pix;
  double pitch, theta_x, theta_y, H;
  float scale;                 // 500 / lambda
  const float *amp;            // [n_pix][n_pix]
  float *phase;                // [n_pix][n_pix]
  int *tab_i;                  // [n_layers][2][n_pix]
  float *tab_f;
  int n_sub, n_valid, slope_off;
  const int32_t *valid;
  const float2 *pre;           // SH: [NF] centred-DFT input phase
  unsigned long long win_ok;   // SH: bit l set if a task's span on layer l < side - 2
  int n_mod, nd, bsz, spt;     // pyramid
  const float2 *gx, *gy, *mask, *twA, *twB;
  float2 *field, *rows, *cols;
  float *part, *det;
};

struct MwParams {
  MwSensor S[kMwMaxSensors];
  MwLayer L[kMwMaxLayers];
  int n_sensors, n_layers, n_tasks, n_ctr;
  const MwTask *tasks;
  int *ctr;                    // [0] ticket, [1] CTAs done, [2] abort, [3..] dependencies
  double t_host;
  const double *t_dev;
  int flat;                    // 1: flat wavefront (reference slopes)
  const float *R;
  int n_modes, n_slopes, r_vec4;
  const float *ref;
  float *slopes, *modes, *mpart;
  int32_t *status;
  int32_t *nf_status;          // non-finite guard: status word, or null when off
  unsigned long long wait_ns;  // limit of one dependency wait
  int stall_task;              // fault injection: this task waits for a count never reached
};

// ---- synchronisation ---------------------------------------------------------
__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu(int *p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 only: wait until *c >= need.  0 if the frame was aborted.
__device__ int mw_wait(const int *c, int need, int *abortf, int32_t *status,
                       unsigned long long limit_ns) {
  if (ld_acquire_gpu(c) >= need) return 1;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(128);
    if (ld_acquire_gpu(c) >= need) return 1;
    if (ld_relaxed_gpu(abortf)) return 0;
    if (global_ns() - t0 > limit_ns) {
      atomicExch(status, SPECULA_ETIMEOUT);
      atomicExch(abortf, 1);
      return 0;
    }
  }
}

// Non-finite guard on a slope pair: a status write only when one is NaN/Inf.
__device__ __forceinline__ void mw_guard(float a, float b, int32_t *nf_status) {
  if (nf_status && !(isfinite(a) && isfinite(b))) atomicExch(nf_status, SPECULA_ENONFINITE);
}

__device__ __forceinline__ float mw_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float4 mw_ld_stream(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// ---- extraction ------------------------------------------------------------------
// Table entries [e0, e1) of [layer][axis][pixel] (same arithmetic as
// k_atmo_coords).  float64 throughput is low on this part, so the tasks are
// small (one entry per thread) and spread over the whole GPU.  Written
// in-kernel, so the readers use L2 loads (__ldcg).
__device__ void mw_coords(const MwParams &P, const MwSensor &S, int e0, int e1) {
  const int n = S.n_pix;
  const double t = P.t_dev ? *P.t_dev : P.t_host;
  for (int e = e0 + threadIdx.x; e < e1; e += kMwThreads) {
    const int l = e / (2 * n), r = e % (2 * n);
    const int axis = r / n, idx = r % n;
    const MwLayer &Ly = P.L[l];
    const double s = __dsub_rn(1.0, __ddiv_rn(Ly.h, S.H));
    const double theta = axis ? S.theta_y : S.theta_x;
    const double v = axis ? Ly.vy : Ly.vx;
    const int side = Ly.side;
    const double x = __dmul_rn(__dsub_rn((double)idx, (double)(n - 1) / 2.0), S.pitch);
    const double off = __dsub_rn(__dmul_rn(Ly.h, theta), __dmul_rn(v, t));
    const double u =
        __dadd_rn(__ddiv_rn(__dadd_rn(__dmul_rn(x, s), off), Ly.pitch), (double)side / 2.0);
    const double u0 = floor(u);
    const double f = __dsub_rn(u, u0);
    long long k = (long long)u0 % side;
    if (k < 0) k += side;
    const size_t o = ((size_t)l * 2 + axis) * n + idx;
    S.tab_i[o] = (int)k;
    S.tab_f[o] = (float)f;
  }
}

// Phase of a block of pupil pixels: bilinear periodic samples summed over the
// layers in order, times 500 / lambda (the arithmetic of k_atmo_extract).
// The block's pixels use ncs distinct columns and nrs distinct rows (their
// "slots"); pixel q < npx (thread q % 256, register q / 256) reads column
// slot cs and row slot rs given by pix(q).  For each chunk of kMwLayerChunk
// layers the CTA first stages the table entries of its slots in shared
// memory (one round of independent L2 loads), then every thread issues the
// screen gathers of all its pixels together.
constexpr int kMwLayerChunk = 8;

//
// With WIN > 0 the caller guarantees that its column slots xf..xl and row
// slots yf..yl are the extreme ones (the sampling coordinate grows with the
// pupil coordinate when the layer is below the guide star): the screen
// window they span, if it holds at most WIN samples, is staged in shared
// memory with coalesced loads and the interpolation reads it there — the
// same samples, so the same result as the direct gathers.
template <int PPT, int WIN, class ColF, class RowF, class PixF>
__device__ __forceinline__ void mw_extract_block(const MwParams &P, const MwSensor &S, int ncs,
                                                 int nrs, ColF colX, RowF rowY, PixF pix, int npx,
                                                 float (&acc)[PPT], int *s_i, float *s_f,
                                                 float *s_win = nullptr, int xf = 0, int xl = 0,
                                                 int yf = 0, int yl = 0) {
#pragma unroll
  for (int i = 0; i < PPT; ++i) acc[i] = 0.f;
  if (P.flat) return;
  const int n = S.n_pix;
  const int per = ncs + nrs;
  for (int l0 = 0; l0 < P.n_layers; l0 += kMwLayerChunk) {
    const int lc = min(kMwLayerChunk, P.n_layers - l0);
    __syncthreads();   // the previous chunk's readers are done
    for (int e = threadIdx.x; e < lc * per; e += kMwThreads) {
      const int l = e / per, r = e - l * per;
      const size_t o = r < ncs ? (size_t)(2 * (l0 + l)) * n + colX(r)
                               : (size_t)(2 * (l0 + l) + 1) * n + rowY(r - ncs);
      s_i[e] = __ldcg(S.tab_i + o);
      s_f[e] = __ldcg(S.tab_f + o);
    }
    __syncthreads();
    for (int l = 0; l < lc; ++l) {
      const float *Sc = P.L[l0 + l].scr;
      const int M = P.L[l0 + l].side;
      const int *ti = s_i + l * per;
      const float *tf = s_f + l * per;
      if (WIN > 0 && ((S.win_ok >> (l0 + l)) & 1ull)) {
        const int x0 = ti[xf], y0 = ti[ncs + yf];
        const int wx = (ti[xl] - x0 + M) % M + 2, wy = (ti[ncs + yl] - y0 + M) % M + 2;
        if (wx * wy <= WIN && wx <= M && wy <= M) {   // uniform over the CTA
          __syncthreads();   // the previous layer's window readers are done
          for (int e = threadIdx.x; e < wx * wy; e += kMwThreads) {
            const int r = e / wx, c = e - r * wx;
            int yy = y0 + r, xx = x0 + c;
            if (yy >= M) yy -= M;
            if (xx >= M) xx -= M;
            s_win[e] = __ldg(Sc + (size_t)yy * M + xx);
          }
          __syncthreads();
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            const int q = threadIdx.x + i * kMwThreads;
            if (q < npx) {
              int cs, rs;
              pix(q, cs, rs);
              int cx = ti[cs] - x0, cy = ti[ncs + rs] - y0;
              if (cx < 0) cx += M;
              if (cy < 0) cy += M;
              if (cx > wx - 2 || cy > wy - 2) {   // never with a valid task split
                atomicExch(P.status, SPECULA_EINVAL);
                cx = min(cx, wx - 2);
                cy = min(cy, wy - 2);
              }
              const float fx = tf[cs], fy = tf[ncs + rs];
              const float *w0 = s_win + cy * wx + cx;
              const float s00 = w0[0], s01 = w0[1], s10 = w0[wx], s11 = w0[wx + 1];
              const float a = s00 + fx * (s01 - s00);
              const float b = s10 + fx * (s11 - s10);
              acc[i] += a + fy * (b - a);
            }
          }
          continue;
        }
      }
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const int q = threadIdx.x + i * kMwThreads;
        if (q < npx) {
          int cs, rs;
          pix(q, cs, rs);
          const int ix0 = ti[cs], iy0 = ti[ncs + rs];
          const float fx = tf[cs], fy = tf[ncs + rs];
          const int ix1 = ix0 + 1 == M ? 0 : ix0 + 1;
          const int iy1 = iy0 + 1 == M ? 0 : iy0 + 1;
          const float s00 = __ldg(Sc + (size_t)iy0 * M + ix0);
          const float s01 = __ldg(Sc + (size_t)iy0 * M + ix1);
          const float s10 = __ldg(Sc + (size_t)iy1 * M + ix0);
          const float s11 = __ldg(Sc + (size_t)iy1 * M + ix1);
          const float a = s00 + fx * (s01 - s00);
          const float b = s10 + fx * (s11 - s10);
          acc[i] += a + fy * (b - a);
        }
      }
    }
  }
}

constexpr int kMwFieldPx = kMwThreads;   // pixels per FIELD task (whole rows)

// Pyramid field of rows [y0, y1) (at most kMwFieldPx pixels, one per
// thread).  A pyramid's pupil samples the screens sparsely (several screen
// samples apart), so there is no window to stage: per chunk of layers the
// table entries go to shared memory, then each thread issues the gathers of
// four layers at once before interpolating them in layer order.
__device__ void mw_field(const MwParams &P, const MwSensor &S, int y0, int y1, float2 *smem) {
  const int n = S.n_pix, nr = y1 - y0, per = n + nr;
  int *s_i = reinterpret_cast<int *>(smem);
  float *s_f = reinterpret_cast<float *>(s_i + kMwLayerChunk * per);
  const int q = threadIdx.x;
  const bool act = q < nr * n;
  const int r = act ? q / n : 0, c = act ? q - r * n : 0;
  float acc = 0.f;
  if (!P.flat) {
    for (int l0 = 0; l0 < P.n_layers; l0 += kMwLayerChunk) {
      const int lc = min(kMwLayerChunk, P.n_layers - l0);
      __syncthreads();
      constexpr int TPT = 4;   // table entries per thread: chunk (n + rows) <= 4 x 256 (host check)
      int vi[TPT];
      float vf[TPT];
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        const int e = threadIdx.x + k * kMwThreads;
        if (e < lc * per) {
          const int l = e / per, rr = e - l * per;
          const size_t o = rr < n ? (size_t)(2 * (l0 + l)) * n + rr
                                  : (size_t)(2 * (l0 + l) + 1) * n + y0 + (rr - n);
          vi[k] = __ldcg(S.tab_i + o);
          vf[k] = __ldcg(S.tab_f + o);
        }
      }
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        const int e = threadIdx.x + k * kMwThreads;
        if (e < lc * per) {
          s_i[e] = vi[k];
          s_f[e] = vf[k];
        }
      }
      __syncthreads();
      if (act) {
        // two layers' gathers in flight, interpolated in layer order
        for (int l = 0; l < lc; l += 2) {
          const bool two = l + 1 < lc;
          const float *Sa = P.L[l0 + l].scr;
          const int Ma = P.L[l0 + l].side;
          const int ia = s_i[l * per + c], ja = s_i[l * per + n + r];
          const float *Sb = two ? P.L[l0 + l + 1].scr : Sa;
          const int Mb = two ? P.L[l0 + l + 1].side : Ma;
          const int lb = two ? l + 1 : l;
          const int ib = s_i[lb * per + c], jb = s_i[lb * per + n + r];
          const int ia1 = ia + 1 == Ma ? 0 : ia + 1, ja1 = ja + 1 == Ma ? 0 : ja + 1;
          const int ib1 = ib + 1 == Mb ? 0 : ib + 1, jb1 = jb + 1 == Mb ? 0 : jb + 1;
          const float a00 = __ldg(Sa + (size_t)ja * Ma + ia), a01 = __ldg(Sa + (size_t)ja * Ma + ia1);
          const float a10 = __ldg(Sa + (size_t)ja1 * Ma + ia), a11 = __ldg(Sa + (size_t)ja1 * Ma + ia1);
          const float b00 = __ldg(Sb + (size_t)jb * Mb + ib), b01 = __ldg(Sb + (size_t)jb * Mb + ib1);
          const float b10 = __ldg(Sb + (size_t)jb1 * Mb + ib), b11 = __ldg(Sb + (size_t)jb1 * Mb + ib1);
          {
            const float fx = s_f[l * per + c], fy = s_f[l * per + n + r];
            const float a = a00 + fx * (a01 - a00);
            const float b = a10 + fx * (a11 - a10);
            acc += a + fy * (b - a);
          }
          if (two) {
            const float fx = s_f[lb * per + c], fy = s_f[lb * per + n + r];
            const float a = b00 + fx * (b01 - b00);
            const float b = b10 + fx * (b11 - b10);
            acc += a + fy * (b - a);
          }
        }
      }
    }
  }
  if (act) {
    const size_t e = (size_t)(y0 + r) * n + c;
    const float ph = acc * S.scale;
    S.phase[e] = ph;
    float sv, cv;
    sincosf(ph, &sv, &cv);
    const float a = __ldg(S.amp + e);
    S.field[e] = make_float2(a * cv, a * sv);
  }
}

// ---- Shack-Hartmann ----------------------------------------------------------------
// Subapertures [v0, v1) (at most kMwShSubPerTask, one subaperture row,
// ascending columns spanning fewer than kMwShSubPerTask: the host split).
// The CTA extracts the phase of their pixels as one strip of SP rows x
// W = kMwShSubPerTask SP column slots (slot c: subaperture c / SP, column
// c % SP), then one warp per subaperture images it: the spot arithmetic of
// k_sh_spots, with the centre of gravity taken in registers.
template <int NF, int SP>
struct MwShSmem {
  static constexpr int W = kMwShSubPerTask * SP;                        // column slots
  static constexpr int kPh = kMwShSubPerTask * SP * SP;                 // floats
  static constexpr int kTab = 2 * kMwLayerChunk * (W + SP);             // int + float
  static constexpr int kWin = 4096;                                     // one screen window
  static constexpr int kFft = kMwWarps * NF * (SP | 1) * 2;            // floats
  static_assert(kFft <= kTab + 2 * kWin, "the FFT exchange reuses the extraction space");
  static_assert((W * SP) % kMwThreads == 0, "whole pixels per thread");
  static constexpr size_t bytes = (size_t)(kPh + kTab + 2 * kWin + 2 * kMwShSubPerTask) * 4;
};

// Strip extraction: per chunk of layers the table entries of the W column
// slots and SP rows go to shared memory; per layer, when the host marked
// the layer's span as shorter than the screen (S.win_ok), the screen window
// the strip samples is staged in shared memory with coalesced row loads
// (the sampling coordinate grows with the pupil coordinate below the guide
// star, so slots 0 and ns SP - 1, rows 0 and SP - 1 bound it) and the
// interpolation reads it there; otherwise it gathers from the screen.  Both
// read the same samples: the result is that of k_atmo_extract.
template <int SP, int PPT>
__device__ __forceinline__ void mw_sh_extract(const MwParams &P, const MwSensor &S, int ns,
                                              const int *s_ab, int *s_i, float *s_f,
                                              float *s_win, int win_cap, float (&acc)[PPT]) {
  constexpr int W = kMwShSubPerTask * SP, PER = W + SP;
#pragma unroll
  for (int i = 0; i < PPT; ++i) acc[i] = 0.f;
  if (P.flat) return;
  const int n = S.n_pix, wc = ns * SP, arow = s_ab[0];
  for (int l0 = 0; l0 < P.n_layers; l0 += kMwLayerChunk) {
    const int lc = min(kMwLayerChunk, P.n_layers - l0);
    __syncthreads();
    // all of this thread's table loads in flight before any store
    constexpr int TPT = (kMwLayerChunk * PER + kMwThreads - 1) / kMwThreads;
    int vi[TPT];
    float vf[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int e = threadIdx.x + k * kMwThreads;
      if (e < lc * PER) {
        const int l = e / PER, r = e - l * PER;
        int pix, axis = 0;
        if (r < W) {
          const int c = r < wc ? r : wc - 1;   // unused slots repeat the last column
          pix = s_ab[kMwShSubPerTask + c / SP] * SP + c % SP;
        } else {
          pix = arow * SP + (r - W);
          axis = 1;
        }
        const size_t o = (size_t)(2 * (l0 + l) + axis) * n + pix;
        vi[k] = __ldcg(S.tab_i + o);
        vf[k] = __ldcg(S.tab_f + o);
      }
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int e = threadIdx.x + k * kMwThreads;
      if (e < lc * PER) {
        s_i[e] = vi[k];
        s_f[e] = vf[k];
      }
    }
    __syncthreads();
    // windows double-buffered: layer l + 1's window is copied (cp.async)
    // while layer l interpolates from the other buffer
    auto win_geom = [&](int l, int &x0, int &y0, int &wx, int &wy) {
      const int *ti = s_i + l * PER;
      const int M = P.L[l0 + l].side;
      x0 = ti[0];
      y0 = ti[W];
      wx = (ti[wc - 1] - x0 + M) % M + 2;
      wy = (ti[W + SP - 1] - y0 + M) % M + 2;
      return ((S.win_ok >> (l0 + l)) & 1ull) && wx * wy <= win_cap;
    };
    auto issue = [&](int l, float *buf) {
      int x0, y0, wx, wy;
      if (!win_geom(l, x0, y0, wx, wy)) return;
      const float *Sc = P.L[l0 + l].scr;
      const int M = P.L[l0 + l].side;
      for (int c = threadIdx.x; c < wx; c += kMwThreads) {
        int xx = x0 + c;
        if (xx >= M) xx -= M;
        for (int r = 0; r < wy; ++r) {
          int yy = y0 + r;
          if (yy >= M) yy -= M;
          cp_async4(buf + r * wx + c, Sc + (size_t)yy * M + xx);
        }
      }
    };
    issue(0, s_win);
    cp_async_commit();
    for (int l = 0; l < lc; ++l) {
      float *cur = s_win + (l & 1) * win_cap;
      if (l + 1 < lc) issue(l + 1, s_win + ((l + 1) & 1) * win_cap);
      cp_async_commit();
      cp_async_wait_1();     // all but the newest group: layer l's window is in
      __syncthreads();
      const float *Sc = P.L[l0 + l].scr;
      const int M = P.L[l0 + l].side;
      const int *ti = s_i + l * PER;
      const float *tf = s_f + l * PER;
      int x0, y0, wx, wy;
      if (win_geom(l, x0, y0, wx, wy)) {   // uniform over the CTA
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const int q = threadIdx.x + i * kMwThreads;
          const int r = q / W, c = q - r * W;
          if (c < wc) {
            int cx = ti[c] - x0, cy = ti[W + r] - y0;
            if (cx < 0) cx += M;
            if (cy < 0) cy += M;
            if (cx > wx - 2 || cy > wy - 2) {   // never with the host's task split
              atomicExch(P.status, SPECULA_EINVAL);
              cx = min(cx, wx - 2);
              cy = min(cy, wy - 2);
            }
            const float fx = tf[c], fy = tf[W + r];
            const float *w0 = cur + cy * wx + cx;
            const float s00 = w0[0], s01 = w0[1], s10 = w0[wx], s11 = w0[wx + 1];
            const float a = s00 + fx * (s01 - s00);
            const float b = s10 + fx * (s11 - s10);
            acc[i] += a + fy * (b - a);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const int q = threadIdx.x + i * kMwThreads;
          const int r = q / W, c = q - r * W;
          if (c < wc) {
            const int ix0 = ti[c], iy0 = ti[W + r];
            const float fx = tf[c], fy = tf[W + r];
            const int ix1 = ix0 + 1 == M ? 0 : ix0 + 1;
            const int iy1 = iy0 + 1 == M ? 0 : iy0 + 1;
            const float s00 = __ldg(Sc + (size_t)iy0 * M + ix0);
            const float s01 = __ldg(Sc + (size_t)iy0 * M + ix1);
            const float s10 = __ldg(Sc + (size_t)iy1 * M + ix0);
            const float s11 = __ldg(Sc + (size_t)iy1 * M + ix1);
            const float a = s00 + fx * (s01 - s00);
            const float b = s10 + fx * (s11 - s10);
            acc[i] += a + fy * (b - a);
          }
        }
      }
      __syncthreads();   // readers of `cur` are done before it is refilled
    }
  }
}

template <int NF, int SP>
__device__ void mw_sh(const MwParams &P, const MwSensor &S, int v0, int v1, float2 *smem) {
  constexpr int OFF = (NF - SP) / 2;
  constexpr int XS = SP | 1;
  using L = MwShSmem<NF, SP>;
  constexpr int W = L::W;
  constexpr int PPT = W * SP / kMwThreads;
  float *ph = reinterpret_cast<float *>(smem);
  float *region = ph + L::kPh;                     // tables + window, then FFT exchange
  float *s_win = region + L::kTab;                 // two windows
  int *s_ab = reinterpret_cast<int *>(s_win + 2 * L::kWin);
  const int ns = v1 - v0;
  for (int k = threadIdx.x; k < ns; k += kMwThreads) {
    const int idx = __ldg(S.valid + v0 + k);
    s_ab[k] = idx / S.n_sub;
    s_ab[kMwShSubPerTask + k] = idx % S.n_sub;
  }
  __syncthreads();
  int *s_i = reinterpret_cast<int *>(region);
  float *s_f = region + kMwLayerChunk * (W + SP);
  float acc[PPT];
  mw_sh_extract<SP, PPT>(P, S, ns, s_ab, s_i, s_f, s_win, L::kWin, acc);
  const int n = S.n_pix;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int q = threadIdx.x + i * kMwThreads;
    const int r = q / W, cs = q - r * W;
    if (cs < ns * SP) {
      const int sub = cs / SP, c = cs % SP;
      const float f = acc[i] * S.scale;
      ph[sub * SP * SP + r * SP + c] = f;
      S.phase[(size_t)(s_ab[sub] * SP + r) * n + (size_t)s_ab[kMwShSubPerTask + sub] * SP + c] = f;
    }
  }
  __syncthreads();
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  float2 *xs = reinterpret_cast<float2 *>(region) + w * (NF * XS);
  for (int sub = w; sub < ns; sub += kMwWarps) {
    const int v = v0 + sub;
    const int a = s_ab[sub], bc = s_ab[kMwShSubPerTask + sub];
    const float *phs = ph + sub * SP * SP;
    float2 vv[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) vv[q] = make_float2(0.f, 0.f);
    if (lane < SP) {
      const float *am = S.amp + (size_t)(a * SP + lane) * n + (size_t)bc * SP;
      const float2 py = __ldg(S.pre + OFF + lane);
#pragma unroll
      for (int c = 0; c < SP; ++c) {
        float sv, cv;
        sincosf(phs[lane * SP + c], &sv, &cv);
        const float A = __ldg(am + c);
        vv[OFF + c] = cmul(cmul(make_float2(A * cv, A * sv), __ldg(S.pre + OFF + c)), py);
      }
    }
    RegDFT<NF, false>::run(vv);
    __syncwarp();
    if (lane < SP) {
#pragma unroll
      for (int k = 0; k < NF; ++k) xs[k * XS + lane] = vv[k];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NF; ++q) vv[q] = make_float2(0.f, 0.f);
    if (lane < NF) {
#pragma unroll
      for (int r = 0; r < SP; ++r) vv[OFF + r] = xs[lane * XS + r];
    }
    RegDFT<NF, false>::run(vv);
    // lane k holds column k of the spot: vv[q] at row q
    float si = 0.f, sx = 0.f, sy = 0.f;
    if (lane < NF) {
      constexpr float inv = 1.0f / (float)(NF * NF);
      const float c = 0.5f * (float)(NF - 1);
      const float xk = (float)lane - c;
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        const float I = (vv[q].x * vv[q].x + vv[q].y * vv[q].y) * inv;
        si += I;
        sx += I * xk;
        sy += I * ((float)q - c);
      }
    }
    si = mw_warp_sum(si);
    sx = mw_warp_sum(sx);
    sy = mw_warp_sum(sy);
    if (lane == 0) {
      float gx = sx / si, gy = sy / si;
      if (P.ref) {
        gx -= P.ref[S.slope_off + v];
        gy -= P.ref[S.slope_off + S.n_valid + v];
      }
      P.slopes[S.slope_off + v] = gx;
      P.slopes[S.slope_off + S.n_valid + v] = gy;
      mw_guard(gx, gy, P.nf_status);
    }
    __syncwarp();
  }
}

// ---- pyramid passes (arithmetic of k_rows_fwd / k_cols / k_rows_inv_part) ------
template <int N1, int N2>
__device__ void mw_rows(const MwSensor &S, int m, int rg, float2 *smem) {
  using Sp = Split<N1, N2>;
  constexpr int N = Sp::N, G = Sp::G, S1 = Sp::S1;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  constexpr int VPC = kMwThreads / G;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  float2 *xb = smem + vec * Sp::XB;
  const int n_pix = S.n_pix;
  const int j = rg * VPC + vec;
  const bool row_ok = j < n_pix;
  const bool in_lane = row_ok && lane < N1;
  float2 r[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  const float2 gyv = row_ok ? __ldg(S.gy + (size_t)m * n_pix + j) : make_float2(0.f, 0.f);
  if (in_lane) {
    const float2 *src = S.field + (size_t)j * n_pix + lane;
    const float2 *g = S.gx + (size_t)m * n_pix + lane;
#pragma unroll
    for (int h = 0; h < QH; ++h) r[Q0 + h] = cmul(cmul(__ldcg(src + N1 * h), __ldg(g + N1 * h)), gyv);
  }
  RegDFT<N2, false>::run(r);
  __syncwarp();
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = cmulc(r[k2], __ldg(S.twA + k2 * N1 + lane));
  }
  __syncwarp();
  if (lane < N2) {
    float2 r2[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xb[lane * S1 + n1];
    RegDFT<N1, false>::run(r2);
    if (row_ok) {
      float2 *dst = S.rows + ((size_t)m * n_pix + j) * N + lane;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) dst[N2 * k1] = r2[k1];
    }
  }
}

template <int N1, int N2> struct MwCols {
  using Sp = Split<N1, N2>;
  static constexpr int TC = kMwThreads / Sp::G;
  // column stride = 1 (mod 16) complex: the row-wise staging of TC = 16
  // columns touches 16 distinct bank pairs
  static constexpr int base = imax3(Sp::N, N2 * Sp::S1, N1 * Sp::S2);
  static constexpr int CS = base + ((1 - base % 16) + 16) % 16;
  static constexpr size_t smem = (size_t)TC * CS * sizeof(float2);
};

template <int N1, int N2>
__device__ void mw_cols(const MwSensor &S, int m, int ct, float2 *smem) {
  using Sp = Split<N1, N2>;
  constexpr int N = Sp::N, G = Sp::G, S1 = Sp::S1, S2 = Sp::S2;
  constexpr int TC = MwCols<N1, N2>::TC, CS = MwCols<N1, N2>::CS;
  constexpr int Q0 = N2 / 4, QH = N2 / 2;
  constexpr int off = N / 4;
  const int n_pix = S.n_pix;
  float2 *s_tile = smem;
  const int col0 = ct * TC;
  const float2 *src = S.rows + (size_t)m * n_pix * N + col0;
#pragma unroll 4
  for (int e = threadIdx.x; e < n_pix * TC; e += kMwThreads) {
    const int c = e % TC, jj = e / TC;
    s_tile[c * CS + off + jj] = __ldcg(src + (size_t)jj * N + c);
  }
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  const float2 mk = __ldg(S.mask + col0 + vec);
  __syncthreads();
  float2 *col = s_tile + vec * CS;
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
    for (int k2 = 0; k2 < N2; ++k2) col[k2 * S1 + lane] = cmulc(r[k2], __ldg(S.twA + k2 * N1 + lane));
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
  if (lane < N2) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) r2[k1] = cmul(r2[k1], cmul(__ldg(S.mask + N2 * k1 + lane), mk));
  }
  RegDFT<N1, true>::run(r2);
  __syncwarp();
  if (lane < N2) {
#pragma unroll
    for (int k2 = 0; k2 < N1; ++k2) col[k2 * S2 + lane] = cmul(r2[k2], __ldg(S.twB + k2 * N2 + lane));
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
    for (int k1 = 0; k1 < N2; ++k1) col[N1 * k1 + lane] = r3[k1];
  }
  __syncthreads();
  float2 *dst = S.cols + (size_t)m * N * N + col0;
  for (int e = threadIdx.x; e < N * TC; e += kMwThreads) {
    const int c = e % TC, y = e / TC;
    dst[(size_t)y * N + c] = s_tile[c * CS + y];
  }
}

// Strips [sg spt, sg spt + spt) of bsz rows each: row IFFT, |.|^2 / n_mod,
// b x b bins -> part[m][strip][.].
template <int N1, int N2>
__device__ void mw_rinv(const MwSensor &S, int m, int sg, float2 *smem) {
  using Sp = Split<N1, N2>;
  constexpr int N = Sp::N, G = Sp::G, S1 = Sp::S1;
  const int vec = threadIdx.x / G, lane = threadIdx.x % G;
  const int bsz = S.bsz, nd = S.nd, spt = S.spt;
  const int strip0 = sg * spt;
  const int n_strips = min(spt, nd - strip0);
  const bool act = vec < n_strips * bsz;
  const int y = strip0 * bsz + (act ? vec : 0);
  float2 *xb = smem + vec * Sp::XB;
  float2 r[N2];
  if (act && lane < N1) {
    const float2 *src = S.cols + ((size_t)m * N + y) * N + lane;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = __ldcg(src + N1 * n2);
  } else {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = make_float2(0.f, 0.f);
  }
  RegDFT<N2, true>::run(r);
  if (lane < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) xb[k2 * S1 + lane] = cmul(r[k2], __ldg(S.twA + k2 * N1 + lane));
  }
  __syncwarp();
  float2 r2[N1];
  if (lane < N2) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r2[n1] = xb[lane * S1 + n1];
  }
  __syncwarp();
  float *s_row = reinterpret_cast<float *>(xb);
  const float scale = 1.0f / (float)S.n_mod;
  if (act && lane < N2) {
    RegDFT<N1, true>::run(r2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      s_row[N2 * k1 + lane] = (r2[k1].x * r2[k1].x + r2[k1].y * r2[k1].y) * scale;
  }
  __syncthreads();
  const float *s_I = reinterpret_cast<const float *>(smem);
  constexpr int RS = 2 * Sp::XB;
  for (int q = threadIdx.x; q < n_strips * nd; q += kMwThreads) {
    const int ls = q / nd, qq = q - ls * nd;
    float v = 0.f;
    for (int rr = 0; rr < bsz; ++rr)
      for (int xx = 0; xx < bsz; ++xx) v += s_I[(ls * bsz + rr) * RS + qq * bsz + xx];
    S.part[((size_t)m * nd + strip0 + ls) * nd + qq] = v;
  }
}

__device__ void mw_bin(const MwSensor &S, int p0, int p1) {
  const int nd2 = S.nd * S.nd;
  for (int p = p0 + threadIdx.x; p < p1; p += kMwThreads) {
    // eight loads in flight, summed in modulation order
    float v = 0.f;
    int m = 0;
    for (; m + 8 <= S.n_mod; m += 8) {
      float t[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) t[k] = __ldcg(S.part + (size_t)(m + k) * nd2 + p);
#pragma unroll
      for (int k = 0; k < 8; ++k) v += t[k];
    }
    for (; m < S.n_mod; ++m) v += __ldcg(S.part + (size_t)m * nd2 + p);
    S.det[p] = v;
  }
}

__device__ void mw_pyr_slopes(const MwParams &P, const MwSensor &S, float *s_w) {
  const int ns = S.n_sub, w2 = 2 * ns;
  const float *d = S.det;
  float part = 0.f;
#pragma unroll 4
  for (int k = threadIdx.x; k < S.n_valid; k += kMwThreads) {
    const int s = __ldg(S.valid + k);
    const int a = s / ns, c = s % ns;
    const float q1 = __ldcg(d + (ns + a) * w2 + ns + c), q2 = __ldcg(d + (ns + a) * w2 + c);
    const float q3 = __ldcg(d + a * w2 + c), q4 = __ldcg(d + a * w2 + ns + c);
    part += ((q1 + q2) + q3) + q4;
  }
  part = mw_warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = part;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < kMwWarps; ++i) t += s_w[i];
  const float T = t / (float)S.n_valid;
  float *o = P.slopes + S.slope_off;
  const float *ref = P.ref ? P.ref + S.slope_off : nullptr;
#pragma unroll 4
  for (int k = threadIdx.x; k < S.n_valid; k += kMwThreads) {
    const int s = __ldg(S.valid + k);
    const int a = s / ns, c = s % ns;
    const float q1 = __ldcg(d + (ns + a) * w2 + ns + c), q2 = __ldcg(d + (ns + a) * w2 + c);
    const float q3 = __ldcg(d + a * w2 + c), q4 = __ldcg(d + a * w2 + ns + c);
    float sx = ((q1 + q4) - (q2 + q3)) / T;
    float sy = ((q1 + q2) - (q3 + q4)) / T;
    if (ref) {
      sx -= ref[k];
      sy -= ref[S.n_valid + k];
    }
    o[k] = sx;
    o[S.n_valid + k] = sy;
    mw_guard(sx, sy, P.nf_status);
  }
}

// ---- reconstructor ---------------------------------------------------------------
// Rows [r0, r1) of R restricted to this sensor's columns, times its slopes
// (staged in shared memory); one warp per row, 8 independent 16-byte loads
// in flight per lane.
__device__ void mw_mvm(const MwParams &P, const MwSensor &S, int sidx, int r0, int r1,
                       float *s_v) {
  const int ns = 2 * S.n_valid, c0 = S.slope_off;
  for (int e = threadIdx.x; e < ns; e += kMwThreads) s_v[e] = __ldcg(P.slopes + c0 + e);
  __syncthreads();
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int row = r0 + w; row < r1; row += kMwWarps) {
    const float *Rr = P.R + (size_t)row * P.n_slopes + c0;
    float acc = 0.f;
    if (P.r_vec4) {
      const float4 *r4 = reinterpret_cast<const float4 *>(Rr);
      const float4 *v4 = reinterpret_cast<const float4 *>(s_v);
      const int n4 = ns / 4;
      for (int j0 = lane; j0 < n4; j0 += 8 * 32) {
        float4 a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          a[u] = (j0 + 32 * u < n4) ? mw_ld_stream(r4 + j0 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + 32 * u;
          if (j < n4) {
            const float4 x = v4[j];
            acc += a[u].x * x.x + a[u].y * x.y + a[u].z * x.z + a[u].w * x.w;
          }
        }
      }
    } else {
      for (int j = lane; j < ns; j += 32) acc += __ldg(Rr + j) * s_v[j];
    }
    acc = mw_warp_sum(acc);
    if (lane == 0) P.mpart[(size_t)sidx * P.n_modes + row] = acc;
  }
}

__device__ void mw_final(const MwParams &P, int r0, int r1) {
  for (int row = r0 + threadIdx.x; row < r1; row += kMwThreads) {
    float v = 0.f;
    for (int s = 0; s < P.n_sensors; ++s) v += __ldcg(P.mpart + (size_t)s * P.n_modes + row);
    P.modes[row] = v;
  }
}

// ---- the persistent kernel ---------------------------------------------------------
template <int PN1, int PN2, int NF, int SP>
__global__ void __launch_bounds__(kMwThreads, 3) k_mwfs(const __grid_constant__ MwParams P) {
  extern __shared__ __align__(16) float2 mw_smem[];
  __shared__ int s_t, s_ok;
  __shared__ float s_w[kMwWarps];
  int *ticket = P.ctr, *exitc = P.ctr + 1, *abortf = P.ctr + 2;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(ticket, 1);
      int ok = 1;
      if (t < P.n_tasks) {
        int wc = P.tasks[t].wait_ctr, wv = P.tasks[t].wait_val;
        if (t == P.stall_task) {       // its own completion count: never reached
          wc = P.tasks[t].done_ctr;
          wv = 0x7fffffff;
        }
        if (ld_relaxed_gpu(abortf)) ok = 0;
        else if (wc >= 0) ok = mw_wait(P.ctr + wc, wv, abortf, P.status, P.wait_ns);
      }
      s_t = t;
      s_ok = ok;
    }
    __syncthreads();
    const int t = s_t;
    if (t >= P.n_tasks || !s_ok) break;
    const MwTask tk = P.tasks[t];
    const MwSensor &S = P.S[tk.sensor];
    switch (tk.type) {
      case MT_COORDS: mw_coords(P, S, tk.a, tk.b); break;
      case MT_FIELD: mw_field(P, S, tk.a, tk.b, mw_smem); break;
      case MT_SH:
        if constexpr (NF > 0) mw_sh<NF, SP>(P, S, tk.a, tk.b, mw_smem);
        break;
      case MT_ROWS: mw_rows<PN1, PN2>(S, tk.a, tk.b, mw_smem); break;
      case MT_COLS: mw_cols<PN1, PN2>(S, tk.a, tk.b, mw_smem); break;
      case MT_RINV: mw_rinv<PN1, PN2>(S, tk.a, tk.b, mw_smem); break;
      case MT_BIN: mw_bin(S, tk.a, tk.b); break;
      case MT_SLOPES: mw_pyr_slopes(P, S, s_w); break;
      case MT_MVM: mw_mvm(P, S, tk.sensor, tk.a, tk.b, reinterpret_cast<float *>(mw_smem)); break;
      case MT_FINAL: mw_final(P, tk.a, tk.b); break;
      default: break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      red_release_gpu(P.ctr + tk.done_ctr, 1);
    }
  }
  // the last CTA to leave resets the counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(exitc, 1) == (int)gridDim.x - 1) {
      for (int i = 3; i < P.n_ctr; ++i) P.ctr[i] = 0;
      P.ctr[0] = 0;
      P.ctr[2] = 0;
      __threadfence();
      P.ctr[1] = 0;
    }
  }
}

template <int PN1, int PN2, int NF, int SP>
static size_t mw_smem_bytes(int max_slopes, int max_field_slots) {
  using Sp = Split<PN1, PN2>;
  size_t b = MwShSmem<NF, SP>::bytes;
  b = std::max(b, (size_t)(kMwThreads / Sp::G) * Sp::XB * sizeof(float2));   // rows, rinv
  b = std::max(b, MwCols<PN1, PN2>::smem);
  b = std::max(b, (size_t)max_slopes * sizeof(float));
  b = std::max(b, (size_t)2 * kMwLayerChunk * max_field_slots * 4);            // field tables
  return (b + 15) / 16 * 16;
}

typedef void (*MwKernel)(MwParams);

struct MwVariant {
  int pn1, pn2, nf, sp;
  MwKernel fn;
  size_t (*smem)(int, int);
};

static const MwVariant kMwVariants[] = {
    {8, 16, 24, 12, k_mwfs<8, 16, 24, 12>, mw_smem_bytes<8, 16, 24, 12>},
    {15, 16, 24, 12, k_mwfs<15, 16, 24, 12>, mw_smem_bytes<15, 16, 24, 12>},
};

}  // namespace specula

using namespace specula;

struct specula_mwfs {
  specula_ctx *ctx = nullptr;
  int device = 0;
  MwParams P;
  const MwVariant *var = nullptr;
  std::vector<std::unique_ptr<DevBuf>> bufs;
  DevBuf tasks, ctr, mpart;
  std::vector<MwTask> host_tasks;
  std::vector<int> n_valid, slope_off, kind, det_n;
  std::vector<std::vector<int32_t>> valid_host;
  int n_slopes = 0;
  int grid = 0, max_grid = 0;
  size_t smem = 0;
  int sm_count = 0, occupancy = 0;
  DevBuf *add(size_t bytes, int *status) {
    bufs.emplace_back(new DevBuf());
    *status = bufs.back()->alloc(bytes);
    return bufs.back().get();
  }
};

namespace {

// Emit A in order and release the (independent of each other) tasks of B
// once the last producer of their dependency went out at least `lag`
// positions earlier (about two waves of CTAs: by the time a CTA takes such
// a task, its dependency has most likely completed, so it does not idle).
// From the first position where some B task is eligible, B tasks leave at a
// steady rate over the rest of A, in the order they became eligible; what is
// left follows A.
void release_when_ready(const std::vector<MwTask> &A, const std::vector<MwTask> &B,
                        const std::vector<int> &produced_total, std::vector<int> &emitted,
                        std::vector<MwTask> &out, int lag) {
  std::vector<long> last_pos(produced_total.size(), -1);
  std::vector<char> pooled(B.size(), 0);
  std::vector<size_t> pool;
  size_t head = 0, n_out = 0;
  long first = -1;
  auto eligible = [&](const MwTask &t, long pos) {
    if (t.wait_ctr < 0) return true;
    return emitted[t.wait_ctr] >= produced_total[t.wait_ctr] && pos - last_pos[t.wait_ctr] >= lag;
  };
  auto refill = [&](long pos) {
    for (size_t i = 0; i < B.size(); ++i)
      if (!pooled[i] && eligible(B[i], pos)) {
        pooled[i] = 1;
        pool.push_back(i);
      }
  };
  auto emit = [&](const MwTask &t) {
    last_pos[t.done_ctr] = (long)out.size();
    out.push_back(t);
    emitted[t.done_ctr]++;
  };
  for (size_t ia = 0; ia < A.size(); ++ia) {
    emit(A[ia]);
    refill((long)out.size());
    if (first < 0 && head < pool.size()) first = (long)ia;
    if (first < 0) continue;
    const double frac = (double)(ia + 1 - first) / (double)(A.size() - first);
    while (head < pool.size() && (double)n_out < frac * B.size()) {
      emit(B[pool[head++]]);
      n_out++;
    }
  }
  refill(1L << 40);
  while (head < pool.size()) emit(B[pool[head++]]);
}

MwTask mk(int type, int sensor, int a, int b, int wait_ctr, int wait_val, int done_ctr) {
  MwTask t;
  t.type = type; t.sensor = sensor; t.a = a; t.b = b;
  t.wait_ctr = wait_ctr; t.wait_val = wait_val; t.done_ctr = done_ctr; t.pad = 0;
  return t;
}

}  // namespace

extern "C" int specula_mwfs_create(specula_ctx *ctx, int32_t n_sensors,
                                   const specula_wfs_desc *sensors, int32_t n_layers,
                                   const specula_layer_desc *layers,
                                   const float *const *screens_dev, int32_t n_modes,
                                   const float *R_dev, specula_mwfs **out) {
  if (!ctx || !sensors || !out || n_sensors < 1 || n_layers < 1 || !layers || !screens_dev)
    return SPECULA_EINVAL;
  if (n_sensors > kMwMaxSensors || n_layers > kMwMaxLayers) return SPECULA_EUNSUPPORTED;
  if (n_modes < 0 || (n_modes > 0 && !R_dev)) return SPECULA_EINVAL;
  *out = nullptr;
  for (int l = 0; l < n_layers; ++l) {
    const specula_layer_desc &L = layers[l];
    if (!screens_dev[l] || L.side < 2 || !(L.pitch_m > 0) || !isfinite(L.height_m) ||
        !isfinite(L.vx_mps) || !isfinite(L.vy_mps))
      return SPECULA_EINVAL;
  }
  // one pyramid FFT side and one SH geometry per system (the kernel variant)
  int pN = 0, nf = 0, sp = 0;
  for (int k = 0; k < n_sensors; ++k) {
    const specula_wfs_desc &d = sensors[k];
    const specula_pupil_desc &pu = d.pupil;
    if (pu.n_pix < 2 || !(pu.pitch_m > 0) || !(pu.obsc_frac >= 0 && pu.obsc_frac < 1))
      return SPECULA_EINVAL;
    if (!(d.source.wavelength_nm > 0) || !(d.source.height_m > 0)) return SPECULA_EINVAL;
    for (int l = 0; l < n_layers; ++l)   // the cone factor 1 - h/H must stay positive
      if (!(layers[l].height_m < d.source.height_m)) return SPECULA_EUNSUPPORTED;
    if (d.kind == SPECULA_WFS_PYR) {
      const specula_pwfs_desc &g = d.pwfs;
      if (g.n_mod < 1 || g.n_sub < 1 || g.pad != 2 || g.pup_dist_px != pu.n_pix ||
          pu.n_pix % g.n_sub)
        return g.n_mod < 1 || g.n_sub < 1 ? SPECULA_EINVAL : SPECULA_EUNSUPPORTED;
      const int N = 2 * pu.n_pix;
      if (pN && pN != N) return SPECULA_EUNSUPPORTED;
      if (pu.n_pix > kMwFieldPx) return SPECULA_EUNSUPPORTED;   // whole rows per FIELD task
      pN = N;
    } else if (d.kind == SPECULA_WFS_SH) {
      const specula_sh_desc &h = d.sh;
      if (h.n_sub < 1 || h.sub_pix < 1 || h.n_sub * h.sub_pix != pu.n_pix) return SPECULA_EINVAL;
      if (nf && (nf != h.fft_n || sp != h.sub_pix)) return SPECULA_EUNSUPPORTED;
      nf = h.fft_n;
      sp = h.sub_pix;
    } else {
      return SPECULA_EINVAL;
    }
  }
  int pn1 = 8, pn2 = 16;
  if (pN && !pwfs_split_for(pN, &pn1, &pn2)) return SPECULA_EUNSUPPORTED;
  const MwVariant *var = nullptr;
  for (const MwVariant &v : kMwVariants)
    if (v.pn1 == pn1 && v.pn2 == pn2 && (nf == 0 || (v.nf == nf && v.sp == sp))) var = &v;
  if (!var) return SPECULA_EUNSUPPORTED;

  SPECULA_CK(cudaSetDevice(ctx->device));
  std::unique_ptr<specula_mwfs> m(new specula_mwfs());
  m->ctx = ctx;
  m->device = ctx->device;
  m->var = var;
  MwParams &P = m->P;
  memset(&P, 0, sizeof(P));
  P.n_sensors = n_sensors;
  P.n_layers = n_layers;
  for (int l = 0; l < n_layers; ++l) {
    P.L[l].scr = screens_dev[l];
    P.L[l].side = layers[l].side;
    P.L[l].pitch = layers[l].pitch_m;
    P.L[l].h = layers[l].height_m;
    P.L[l].vx = layers[l].vx_mps;
    P.L[l].vy = layers[l].vy_mps;
  }
  static_assert(Split<8, 16>::G == 16 && Split<15, 16>::G == 16, "one vector width");
  const int G = 16;   // lanes per vector of both supported pyramid splits
  int st = SPECULA_OK;
  int off = 0, max_slopes = 0, max_field_slots = 0;
  for (int k = 0; k < n_sensors; ++k) {
    const specula_wfs_desc &d = sensors[k];
    MwSensor &S = P.S[k];
    const int n = d.pupil.n_pix;
    S.kind = d.kind;
    S.n_pix = n;
    S.pitch = d.pupil.pitch_m;
    S.theta_x = d.source.theta_x_rad;
    S.theta_y = d.source.theta_y_rad;
    S.H = d.source.height_m;
    S.scale = (float)(500.0 / d.source.wavelength_nm);
    std::vector<uint8_t> mk8((size_t)n * n);
    host_pupil_mask(n, d.pupil.obsc_frac, mk8.data());
    std::vector<float> ampf(mk8.begin(), mk8.end());
    DevBuf *b;
    if ((b = m->add(ampf.size() * 4, &st)), st) return st;
    SPECULA_CK(cudaMemcpy(b->p, ampf.data(), ampf.size() * 4, cudaMemcpyHostToDevice));
    S.amp = b->as<float>();
    if ((b = m->add((size_t)n * n * 4, &st)), st) return st;
    SPECULA_CK(cudaMemset(b->p, 0, b->bytes));
    S.phase = b->as<float>();
    if ((b = m->add((size_t)n_layers * 2 * n * 4, &st)), st) return st;
    S.tab_i = b->as<int>();
    if ((b = m->add((size_t)n_layers * 2 * n * 4, &st)), st) return st;
    S.tab_f = b->as<float>();
    const int nsub = d.kind == SPECULA_WFS_PYR ? d.pwfs.n_sub : d.sh.n_sub;
    std::vector<int32_t> idx((size_t)nsub * nsub);
    int32_t nv = 0;
    host_valid_subaps(n, d.pupil.obsc_frac, nsub, idx.data(), &nv);
    if (nv < 1) return SPECULA_EINVAL;
    if ((b = m->add((size_t)nv * 4, &st)), st) return st;
    SPECULA_CK(cudaMemcpy(b->p, idx.data(), (size_t)nv * 4, cudaMemcpyHostToDevice));
    S.valid = b->as<int32_t>();
    S.n_sub = nsub;
    S.n_valid = nv;
    S.slope_off = off;
    off += 2 * nv;
    max_slopes = std::max(max_slopes, 2 * nv);
    m->n_valid.push_back(nv);
    m->valid_host.emplace_back(idx.begin(), idx.begin() + nv);
    m->slope_off.push_back(S.slope_off);
    m->kind.push_back(d.kind);
    if (d.kind == SPECULA_WFS_SH) {
      const int NF = d.sh.fft_n;
      std::vector<float2> pre(NF);
      for (int q = 0; q < NF; ++q) {
        const long long r = ((long long)(NF - 1) * q) % (2 * NF);
        const double ang = M_PI * (double)r / (double)NF;
        pre[q] = make_float2((float)cos(ang), (float)sin(ang));
      }
      if ((b = m->add(NF * sizeof(float2), &st)), st) return st;
      SPECULA_CK(cudaMemcpy(b->p, pre.data(), NF * sizeof(float2), cudaMemcpyHostToDevice));
      S.pre = b->as<float2>();
      m->det_n.push_back(0);
      // a task spans < kMwShSubPerTask subapertures of one row: its sampling
      // span on layer l is at most (16 sub_pix - 1) r + 2 screen samples,
      // r = pupil pitch (1 - h/H) / layer pitch; the window path needs it
      // below the side, where the wrapped width equals the true width
      S.win_ok = 0;
      for (int l = 0; l < n_layers; ++l) {
        const double cone = 1.0 - layers[l].height_m / d.source.height_m;
        const double r = d.pupil.pitch_m * cone / layers[l].pitch_m;
        const double span = (kMwShSubPerTask * d.sh.sub_pix - 1) * r + 3.0;
        if (span < (double)layers[l].side - 2.0) S.win_ok |= 1ull << l;
      }
    } else {
      const specula_pwfs_desc &g = d.pwfs;
      const int N = 2 * n;
      PwfsTablesHost T;
      pwfs_host_tables(n, N, pn1, pn2, g.n_mod, g.mod_amp, g.pup_dist_px, &T);
      const std::vector<float2> *tabs[5] = {&T.gx, &T.gy, &T.mask, &T.twA, &T.twB};
      const float2 **dst[5] = {&S.gx, &S.gy, &S.mask, &S.twA, &S.twB};
      for (int q = 0; q < 5; ++q) {
        if ((b = m->add(tabs[q]->size() * sizeof(float2), &st)), st) return st;
        SPECULA_CK(cudaMemcpy(b->p, tabs[q]->data(), b->bytes, cudaMemcpyHostToDevice));
        *dst[q] = b->as<float2>();
      }
      S.n_mod = g.n_mod;
      S.nd = 2 * g.n_sub;
      S.bsz = n / g.n_sub;
      S.spt = (kMwThreads / G) / S.bsz;
      if (S.spt < 1) return SPECULA_EUNSUPPORTED;
      if ((b = m->add((size_t)n * n * sizeof(float2), &st)), st) return st;
      S.field = b->as<float2>();
      if ((b = m->add((size_t)g.n_mod * n * N * sizeof(float2), &st)), st) return st;
      S.rows = b->as<float2>();
      if ((b = m->add((size_t)g.n_mod * N * N * sizeof(float2), &st)), st) return st;
      S.cols = b->as<float2>();
      if ((b = m->add((size_t)g.n_mod * S.nd * S.nd * 4, &st)), st) return st;
      S.part = b->as<float>();
      if ((b = m->add((size_t)S.nd * S.nd * 4, &st)), st) return st;
      SPECULA_CK(cudaMemset(b->p, 0, b->bytes));
      S.det = b->as<float>();
      m->det_n.push_back(S.nd * S.nd);
    }
  }
  m->n_slopes = off;
  P.n_modes = n_modes;
  P.n_slopes = off;
  P.R = R_dev;
  bool v4 = (off % 4 == 0) && ((uintptr_t)R_dev % 16 == 0);
  for (int k = 0; k < n_sensors; ++k)
    v4 = v4 && (P.S[k].slope_off % 4 == 0) && ((2 * P.S[k].n_valid) % 4 == 0);
  P.r_vec4 = v4 ? 1 : 0;
  if (n_modes > 0 && (st = m->mpart.alloc((size_t)n_sensors * n_modes * 4))) return st;
  P.mpart = m->mpart.as<float>();

  // ---- task list -----------------------------------------------------------------
  int nctr = 3;
  auto new_ctr = [&]() { return nctr++; };
  std::vector<int> c_coords(n_sensors), n_coords(n_sensors, 0), c_field(n_sensors, -1),
      n_field(n_sensors, 0), c_sh(n_sensors, -1), n_sh(n_sensors, 0), c_slopes(n_sensors, -1),
      c_rinv(n_sensors, -1), c_bin(n_sensors, -1), n_binv(n_sensors, 0);
  std::vector<std::vector<int>> c_rows(n_sensors), c_cols(n_sensors);
  std::vector<MwTask> L_coords, L_field, L_pyr, L_sh, L_mvm, L_final;
  std::vector<std::vector<MwTask>> L_sh_by(n_sensors);
  const int TC = kMwThreads / G, VPC = kMwThreads / G;
  for (int pass = 0; pass < 2; ++pass)   // pyramids first, then SH
    for (int k = 0; k < n_sensors; ++k) {
      if ((pass == 0) != (m->kind[k] == SPECULA_WFS_PYR)) continue;
      const int n = P.S[k].n_pix;
      c_coords[k] = new_ctr();
      const int ne = n_layers * 2 * n;
      for (int e0 = 0; e0 < ne; e0 += kMwCoordsPerTask) {
        L_coords.push_back(mk(MT_COORDS, k, e0, std::min(ne, e0 + kMwCoordsPerTask), -1, 0,
                              c_coords[k]));
        n_coords[k]++;
      }
    }
  for (int k = 0; k < n_sensors; ++k) {
    const MwSensor &S = P.S[k];
    const int n = S.n_pix;
    if (m->kind[k] == SPECULA_WFS_SH) {
      c_sh[k] = new_ctr();
      // runs of valid subapertures in one row spanning < 16 columns, so a
      // task's screen window stays small
      const std::vector<int32_t> &vl = m->valid_host[k];
      int v0 = 0;
      while (v0 < S.n_valid) {
        const int a0 = vl[v0] / S.n_sub, b0 = vl[v0] % S.n_sub;
        int v1 = v0 + 1;
        while (v1 < S.n_valid && v1 - v0 < kMwShSubPerTask && vl[v1] / S.n_sub == a0 &&
               vl[v1] % S.n_sub - b0 < kMwShSubPerTask)
          ++v1;
        L_sh_by[k].push_back(mk(MT_SH, k, v0, v1, c_coords[k], n_coords[k], c_sh[k]));
        n_sh[k]++;
        v0 = v1;
      }
      continue;
    }
    const int N = 2 * n;
    c_field[k] = new_ctr();
    const int rpt = std::max(1, kMwFieldPx / n);
    max_field_slots = std::max(max_field_slots, n + rpt);
    if (kMwLayerChunk * (n + rpt) > 4 * kMwThreads) return SPECULA_EUNSUPPORTED;
    for (int y0 = 0; y0 < n; y0 += rpt) {
      L_field.push_back(mk(MT_FIELD, k, y0, std::min(n, y0 + rpt), c_coords[k], n_coords[k],
                           c_field[k]));
      n_field[k]++;
    }
    const int nrg = (n + VPC - 1) / VPC, nct = N / TC, nsg = (S.nd + S.spt - 1) / S.spt;
    c_rinv[k] = new_ctr();
    for (int mm = 0; mm < S.n_mod; ++mm) {
      c_rows[k].push_back(new_ctr());
      c_cols[k].push_back(new_ctr());
    }
    for (int mm = 0; mm < S.n_mod; ++mm)
      for (int rg = 0; rg < nrg; ++rg)
        L_pyr.push_back(mk(MT_ROWS, k, mm, rg, c_field[k], n_field[k], c_rows[k][mm]));
    for (int mm = 0; mm < S.n_mod; ++mm)
      for (int ct = 0; ct < nct; ++ct)
        L_pyr.push_back(mk(MT_COLS, k, mm, ct, c_rows[k][mm], nrg, c_cols[k][mm]));
    for (int mm = 0; mm < S.n_mod; ++mm)
      for (int sg = 0; sg < nsg; ++sg)
        L_pyr.push_back(mk(MT_RINV, k, mm, sg, c_cols[k][mm], nct, c_rinv[k]));
    c_bin[k] = new_ctr();
    const int nd2 = S.nd * S.nd;
    for (int p0 = 0; p0 < nd2; p0 += kMwBinPerTask) {
      L_pyr.push_back(mk(MT_BIN, k, p0, std::min(nd2, p0 + kMwBinPerTask), c_rinv[k],
                         S.n_mod * nsg, c_bin[k]));
      n_binv[k]++;
    }
    c_slopes[k] = new_ctr();
    L_pyr.push_back(mk(MT_SLOPES, k, 0, 0, c_bin[k], n_binv[k], c_slopes[k]));
  }
  const int c_mvm = new_ctr(), c_final = new_ctr();
  int n_mvm = 0;
  if (n_modes > 0) {
    // pyramids' MVM first: their slopes come first in the ALU list
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < n_sensors; ++k) {
        const bool pyr = m->kind[k] == SPECULA_WFS_PYR;
        if ((pass == 0) != pyr) continue;
        for (int r0 = 0; r0 < n_modes; r0 += kMwMvmRows) {
          L_mvm.push_back(mk(MT_MVM, k, r0, std::min(n_modes, r0 + kMwMvmRows),
                             pyr ? c_slopes[k] : c_sh[k], pyr ? 1 : n_sh[k], c_mvm));
          n_mvm++;
        }
      }
    for (int r0 = 0; r0 < n_modes; r0 += kMwFinalRows)
      L_final.push_back(mk(MT_FINAL, 0, r0, std::min(n_modes, r0 + kMwFinalRows), c_mvm, n_mvm,
                           c_final));
  }
  // producers per counter, for the merge
  std::vector<int> produced(nctr, 0), emitted(nctr, 0);
  auto count = [&](const std::vector<MwTask> &v) { for (auto &t : v) produced[t.done_ctr]++; };
  count(L_coords); count(L_field); count(L_pyr); count(L_mvm); count(L_final);
  for (auto &v : L_sh_by) count(v);
  std::vector<MwTask> A, order;
  for (auto &t : L_coords) { order.push_back(t); emitted[t.done_ctr]++; }
  for (auto &t : L_field) { order.push_back(t); emitted[t.done_ctr]++; }
  // SH sensors one after another (each finishes early and its MVM tasks can
  // stream R from HBM while the rest compute), then the pyramid passes, whose
  // dependency chains the MVM tasks fill; the pyramids' own MVM tasks end
  // the frame.
  for (int k = 0; k < n_sensors; ++k) A.insert(A.end(), L_sh_by[k].begin(), L_sh_by[k].end());
  A.insert(A.end(), L_pyr.begin(), L_pyr.end());
  int sms = 0;
  SPECULA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  release_when_ready(A, L_mvm, produced, emitted, order, 4 * sms);
  for (auto &t : L_final) { order.push_back(t); emitted[t.done_ctr]++; }
  // every dependency precedes its consumer
  {
    std::vector<int> seen(nctr, 0);
    for (auto &t : order) {
      if (t.wait_ctr >= 0 && seen[t.wait_ctr] < t.wait_val) return SPECULA_EINVAL;
      seen[t.done_ctr]++;
    }
  }
  m->host_tasks = order;
  if ((st = m->tasks.upload(order.data(), order.size() * sizeof(MwTask)))) return st;
  if ((st = m->ctr.alloc((size_t)nctr * 4))) return st;
  SPECULA_CK(cudaMemset(m->ctr.p, 0, m->ctr.bytes));
  P.tasks = m->tasks.as<MwTask>();
  P.n_tasks = (int)order.size();
  P.ctr = m->ctr.as<int>();
  P.n_ctr = nctr;
  P.status = ctx->status_dev;
  P.wait_ns = kMwWaitNs;
  P.stall_task = -1;

  m->smem = var->smem(max_slopes, max_field_slots);
  if (m->smem > 227 * 1024) return SPECULA_EUNSUPPORTED;
  if ((st = ensure_dynamic_smem((const void *)var->fn, m->smem))) return st;
  int occ = 0;
  SPECULA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, var->fn, kMwThreads, m->smem));
  if (occ < 1) return SPECULA_EUNSUPPORTED;
  m->sm_count = sms;
  m->occupancy = occ;
  m->max_grid = sms * occ;
  m->grid = std::min(m->max_grid, P.n_tasks);
  SPECULA_CK(cudaDeviceSynchronize());
  *out = m.release();
  return SPECULA_OK;
}

extern "C" int specula_mwfs_destroy(specula_mwfs *m) {
  if (!m) return SPECULA_EINVAL;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  delete m;
  return SPECULA_OK;
}

extern "C" int specula_mwfs_info(const specula_mwfs *m, int32_t sensor, int32_t *n_valid,
                                 int32_t *slope_offset, int32_t *n_slopes_total) {
  if (!m) return SPECULA_EINVAL;
  if (n_slopes_total) *n_slopes_total = m->n_slopes;
  if (sensor < 0) return SPECULA_OK;
  if (sensor >= m->P.n_sensors) return SPECULA_EINVAL;
  if (n_valid) *n_valid = m->n_valid[sensor];
  if (slope_offset) *slope_offset = m->slope_off[sensor];
  return SPECULA_OK;
}

extern "C" int specula_mwfs_schedule(const specula_mwfs *m, int32_t *n_tasks, int32_t *grid,
                                     int32_t *max_grid) {
  if (!m) return SPECULA_EINVAL;
  if (n_tasks) *n_tasks = m->P.n_tasks;
  if (grid) *grid = m->grid;
  if (max_grid) *max_grid = m->max_grid;
  return SPECULA_OK;
}

extern "C" int specula_mwfs_set_grid(specula_mwfs *m, int32_t ctas) {
  if (!m || ctas < 0) return SPECULA_EINVAL;
  m->grid = ctas == 0 ? std::min(m->max_grid, m->P.n_tasks) : std::min(ctas, m->max_grid);
  return SPECULA_OK;
}

extern "C" int specula_mwfs_set_wait(specula_mwfs *m, int64_t limit_ns, int32_t stall_task) {
  if (!m || limit_ns < 0 || limit_ns > kMwWaitMaxNs) return SPECULA_EINVAL;
  if (stall_task < -1 || stall_task >= m->P.n_tasks) return SPECULA_EINVAL;
  m->P.wait_ns = limit_ns == 0 ? kMwWaitNs : (unsigned long long)limit_ns;
  m->P.stall_task = stall_task;
  return SPECULA_OK;
}

static int mwfs_launch(specula_mwfs *m, double t_s, const double *t_dev, const float *ref_dev,
                       float *slopes_dev, float *modes_dev, int flat, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  MwParams P = m->P;
  P.t_host = t_s;
  P.t_dev = t_dev;
  P.flat = flat;
  P.ref = ref_dev;
  P.slopes = slopes_dev;
  P.modes = modes_dev;
  P.nf_status = m->ctx->guard ? m->ctx->status_dev : nullptr;
  SPECULA_LAUNCH(m->ctx, SPECULA_K_MWFS, st,
                 m->var->fn<<<m->grid, kMwThreads, m->smem, st>>>(P));
  return SPECULA_OK;
}

extern "C" int specula_mwfs_frame(specula_mwfs *m, double t_s, const double *t_dev,
                                  const float *ref_dev, float *slopes_dev, float *modes_dev,
                                  void *stream) {
  if (!m || !slopes_dev) return SPECULA_EINVAL;
  if (!t_dev && !isfinite(t_s)) return SPECULA_EINVAL;
  if ((m->P.n_modes > 0) != (modes_dev != nullptr)) return SPECULA_EINVAL;
  return mwfs_launch(m, t_s, t_dev, ref_dev, slopes_dev, modes_dev, 0, stream);
}

extern "C" int specula_mwfs_reference(specula_mwfs *m, float *ref_dev, float *modes_dev,
                                      void *stream) {
  if (!m || !ref_dev) return SPECULA_EINVAL;
  if ((m->P.n_modes > 0) != (modes_dev != nullptr)) return SPECULA_EINVAL;
  return mwfs_launch(m, 0.0, nullptr, nullptr, ref_dev, modes_dev, 1, stream);
}

extern "C" int specula_mwfs_read(const specula_mwfs *m, int32_t sensor, int32_t what,
                                 float *dst_dev, void *stream) {
  if (!m || !dst_dev || sensor < 0 || sensor >= m->P.n_sensors) return SPECULA_EINVAL;
  const MwSensor &S = m->P.S[sensor];
  if (what == SPECULA_MWFS_PHASE)
    SPECULA_CK(cudaMemcpyAsync(dst_dev, S.phase, (size_t)S.n_pix * S.n_pix * 4,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  else if (what == SPECULA_MWFS_DETECTOR && S.kind == SPECULA_WFS_PYR)
    SPECULA_CK(cudaMemcpyAsync(dst_dev, S.det, (size_t)S.nd * S.nd * 4,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  else
    return SPECULA_EINVAL;
  return SPECULA_OK;
}
