// Internal declarations shared by the translation units of libspecula_gb300.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <vector>

#include "../../include/specula_gb300.h"

namespace specula {
// the CUDA error behind the calling thread's last SPECULA_ECUDA (api.cu)
void note_cuda_error(cudaError_t e, const char *file, int line);
}

#define SPECULA_CK(call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) {                               \
      specula::note_cuda_error(e_, __FILE__, __LINE__);    \
      return SPECULA_ECUDA;                                \
    }                                                      \
  } while (0)

#define SPECULA_CK_LAUNCH()                                \
  do {                                                     \
    cudaError_t e_ = cudaGetLastError();                   \
    if (e_ != cudaSuccess) {                               \
      specula::note_cuda_error(e_, __FILE__, __LINE__);    \
      return SPECULA_ECUDA;                                \
    }                                                      \
  } while (0)

namespace specula {

// Every buffer the library allocates carries kGuardBytes of a fixed pattern
// past its end.  A kernel that writes past its workspace lands there rather
// than in a neighbouring allocation, which would not fault;
// specula_check_guards compares the bands (api.cu keeps the live buffers).
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
struct DevBuf;
void guard_register(DevBuf *b);
void guard_unregister(DevBuf *b);

// A device buffer owned by a plan.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  int device = -1;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (!p) return;
    guard_unregister(this);
    cudaFree(p);
    p = nullptr;
  }
  int alloc(size_t n) {
    release();
    bytes = n;
    if (n == 0) return SPECULA_OK;
    if (cudaMalloc(&p, n + kGuardBytes) != cudaSuccess) {
      p = nullptr;
      return SPECULA_ENOMEM;
    }
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaMemset(static_cast<char *>(p) + n, kGuardByte, kGuardBytes) != cudaSuccess) {
      cudaFree(p);
      p = nullptr;
      return SPECULA_ECUDA;
    }
    guard_register(this);
    return SPECULA_OK;
  }
  int upload(const void *h, size_t n) {
    int s = alloc(n);
    if (s) return s;
    return cudaMemcpy(p, h, n, cudaMemcpyHostToDevice) == cudaSuccess ? SPECULA_OK : SPECULA_ECUDA;
  }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// Pyramid plan: tables and the per-chunk intermediate workspace.
struct PwfsPlan {
  int n_pix, pad, n_mod, n_sub, pup_dist;
  double mod_amp;
  int N, N1, N2;
  int chunk;            // modulation items per pipeline chunk
  int ka;               // items per row group in the row-forward pass
  int nbw;              // field slots: batch elements one chunk can touch
  int blockA, blockB, blockC;
  size_t smemA, smemB, smemC;
  int passes;           // 2: row filter + column filter/bins; 3: rows, cols, rows
  int nc;               // row-filter slots per batch element (distinct cosines)
  int slot_lo = 0;      // cosine slots [slot_lo, slot_hi) imaged (slot_hi < 0: all)
  int slot_hi = -1;
  bool two_ok;          // the two-pass form fits this geometry
  int blockR, blockK;   // two-pass blocks (K: TC columns x G lanes)
  size_t smemR, smemK;
  int csK = 0;                      // column stride of the column-pass tile (complex)
  // a detector pixel is fp / fq grid pixels (N / (pad n_sub) in lowest
  // terms; fq = 1: fp x fp binning, else area-weighted rebinning)
  int fp = 1, fq = 1;
  DevBuf gx, gy;        // [n_mod][n_pix] float2: tilt x pre-phase (x and y parts)
  DevBuf mask;          // [N] float2: pyramid mask factor per axis, x (1/N)
  DevBuf twA, twB;      // [N] float2: inter-step twiddles (cos, sin)
  DevBuf field;         // [nbw][n_pix][n_pix] float2: E = amp exp(i phase)
  DevBuf rows;          // [chunk][n_pix][N] float2: after the row transform
  DevBuf cols;          // [chunk][N][N] float2: after the column pass (three-pass form)
  DevBuf part;          // [chunk][nd][nd] float: binned intensity per item
  // per-call settings of the polychromatic image (defaults: a plain image):
  // the phase is multiplied by run_phase_scale and the detector becomes
  // run_beta det + run_alpha image
  float run_phase_scale = 1.f, run_alpha = 1.f, run_beta = 0.f;
  // shifted-mask form (SPECULA_PWFS_FORM_SHIFTED)
  int form = 0;
  int sm_blockK = 0, sm_chunk = 0;
  size_t sm_smemK = 0, sm_smemR = 0, sm_smemC = 0;
  DevBuf sm_pre;        // [Np] float2: centred-DFT input phase over the pupil
  DevBuf sm_mx, sm_my;  // [nc][N], [n_mod][N] float2: shifted mask factors / N
  DevBuf sm_frows;      // [Np][N] float2: after the forward row transform
  DevBuf sm_fspec;      // [N][N] float2: the field's spectrum
  DevBuf sm_rows;       // [sm_chunk][N][N] float2 (+2): after the inverse row transform
  DevBuf sm_part;       // [n_mod][nd][nd] float: binned intensity per point
  // two-pass form with packed-pair arithmetic (passes == 4, pwfs_pair.cu)
  bool pair_ok = false;
  int pair_blockR = 0, pair_blockK = 0;
  size_t pair_smemR = 0, pair_smemK = 0;
  DevBuf twA2, twB2;    // [N] float4 (re, re, im, im): inter-step twiddles
  DevBuf mask2;         // [N] float4: mask factor per axis, x (1/N)
  DevBuf gx2;           // [n_mod][n_pix] float4: x factor of the tilt x pre-phase
  DevBuf pair_units;    // [n_pair_units] int4: (slot a, point a, slot b, point b or -1)
  DevBuf gyp;           // [n_pair_units][n_pix] float4: the units' y factors (re_a, re_b, im_a, im_b)
  int n_pair_units = 0;
  int pair_units_for = -1;   // the slot range the unit table was built for
  std::vector<float2> gy_host;
  // DFT-as-GEMM forms (pwfs_dftgemm.cu)
  int dg_form = -1;     // the form the operator below was built for
  int dg_M1 = 0, dg_M2 = 0;
  DevBuf dg_B;          // [2N][6 n_pix] split operator (bf16 or float32/tf32)
  DevBuf dg_A1, dg_A2;  // split operands of the row and column GEMMs
  DevBuf dg_C1, dg_C2;  // [M][2N] float32 products
  DevBuf dg_work;       // split-K partials of the row GEMM
};

struct ShPlan {
  int n_pix, n_sub, sub_pix, fft_n;
  double obsc = 0.0;   // the pupil's obscuration (the valid list depends on it)
  int n_valid;
  int sub_lo = 0, sub_hi = -1;   // imaged valid subapertures [sub_lo, sub_hi) (-1: all)
  DevBuf valid;         // [n_valid] int32
  DevBuf pre;           // [fft_n] float2: centred-DFT input phase
  DevBuf tw;            // [fft_n] float2 twiddles
};

}  // namespace specula

// capacity of the per-context extraction coordinate table
#define SPECULA_ATMO_MAX_LAYERS 64
#define SPECULA_ATMO_MAX_PIX 8192

struct specula_ctx {
  int device = 0;
  int32_t *status_dev = nullptr;
  double *loop_part = nullptr;      // [kLoopMaxBlocks][5] closed-loop statistics partials
  bool guard = true;                // slope kernels record non-finite outputs
  int *atmo_tab_i = nullptr;        // [64][2][8192] screen sample index
  float *atmo_tab_f = nullptr;      // [64][2][8192] interpolation fraction
  std::vector<std::unique_ptr<specula::PwfsPlan>> pwfs;
  std::vector<std::unique_ptr<specula::ShPlan>> sh;
  // tracing: kernels launched, and optional per-kernel CUDA-event pairs
  int64_t launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev;      // 2 per record
  size_t ev_next = 0;
  std::vector<int> rec_kid;         // kernel id of record i (events 2i, 2i+1)
  // batched bf16 reconstructor products: the slopes' bf16 halves and the
  // split-K partials (grown on demand outside stream capture)
  specula::DevBuf recon_ws;
  // one wavelength's spots of the polychromatic Shack-Hartmann (grown on
  // demand outside stream capture)
  specula::DevBuf sh_poly_ws;
};

namespace specula {

// Bracket one kernel launch with events on its stream when tracing is on.
inline int prof_begin(specula_ctx *c, cudaStream_t st) {
  c->launches++;
  if (!c->prof || c->ev_next + 2 > c->ev.size()) return -1;
  const int slot = (int)c->ev_next;
  c->ev_next += 2;
  cudaEventRecord(c->ev[slot], st);
  return slot;
}
inline void prof_end(specula_ctx *c, int slot, int kid, cudaStream_t st) {
  if (slot < 0) return;
  cudaEventRecord(c->ev[slot + 1], st);
  c->rec_kid.push_back(kid);   // capacity reserved when tracing is enabled
}

#define SPECULA_LAUNCH(ctx, kid, st, ...)            \
  do {                                               \
    const int slot_ = prof_begin((ctx), (st));       \
    __VA_ARGS__;                                     \
    SPECULA_CK_LAUNCH();                             \
    prof_end((ctx), slot_, (kid), (st));             \
  } while (0)
// per-translation-unit device initialisation (constant tables)
int pwfs_init_device();
int sh_init_device();
int mwfs_init_device();
// float64 helpers of the calibration file, shared with the infinite screens:
// C[i][j] = sum_k X(i,k) d(k) Y(k,j), X(i,k) = X[i xi + k xk], Y(k,j) = Y[k yk + j yj]
// (d may be NULL); and the Jacobi eigen-decomposition of a symmetric matrix
// (eigenvalues on G's diagonal, eigenvectors in V's columns).
int gemm_f64(specula_ctx *ctx, cudaStream_t st, const double *X, long xi, long xk,
             const double *Y, long yk, long yj, const double *d, double *C, int M, int N, int K);
int sym_eig_f64(specula_ctx *ctx, cudaStream_t st, double *G, double *V, int n);
constexpr int kLoopMaxBlocks = 512;
int loop_alloc_workspace(specula_ctx *ctx);
int pwfs_shifted_init_device();
int pwfs_shifted_prepare(PwfsPlan *p);
int pwfs_shifted_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                     int n_batch, float *det, cudaStream_t st);
int pwfs_bin_reduce(specula_ctx *ctx, const float *part, float *det, int nd2, int n_mod,
                    float alpha, float beta, cudaStream_t st);
// the field of batch elements fb .. fb + nb - 1 into the plan's field slots,
// and their detectors from the plan's per-point bins
int pwfs_field_launch(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                      int fb, int nb, cudaStream_t st);
int pwfs_bin_reduce_range(specula_ctx *ctx, PwfsPlan *p, float *det, int nd2, int b0, int nb,
                          cudaStream_t st);
struct PwfsTablesHost;
int pwfs_pair_init_device();
int pwfs_dftgemm_prepare(PwfsPlan *p, int form);
int pwfs_dftgemm_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                     int n_batch, float *det, cudaStream_t st);
int pwfs_pair_configure(PwfsPlan *p);
int pwfs_pair_tables(PwfsPlan *p, const PwfsTablesHost &T);
int pwfs_pair_run(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                  int n_batch, float *det, cudaStream_t st);
int atmo_alloc_tables(specula_ctx *ctx);

// launchers implemented in the kernel translation units
int pwfs_plan_build(specula_ctx *ctx, const specula_pupil_desc *pupil,
                    const specula_pwfs_desc *pwfs, PwfsPlan **out);
PwfsPlan *pwfs_plan_find(specula_ctx *ctx, const specula_pupil_desc *pupil,
                         const specula_pwfs_desc *pwfs);
int pwfs_set_tiles(PwfsPlan *p, int chunk, int ka, int passes);
int pwfs_autotune(specula_ctx *ctx, PwfsPlan *p, const float *amp, const float *phase,
                  int n_batch, float *det, cudaStream_t st, int reps, size_t max_ws_bytes,
                  int *best_chunk, int *best_ka, int *best_passes);
int pwfs_run(specula_ctx *ctx, PwfsPlan *plan, const float *amp, const float *phase,
             int n_batch, float *det, cudaStream_t st);
int sh_plan_build(specula_ctx *ctx, const specula_pupil_desc *pupil,
                  const specula_sh_desc *sh, ShPlan **out);
ShPlan *sh_plan_find(specula_ctx *ctx, const specula_pupil_desc *pupil,
                     const specula_sh_desc *sh);
int sh_run(specula_ctx *ctx, ShPlan *plan, const float *amp, const float *phase,
           int n_batch, float *spots, cudaStream_t st, float phase_scale = 1.0f);
// out = (first ? 0 : out) + weight ratio^2 W spots W^T for n_spots fft_n^2
// spots of one wavelength (ratio = lambda_ref / lambda): the polychromatic SH
int sh_poly_acc(specula_ctx *ctx, int fft_n, const float *spots, int n_spots, double ratio,
                double weight, bool first, float *out, cudaStream_t st);

// Raise (never lower) a kernel's dynamic shared-memory limit to `bytes` on
// the current device.  The limit belongs to the function, shared by every
// plan that launches it, so a later plan with a smaller need must not shrink
// what an earlier one relies on.  Needs up to 48 KB need no call.
int ensure_dynamic_smem(const void *fn, size_t bytes);

int gemm_check(const void *A, const void *B, int M, int N, int K, bool tf32 = false);
int gemm_splits(int K, int want, bool tf32 = false);
int gemm_tf32_tn(specula_ctx *ctx, const float *A, const float *B, int M, int N, int K, float *C,
                 int splits, float *work, cudaStream_t st);
int gemm_bf16_tn(specula_ctx *ctx, const void *A, const void *B, int M, int N, int K, float *C,
                 int splits, float *work, cudaStream_t st);
// C = sum over t < n_terms (<= 3) of A_t B_t^T, one accumulation on the
// tensor cores (split-precision products); every A_t is M x K, every B_t is
// N x K, bf16, row-major
int gemm_bf16_terms(specula_ctx *ctx, int n_terms, const void *const *A, const void *const *B,
                    int M, int N, int K, float *C, int splits, float *work, cudaStream_t st);

int slopes_pyr_run(specula_ctx *ctx, const int32_t *idx, int n_sub, int n_valid,
                   const float *det, const float *ref, int n_batch, float *out, cudaStream_t st);

bool pwfs_split_for(int N, int *N1, int *N2);

// host geometry (api.cu)
int host_pupil_mask(int n, double obsc, uint8_t *mask);
int host_valid_subaps(int n, double obsc, int n_sub, int32_t *idx, int32_t *n_valid);
}  // namespace specula
