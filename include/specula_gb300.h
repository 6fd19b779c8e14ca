/*
 * specula_gb300 — C ABI of the GB300-native wavefront-sensor hot path.
 *
 * One frame of an adaptive-optics simulation's sensing chain, as the paper's
 * processing objects compute it (App. A, Tab. 4): AtmoEvolution +
 * AtmoPropagation (layer extraction), ModulatedPyramid / SH (sensor image),
 * CCD (binning, noise off), PyrSlopec / ShSlopec (slopes) and Modalrec
 * (reconstructor matrix-vector product), with the parameters of App. B,
 * Listing 2.  The paper prints no equation for these objects; the formulas
 * each call implements are stated beside it.
 *
 * Conventions shared by every call
 *  - Arrays are row-major [y][x].  Grids are centred: sample i of a side-n grid
 *    sits at i - (n-1)/2.
 *  - "*_dev" pointers are device memory owned by the caller; "*_host" pointers
 *    are host memory owned by the caller.  The library keeps no pointer
 *    beyond the call unless a plan call says so.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Per-frame
 *    calls (atmo_extract, pwfs_image, sh_image, slopes, recon) only enqueue
 *    kernels: they allocate nothing and never synchronise the host, so they
 *    can be captured into a CUDA graph (the rule of Sect. 2.3 for a
 *    processing object's trigger phase).  Plan calls may allocate.
 *  - Every call validates its arguments on the host and returns a negative
 *    status before launching anything.  Device-side conditions (non-finite
 *    guard, bounded waits) are recorded in a per-context status word read by
 *    specula_ctx_status.
 *  - One context per device per host thread; calls on one context are not
 *    thread-safe.
 */
#ifndef SPECULA_GB300_H
#define SPECULA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define SPECULA_OK            0
#define SPECULA_EINVAL       -1  /* bad argument (null pointer, size, range)   */
#define SPECULA_ENOMEM       -2  /* device or host allocation failed           */
#define SPECULA_ECUDA        -3  /* a CUDA runtime call failed                 */
#define SPECULA_ETIMEOUT     -4  /* a bounded device wait expired              */
#define SPECULA_EUNSUPPORTED -5  /* valid request outside the built sizes      */
#define SPECULA_ENONFINITE   -6  /* non-finite value seen by a guarded kernel  */
#define SPECULA_ENOPLAN      -7  /* per-frame call without a matching plan     */

/* Human-readable text of a status code (static storage; never NULL). */
const char *specula_strerror(int status);

/* Text of the CUDA error behind the calling thread's last SPECULA_ECUDA
 * (error name, description, source location); "" if none yet.  Static
 * thread-local storage, valid until the thread's next failing call. */
const char *specula_last_cuda_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int specula_version(void);

/* ---- descriptors -------------------------------------------------------- */

/* Telescope pupil sampled on n_pix x n_pix pixels of pitch_m metres with a
 * central obscuration obsc_frac of the diameter (PupilStop, App. A, Tab. 3;
 * Listing 2 `pixel_pupil`, `pixel_pitch`). */
typedef struct {
  int32_t n_pix;
  double pitch_m;
  double obsc_frac;
} specula_pupil_desc;

/* Guide star: direction (radians on sky), height (INFINITY for a natural
 * star; finite for a laser star, which compresses each layer's footprint by
 * 1 - h/height) and wavelength (Source, App. A, Tab. 3; Listing 2
 * `polar_coordinates`, `wavelengthInNm`). */
typedef struct {
  double theta_x_rad, theta_y_rad, height_m, wavelength_nm;
} specula_source_desc;

/* One frozen-flow turbulence layer: side x side screen of pitch_m metres at
 * height_m, translated by the wind (vx, vy) m/s (Layer, App. A, Tab. 3;
 * AtmoEvolution in Listing 2). */
typedef struct {
  int32_t side;
  double pitch_m, height_m, vx_mps, vy_mps;
} specula_layer_desc;

/* Modulated pyramid (ModulatedPyramid, Listing 2): FFT side N = pad * n_pix;
 * n_mod modulation points on a circle of mod_amp lambda/D; a pad n_sub
 * detector (output_resolution) with n_sub pixels across each pupil image;
 * pup_dist_px = separation of the pupil images' centres in grid pixels.
 * A detector pixel is b = n_pix / n_sub grid pixels: a whole b is b x b
 * binning; a fractional b (the SOUL example: 220 / 40 = 5.5) is
 * area-weighted rebinning, each detector pixel collecting the overlapped
 * area of every grid pixel, the intensity constant over a grid pixel.
 * Supported: pad 2-4 with N one of 64, 128, 240, 320, 660 (pad 3 or 4),
 * 960, 1600 (pad 4: the ANDES grid of Sect. 6, Tab. 2, a 400 px pupil);
 * pup_dist_px + n_pix <= N (the images inside the grid); column tiles of
 * whole detector pixels within 352 threads (128 at N = 1600);
 * SPECULA_EUNSUPPORTED else.  With pad 2 and pup_dist_px = n_pix the four
 * images tile the grid (quadrant slopes); otherwise read the slopes with
 * SPECULA_SLOPES_PYR_MAPS.
 * The three-pass, shifted-mask, paired and DFT-as-GEMM forms need pad 2 and
 * a whole b. */
typedef struct {
  int32_t pad, n_mod, n_sub, pup_dist_px;
  double mod_amp;
} specula_pwfs_desc;

/* Shack-Hartmann (SH / Lenslet, App. A, Tabs. 3-4): n_sub x n_sub lenslets of
 * sub_pix pupil pixels, each imaged with an fft_n x fft_n DFT. */
typedef struct {
  int32_t n_sub, sub_pix, fft_n;
} specula_sh_desc;

#define SPECULA_SLOPES_PYR      0
#define SPECULA_SLOPES_SH       1
#define SPECULA_SLOPES_PYR_MAPS 2

/* Slope computer (PyrSlopec / ShSlopec, App. A, Tab. 4).  subap_idx_dev lists
 * the valid subapertures as a * n_sub + b (row a, column b), ascending; for
 * SH, the image holds one fft_n^2 spot per listed subaperture.  For
 * PYR_MAPS, subap_idx_dev holds 4 n_valid detector linear indices (the
 * subapertures' pixels in images Q1, Q2, Q3, Q4, one block each; see
 * specula_pyr_image_index_host) and n_sub is the detector side. */
typedef struct {
  int32_t kind;            /* SPECULA_SLOPES_PYR, _SH or _PYR_MAPS      */
  int32_t n_sub;           /* subapertures across one pupil image (PYR,
                              SH); detector side (PYR_MAPS)             */
  int32_t n_valid;         /* entries of subap_idx_dev                  */
  int32_t fft_n;           /* SH spot side (ignored for PYR)            */
  const int32_t *subap_idx_dev;
} specula_slopec_desc;

#define SPECULA_PREC_FP32   0   /* R in float32                                   */
#define SPECULA_PREC_BF16   1   /* R rounded to bfloat16                          */
#define SPECULA_PREC_BF16X2 2   /* R = hi + lo, both bfloat16 (split precision)   */

/* Linear modal reconstructor (Modalrec / Recmat, Listing 2 `recmat_object`):
 * R is n_modes x n_slopes, row-major.  FP32: R_dev is float*.  BF16: R_dev is
 * the bfloat16 copy.  BF16X2: R_dev = hi, R_lo_dev = lo (see
 * specula_recon_convert). */
typedef struct {
  int32_t n_modes, n_slopes, precision;
  const void *R_dev;
  const void *R_lo_dev;
} specula_recon_desc;

/* ---- context -------------------------------------------------------------- */
typedef struct specula_ctx specula_ctx;

/* Create a context on CUDA device `device`: selects the device, uploads the
 * FFT codelet twiddle tables and allocates the device status word.
 * May allocate.  *out is set on success. */
int specula_ctx_create(specula_ctx **out, int device);

/* Destroy a context and every plan it owns.  Synchronises the device. */
int specula_ctx_destroy(specula_ctx *ctx);

/* Wait for the device, return the device status word (SPECULA_OK if no
 * device-side condition was recorded) in *device_status and clear it. */
int specula_ctx_status(specula_ctx *ctx, int32_t *device_status);

/* Non-finite guard (on by default).  While on, every slope computer (the
 * pyramid and Shack-Hartmann slope calls, the slope stages of the
 * multi-sensor launch) records SPECULA_ENONFINITE in the device status word
 * when one of its outputs is NaN or infinite (a NaN in a phase screen, a
 * dark pupil).  The outputs are still written.  `on` is 0 or 1; takes effect
 * for launches made after the call. */
int specula_ctx_set_guard(specula_ctx *ctx, int32_t on);

/* Workspace guard bands (failure detection of this library; the paper has
 * no counterpart).  Every device buffer the library allocates (plan
 * tables and workspaces, the multi-sensor and learned-reconstructor buffers)
 * is followed by 256 bytes of the pattern 0xA5.  A kernel that writes past
 * its workspace stays inside the allocation, so the write does not fault;
 * this call finds it afterwards.  Synchronises the device, then compares the
 * band of every live library buffer on the context's device: *n_checked =
 * the buffers compared, *n_bad = those whose band changed (0 when no kernel
 * wrote out of bounds).  Host-synchronous; not for use inside a capture.
 * Buffers the caller owns (inputs, outputs) are not covered. */
int specula_check_guards(specula_ctx *ctx, int32_t *n_checked, int32_t *n_bad);

/* ---- tracing -----------------------------------------------------------------
 * LoopControl reports the simulation speed (Sect. 2.4); these calls give the
 * per-kernel view behind it.  Kernel ids: */
#define SPECULA_K_PWFS_ROWS_FWD 0   /* pyramid pass A: field, tilt, row FFT       */
#define SPECULA_K_PWFS_COLS     1   /* pyramid pass B: column FFT, mask, IFFT     */
#define SPECULA_K_PWFS_ROWS_INV 2   /* pyramid pass C: row IFFT, |E|^2, binning   */
#define SPECULA_K_ATMO          3   /* layer extraction                           */
#define SPECULA_K_SLOPES        4   /* slope computers                            */
#define SPECULA_K_RECON         5   /* reconstructor MVM                          */
#define SPECULA_K_SH            6   /* Shack-Hartmann spots                       */
#define SPECULA_K_PWFS_FIELD    7   /* pyramid: field E = amp exp(i phase)        */
#define SPECULA_K_PWFS_BIN      8   /* pyramid: per-item bins -> detector         */
#define SPECULA_K_CALIB         9   /* calibration kernels (IM, float64 algebra)  */
#define SPECULA_K_GEMM          10  /* tcgen05 BF16 GEMM and split-K reduction    */
#define SPECULA_K_MLP           11  /* learned-reconstructor element-wise kernels */
#define SPECULA_K_MWFS          12  /* multi-sensor frame, one persistent launch  */
#define SPECULA_K_PWFS_ROWFILT  13  /* pyramid two-pass form: row filter          */
#define SPECULA_K_PWFS_COLFILT  14  /* pyramid two-pass form: column filter, bins */
#define SPECULA_K_PWFS_SM_FWD   15  /* shifted-mask form: forward 2-D transform   */
#define SPECULA_K_PWFS_SM_ROWS  16  /* shifted-mask form: row pass                */
#define SPECULA_K_PWFS_SM_COLS  17  /* shifted-mask form: column pass, bins       */
#define SPECULA_K_LOOP          18  /* closed loop: mirror shape, residual, update */
#define SPECULA_K_CCD           19  /* detector photon and readout noise          */
#define SPECULA_K_INFSCREEN     20  /* infinite screens: set-up and line growth   */
#define SPECULA_K_PEAK          21  /* fused multiply-add rate probe              */
#define SPECULA_K_PWFS_DFTGEMM  22  /* pyramid DFT-as-GEMM form: packing, bins    */
#define SPECULA_K_COUNT         23

/* Enable (capacity > 0: room for that many kernel records; allocates CUDA
 * events; set-up call) or disable (capacity = 0) per-kernel event timing.
 * While enabled, each kernel a per-frame call launches is bracketed by a pair
 * of events recorded on its own stream (eager launches only; do not enable
 * while capturing a graph).  Records beyond capacity are dropped. */
int specula_prof_enable(specula_ctx *ctx, int32_t capacity);

/* Synchronise, then return for each kernel id k < SPECULA_K_COUNT the summed
 * elapsed milliseconds ms_host[k] and the number of records n_host[k] since
 * the last read (arrays of SPECULA_K_COUNT entries), and clear the records. */
int specula_prof_read(specula_ctx *ctx, double *ms_host, int64_t *n_host);

/* Arithmetic peak probe (a measurement utility; the paper has no
 * counterpart): n_ctas CTAs of 256 threads; each thread runs 8
 * independent fused multiply-add chains of n_iter steps in float32 (bits 32)
 * or float64 (bits 64) and writes one value to sink_dev (n_ctas * 256
 * elements of that type).  Work: 2 * 8 * n_iter * 256 * n_ctas flops; timed
 * with events on the stream it gives the part's FMA rate (the roof of
 * CUDA-core arithmetic).  n_ctas 1..65535, n_iter 1..2^24.  One kernel. */
int specula_fma_probe(specula_ctx *ctx, int32_t bits, int32_t n_ctas, int32_t n_iter,
                      void *sink_dev, void *stream);

/* Number of kernels this context has launched since it was created. */
int specula_launch_count(specula_ctx *ctx, int64_t *count);

/* ---- frame graphs ---------------------------------------------------------------
 * The processing objects' trigger phase is captured once into a CUDA graph
 * and replayed every time step (Sect. 2.3, `build_stream`).  begin starts a
 * thread-local capture on `stream` (a created stream, not the legacy NULL
 * stream); every per-frame call issued on that stream until end is
 * recorded, not run; end instantiates the graph.  A frame that must advance
 * in time reads t from device memory (specula_atmo_extract t_dev), which the
 * caller updates before each launch.  Tracing must be disabled while
 * capturing.  begin/end may allocate; launch only enqueues. */
typedef struct specula_graph specula_graph;
int specula_graph_begin(specula_ctx *ctx, void *stream);
int specula_graph_end(specula_ctx *ctx, void *stream, specula_graph **out);
int specula_graph_launch(specula_graph *graph, void *stream);
/* Number of kernel nodes in the graph. */
int specula_graph_kernel_count(specula_graph *graph, int64_t *count);
int specula_graph_destroy(specula_graph *graph);

/* ---- integer geometry (host; bit-exact; no GPU needed) ---------------------
 * Pupil stop (PupilStop): pixel (j, i) is inside iff
 *   r4 = (2i - n + 1)^2 + (2j - n + 1)^2 <= n^2  and  r4 > (obsc * n)^2,
 * the last bound as the float64 product e * e, e = obsc_frac * n_pix.
 * Writes n_pix^2 bytes (1 inside, 0 outside) to mask_host. */
int specula_pupil_mask_host(const specula_pupil_desc *pupil, uint8_t *mask_host);

/* Valid subapertures (PupData / SubapData; PyrPupdataCalibrator /
 * ShSubapCalibrator, App. A, Tab. 4; geometric reading of the flux threshold):
 * a subaperture of b x b pupil pixels (b = n_pix / n_sub, whole or
 * fractional; 1 <= n_sub <= n_pix) is valid iff at least half of its area is
 * inside the stop, evaluated exactly with each pixel's overlap of the
 * subaperture in units of 1 / n_sub (for a whole b: 2 * (pixels inside) >=
 * b^2).  Writes the ascending linear indices a * n_sub + b to idx_host
 * (capacity n_sub^2) and their count to *n_valid. */
int specula_valid_subaps_host(const specula_pupil_desc *pupil, int32_t n_sub,
                              int32_t *idx_host, int32_t *n_valid);

/* Detector indices of the four pupil images of each valid subaperture for
 * any padding and image separation (PyrPupdataCalibrator; the SOUL example's
 * pup_diam / pup_dist / output_resolution, App. B, Listing 2).  The padded
 * grid (pad n_pix) sampled in detector pixels of b x b grid pixels (b =
 * n_pix / n_sub) is an n_det = pad n_sub detector; image Q, n_sub pixels wide, is centred
 * d = pup_dist_px / (2 b) pixels from the detector centre along (sx, sy) =
 * (+,+) Q1, (-,+) Q2, (-,-) Q3, (+,-) Q4 (face (+x, +y) to larger row and
 * column); subaperture (a, c) of image Q is at row n_det/2 + sy d - n_sub/2
 * + a, column n_det/2 + sx d - n_sub/2 + c.  Writes 4 n_valid indices (Q1
 * block first) to idx_host (capacity 4 n_sub^2) and *n_valid.
 * SPECULA_EUNSUPPORTED unless the image corners are whole detector pixels
 * (pup_dist_px / b = pup_dist_px n_sub / n_pix a whole number, it minus
 * n_sub and n_det even) and the images lie on the detector; b may be
 * fractional (the SOUL example: 220 px pupil, 40 subapertures, 5.5 grid
 * pixels per detector pixel, pup_dist_px 264 -> images 48 pixels apart).  With pad 2 and pup_dist_px = n_pix the
 * blocks are the quadrant layout of SPECULA_SLOPES_PYR. */
int specula_pyr_image_index_host(const specula_pupil_desc *pupil, int32_t pad,
                                 int32_t pup_dist_px, int32_t n_sub, int32_t *idx_host,
                                 int32_t *n_valid);

/* Modulation points (ModulatedPyramid `mod_amp`): theta_m = (2 pi m) / n_mod,
 * m = 0..n_mod-1, counter-clockwise from +x; writes cos/sin in float64. */
int specula_mod_table_host(int32_t n_mod, double *cos_host, double *sin_host);

/* ---- integer geometry on the device ----------------------------------------
 * Same rules as the host versions, computed by kernels (bit-exact). */
int specula_pupil_mask(specula_ctx *ctx, const specula_pupil_desc *pupil,
                       float *amp_dev, void *stream);
/* idx_dev: capacity n_sub^2 int32; n_valid_dev: one int32. */
int specula_valid_subaps(specula_ctx *ctx, const specula_pupil_desc *pupil,
                         int32_t n_sub, int32_t *idx_dev, int32_t *n_valid_dev,
                         void *stream);

/* ---- phase screens (set-up; may allocate) -----------------------------------
 * Von Karman screen by the FFT method (AtmoEvolution, App. A, Tab. 4; Listing
 * 2 `L0`, `Cn2`, `seed`), radians at 500 nm:
 *   Phi(f) = 0.023 r0^(-5/3) (|f|^2 + L0^-2)^(-11/6), Phi(0) = 0;
 *   screen[y][x] = Re sum_k c_k sqrt(Phi(f_k)) df exp(2 pi i f_k.(x,y) pitch),
 * f_k = signed FFT index / (side pitch), df = 1 / (side pitch); plus three
 * levels of subharmonics (spacing df/3^p, the eight non-zero offsets of a
 * 3 x 3 grid, same amplitude rule) whose sum has its mean removed.
 * noise_dev: side*side complex float64 (interleaved re, im), element
 * [ky][kx] for FFT indices (ky, kx).  noise_sub_host: 3*3*3 complex float64
 * [p][b][a] for level p+1, offset (a-1, b-1).  L0_m = INFINITY: Kolmogorov.
 * Computed in float64 on the device and rounded to float32 once.  side must
 * be a power of two in [32, 4096]. */
int specula_screen_generate(specula_ctx *ctx, int32_t side, double pitch_m,
                            double r0_m, double L0_m, const double *noise_dev,
                            const double *noise_sub_host, float *screen_dev,
                            void *stream);

/* Counter-based normals (Philox4x32-10, Salmon et al., SC 2011; uniforms
 * (x + 0.5) 2^-32, Box-Muller): for sample b in [sample0, sample0 +
 * n_samples), n_per_sample complex values, element 2i and 2i+1 from counter
 * (i low, i high, b, stream_id) with key (seed low, seed high).  out_dev:
 * n_samples * n_per_sample complex float64, interleaved. */
int specula_rng_complex(specula_ctx *ctx, uint64_t seed, int32_t sample0, int32_t n_samples,
                        int32_t stream_id, int64_t n_per_sample, double *out_dev, void *stream);

/* Batch of independent von Karman screens (same construction as
 * specula_screen_generate) whose noise is drawn on the device: screen b uses
 * the Philox complex normals of sample sample0 + b, stream 0 for the FFT
 * grid (element ky * side + kx) and stream 1 for the 27 subharmonic values
 * (element (p * 3 + b) * 3 + a).  screens_dev: n_screens * side^2 floats.
 * Set-up call: allocates at most 1 GiB of float64 work arrays. */
int specula_screen_generate_batch(specula_ctx *ctx, int32_t n_screens, int32_t side,
                                  double pitch_m, double r0_m, double L0_m, uint64_t seed,
                                  int32_t sample0, float *screens_dev, void *stream);

/* Random pupil phases from screens (AtmoRandomPhase, App. A, Tab. 4):
 * phase[b][j][i] = scale[b] * screen[b][j + o][i + o], o = (side - n_pix)/2,
 * for n screens; scale_dev: n floats (e.g. (r0_ref / r0_b)^(5/6) 500 /
 * lambda). */
int specula_random_phase(specula_ctx *ctx, const float *screens_dev, int32_t n, int32_t side,
                         int32_t n_pix, const float *scale_dev, float *phase_dev, void *stream);

/* ---- infinite phase screens ----------------------------------------------
 * InfinitePhaseScreen (Tab. 3) and AtmoInfiniteEvolution (Tab. 4).  The paper
 * names them without their construction; this follows the conditional growth
 * of Assemat, Wilson and Gendron (Optics Express 14, 988, 2006).  A screen is
 * a side x side ring: line L (a row, axis 0, or a column, axis 1) sits at
 * slot L mod side (rows: screen[slot][*], columns: screen[*][slot]).  It grows
 * one line at a time.  Each new line Z is drawn from its Gaussian distribution
 * given the stencil X: the n_st lines behind it, nearest first, full width.
 *   Z = A X + b_scale B b,   A = C_ZX C_XX^+,   B = (C_ZZ - A C_XZ)^(1/2).
 * Extraction reads such a ring unchanged: specula_atmo_extract's periodic
 * addressing is the ring's. */

/* Set-up: the operators of the draw.  C is the von Karman phase covariance, in
 * rad^2 at 500 nm, of the spectrum of specula_screen_generate:
 *   C(r) = 0.023 (2 pi / (2^(5/6) Gamma(11/6))) (L0/r0)^(5/3) x^(5/6) K_5/6(x),
 *   x = 2 pi r / L0.
 * Pixel p of a line lies at p pitch_m along it, and stencil line d (1..n_st)
 * lies d pitch_m behind the new line; X index (d - 1) side + p.  C_XX^+ drops
 * the eigenvalues at or below rcond times the largest.  B is the symmetric
 * square root, with negative round-off eigenvalues set to 0.
 * A_dev: side x (n_st side) floats, B_dev: side x side floats, row-major.
 * A64_dev, B64_dev: optional float64 copies (NULL to skip).
 * side 2..1024, n_st 1..4 and n_st < side, pitch_m, r0_m and L0_m finite and
 * > 0, 0 < rcond < 1; else SPECULA_EINVAL.  A does not depend on r0, and B
 * scales as r0^(-5/6): operators built for one r0 serve any layer through
 * b_scale = (r0 / r0_layer)^(5/6).
 * Set-up call: allocates float64 work arrays (about 3 (n_st side)^2 doubles),
 * runs Jacobi eigen-decompositions and synchronises the stream. */
int specula_infscreen_operators(specula_ctx *ctx, int32_t side, int32_t n_st, double pitch_m,
                                double r0_m, double L0_m, double rcond, float *A_dev,
                                float *B_dev, double *A64_dev, double *B64_dev, void *stream);

#define SPECULA_INF_MAX_TASKS 32
typedef struct {
  float *screen_dev;      /* side x side float ring screen                      */
  const float *A_dev;     /* operators of specula_infscreen_operators           */
  const float *B_dev;
  float b_scale;          /* noise scale, (r0_ops / r0_layer)^(5/6)             */
  int32_t axis;           /* 0: add a row, 1: add a column                      */
  int32_t direction;      /* +1: stencil lines L-1, L-2, ..; -1: L+1, L+2, ..   */
  int32_t stream_id;      /* Philox counter word 3 (one per layer)              */
  int64_t line;           /* the line L written (signed)                        */
} specula_inf_line;

/* Per-frame call: write one new line in each of n_tasks ring screens (0..32,
 * distinct screen_dev, all of this side and n_st).  The noise b of line L:
 * element p is normal (p mod 4) of the Philox4x32-10 counter (p / 4, L low 32
 * bits, L high 32 bits, stream_id), key = seed, by Box-Muller with the
 * uniforms (x + 0.5) 2^-32 (the transform of specula_rng_complex, evaluated
 * here in float32).  If noise_dev is not NULL it is used instead:
 * n_tasks x side floats, row t for task t.  The two dot products run in
 * float32.  A line that depends on another line of the same screen needs a
 * later call.  Enqueues one kernel; no allocation, no synchronisation.
 * Errors: SPECULA_EINVAL for a bad size, axis, direction or repeated screen. */
int specula_infscreen_lines(specula_ctx *ctx, int32_t side, int32_t n_st, int32_t n_tasks,
                            const specula_inf_line *tasks, uint64_t seed, const float *noise_dev,
                            void *stream);

/* Ring planner (host only, no GPU): the lines a set of layers must grow so
 * that each ring window covers its pupil footprint at time t.  For layer l
 * and axis a (0: rows = y, 1: columns = x), lo[2 l + a] is the lowest line in
 * the ring's window [lo, lo + side - 1].  A fresh ring from an FFT screen has
 * lo = 0.  The footprint is the range of floor(u) that the extraction reads,
 *   u = ((x s) + ((h theta) - (v t))) / pitch + side / 2,
 * at the two pupil edges x = -+(n_pix - 1) / 2 pupil pitch, s = 1 - h / H, plus
 * the bilinear neighbour, widened by `margin` lines on each side (0..64).  The
 * moves are listed per layer in order: columns, then rows, each in growth
 * order.  Growing down (direction -1) writes line lo - 1 from lines lo,
 * lo + 1, ...; growing up writes line lo + side from the lines below it.  On
 * success lo is updated and *n_moves is set.  If more than max_moves are
 * needed, the call returns SPECULA_EUNSUPPORTED, sets *n_moves to the count
 * needed and leaves lo unchanged.  A footprint wider than the ring, or more
 * than 2^20 lines for one layer and axis, also gives SPECULA_EUNSUPPORTED.  n_layers 0..32; layers' side is ignored (the ring's
 * side is `side`). */
typedef struct {
  int32_t layer, axis, direction;
  int64_t line;
} specula_inf_move;
int specula_infscreen_plan(int32_t n_layers, const specula_layer_desc *layers,
                           const specula_source_desc *source, const specula_pupil_desc *pupil,
                           int32_t side, int32_t margin, double t, int64_t *lo,
                           int32_t max_moves, specula_inf_move *moves, int32_t *n_moves);

/* Per-frame call: plan as specula_infscreen_plan (no move limit), then grow
 * the lines.  Round k is one specula_infscreen_lines call carrying the k-th
 * move of every layer, with stream_id = 2 layer + axis and b_scale[l].
 * screens_dev, A_dev, B_dev: host arrays of n_layers device pointers (rings
 * of this side; operators of this side and n_st).  *n_calls (may be NULL)
 * is set to the number of calls.  lo is updated once every call has been
 * enqueued.  Enqueues kernels only; host work is the plan. */
int specula_infscreen_advance(specula_ctx *ctx, int32_t n_layers, const specula_layer_desc *layers,
                              const specula_source_desc *source, const specula_pupil_desc *pupil,
                              int32_t side, int32_t n_st, int32_t margin,
                              float *const *screens_dev, const float *const *A_dev,
                              const float *const *B_dev, const float *b_scale, int64_t *lo,
                              double t, uint64_t seed, int32_t *n_calls, void *stream);

/* ---- per-frame calls ------------------------------------------------------- */

/* Layer extraction (AtmoEvolution + AtmoPropagation, geometric propagation):
 *   phase[j][i] = (500 / lambda) sum_l bilinear_periodic(S_l, u_l(i), v_l(j))
 *   u = ((x_i * s) + ((h * theta_x) - (vx * t))) / pitch_l + side_l / 2,
 *   x_i = (i - (n_pix - 1) / 2) * pupil pitch, s = 1 - h / H,
 * with floor(u) and the fraction decided in float64 exactly in this
 * operation order, the interpolation in float32.  t = *t_dev if t_dev is not
 * NULL (device double, for graph replay), else t_s.  screens_dev is a host
 * array of n_layers device pointers (side_l^2 floats each).  n_layers <= 64.
 * phase_dev: n_pix^2 floats, radians at the source wavelength. */
int specula_atmo_extract(specula_ctx *ctx, int32_t n_layers,
                         const specula_layer_desc *layers,
                         const float *const *screens_dev,
                         const specula_source_desc *source,
                         const specula_pupil_desc *pupil, double t_s,
                         const double *t_dev, float *phase_dev, void *stream);

/* Allocation-free layer extraction (the paper has no counterpart: this is a
 * library convenience).  Computes exactly what specula_atmo_extract computes,
 * without a context, for callers that cannot call cudaMalloc — a host that
 * only enqueues work into its own CUDA graphs, a real-time loop that forbids
 * allocation after start-up, an embedding that owns all device memory.
 * The coordinate table lives in a fixed device array of 8 MiB (64 layers x 2
 * axes x 8192 pixels of int32 index + float32 fraction) that every GPU which
 * loads the library holds until the process exits; n_layers > 64 or
 * n_pix > 8192 returns SPECULA_EUNSUPPORTED.  Runs on the calling thread's
 * current device.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress): make that call before any stream capture.
 * All calls share the array, so calls whose kernels overlap on the GPU race
 * and must be ordered by the caller.  The address is kept per device for
 * the rest of the process: after a cudaDeviceReset (or anything else that
 * destroys and recreates the device's primary context) it is stale, and this
 * entry point must not be used on that device again.  Allocates nothing. */
int specula_atmo_extract_noalloc(int32_t n_layers, const specula_layer_desc *layers,
                                 const float *const *screens_dev,
                                 const specula_source_desc *source,
                                 const specula_pupil_desc *pupil, double t_s,
                                 const double *t_dev, float *phase_dev, void *stream);

/* Build (or reuse) the tables and workspace of a pyramid geometry: modulation
 * tilt tables, pyramid-mask tables and FFT twiddles, computed in float64 on
 * the host and rounded once to float32.  May allocate.  Supported FFT sides
 * N = pad * n_pix: 64, 128, 240, 320, 660, 960, 1600. */
int specula_pwfs_plan(specula_ctx *ctx, const specula_pupil_desc *pupil,
                      const specula_pwfs_desc *pwfs);

/* Tile choice of a pyramid plan (the autotuner's knobs): `chunk` = number of
 * (batch element, modulation point) items whose intermediates are kept in
 * the workspace at once (the pipeline runs chunk by chunk, so a chunk that
 * fits L2 keeps the intermediates on chip); `ka` = modulation items handled
 * per warp in the row-transform pass (amortises the field's sincos);
 * `passes` = the form of the 2D filter IDFT2(M . DFT2(P)): 3 = row FFTs,
 * column FFT + mask + inverse, row inverse FFTs + |.|^2 + bins; 2 = the
 * separable form (the mask is Mx(u) My(v)): row FFT + x mask + row inverse,
 * then column FFT + y mask + column inverse + |.|^2 + bins, without the
 * N x N intermediate; 4 = the separable form evaluated with packed float32
 * pairs (two transforms per thread: two pupil rows in the row filter, the
 * two modulation points of one cosine in the column filter; pad 2 with
 * touching pupil images, N = 320 or 960; runs whole batch elements, so the
 * chunk is rounded down to a multiple of n_mod / 2 + 1 slots, at least one
 * element).  All compute the same image (float rounding aside).
 * set: may reallocate the workspace (set-up call); chunk in [1, 4096], ka in
 * [1, 64], passes 2, 3 or 4 (2 and 4 return SPECULA_EUNSUPPORTED where their
 * column tile does not fit or the geometry is not supported).  get: reads
 * the current values. */
int specula_pwfs_set_tiles(specula_ctx *ctx, const specula_pupil_desc *pupil,
                           const specula_pwfs_desc *pwfs, int32_t chunk, int32_t ka,
                           int32_t passes);
int specula_pwfs_get_tiles(specula_ctx *ctx, const specula_pupil_desc *pupil,
                           const specula_pwfs_desc *pwfs, int32_t *chunk, int32_t *ka,
                           int32_t *passes);

/* Imaged modulation slots of a pyramid plan (set-up call; synchronises).
 * Slot c (0 <= c <= n_mod / 2) holds the points m = c and m = n_mod - c,
 * which share a modulation cosine.  After this call, specula_pwfs_image
 * images only the points of slots [slot_begin, slot_end) and still
 * normalises by 1 / n_mod.  So the detectors of disjoint slot ranges that
 * cover 0 .. n_mod / 2 add up to the full image: the modulation-point
 * partition of one frame across GPUs, summed by a reduction.  The range
 * [0, n_mod / 2 + 1) restores the full image.  A partial range needs the
 * two-pass tilt form (SPECULA_EUNSUPPORTED from specula_pwfs_image
 * otherwise) and is refused by the autotuner.  Errors: SPECULA_EINVAL for
 * an empty or out-of-range interval, SPECULA_ENOPLAN without a plan. */
int specula_pwfs_set_slots(specula_ctx *ctx, const specula_pupil_desc *pupil,
                           const specula_pwfs_desc *pwfs, int32_t slot_begin, int32_t slot_end);

/* Modulation form of a pyramid plan (set-up call; may allocate).
 *  SPECULA_PWFS_FORM_TILT (default): the modulation steps as listed for
 *    ModulatedPyramid (App. A, Tab. 4): per point, tilt the field, forward
 *    2-D transform, mask, inverse transform, |.|^2.
 *  SPECULA_PWFS_FORM_SHIFTED: one forward 2-D transform per image; per point
 *    the analytic mask at the frequencies moved by -s_m, s_m = mod_amp pad
 *    (cos t_m, sin t_m) bins, inverse transform, |.|^2.  A different
 *    discretisation: it equals the tilt form where no shifted frequency wraps
 *    and differs by the spectrum's wrapped wings otherwise (at pad 2, 13-16 %
 *    of the peak normalised intensity for a flat wavefront on 64-120 px
 *    pupils).  Needs pad = 2 and the sizes of the two-pass form;
 *    SPECULA_EUNSUPPORTED else.
 *  SPECULA_PWFS_FORM_DFTGEMM_BF16, SPECULA_PWFS_FORM_DFTGEMM_TF32: the
 *    modulation steps of the tilt form with the separable filter of every
 *    row and every column (forward DFT of the pupil's half, mask, inverse
 *    DFT: one N x n_pix complex operator, built in float64) applied as a
 *    dense product on the tensor cores: one real GEMM per axis (the complex
 *    product in its real embedding) with three-term split precision
 *    (A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi) in bf16 or tf32 operands and
 *    float32 accumulation; then |.|^2 / n_mod and the bins.  The DFT-as-GEMM
 *    variant for small padded grids: N <= 512, 2N a multiple of 128,
 *    6 n_pix a multiple of 64 (bf16) or 32 (tf32); SPECULA_EUNSUPPORTED
 *    else, and for slot ranges.  Allocates the operator and its workspace
 *    (for the 320^2 grid of the 8 m system about 45 MB).
 * specula_pwfs_image then computes the image in the plan's form.  The
 * autotuner and the tile settings apply to the tilt form; autotune on a
 * plan in another form returns SPECULA_EUNSUPPORTED. */
#define SPECULA_PWFS_FORM_TILT    0
#define SPECULA_PWFS_FORM_SHIFTED 1
#define SPECULA_PWFS_FORM_DFTGEMM_BF16 2
#define SPECULA_PWFS_FORM_DFTGEMM_TF32 3
int specula_pwfs_set_form(specula_ctx *ctx, const specula_pupil_desc *pupil,
                          const specula_pwfs_desc *pwfs, int32_t form);

/* Autotuner: time every candidate (passes in {2, 3, 4}; chunk in
 * {1,2,3,4,6,8,12,16,24,32,48,64} up to the batch's item count and with
 * workspace <= max_workspace_bytes, for passes 4 whole batch elements
 * {1, 2, 4, ...} up to the batch; ka in {1, 2}) with CUDA events over
 * `reps` images of the caller's inputs on
 * `stream`, keep the fastest in the plan and return it.  Set-up call: may
 * reallocate the workspace and synchronises the stream.  det_dev is
 * overwritten. */
int specula_pwfs_autotune(specula_ctx *ctx, const specula_pupil_desc *pupil,
                          const specula_pwfs_desc *pwfs, const float *amp_dev,
                          const float *phase_dev, int32_t n_batch, float *det_dev,
                          int32_t reps, int64_t max_workspace_bytes, int32_t *chunk,
                          int32_t *ka, int32_t *passes, void *stream);

/* Modulated pyramid image (ModulatedPyramid + CCD, noise off).  For each of
 * n_batch phase maps and each modulation point m:
 *   E_m = amp exp(i phase) exp(2 pi i r (x cos t_m + y sin t_m) / n_pix),
 * centred in an N x N zero grid; F = centred DFT; F *= exp(-2 pi i c (|u| +
 * |v|) / N), c = pup_dist / 2; O = inverse centred DFT (1/N^2);
 * I = (1/n_mod) sum_m |O|^2; det = b x b block sums of I, b = n_pix / n_sub.
 * amp_dev: n_pix^2 floats (shared by the batch); phase_dev: n_batch *
 * n_pix^2 floats; det_dev: n_batch * (N/b)^2 floats.  n_sub = n_pix gives
 * the unbinned N x N intensity.  Requires a plan (else SPECULA_ENOPLAN). */
int specula_pwfs_image(specula_ctx *ctx, const specula_pupil_desc *pupil,
                       const specula_pwfs_desc *pwfs, const float *amp_dev,
                       const float *phase_dev, int32_t n_batch, float *det_dev,
                       void *stream);

/* Polychromatic pyramid image (PolyCromPyramid, App. A, Tab. 4): for n_batch
 * phase maps in radians at the reference wavelength,
 *   det = sum over i of weight[i] image_i,
 * image_i the image above at lambda_i: phase times ratio[i] = lambda_ref /
 * lambda_i and the modulation radius mod_amp ratio[i] (lambda_i / D); the
 * pupil images' separation pup_dist is geometric and the same at every
 * wavelength.  ratio, weight: n_lambda host doubles (1 <= n_lambda <= 64,
 * ratio > 0).  Needs a plan for every wavelength: the descriptor with
 * mod_amp = pwfs->mod_amp * ratio[i] (SPECULA_ENOPLAN else, checked before
 * anything is enqueued).  Per-frame call: enqueues only. */
int specula_pwfs_image_poly(specula_ctx *ctx, const specula_pupil_desc *pupil,
                            const specula_pwfs_desc *pwfs, int32_t n_lambda, const double *ratio,
                            const double *weight, const float *amp_dev, const float *phase_dev,
                            int32_t n_batch, float *det_dev, void *stream);

/* Build (or reuse) the tables of a Shack-Hartmann geometry and its valid
 * subaperture list (host rule above).  May allocate.  Supported (fft_n,
 * sub_pix): (24, 12), (16, 8), and Sect. 6 Tab. 2's spot sizes (56, 8) (the
 * SCAO SH: 20 x 20 lenslets on a 160 px pupil) and (68, 4) (ERIS: 40 x 40
 * on 160 px), whose transforms are wider than a warp (56 = 8 x 7, 68 = 4 x
 * 17, prime-factor form).  *n_valid receives the count. */
int specula_sh_plan(specula_ctx *ctx, const specula_pupil_desc *pupil,
                    const specula_sh_desc *sh, int32_t *n_valid);

/* Shack-Hartmann spots (SH): for each valid subaperture (ascending index), its
 * sub_pix^2 block of E = amp exp(i phase) is centred in an fft_n^2 zero grid;
 * spot = |centred DFT|^2 / fft_n^2.  spots_dev: n_batch * n_valid * fft_n^2
 * floats.  Requires a plan. */
int specula_sh_image(specula_ctx *ctx, const specula_pupil_desc *pupil,
                     const specula_sh_desc *sh, const float *amp_dev,
                     const float *phase_dev, int32_t n_batch, float *spots_dev,
                     void *stream);

/* Polychromatic Shack-Hartmann spots (PolyChromSH, App. A, Tab. 4): for
 * n_batch phase maps in radians at the reference wavelength,
 *   spots = sum over i (in order) of weight[i] ratio[i]^2 W_i S_i W_i^T,
 * S_i the spots above at lambda_i (phase times ratio[i] = lambda_ref /
 * lambda_i, the same fft_n, so a spot pixel is lambda_i / (fft_n d) = 1 /
 * ratio[i] reference pixels) and W_i[o][j] the overlap of reference pixel o,
 * [o - fft_n/2 - 1/2, o - fft_n/2 + 1/2), with spot pixel j, [(j - fft_n/2 -
 * 1/2) / ratio, (j - fft_n/2 + 1/2) / ratio), both centred on the zero
 * frequency: the detector integrates each wavelength's piecewise-constant
 * spot over its own pixels; light beyond a subaperture's fft_n window is
 * dropped (a field stop per subaperture).  ratio[i] = 1 reproduces
 * specula_sh_image.  ratio, weight: n_lambda host doubles (1 <= n_lambda
 * <= 64, ratio > 0).  spots_dev as specula_sh_image (the plan's imaged
 * range).  Uses a context workspace of one wavelength's spots: reserve it
 * with specula_sh_poly_reserve (set-up call) so that per-frame calls never
 * allocate; a call that finds it too small grows it (synchronising the
 * stream), or returns SPECULA_EUNSUPPORTED inside stream capture.  fft_n 24
 * or 16. */
int specula_sh_image_poly(specula_ctx *ctx, const specula_pupil_desc *pupil,
                          const specula_sh_desc *sh, int32_t n_lambda, const double *ratio,
                          const double *weight, const float *amp_dev, const float *phase_dev,
                          int32_t n_batch, float *spots_dev, void *stream);

/* Set-up call (may allocate; synchronises the device when it grows): size
 * the polychromatic SH workspace for batches up to max_batch of this plan's
 * valid subapertures.  SPECULA_ENOPLAN without a plan. */
int specula_sh_poly_reserve(specula_ctx *ctx, const specula_pupil_desc *pupil,
                            const specula_sh_desc *sh, int32_t max_batch);

/* Imaged subapertures of a Shack-Hartmann plan (set-up call; synchronises):
 * after this call specula_sh_image computes the spots of the valid
 * subapertures sub_begin .. sub_end - 1 only (positions in the ascending
 * valid list), compact: n_batch * (sub_end - sub_begin) * fft_n^2 floats.
 * Their slopes are specula_slopes over the same count; the slope vectors of
 * disjoint blocks that cover the list, each laid out all x then all y, make
 * up the full vector.  This is the subaperture partition of one sensor
 * across GPUs, the analogue of the paper's DistributedSH (Sect. 6; App. A,
 * Tab. 4), joined by an all-gather of slopes.  [0, n_valid) restores the
 * whole sensor.  Errors: SPECULA_EINVAL for a range outside [0, n_valid],
 * SPECULA_ENOPLAN without a plan. */
int specula_sh_set_range(specula_ctx *ctx, const specula_pupil_desc *pupil,
                         const specula_sh_desc *sh, int32_t sub_begin, int32_t sub_end);

/* Slopes (PyrSlopec / ShSlopec).  Output per batch element: all x slopes of
 * the listed subapertures, then all y slopes (2 * n_valid floats).
 *  PYR: img is the 2 n_sub x 2 n_sub detector; with Q1 (+x,+y) at
 *   (n_sub + a, n_sub + b), Q2 (-x,+y) at (n_sub + a, b), Q3 (-x,-y) at
 *   (a, b), Q4 (+x,-y) at (a, n_sub + b):
 *   Sx = ((Q1 + Q4) - (Q2 + Q3)) / T, Sy = ((Q1 + Q2) - (Q3 + Q4)) / T,
 *   T = mean over the listed subapertures of Q1 + Q2 + Q3 + Q4.
 *  PYR_MAPS: the same slopes with Q1..Q4 read at the listed detector
 *   indices (any padding and image separation); an index outside the
 *   n_sub x n_sub detector reads pixel 0 and records SPECULA_EINVAL.
 *  SH: img holds n_valid spots of fft_n^2; centre of gravity over the whole
 *   window, x = j - (fft_n - 1)/2 pixels.
 * ref_dev (nullable): 2 * n_valid reference slopes subtracted from each
 * batch element.  Reductions run in a fixed order (bit-reproducible). */
int specula_slopes(specula_ctx *ctx, const specula_slopec_desc *slopec,
                   const float *img_dev, const float *ref_dev, int32_t n_batch,
                   float *slopes_dev, void *stream);

/* Modal reconstruction (Modalrec): modes[b] = R slopes[b] for n_batch slope
 * vectors of n_slopes floats; modes_dev: n_batch * n_modes floats.
 * Accumulation in float32 for every precision.  FP32 runs on the CUDA
 * cores at every batch.  BF16 and BF16X2 (n_slopes a multiple of 8, 16-byte
 * aligned operands) run on the CUDA cores below 32 vectors; from 32 on, the
 * slopes are split into bfloat16 halves xh + xl in a context-owned
 * workspace and one tensor-core GEMM forms xh Rh^T + xh Rl^T + xl Rh^T
 * (BF16X2) or (xh + xl) Rh^T (BF16).  That workspace grows on the first
 * batched call of a new size, which synchronises the stream; inside stream
 * capture a call that would grow it returns SPECULA_EUNSUPPORTED.
 * specula_recon_reserve sizes it in advance, so per-frame calls then never
 * allocate. */
int specula_recon(specula_ctx *ctx, const specula_recon_desc *rec,
                  const float *slopes_dev, int32_t n_batch, float *modes_dev,
                  void *stream);

/* Set-up call (may allocate; synchronises the device when it grows): size
 * the context workspace of the batched bf16 products of rec for every batch
 * up to max_batch (no-op for SPECULA_PREC_FP32 and batches below 32). */
int specula_recon_reserve(specula_ctx *ctx, const specula_recon_desc *rec, int32_t max_batch);

/* Reduced-precision copies of a float32 R: BF16 writes hi = bf16(R) (round to
 * nearest even); BF16X2 also writes lo = bf16(R - float(hi)).  hi_dev / lo_dev
 * hold n_modes * n_slopes uint16 each (lo_dev unused for BF16). */
int specula_recon_convert(specula_ctx *ctx, int32_t n_modes, int32_t n_slopes,
                          const float *R_dev, int32_t precision, void *hi_dev,
                          void *lo_dev, void *stream);

/* ---- multi-sensor system in one persistent launch ---------------------------
 * All wavefront sensors of a system (Shack-Hartmann and pyramids of different
 * sizes, each with its own guide star), their slopes and the reconstructor
 * product on the concatenated slopes, computed by one kernel launch per
 * frame (the multi-sensor systems of Sect. 6, Tab. 2; App. A, Tab. 4:
 * AtmoPropagation per source, SH / ModulatedPyramid, ShSlopec / PyrSlopec,
 * Modalrec).  Each sensor computes what the single-sensor calls compute:
 * specula_atmo_extract for its source, then specula_sh_image +
 * SPECULA_SLOPES_SH (centre of gravity taken directly from the spot, which is
 * not stored) or specula_pwfs_image + SPECULA_SLOPES_PYR; the reconstructor
 * is modes = R slopes with R n_modes x n_slopes float32, summed per sensor
 * then over sensors in sensor order.  Every sensor's valid subapertures come
 * from the geometric rule of specula_valid_subaps_host.  Built kernel
 * variants: pyramids with FFT side 128 or 240 (one side per system, pad 2,
 * pup_dist_px = n_pix, b = n_pix / n_sub <= 16); SH with sub_pix 12 and
 * fft_n 24.  Up to 16 sensors and 64 layers. */
#define SPECULA_WFS_PYR 0
#define SPECULA_WFS_SH  1
typedef struct {
  int32_t kind;                 /* SPECULA_WFS_PYR or SPECULA_WFS_SH   */
  specula_pupil_desc pupil;
  specula_source_desc source;
  specula_pwfs_desc pwfs;       /* kind PYR                            */
  specula_sh_desc sh;           /* kind SH                             */
} specula_wfs_desc;
typedef struct specula_mwfs specula_mwfs;

/* Plan the system (set-up call: allocates, synchronises).  screens_dev is a
 * host array of n_layers device pointers and R_dev (n_modes x n_slopes
 * float32, NULL when n_modes = 0) is device memory; the library keeps these
 * pointers, so they must stay valid until specula_mwfs_destroy.  Slopes are
 * concatenated in sensor order, each sensor's block all x then all y
 * (specula_mwfs_info gives the offsets). */
int specula_mwfs_create(specula_ctx *ctx, int32_t n_sensors, const specula_wfs_desc *sensors,
                        int32_t n_layers, const specula_layer_desc *layers,
                        const float *const *screens_dev, int32_t n_modes, const float *R_dev,
                        specula_mwfs **out);
int specula_mwfs_destroy(specula_mwfs *mwfs);
/* Per-sensor valid-subaperture count and slope offset (sensor >= 0), and
 * the total slope count (any sensor; pass -1 for the total only). */
int specula_mwfs_info(const specula_mwfs *mwfs, int32_t sensor, int32_t *n_valid,
                      int32_t *slope_offset, int32_t *n_slopes_total);
/* Number of tasks of one frame, CTAs launched, and the most CTAs that fit
 * on the device at once. */
int specula_mwfs_schedule(const specula_mwfs *mwfs, int32_t *n_tasks, int32_t *grid,
                          int32_t *max_grid);
/* CTAs per launch (0: as many as fit); the frame's result does not depend on
 * it except for float rounding order, which it does not change either
 * (every reduction has a fixed order). */
int specula_mwfs_set_grid(specula_mwfs *mwfs, int32_t ctas);
/* Limit of one dependency wait inside the launch, in ns (0: the default of
 * 2 s; at most 10 s), and fault injection for tests of the failure path:
 * task `stall_task` (0 .. n_tasks-1; -1: none) waits for an arrival count
 * that never comes.  That wait expires after limit_ns, records
 * SPECULA_ETIMEOUT in the context status word and makes every CTA leave;
 * the launch's outputs are then undefined and the next launch starts from
 * clean counters.  Takes effect for launches made after the call (a
 * captured graph keeps the values of its capture). */
int specula_mwfs_set_wait(specula_mwfs *mwfs, int64_t limit_ns, int32_t stall_task);
/* One frame at time t (t = *t_dev if t_dev is not NULL): slopes_dev
 * (n_slopes floats) minus ref_dev (nullable, same layout), and modes_dev
 * (n_modes floats; must be NULL exactly when n_modes = 0).  Per-frame call:
 * enqueues one kernel, allocates nothing.  A dependency wait longer than the
 * limit (2 s unless set) ends the launch early with SPECULA_ETIMEOUT in the
 * context status word. */
int specula_mwfs_frame(specula_mwfs *mwfs, double t_s, const double *t_dev,
                       const float *ref_dev, float *slopes_dev, float *modes_dev, void *stream);
/* Slopes of a flat wavefront (no layers), no reference subtracted: the
 * reference slopes of every sensor in one launch. */
int specula_mwfs_reference(specula_mwfs *mwfs, float *ref_dev, float *modes_dev, void *stream);
/* Copy sensor `sensor`'s last phase (n_pix^2 floats, radians at its
 * wavelength; a Shack-Hartmann sensor's phase is computed on the pixels of
 * its valid subapertures only and is 0 elsewhere) or pyramid detector
 * ((2 n_sub)^2 floats) into dst_dev. */
#define SPECULA_MWFS_PHASE    0
#define SPECULA_MWFS_DETECTOR 1
int specula_mwfs_read(const specula_mwfs *mwfs, int32_t sensor, int32_t what, float *dst_dev,
                      void *stream);

/* ---- tensor-core GEMM ---------------------------------------------------------
 * C[M][N] = A[M][K] . B[N][K]^T with A, B bfloat16 row-major (both K-major),
 * accumulated in float32 on the tcgen05 tensor cores; C float32 row-major.
 * The dense contractions of the learned reconstructor and the batched bf16
 * reconstructor products use it (the paper's own reconstructor, Modalrec,
 * is the MVM above).  Any M, N >= 1; K a multiple of 8 (rows of a multiple
 * of 16 bytes); A and B 16-byte aligned (else SPECULA_EINVAL; a K that is
 * not a multiple of 8 gives SPECULA_EUNSUPPORTED).  A persistent grid of at
 * most one CTA per SM works through 128 x 256 output tiles (128 x 128 where
 * N is a multiple of 128 but not of 256).  splits > 1 divides K into slices
 * computed as separate work items whose float32 partials go to work_dev
 * (splits * M * N floats, caller-owned) and are summed in slice order.
 * Per-frame call: enqueues only. */
int specula_gemm_bf16(specula_ctx *ctx, const void *A_dev, const void *B_dev, int32_t M,
                      int32_t N, int32_t K, float *C_dev, int32_t splits, float *work_dev,
                      void *stream);

/* The same product with tf32 operands (kind::tf32): A, B float32 row-major,
 * of which the tensor cores use the tf32 part (sign, 8-bit exponent, 10-bit
 * mantissa; the low 13 bits are ignored, so callers round to tf32 first
 * where rounding matters).  K a multiple of 4; otherwise as
 * specula_gemm_bf16.  It serves the tf32 split-precision DFT-as-GEMM
 * pyramid form and the measured tf32 rate.  Per-frame call: enqueues only. */
int specula_gemm_tf32(specula_ctx *ctx, const float *A_dev, const float *B_dev, int32_t M,
                      int32_t N, int32_t K, float *C_dev, int32_t splits, float *work_dev,
                      void *stream);

/* ---- learned reconstructor ----------------------------------------------------
 * A perceptron slopes -> modal coefficients, n_in -> n_h1 -> n_h2 -> n_out with
 * exact-erf GELU between layers (not in the paper, whose reconstructor is
 * the linear Modalrec; a nonlinear alternative to it, trained on pairs the
 * simulator generates).  FP32 master weights and Adam moments, bf16 copies for
 * the tcgen05 GEMMs, FP32 accumulation.  Hidden widths must be multiples of
 * 128; the input/output widths and the batch are padded internally.
 * create/destroy/set/get may allocate and synchronise; forward, backward and
 * adam only enqueue.  One model per stream at a time.  The model keeps a
 * pointer to its context: destroy it before the context (destroy itself
 * does not touch the context, so a late destroy is harmless, but any other
 * call on a model whose context is gone is undefined). */
typedef struct specula_mlp specula_mlp;
int specula_mlp_create(specula_ctx *ctx, int32_t n_in, int32_t n_h1, int32_t n_h2,
                       int32_t n_out, int32_t batch_max, specula_mlp **out);
int specula_mlp_destroy(specula_mlp *mlp);
/* layer l in {0,1,2}: W_host (out x in, row-major) and b_host (out) floats;
 * set resets that layer's Adam moments and the step count. */
int specula_mlp_set_layer(specula_mlp *mlp, int32_t layer, const float *W_host,
                          const float *b_host);
int specula_mlp_get_layer(specula_mlp *mlp, int32_t layer, float *W_host, float *b_host);
/* gradient of the last backward for layer l (same layouts as get_layer) */
int specula_mlp_get_grad(specula_mlp *mlp, int32_t layer, float *dW_host, float *db_host);
/* Y_dev (nullable): batch x n_out floats; X_dev: batch x n_in floats. */
int specula_mlp_forward(specula_mlp *mlp, const float *X_dev, int32_t batch, float *Y_dev,
                        void *stream);
/* Inference only (keeps no state for backward): Y_dev = the network applied
 * to X_dev.  For batch <= 4 each layer streams its bf16 weight rows once
 * against the float32 inputs (one warp per output, float32 accumulation and
 * activations): the way to run the network inside a frame.  Larger batches
 * run as specula_mlp_forward (whose tensor-core GEMMs take bf16 activations,
 * so results differ at the bf16 level).  Per-frame call: enqueues only. */
int specula_mlp_infer(specula_mlp *mlp, const float *X_dev, int32_t batch, float *Y_dev,
                      void *stream);
/* Gradients of loss = mean over batch and outputs of (Y - T)^2 for the last
 * forward (same batch); T_dev: batch x n_out floats; loss_dev (nullable): one
 * float. */
int specula_mlp_backward(specula_mlp *mlp, const float *T_dev, int32_t batch, float *loss_dev,
                         void *stream);
/* Adam on every parameter with the last gradients: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, w -= lr sqrt(1-b2^t)/(1-b1^t) m / (sqrt(v) + eps). */
int specula_mlp_adam(specula_mlp *mlp, float lr, float b1, float b2, float eps, void *stream);

/* Per-column statistics and affine maps for standardising the learned
 * reconstructor's inputs and outputs.  col_stats: mean and (population)
 * standard deviation of each column of X (rows x cols floats), summed in
 * float64 in row order.  affine_cols: out[r][c] = (X[r][c] - shift[c]) *
 * mul[c] (out may equal X). */
int specula_col_stats(specula_ctx *ctx, const float *X_dev, int32_t rows, int32_t cols,
                      float *mean_dev, float *std_dev, void *stream);
int specula_affine_cols(specula_ctx *ctx, const float *X_dev, int64_t rows, int32_t cols,
                        const float *shift_dev, const float *mul_dev, float *out_dev,
                        void *stream);

/* ---- calibration (set-up calls: may allocate, synchronise the stream) ------
 * Modal basis (stands in for the non-public KL files of Listing 2,
 * `ifunc_object`): Zernike modes in Noll order without piston, j = 2 ..
 * n_modes + 1, sqrt(n+1) R_n^|m|(rho) (x sqrt 2 cos/sin |m| theta for m != 0,
 * cos for even j), rho = |(x, y)| / (n_pix / 2) at centred pixel coordinates,
 * theta = atan2(y, x), zero outside the pupil stop.  Evaluated in float64.
 * basis_host: n_modes * n_pix^2 doubles; basis_dev: the same as float32. */
int specula_modal_basis_host(const specula_pupil_desc *pupil, int32_t n_modes,
                             double *basis_host);
int specula_modal_basis(specula_ctx *ctx, const specula_pupil_desc *pupil, int32_t n_modes,
                        float *basis_dev, void *stream);

/* Push-pull interaction matrix (ImCalibrator + PushPullGenerator, App. A,
 * Tab. 4): IM[s][j] = (S_s(+a Z_j) - S_s(-a Z_j)) / (2a), S the pyramid slopes
 * (kind PYR or PYR_MAPS, no reference) of the phase +-a Z_j, a = push_amp radians at the
 * WFS wavelength.  basis_dev: n_modes * n_pix^2 floats; im_dev: n_slopes *
 * n_modes doubles, row-major (n_slopes = 2 n_valid).  Requires a pyramid
 * plan.  Allocates a 16-mode workspace for the call. */
int specula_calib_intmat(specula_ctx *ctx, const specula_pupil_desc *pupil,
                         const specula_pwfs_desc *pwfs, const float *amp_dev,
                         const float *basis_dev, int32_t n_modes, double push_amp,
                         const specula_slopec_desc *slopec, double *im_dev, void *stream);

/* Truncated pseudo-inverse in float64 on the GPU (RecCalibrator, App. A,
 * Tab. 4): A is m x n row-major (device doubles); R = V diag(1/lambda) V^T
 * A^T with (lambda, V) the eigen-pairs of A^T A (parallel cyclic Jacobi) and
 * eigenvalues <= rcond^2 lambda_max discarded — the Moore-Penrose inverse with
 * singular values below rcond sigma_max dropped.  R_dev: n x m doubles;
 * R32_dev (nullable): the same rounded to float32; *rank: kept count.
 * n <= 8192, 0 < rcond < 1. */
int specula_pinv_fp64(specula_ctx *ctx, const double *A_dev, int32_t m, int32_t n,
                      double rcond, double *R_dev, float *R32_dev, int32_t *rank,
                      void *stream);

/* ---- detector noise (per-frame call: enqueue only, allocates nothing) ------
 * CCD object (App. A, Tab. 4; App. B, Listing 2: photon_noise,
 * readout_noise, quantum_eff): pixel p of out_dev = k + ron g, with
 * k ~ Poisson(det_dev[p] scale) (scale = photons per frame x quantum
 * efficiency / pupil pixels, det_dev the noise-free detector image) and g a
 * standard normal.  Draws from Philox4x32-10, counter (p, frame, block,
 * stream), key = seed, uniform (x + 1/2) 2^-32 of a word x: up to a mean of
 * 30 the multiplicative method (the number of uniforms whose running product
 * stays above exp(-lambda), at most 1000; stream 2; uniforms, product and
 * threshold in float32, so a count may differ by one from the float64
 * statement of the method where the product ends within a few roundings of
 * the threshold), above it floor(lambda + sqrt(lambda) g0 + 1/2) clamped at 0;
 * (g0, g) is the float32 Box-Muller pair of words 0 and 1 of block 0 of
 * stream 3.  Reproducible per (seed, frame); the frame index is
 * frame + *frame_dev when frame_dev (one device uint32, nullable) is given,
 * so a captured graph draws new noise when the caller advances *frame_dev.
 * n floats in and out (out may alias det); scale >= 0, ron >= 0. */
int specula_ccd(specula_ctx *ctx, int32_t n, const float *det_dev, double scale, double ron,
                uint64_t seed, uint32_t frame, const uint32_t *frame_dev, float *out_dev,
                void *stream);

/* Detector sampling at a non-integer pixel ratio (a pyramid output_resolution
 * that is not a whole fraction of the padded grid, Listing 2): area-weighted
 * rebinning of n_batch square images n_in x n_in to n_out x n_out,
 *   out[J][I] = sum_j sum_i wy(J, j) wx(I, i) in[j][i],
 *   w(I, i) = |[i, i + 1) n [I b, (I + 1) b)|,   b = n_in / n_out,
 * the grid pixel's area that detector pixel I collects (flux is kept; an
 * integer b is b x b binning).  The overlaps are exact integers in units of
 * 1/n_out; the sums run in float32, row by row in index order, scaled by
 * 1/n_out^2.  in_dev, out_dev: n_batch images, row-major.  1 <= n_in, n_out
 * <= 4096 (n_out > n_in spreads each grid pixel over several detector
 * pixels); n_batch 0 is a no-op.  Per-frame call: one kernel. */
int specula_rebin(specula_ctx *ctx, const float *in_dev, int32_t n_in, int32_t n_out,
                  int32_t n_batch, float *out_dev, void *stream);

/* ---- closed loop (per-frame calls: enqueue only, allocate nothing) ---------
 * The closed-loop objects of the SOUL example (App. B, Listing 2: a DM with a
 * modal influence-function basis, an IirFilter integrator, the ":-1" delayed
 * connection of Sect. 2.2).  Step k of a loop:
 *   residual = phi_atm(t_k) - B^T c_{k-1}        (specula_dm_shape, then
 *                                                 specula_loop_residual)
 *   m = R (slopes(residual) - reference)         (pyramid, slopes, recon calls)
 *   c_k = (1 - leak) c_{k-1} + gain m            (specula_loop_integrate)
 * All sums run in a fixed order: a loop is bit-reproducible. */

/* phase_dev[p] = sum over j (in order) of cmd_dev[j] basis_dev[j][p]:
 * basis n_modes x n_pix2 row-major floats (zero outside the pupil), cmd
 * n_modes floats, phase n_pix2 floats (radians at the sensor wavelength).
 * n_modes <= 12288 (SPECULA_EUNSUPPORTED above). */
int specula_dm_shape(specula_ctx *ctx, int32_t n_modes, int32_t n_pix2, const float *basis_dev,
                     const float *cmd_dev, float *phase_dev, void *stream);

/* resid_dev = atm_dev - dm_dev (n_pix2 floats each) and, over the pupil
 * (weights amp_dev), stats_dev[0] = the residual's RMS with its piston
 * removed and stats_dev[1] = the Strehl ratio at the science wavelength,
 * |sum amp exp(i r wfs_over_sci)|^2 / (sum amp)^2, with wfs_over_sci =
 * lambda_wfs / lambda_sci > 0 (two device doubles; float64 partial sums in
 * a fixed order).  Uses the context's statistics workspace: calls on one
 * context must not overlap on the GPU. */
int specula_loop_residual(specula_ctx *ctx, int32_t n_pix2, const float *amp_dev,
                          const float *atm_dev, const float *dm_dev, double wfs_over_sci,
                          float *resid_dev, double *stats_dev, void *stream);

/* cmd_dev = (1 - leak) cmd_dev + gain modes_dev (n_modes floats each);
 * 0 <= leak <= 1. */
int specula_loop_integrate(specula_ctx *ctx, int32_t n_modes, float gain, float leak,
                           const float *modes_dev, float *cmd_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPECULA_GB300_H */
