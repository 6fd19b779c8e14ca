// Context, status codes, integer geometry and argument validation of the
// C ABI (include/specula_gb300.h).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <unordered_set>
#include <utility>

#include <vector>

#include <algorithm>

#include "internal.h"

using namespace specula;

extern "C" const char *specula_strerror(int s) {
  switch (s) {
    case SPECULA_OK: return "ok";
    case SPECULA_EINVAL: return "invalid argument";
    case SPECULA_ENOMEM: return "out of memory";
    case SPECULA_ECUDA: return "CUDA runtime error";
    case SPECULA_ETIMEOUT: return "bounded device wait expired";
    case SPECULA_EUNSUPPORTED: return "size or option not supported by this library";
    case SPECULA_ENONFINITE: return "non-finite value detected";
    case SPECULA_ENOPLAN: return "no plan for this geometry (call the plan function first)";
    default: return "unknown status";
  }
}

extern "C" int specula_version(void) { return 100; }

extern "C" int specula_ctx_create(specula_ctx **out, int device) {
  if (!out) return SPECULA_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) return SPECULA_ECUDA;
  if (device < 0 || device >= n) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(device));
  specula_ctx *c = new (std::nothrow) specula_ctx();
  if (!c) return SPECULA_ENOMEM;
  c->device = device;
  if (cudaMalloc(&c->status_dev, sizeof(int32_t)) != cudaSuccess) {
    delete c;
    return SPECULA_ENOMEM;
  }
  if (cudaMemset(c->status_dev, 0, sizeof(int32_t)) != cudaSuccess) {
    cudaFree(c->status_dev);
    delete c;
    return SPECULA_ECUDA;
  }
  int s = pwfs_init_device();
  if (!s) s = sh_init_device();
  if (!s) s = mwfs_init_device();
  if (!s) s = pwfs_shifted_init_device();
  if (!s) s = pwfs_pair_init_device();
  if (!s) s = atmo_alloc_tables(c);
  if (!s) s = loop_alloc_workspace(c);
  if (s) {
    cudaFree(c->status_dev);
    if (c->loop_part) cudaFree(c->loop_part);
    if (c->atmo_tab_i) cudaFree(c->atmo_tab_i);
    if (c->atmo_tab_f) cudaFree(c->atmo_tab_f);
    delete c;
    return s;
  }
  *out = c;
  return SPECULA_OK;
}

static void prof_free(specula_ctx *ctx) {
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  ctx->ev.clear();
  ctx->ev_next = 0;
  ctx->rec_kid.clear();
  ctx->prof = false;
}

extern "C" int specula_ctx_destroy(specula_ctx *ctx) {
  if (!ctx) return SPECULA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  prof_free(ctx);
  ctx->pwfs.clear();
  ctx->sh.clear();
  if (ctx->status_dev) cudaFree(ctx->status_dev);
  if (ctx->loop_part) cudaFree(ctx->loop_part);
  if (ctx->atmo_tab_i) cudaFree(ctx->atmo_tab_i);
  if (ctx->atmo_tab_f) cudaFree(ctx->atmo_tab_f);
  delete ctx;
  return SPECULA_OK;
}

extern "C" int specula_prof_enable(specula_ctx *ctx, int32_t capacity) {
  if (!ctx || capacity < 0 || capacity > (1 << 20)) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());
  prof_free(ctx);
  if (capacity == 0) return SPECULA_OK;
  ctx->ev.resize(2 * (size_t)capacity);
  for (auto &e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      prof_free(ctx);
      return SPECULA_ECUDA;
    }
  ctx->rec_kid.reserve(capacity);
  ctx->prof = true;
  return SPECULA_OK;
}

extern "C" int specula_prof_read(specula_ctx *ctx, double *ms_host, int64_t *n_host) {
  if (!ctx || !ms_host || !n_host) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());
  for (int k = 0; k < SPECULA_K_COUNT; ++k) {
    ms_host[k] = 0.0;
    n_host[k] = 0;
  }
  for (size_t i = 0; i < ctx->rec_kid.size(); ++i) {
    float ms = 0.f;
    SPECULA_CK(cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    const int k = ctx->rec_kid[i];
    if (k >= 0 && k < SPECULA_K_COUNT) {
      ms_host[k] += ms;
      n_host[k] += 1;
    }
  }
  ctx->rec_kid.clear();
  ctx->ev_next = 0;
  return SPECULA_OK;
}

struct specula_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

extern "C" int specula_graph_begin(specula_ctx *ctx, void *stream) {
  if (!ctx || !stream) return SPECULA_EINVAL;
  if (ctx->prof) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal));
  return SPECULA_OK;
}

extern "C" int specula_graph_end(specula_ctx *ctx, void *stream, specula_graph **out) {
  if (!ctx || !stream || !out) return SPECULA_EINVAL;
  *out = nullptr;
  cudaGraph_t g = nullptr;
  SPECULA_CK(cudaStreamEndCapture((cudaStream_t)stream, &g));
  specula_graph *sg = new (std::nothrow) specula_graph();
  if (!sg) {
    cudaGraphDestroy(g);
    return SPECULA_ENOMEM;
  }
  sg->graph = g;
  sg->device = ctx->device;
  if (cudaGraphInstantiate(&sg->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    delete sg;
    return SPECULA_ECUDA;
  }
  *out = sg;
  return SPECULA_OK;
}

extern "C" int specula_graph_launch(specula_graph *graph, void *stream) {
  if (!graph || !graph->exec) return SPECULA_EINVAL;
  SPECULA_CK(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
  return SPECULA_OK;
}

extern "C" int specula_graph_kernel_count(specula_graph *graph, int64_t *count) {
  if (!graph || !count) return SPECULA_EINVAL;
  size_t n = 0;
  SPECULA_CK(cudaGraphGetNodes(graph->graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) SPECULA_CK(cudaGraphGetNodes(graph->graph, nodes.data(), &n));
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    SPECULA_CK(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *count = k;
  return SPECULA_OK;
}

extern "C" int specula_graph_destroy(specula_graph *graph) {
  if (!graph) return SPECULA_EINVAL;
  cudaSetDevice(graph->device);
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
  return SPECULA_OK;
}

extern "C" int specula_launch_count(specula_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return SPECULA_EINVAL;
  *count = ctx->launches;
  return SPECULA_OK;
}

extern "C" int specula_ctx_status(specula_ctx *ctx, int32_t *device_status) {
  if (!ctx || !device_status) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());
  int32_t v = 0;
  SPECULA_CK(cudaMemcpy(&v, ctx->status_dev, sizeof(v), cudaMemcpyDeviceToHost));
  SPECULA_CK(cudaMemset(ctx->status_dev, 0, sizeof(int32_t)));
  *device_status = v;
  return SPECULA_OK;
}

extern "C" int specula_ctx_set_guard(specula_ctx *ctx, int32_t on) {
  if (!ctx || (on != 0 && on != 1)) return SPECULA_EINVAL;
  ctx->guard = on != 0;
  return SPECULA_OK;
}

// ---- workspace guard bands ----------------------------------------------------

namespace specula {
// Never destroyed: buffers may outlive static destruction at exit.
static std::mutex &guard_mu() {
  static std::mutex *m = new std::mutex;
  return *m;
}
static std::unordered_set<DevBuf *> &guard_set() {
  static std::unordered_set<DevBuf *> *s = new std::unordered_set<DevBuf *>;
  return *s;
}
void guard_register(DevBuf *b) {
  std::lock_guard<std::mutex> g(guard_mu());
  guard_set().insert(b);
}
void guard_unregister(DevBuf *b) {
  std::lock_guard<std::mutex> g(guard_mu());
  guard_set().erase(b);
}
}  // namespace specula

extern "C" int specula_check_guards(specula_ctx *ctx, int32_t *n_checked, int32_t *n_bad) {
  if (!ctx || !n_checked || !n_bad) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> g(guard_mu());
  unsigned char h[kGuardBytes];
  int32_t nc = 0, nb = 0;
  for (DevBuf *b : guard_set()) {
    if (b->device != ctx->device) continue;
    SPECULA_CK(cudaMemcpy(h, static_cast<const char *>(b->p) + b->bytes, kGuardBytes,
                          cudaMemcpyDeviceToHost));
    ++nc;
    for (size_t i = 0; i < kGuardBytes; ++i)
      if (h[i] != kGuardByte) {
        ++nb;
        break;
      }
  }
  *n_checked = nc;
  *n_bad = nb;
  return SPECULA_OK;
}

// ---- integer geometry --------------------------------------------------------

namespace specula {
static thread_local char t_last_error[256] = "";
void note_cuda_error(cudaError_t e, const char *file, int line) {
  const char *f = strrchr(file, '/');
  snprintf(t_last_error, sizeof(t_last_error), "%s (%s) at %s:%d", cudaGetErrorName(e),
           cudaGetErrorString(e), f ? f + 1 : file, line);
}
}  // namespace specula

extern "C" const char *specula_last_cuda_error(void) { return specula::t_last_error; }

namespace specula {
int ensure_dynamic_smem(const void *fn, size_t bytes) {
  if (bytes <= 48 * 1024) return SPECULA_OK;
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> cur;
  int dev = 0;
  SPECULA_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t &c = cur[std::make_pair(dev, fn)];
  if (bytes > c) {
    SPECULA_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    c = bytes;
  }
  return SPECULA_OK;
}
}  // namespace specula

namespace specula {

int host_pupil_mask(int n, double obsc, uint8_t *mask) {
  const double e = obsc * (double)n;
  const double thr = e * e;
  const int64_t nn = (int64_t)n * n;
  for (int j = 0; j < n; ++j) {
    const int64_t dy = 2 * (int64_t)j - n + 1;
    for (int i = 0; i < n; ++i) {
      const int64_t dx = 2 * (int64_t)i - n + 1;
      const int64_t r4 = dx * dx + dy * dy;
      mask[(size_t)j * n + i] = (r4 <= nn && (double)r4 > thr) ? 1 : 0;
    }
  }
  return SPECULA_OK;
}

// A subaperture (n / n_sub pupil pixels a side, whole or fractional) is valid
// iff at least half of its area is in the stop: with ov(i, A) the overlap of
// pixel i with subaperture A in units of 1 / n_sub,
// 2 sum ov(y, A) ov(x, C) mask[y][x] >= n^2, exact in integers (for a whole
// side b it is 2 count >= b^2).
int host_valid_subaps(int n, double obsc, int n_sub, int32_t *idx, int32_t *n_valid) {
  std::vector<uint8_t> m((size_t)n * n);
  host_pupil_mask(n, obsc, m.data());
  auto ov = [&](int i, int A) -> int64_t {
    const int64_t lo = std::max<int64_t>((int64_t)i * n_sub, (int64_t)A * n);
    const int64_t hi = std::min<int64_t>((int64_t)(i + 1) * n_sub, (int64_t)(A + 1) * n);
    return hi > lo ? hi - lo : 0;
  };
  int cnt = 0;
  for (int a = 0; a < n_sub; ++a) {
    const int y0 = (int)((int64_t)a * n / n_sub), y1 = (int)(((int64_t)(a + 1) * n + n_sub - 1) / n_sub);
    for (int c = 0; c < n_sub; ++c) {
      const int x0 = (int)((int64_t)c * n / n_sub), x1 = (int)(((int64_t)(c + 1) * n + n_sub - 1) / n_sub);
      int64_t in = 0;
      for (int y = y0; y < y1; ++y) {
        const int64_t wy = ov(y, a);
        for (int x = x0; x < x1; ++x)
          if (m[(size_t)y * n + x]) in += wy * ov(x, c);
      }
      if (2 * in >= (int64_t)n * n) idx[cnt++] = a * n_sub + c;
    }
  }
  *n_valid = cnt;
  return SPECULA_OK;
}

}  // namespace specula

static int check_pupil(const specula_pupil_desc *p) {
  if (!p) return SPECULA_EINVAL;
  if (p->n_pix < 2 || p->n_pix > 8192) return SPECULA_EINVAL;
  if (!(p->obsc_frac >= 0.0 && p->obsc_frac < 1.0)) return SPECULA_EINVAL;
  if (!(p->pitch_m > 0.0) || !isfinite(p->pitch_m)) return SPECULA_EINVAL;
  return SPECULA_OK;
}

extern "C" int specula_pupil_mask_host(const specula_pupil_desc *pupil, uint8_t *mask_host) {
  int s = check_pupil(pupil);
  if (s) return s;
  if (!mask_host) return SPECULA_EINVAL;
  return host_pupil_mask(pupil->n_pix, pupil->obsc_frac, mask_host);
}

extern "C" int specula_valid_subaps_host(const specula_pupil_desc *pupil, int32_t n_sub,
                                         int32_t *idx_host, int32_t *n_valid) {
  int s = check_pupil(pupil);
  if (s) return s;
  if (!idx_host || !n_valid || n_sub < 1 || n_sub > pupil->n_pix) return SPECULA_EINVAL;
  return host_valid_subaps(pupil->n_pix, pupil->obsc_frac, n_sub, idx_host, n_valid);
}

extern "C" int specula_pyr_image_index_host(const specula_pupil_desc *pupil, int32_t pad,
                                            int32_t pup_dist_px, int32_t n_sub,
                                            int32_t *idx_host, int32_t *n_valid) {
  int s = check_pupil(pupil);
  if (s) return s;
  if (!idx_host || !n_valid || n_sub < 1 || n_sub > pupil->n_pix || pad < 1) return SPECULA_EINVAL;
  // image centres 2 d = pup_dist / b detector pixels apart, b = n_pix / n_sub
  // grid pixels per detector pixel (whole or fractional)
  const int n_det = pad * n_sub;
  if (pup_dist_px < 0 || ((int64_t)pup_dist_px * n_sub) % pupil->n_pix) return SPECULA_EUNSUPPORTED;
  const int two_d = (int)((int64_t)pup_dist_px * n_sub / pupil->n_pix);
  if ((two_d - n_sub) % 2 || n_det % 2) return SPECULA_EUNSUPPORTED;
  std::vector<int32_t> valid((size_t)n_sub * n_sub);
  int32_t nv = 0;
  if ((s = host_valid_subaps(pupil->n_pix, pupil->obsc_frac, n_sub, valid.data(), &nv))) return s;
  const int sxs[4] = {1, -1, -1, 1}, sys[4] = {1, 1, -1, -1};
  for (int q = 0; q < 4; ++q) {
    const int r0 = (n_det + sys[q] * two_d - n_sub) / 2, c0 = (n_det + sxs[q] * two_d - n_sub) / 2;
    if (r0 < 0 || r0 + n_sub > n_det || c0 < 0 || c0 + n_sub > n_det) return SPECULA_EUNSUPPORTED;
    for (int k = 0; k < nv; ++k) {
      const int a = valid[k] / n_sub, c = valid[k] % n_sub;
      idx_host[(size_t)q * nv + k] = (r0 + a) * n_det + (c0 + c);
    }
  }
  *n_valid = nv;
  return SPECULA_OK;
}

extern "C" int specula_mod_table_host(int32_t n_mod, double *cos_host, double *sin_host) {
  if (n_mod < 1 || !cos_host || !sin_host) return SPECULA_EINVAL;
  for (int m = 0; m < n_mod; ++m) {
    const double th = 2.0 * M_PI * m / n_mod;
    cos_host[m] = cos(th);
    sin_host[m] = sin(th);
  }
  return SPECULA_OK;
}

// Device versions of the integer rules.
__global__ void k_pupil_mask(int n, double thr, float *amp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n || j >= n) return;
  const long long dx = 2LL * i - n + 1, dy = 2LL * j - n + 1;
  const long long r4 = dx * dx + dy * dy;
  amp[(size_t)j * n + i] = (r4 <= (long long)n * n && (double)r4 > thr) ? 1.0f : 0.0f;
}

// One CTA: count pupil pixels per subaperture, flag, ordered compaction.
__global__ void k_valid_subaps(int n, double thr, int n_sub, int32_t *idx, int32_t *n_valid) {
  __shared__ int32_t s_scan[1024];
  const int b = n / n_sub;
  const int total = n_sub * n_sub;
  const int per = (total + blockDim.x - 1) / blockDim.x;   // <= 16 (n_sub <= 128)
  const int t = threadIdx.x;
  uint32_t flags = 0;
  int mine = 0;
  for (int q = 0; q < per; ++q) {
    const int s = t * per + q;
    if (s >= total) break;
    const int a = s / n_sub, c = s % n_sub;
    int in = 0;
    for (int y = 0; y < b; ++y) {
      const long long dy = 2LL * (a * b + y) - n + 1;
      for (int x = 0; x < b; ++x) {
        const long long dx = 2LL * (c * b + x) - n + 1;
        const long long r4 = dx * dx + dy * dy;
        in += (r4 <= (long long)n * n && (double)r4 > thr) ? 1 : 0;
      }
    }
    if (2 * in >= b * b) { flags |= 1u << q; ++mine; }
  }
  s_scan[t] = mine;
  __syncthreads();
  // inclusive Hillis-Steele scan
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = (t >= off) ? s_scan[t - off] : 0;
    __syncthreads();
    s_scan[t] += v;
    __syncthreads();
  }
  int pos = s_scan[t] - mine;
  for (int q = 0; q < per; ++q) {
    const int s = t * per + q;
    if (s >= total) break;
    if (flags & (1u << q)) idx[pos++] = s;
  }
  if (t == blockDim.x - 1) *n_valid = s_scan[t];
}

extern "C" int specula_pupil_mask(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                  float *amp_dev, void *stream) {
  if (!ctx || !amp_dev) return SPECULA_EINVAL;
  int s = check_pupil(pupil);
  if (s) return s;
  const int n = pupil->n_pix;
  const double e = pupil->obsc_frac * (double)n;
  dim3 grid((n + 127) / 128, n);
  k_pupil_mask<<<grid, 128, 0, (cudaStream_t)stream>>>(n, e * e, amp_dev);
  SPECULA_CK_LAUNCH();
  return SPECULA_OK;
}

extern "C" int specula_valid_subaps(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                    int32_t n_sub, int32_t *idx_dev, int32_t *n_valid_dev,
                                    void *stream) {
  if (!ctx || !idx_dev || !n_valid_dev) return SPECULA_EINVAL;
  int s = check_pupil(pupil);
  if (s) return s;
  if (n_sub < 1 || n_sub > 128 || pupil->n_pix % n_sub) return SPECULA_EINVAL;
  const int n = pupil->n_pix;
  const double e = pupil->obsc_frac * (double)n;
  k_valid_subaps<<<1, 1024, 0, (cudaStream_t)stream>>>(n, e * e, n_sub, idx_dev, n_valid_dev);
  SPECULA_CK_LAUNCH();
  return SPECULA_OK;
}

// ---- pyramid / SH dispatch -----------------------------------------------------

static int check_pwfs(const specula_pupil_desc *pupil, const specula_pwfs_desc *p) {
  int s = check_pupil(pupil);
  if (s) return s;
  if (!p) return SPECULA_EINVAL;
  if (p->pad < 1 || p->n_mod < 1 || p->n_mod > 4096 || p->n_sub < 1) return SPECULA_EINVAL;
  if (p->n_sub > pupil->n_pix) return SPECULA_EINVAL;
  if (!(p->mod_amp >= 0.0) || !isfinite(p->mod_amp)) return SPECULA_EINVAL;
  // padding 2-4; the four pupil images (n_pix wide, centres pup_dist apart)
  // inside the padded grid
  if (p->pad < 2 || p->pad > 4) return SPECULA_EUNSUPPORTED;
  if (p->pup_dist_px < 1 || p->pup_dist_px + pupil->n_pix > p->pad * pupil->n_pix)
    return SPECULA_EUNSUPPORTED;
  return SPECULA_OK;
}

extern "C" int specula_pwfs_plan(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                 const specula_pwfs_desc *pwfs) {
  if (!ctx) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  if (pwfs_plan_find(ctx, pupil, pwfs)) return SPECULA_OK;
  SPECULA_CK(cudaSetDevice(ctx->device));
  PwfsPlan *p = nullptr;
  return pwfs_plan_build(ctx, pupil, pwfs, &p);
}

extern "C" int specula_pwfs_set_tiles(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                      const specula_pwfs_desc *pwfs, int32_t chunk, int32_t ka,
                                      int32_t passes) {
  if (!ctx) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  if (chunk < 1 || chunk > 4096 || ka < 1 || ka > 64) return SPECULA_EINVAL;
  if (passes < 2 || passes > 4) return SPECULA_EINVAL;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  SPECULA_CK(cudaSetDevice(ctx->device));
  return pwfs_set_tiles(p, chunk, ka, passes);
}

extern "C" int specula_pwfs_set_form(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                     const specula_pwfs_desc *pwfs, int32_t form) {
  if (!ctx) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  if (form < SPECULA_PWFS_FORM_TILT || form > SPECULA_PWFS_FORM_DFTGEMM_TF32) return SPECULA_EINVAL;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  SPECULA_CK(cudaSetDevice(ctx->device));
  if (form == SPECULA_PWFS_FORM_SHIFTED && !p->sm_chunk) {
    SPECULA_CK(cudaDeviceSynchronize());
    if ((s = pwfs_shifted_prepare(p))) return s;
  }
  if ((form == SPECULA_PWFS_FORM_DFTGEMM_BF16 || form == SPECULA_PWFS_FORM_DFTGEMM_TF32) &&
      p->dg_form != form) {
    SPECULA_CK(cudaDeviceSynchronize());
    if ((s = pwfs_dftgemm_prepare(p, form))) return s;
  }
  p->form = form;
  return SPECULA_OK;
}

extern "C" int specula_pwfs_set_slots(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                      const specula_pwfs_desc *pwfs, int32_t slot_begin,
                                      int32_t slot_end) {
  if (!ctx) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  if (slot_begin < 0 || slot_end <= slot_begin || slot_end > p->nc) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());   // the workspace may be in use
  const bool all = slot_begin == 0 && slot_end == p->nc;
  p->slot_lo = all ? 0 : slot_begin;
  p->slot_hi = all ? -1 : slot_end;
  if (p->part.p) SPECULA_CK(cudaMemset(p->part.p, 0, p->part.bytes));
  return SPECULA_OK;
}

extern "C" int specula_pwfs_autotune(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                     const specula_pwfs_desc *pwfs, const float *amp_dev,
                                     const float *phase_dev, int32_t n_batch, float *det_dev,
                                     int32_t reps, int64_t max_workspace_bytes, int32_t *chunk,
                                     int32_t *ka, int32_t *passes, void *stream) {
  if (!ctx || !amp_dev || !phase_dev || !det_dev || !chunk || !ka || !passes)
    return SPECULA_EINVAL;
  if (n_batch < 1 || reps < 1 || reps > 1000 || max_workspace_bytes < 1) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  if (p->form != SPECULA_PWFS_FORM_TILT || p->slot_hi >= 0) return SPECULA_EUNSUPPORTED;
  SPECULA_CK(cudaSetDevice(ctx->device));
  int bc = 0, bk = 0, bp = 0;
  s = pwfs_autotune(ctx, p, amp_dev, phase_dev, n_batch, det_dev, (cudaStream_t)stream, reps,
                    (size_t)max_workspace_bytes, &bc, &bk, &bp);
  if (s) return s;
  *chunk = bc;
  *ka = bk;
  *passes = bp;
  return SPECULA_OK;
}

extern "C" int specula_pwfs_get_tiles(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                      const specula_pwfs_desc *pwfs, int32_t *chunk, int32_t *ka,
                                      int32_t *passes) {
  if (!ctx || !chunk || !ka || !passes) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  *chunk = p->chunk;
  *ka = p->ka;
  *passes = p->passes;
  return SPECULA_OK;
}

extern "C" int specula_pwfs_image(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                  const specula_pwfs_desc *pwfs, const float *amp_dev,
                                  const float *phase_dev, int32_t n_batch, float *det_dev,
                                  void *stream) {
  if (!ctx || !amp_dev || !phase_dev || !det_dev || n_batch < 0) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  if (n_batch == 0) return SPECULA_OK;
  return pwfs_run(ctx, p, amp_dev, phase_dev, n_batch, det_dev, (cudaStream_t)stream);
}

extern "C" int specula_pwfs_image_poly(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                       const specula_pwfs_desc *pwfs, int32_t n_lambda,
                                       const double *ratio, const double *weight,
                                       const float *amp_dev, const float *phase_dev,
                                       int32_t n_batch, float *det_dev, void *stream) {
  if (!ctx || !amp_dev || !phase_dev || !det_dev || !ratio || !weight || n_batch < 0)
    return SPECULA_EINVAL;
  if (n_lambda < 1 || n_lambda > 64) return SPECULA_EINVAL;
  int s = check_pwfs(pupil, pwfs);
  if (s) return s;
  // every wavelength's plan first (mod_amp in its own lambda / D), so that a
  // missing one fails before anything is enqueued
  PwfsPlan *plans[64];
  for (int i = 0; i < n_lambda; ++i) {
    if (!(ratio[i] > 0.0) || !isfinite(ratio[i]) || !isfinite(weight[i])) return SPECULA_EINVAL;
    specula_pwfs_desc d = *pwfs;
    d.mod_amp = pwfs->mod_amp * ratio[i];
    if ((s = check_pwfs(pupil, &d))) return s;
    if (!(plans[i] = pwfs_plan_find(ctx, pupil, &d))) return SPECULA_ENOPLAN;
  }
  if (n_batch == 0) return SPECULA_OK;
  for (int i = 0; i < n_lambda; ++i) {
    PwfsPlan *p = plans[i];
    p->run_phase_scale = (float)ratio[i];
    p->run_alpha = (float)weight[i];
    p->run_beta = i == 0 ? 0.f : 1.f;
    s = pwfs_run(ctx, p, amp_dev, phase_dev, n_batch, det_dev, (cudaStream_t)stream);
    p->run_phase_scale = 1.f;
    p->run_alpha = 1.f;
    p->run_beta = 0.f;
    if (s) return s;
  }
  return SPECULA_OK;
}

static int check_sh(const specula_pupil_desc *pupil, const specula_sh_desc *sh) {
  int s = check_pupil(pupil);
  if (s) return s;
  if (!sh || sh->n_sub < 1 || sh->sub_pix < 1 || sh->fft_n < sh->sub_pix) return SPECULA_EINVAL;
  if (sh->n_sub * sh->sub_pix != pupil->n_pix) return SPECULA_EINVAL;
  if (!((sh->fft_n == 24 && sh->sub_pix == 12) || (sh->fft_n == 16 && sh->sub_pix == 8) ||
        (sh->fft_n == 56 && sh->sub_pix == 8) || (sh->fft_n == 68 && sh->sub_pix == 4)))
    return SPECULA_EUNSUPPORTED;
  return SPECULA_OK;
}

extern "C" int specula_sh_plan(specula_ctx *ctx, const specula_pupil_desc *pupil,
                               const specula_sh_desc *sh, int32_t *n_valid) {
  if (!ctx) return SPECULA_EINVAL;
  int s = check_sh(pupil, sh);
  if (s) return s;
  ShPlan *p = sh_plan_find(ctx, pupil, sh);
  if (!p) {
    SPECULA_CK(cudaSetDevice(ctx->device));
    s = sh_plan_build(ctx, pupil, sh, &p);
    if (s) return s;
  }
  if (n_valid) *n_valid = p->n_valid;
  return SPECULA_OK;
}

extern "C" int specula_sh_set_range(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                    const specula_sh_desc *sh, int32_t sub_begin,
                                    int32_t sub_end) {
  if (!ctx) return SPECULA_EINVAL;
  int s = check_sh(pupil, sh);
  if (s) return s;
  ShPlan *p = sh_plan_find(ctx, pupil, sh);
  if (!p) return SPECULA_ENOPLAN;
  if (sub_begin < 0 || sub_end < sub_begin || sub_end > p->n_valid) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());   // calls in flight use the old range
  p->sub_lo = sub_begin;
  p->sub_hi = (sub_begin == 0 && sub_end == p->n_valid) ? -1 : sub_end;
  return SPECULA_OK;
}

extern "C" int specula_sh_image(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                const specula_sh_desc *sh, const float *amp_dev,
                                const float *phase_dev, int32_t n_batch, float *spots_dev,
                                void *stream) {
  if (!ctx || !amp_dev || !phase_dev || !spots_dev || n_batch < 0) return SPECULA_EINVAL;
  int s = check_sh(pupil, sh);
  if (s) return s;
  ShPlan *p = sh_plan_find(ctx, pupil, sh);
  if (!p) return SPECULA_ENOPLAN;
  if (n_batch == 0) return SPECULA_OK;
  return sh_run(ctx, p, amp_dev, phase_dev, n_batch, spots_dev, (cudaStream_t)stream);
}

extern "C" int specula_sh_poly_reserve(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                       const specula_sh_desc *sh, int32_t max_batch) {
  if (!ctx || max_batch < 0) return SPECULA_EINVAL;
  int s = check_sh(pupil, sh);
  if (s) return s;
  ShPlan *p = sh_plan_find(ctx, pupil, sh);
  if (!p) return SPECULA_ENOPLAN;
  const size_t need = (size_t)p->n_valid * max_batch * sh->fft_n * sh->fft_n * sizeof(float);
  if (ctx->sh_poly_ws.bytes >= need) return SPECULA_OK;
  SPECULA_CK(cudaSetDevice(ctx->device));
  SPECULA_CK(cudaDeviceSynchronize());   // calls in flight may use the old workspace
  return ctx->sh_poly_ws.alloc(need);
}

extern "C" int specula_sh_image_poly(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                     const specula_sh_desc *sh, int32_t n_lambda,
                                     const double *ratio, const double *weight,
                                     const float *amp_dev, const float *phase_dev,
                                     int32_t n_batch, float *spots_dev, void *stream) {
  if (!ctx || !amp_dev || !phase_dev || !spots_dev || n_batch < 0 || !ratio || !weight)
    return SPECULA_EINVAL;
  if (n_lambda < 1 || n_lambda > 64) return SPECULA_EINVAL;
  for (int i = 0; i < n_lambda; ++i)
    if (!(ratio[i] > 0.0) || !isfinite(ratio[i]) || !isfinite(weight[i])) return SPECULA_EINVAL;
  int s = check_sh(pupil, sh);
  if (s) return s;
  ShPlan *p = sh_plan_find(ctx, pupil, sh);
  if (!p) return SPECULA_ENOPLAN;
  if (sh->fft_n != 24 && sh->fft_n != 16) return SPECULA_EUNSUPPORTED;
  const int nv = (p->sub_hi < 0 ? p->n_valid : p->sub_hi) - p->sub_lo;
  const size_t n_spots = (size_t)nv * n_batch;
  if (n_spots == 0) return SPECULA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = n_spots * sh->fft_n * sh->fft_n * sizeof(float);
  if (ctx->sh_poly_ws.bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SPECULA_CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SPECULA_EUNSUPPORTED;   // grow before capture
    SPECULA_CK(cudaStreamSynchronize(st));
    if ((s = ctx->sh_poly_ws.alloc(need))) return s;
  }
  float *ws = ctx->sh_poly_ws.as<float>();
  for (int i = 0; i < n_lambda; ++i) {
    if ((s = sh_run(ctx, p, amp_dev, phase_dev, n_batch, ws, st, (float)ratio[i]))) return s;
    if ((s = sh_poly_acc(ctx, sh->fft_n, ws, (int)n_spots, ratio[i], weight[i], i == 0,
                         spots_dev, st)))
      return s;
  }
  return SPECULA_OK;
}
