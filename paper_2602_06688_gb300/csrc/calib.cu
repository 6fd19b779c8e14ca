// Calibration: modal basis, push-pull interaction matrix, FP64 pseudo-inverse.
//
// ImCalibrator / RecCalibrator / PushPullGenerator (App. A, Tab. 4) and the
// Intmat / Recmat data objects (Tab. 3); the modal basis stands in for the KL
// files of App. B, Listing 2, which are not public.
//
//  * basis: Zernike modes in Noll order without piston (j = 2 .. n_modes+1),
//    unit RMS on the unit disk, sampled at pupil pixel centres, zero outside
//    the stop; radial polynomials by Kintner's recurrence, evaluated in
//    float64 (on the device, one thread per pixel; the host variant runs the
//    same routine), stored as float32.
//  * IM[:, j] = (s(+a Z_j) - s(-a Z_j)) / (2 a): batches of 16 modes, 32 phase
//    maps, run through the pyramid and slope kernels; columns formed in
//    float64 from the float32 slopes.
//  * R = pinv(A) with eigenvalues of A^T A below rcond^2 lambda_max discarded
//    (singular values below rcond sigma_max): Gram matrix by a float64 GEMM,
//    eigen-decomposition by parallel cyclic Jacobi (round-robin pairs, one
//    rotation per disjoint pair per round), R = V diag(1/lambda) V^T A^T.
//    Float64 throughout, on the GPU (a set-up cost).
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace specula {

// ---------------------------------------------------------------- basis

static void noll_nm(int j, int *n_out, int *m_out) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 < j) ++n;
  const int k = j - n * (n + 1) / 2 - 1;
  const int mabs = (n % 2 == 0) ? 2 * ((k + 1) / 2) : 2 * (k / 2) + 1;
  *n_out = n;
  *m_out = (mabs == 0 || j % 2 == 0) ? mabs : -mabs;
}

// Mode slots of every (n, |m|) up to the radial order of the last mode:
// tab[n (n_max + 1) + |m|] = (q of the cosine or m = 0 mode, q of the sine
// mode), q = j - 2, -1 where absent or beyond n_modes.
static int modal_table(int n_modes, std::vector<int2> *tab) {
  int n_max, m_last;
  noll_nm(n_modes + 1, &n_max, &m_last);
  tab->assign((size_t)(n_max + 1) * (n_max + 1), make_int2(-1, -1));
  for (int j = 2; j <= n_modes + 1; ++j) {
    int n, m;
    noll_nm(j, &n, &m);
    int2 &e = (*tab)[(size_t)n * (n_max + 1) + (m < 0 ? -m : m)];
    if (m < 0)
      e.y = j - 2;
    else
      e.x = j - 2;
  }
  return n_max;
}

// Every Zernike value of one pupil pixel (dx, dy from the centre, rho =
// |(dx, dy)| / half <= 1): the radial polynomials R_n^m by Kintner's
// recurrence in n for each m (stable at the high radial orders a 4000-mode
// basis needs, where the alternating factorial sum cancels catastrophically
// in float64),
//   R_m^m = rho^m,  R_{m+2}^m = ((m + 2) rho^2 - (m + 1)) rho^m,
//   K1 R_p^m = (K2 rho^2 + K3) R_{p-2}^m + K4 R_{p-4}^m,
//   K1 = (p + m)(p - m)(p - 2) / 2,  K2 = 2 p (p - 1)(p - 2),
//   K3 = -m^2 (p - 1) - p (p - 1)(p - 2),  K4 = -p (p + m - 2)(p - m - 2) / 2,
// and cos / sin (m theta) by angle addition; emit(q, value) per mode slot.
template <class Emit>
__host__ __device__ inline void zernike_pixel(double dx, double dy, double half, int n_max,
                                              const int2 *tab, Emit &emit) {
  const double r = sqrt(dx * dx + dy * dy);
  const double rho = r / half, rho2 = rho * rho;
  const double c1 = r > 0.0 ? dx / r : 1.0, s1 = r > 0.0 ? dy / r : 0.0;
  double cm = 1.0, sm = 0.0, rm = 1.0;   // cos, sin of m theta; rho^m
  for (int m = 0; m <= n_max; ++m) {
    double rp4 = 0.0, rp2 = 0.0;
    for (int p = m; p <= n_max; p += 2) {
      double R;
      if (p == m) {
        R = rm;
      } else if (p == m + 2) {
        R = ((m + 2) * rho2 - (m + 1)) * rm;
      } else {
        const double k1 = 0.5 * (double)(p + m) * (double)(p - m) * (double)(p - 2);
        const double k2 = 2.0 * p * (double)(p - 1) * (double)(p - 2);
        const double k3 = -(double)m * m * (double)(p - 1) - (double)p * (p - 1) * (double)(p - 2);
        const double k4 = -0.5 * p * (double)(p + m - 2) * (double)(p - m - 2);
        R = ((k2 * rho2 + k3) * rp2 + k4 * rp4) / k1;
      }
      rp4 = rp2;
      rp2 = R;
      const int2 e = tab[(size_t)p * (n_max + 1) + m];
      if (m == 0) {
        if (e.x >= 0) emit(e.x, sqrt((double)(p + 1)) * R);
      } else {
        const double a = sqrt(2.0 * (p + 1)) * R;
        if (e.x >= 0) emit(e.x, a * cm);
        if (e.y >= 0) emit(e.y, a * sm);
      }
    }
    const double cn = cm * c1 - sm * s1, sn = sm * c1 + cm * s1;
    cm = cn;
    sm = sn;
    rm *= rho;
  }
}

struct EmitHost {
  double *out;
  size_t stride, p;
  __host__ __device__ void operator()(int q, double v) { out[(size_t)q * stride + p] = v; }
};
struct EmitDev {
  float *out;
  size_t stride, p;
  __device__ void operator()(int q, double v) { out[(size_t)q * stride + p] = (float)v; }
};

// The basis of a pupil on the device: one thread per pixel; zero outside
// the stop (the integer rule of specula_pupil_mask).
__global__ void k_modal_basis(int n, double thr, int n_modes, int n_max,
                              const int2 *__restrict__ tab, float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const size_t np2 = (size_t)n * n, p = (size_t)j * n + i;
  const long long dx = 2LL * i - n + 1, dy = 2LL * j - n + 1;
  const long long r4 = dx * dx + dy * dy;
  if (!(r4 <= (long long)n * n && (double)r4 > thr)) {
    for (int q = 0; q < n_modes; ++q) out[(size_t)q * np2 + p] = 0.f;
    return;
  }
  EmitDev em{out, np2, p};
  zernike_pixel(0.5 * (double)dx, 0.5 * (double)dy, 0.5 * n, n_max, tab, em);
}

int modal_basis_host(int n_pix, double obsc, int n_modes, double *out) {
  std::vector<uint8_t> mask((size_t)n_pix * n_pix);
  host_pupil_mask(n_pix, obsc, mask.data());
  std::vector<int2> tab;
  const int n_max = modal_table(n_modes, &tab);
  const size_t np2 = (size_t)n_pix * n_pix;
  for (int y = 0; y < n_pix; ++y)
    for (int x = 0; x < n_pix; ++x) {
      const size_t p = (size_t)y * n_pix + x;
      if (!mask[p]) {
        for (int q = 0; q < n_modes; ++q) out[(size_t)q * np2 + p] = 0.0;
        continue;
      }
      EmitHost em{out, np2, p};
      zernike_pixel(x - (n_pix - 1) / 2.0, y - (n_pix - 1) / 2.0, n_pix / 2.0, n_max, tab.data(),
                    em);
    }
  return SPECULA_OK;
}

// ---------------------------------------------------------------- push-pull IM

__global__ void k_pushpull(const float *__restrict__ basis, int npix2, int j0, int nq, float a,
                           float *__restrict__ phase) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)npix2 * nq) return;
  const int q = (int)(e / npix2);
  const size_t p = e % npix2;
  const float z = basis[(size_t)(j0 + q) * npix2 + p];
  phase[(size_t)(2 * q) * npix2 + p] = a * z;
  phase[(size_t)(2 * q + 1) * npix2 + p] = -a * z;
}

__global__ void k_im_cols(const float *__restrict__ sl, int n_slopes, int n_modes, int j0, int nq,
                          double a, double *__restrict__ im) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_slopes * nq) return;
  const int q = e / n_slopes, s = e % n_slopes;
  const double d = (double)sl[(size_t)(2 * q) * n_slopes + s] -
                   (double)sl[(size_t)(2 * q + 1) * n_slopes + s];
  im[(size_t)s * n_modes + j0 + q] = d / (2.0 * a);
}

// ---------------------------------------------------------------- float64 GEMM
// C[i][j] = sum_k X(i,k) d(k) Y(k,j), X(i,k) = X[i xi + k xk], Y(k,j) = Y[k yk + j yj]
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm_f64(const double *__restrict__ X, long xi, long xk,
                                                  const double *__restrict__ Y, long yk, long yj,
                                                  const double *__restrict__ d, double *__restrict__ C,
                                                  int M, int N, int K) {
  __shared__ double Xs[GK][GT + 1], Ys[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e / GT, ii = e % GT;
      const int k = k0 + kk;
      const int i = i0 + ii, j = j0 + ii;
      double xv = 0.0, yv = 0.0;
      if (k < K && i < M) xv = X[i * xi + k * xk] * (d ? d[k] : 1.0);
      if (k < K && j < N) yv = Y[k * yk + j * yj];
      Xs[kk][ii] = xv;
      Ys[kk][ii] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double xr[4], yr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xr[u] = Xs[kk][ty + 16 * u];
        yr[u] = Ys[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xr[u], yr[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < M && j < N) C[(size_t)i * N + j] = acc[u][v];
    }
}

int gemm_f64(specula_ctx *ctx, cudaStream_t st, const double *X, long xi, long xk,
             const double *Y, long yk, long yj, const double *d, double *C, int M, int N, int K) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                 k_gemm_f64<<<grid, 256, 0, st>>>(X, xi, xk, Y, yk, yj, d, C, M, N, K));
  return SPECULA_OK;
}

// ---------------------------------------------------------------- Jacobi
// Round r of the circle method on np (even) slots: slot 0 holds index 0, slot
// k >= 1 holds ((k - 1 + r) mod (np - 1)) + 1; pair i = (slot i, slot np-1-i).
__device__ __forceinline__ int rr_index(int slot, int r, int np) {
  return slot == 0 ? 0 : ((slot - 1 + r) % (np - 1)) + 1;
}

__global__ void k_jacobi_params(const double *__restrict__ G, int n, int np, int r,
                                int2 *__restrict__ pq, double2 *__restrict__ cs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np / 2) return;
  int p = rr_index(i, r, np), q = rr_index(np - 1 - i, r, np);
  if (p > q) { const int t = p; p = q; q = t; }
  double c = 1.0, s = 0.0;
  if (q < n) {
    const double apq = G[(size_t)p * n + q];
    if (apq != 0.0) {
      const double app = G[(size_t)p * n + p], aqq = G[(size_t)q * n + q];
      const double th = (aqq - app) / (2.0 * apq);
      const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      c = 1.0 / sqrt(t * t + 1.0);
      s = t * c;
    }
  } else {
    q = p;   // dummy partner (odd n): identity
  }
  pq[i] = make_int2(p, q);
  cs[i] = make_double2(c, s);
}

// G <- J^T G: rows p, q of each pair
__global__ void k_jacobi_rows(double *__restrict__ G, int n, const int2 *__restrict__ pq,
                              const double2 *__restrict__ cs) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int2 e = pq[i];
  if (j >= n || e.x == e.y) return;
  const double2 r = cs[i];
  const double gp = G[(size_t)e.x * n + j], gq = G[(size_t)e.y * n + j];
  G[(size_t)e.x * n + j] = r.x * gp - r.y * gq;
  G[(size_t)e.y * n + j] = r.y * gp + r.x * gq;
}

// G <- G J and V <- V J: columns p, q of each pair
// Column rotations: one grid row per matrix row, threads over the pairs, so
// every matrix row is read and written once per round (the rows are 8 n
// bytes; a thread per row and pair would scatter sector-sized accesses).
__global__ void k_jacobi_cols(double *__restrict__ G, double *__restrict__ V, int n, int npairs,
                              const int2 *__restrict__ pq, const double2 *__restrict__ cs) {
  const int row = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const int2 e = pq[i];
  if (e.x == e.y) return;
  const double2 r = cs[i];
  double *g = G + (size_t)row * n;
  double gp = g[e.x], gq = g[e.y];
  g[e.x] = r.x * gp - r.y * gq;
  g[e.y] = r.y * gp + r.x * gq;
  double *v = V + (size_t)row * n;
  gp = v[e.x];
  gq = v[e.y];
  v[e.x] = r.x * gp - r.y * gq;
  v[e.y] = r.y * gp + r.x * gq;
}

// off-diagonal and total squared norms (one CTA, fixed order)
__global__ void k_offnorm(const double *__restrict__ G, int n, double *__restrict__ out) {
  __shared__ double so[256], st[256];
  double o = 0.0, t = 0.0;
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
    const double v = G[e];
    const size_t r = e / n, c = e % n;
    t += v * v;
    if (r != c) o += v * v;
  }
  so[threadIdx.x] = o;
  st[threadIdx.x] = t;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      so[threadIdx.x] += so[threadIdx.x + h];
      st[threadIdx.x] += st[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = so[0];
    out[1] = st[0];
  }
}

__global__ void k_identity(double *__restrict__ V, int n) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < (size_t)n * n) V[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// d[k] = 1/lambda_k for kept eigenvalues, else 0; count in rank
__global__ void k_inv_eigs(const double *__restrict__ G, int n, double rcond,
                           double *__restrict__ d, int *__restrict__ rank) {
  __shared__ double s_max;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, G[(size_t)k * n + k]);
    s_max = mx;
    *rank = 0;
  }
  __syncthreads();
  const double thr = rcond * rcond * s_max;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double l = G[(size_t)k * n + k];
    const bool keep = l > thr && l > 0.0;
    d[k] = keep ? 1.0 / l : 0.0;
    if (keep) atomicAdd(rank, 1);
  }
}

__global__ void k_f64_to_f32(const double *__restrict__ a, float *__restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Eigen-decomposition of the symmetric n x n float64 matrix G (row-major) by
// parallel cyclic Jacobi: on return G's diagonal holds the eigenvalues and the
// columns of V the eigenvectors.  Sweeps until the off-diagonal squared norm
// is below 1e-30 of the total (at most 40); synchronises the stream per sweep.
int sym_eig_f64(specula_ctx *ctx, cudaStream_t st, double *G_, double *V_, int n) {
  DevBuf PQ, CS, NRM;
  const int np = n + (n & 1);
  int s;
  if ((s = PQ.alloc((size_t)np / 2 * sizeof(int2)))) return s;
  if ((s = CS.alloc((size_t)np / 2 * sizeof(double2)))) return s;
  if ((s = NRM.alloc(2 * sizeof(double)))) return s;
  SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                 k_identity<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, st>>>(V_, n));
  const int npairs = np / 2;
  const dim3 gr((n + 255) / 256, npairs);
  const dim3 gc((npairs + 255) / 256, n);
  for (int sweep = 0; sweep < 40; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                     k_jacobi_params<<<(npairs + 127) / 128, 128, 0, st>>>(
                         G_, n, np, r, PQ.as<int2>(), CS.as<double2>()));
      SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                     k_jacobi_rows<<<gr, 256, 0, st>>>(G_, n, PQ.as<int2>(),
                                                       CS.as<double2>()));
      SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                     k_jacobi_cols<<<gc, 256, 0, st>>>(G_, V_, n, npairs, PQ.as<int2>(),
                                                       CS.as<double2>()));
    }
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_offnorm<<<1, 256, 0, st>>>(G_, n, NRM.as<double>()));
    double h[2];
    SPECULA_CK(cudaMemcpyAsync(h, NRM.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    SPECULA_CK(cudaStreamSynchronize(st));
    if (!(h[0] > 1e-30 * h[1])) break;
  }
  return SPECULA_OK;
}

}  // namespace specula

using namespace specula;

extern "C" int specula_modal_basis_host(const specula_pupil_desc *pupil, int32_t n_modes,
                                        double *basis_host) {
  if (!pupil || !basis_host || n_modes < 1 || n_modes > 20000) return SPECULA_EINVAL;
  if (pupil->n_pix < 2 || pupil->n_pix > 8192 || !(pupil->obsc_frac >= 0 && pupil->obsc_frac < 1))
    return SPECULA_EINVAL;
  return modal_basis_host(pupil->n_pix, pupil->obsc_frac, n_modes, basis_host);
}

extern "C" int specula_modal_basis(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                   int32_t n_modes, float *basis_dev, void *stream) {
  if (!ctx || !basis_dev) return SPECULA_EINVAL;
  if (!pupil || n_modes < 1 || n_modes > 20000 || pupil->n_pix < 2 || pupil->n_pix > 8192)
    return SPECULA_EINVAL;
  if (!(pupil->obsc_frac >= 0 && pupil->obsc_frac < 1)) return SPECULA_EINVAL;
  std::vector<int2> tab;
  const int n_max = modal_table(n_modes, &tab);
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf T;
  int s;
  if ((s = T.upload(tab.data(), tab.size() * sizeof(int2)))) return s;
  const int n = pupil->n_pix;
  const double e = pupil->obsc_frac * (double)n;
  SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                 k_modal_basis<<<dim3((n + 127) / 128, n), 128, 0, st>>>(
                     n, e * e, n_modes, n_max, T.as<int2>(), basis_dev));
  SPECULA_CK(cudaStreamSynchronize(st));   // the table is freed on return
  return SPECULA_OK;
}

extern "C" int specula_calib_intmat(specula_ctx *ctx, const specula_pupil_desc *pupil,
                                    const specula_pwfs_desc *pwfs, const float *amp_dev,
                                    const float *basis_dev, int32_t n_modes, double push_amp,
                                    const specula_slopec_desc *slopec, double *im_dev,
                                    void *stream) {
  if (!ctx || !pupil || !pwfs || !amp_dev || !basis_dev || !slopec || !im_dev) return SPECULA_EINVAL;
  if (n_modes < 1 || !(push_amp > 0) || !isfinite(push_amp)) return SPECULA_EINVAL;
  if ((slopec->kind != SPECULA_SLOPES_PYR && slopec->kind != SPECULA_SLOPES_PYR_MAPS) ||
      !slopec->subap_idx_dev || slopec->n_valid < 1)
    return SPECULA_EINVAL;
  PwfsPlan *p = pwfs_plan_find(ctx, pupil, pwfs);
  if (!p) return SPECULA_ENOPLAN;
  // quadrant slopes: n_sub subapertures per image; image maps: the detector side
  if (slopec->n_sub != (slopec->kind == SPECULA_SLOPES_PYR ? pwfs->n_sub : pwfs->pad * pwfs->n_sub))
    return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int MB = 16;
  const int npix2 = pupil->n_pix * pupil->n_pix;
  const int nd = pwfs->pad * pwfs->n_sub;
  const int ns = 2 * slopec->n_valid;
  DevBuf ph, det, sl;
  int s;
  if ((s = ph.alloc((size_t)2 * MB * npix2 * sizeof(float)))) return s;
  if ((s = det.alloc((size_t)2 * MB * nd * nd * sizeof(float)))) return s;
  if ((s = sl.alloc((size_t)2 * MB * ns * sizeof(float)))) return s;
  for (int j0 = 0; j0 < n_modes; j0 += MB) {
    const int nq = std::min(MB, n_modes - j0);
    const size_t tot = (size_t)npix2 * nq;
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_pushpull<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
                       basis_dev, npix2, j0, nq, (float)push_amp, ph.as<float>()));
    if ((s = pwfs_run(ctx, p, amp_dev, ph.as<float>(), 2 * nq, det.as<float>(), st))) return s;
    if ((s = specula_slopes(ctx, slopec, det.as<float>(), nullptr, 2 * nq, sl.as<float>(), st)))
      return s;
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_im_cols<<<(ns * nq + 255) / 256, 256, 0, st>>>(sl.as<float>(), ns, n_modes,
                                                                      j0, nq, push_amp, im_dev));
  }
  SPECULA_CK(cudaStreamSynchronize(st));   // the workspace is freed on return
  return SPECULA_OK;
}

extern "C" int specula_pinv_fp64(specula_ctx *ctx, const double *A_dev, int32_t m, int32_t n,
                                 double rcond, double *R_dev, float *R32_dev, int32_t *rank,
                                 void *stream) {
  if (!ctx || !A_dev || !R_dev || !rank) return SPECULA_EINVAL;
  if (m < 1 || n < 1 || n > 8192 || !(rcond > 0) || !(rcond < 1)) return SPECULA_EINVAL;
  SPECULA_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf G, V, D, RK;
  int s;
  if ((s = G.alloc((size_t)n * n * sizeof(double)))) return s;
  if ((s = V.alloc((size_t)n * n * sizeof(double)))) return s;
  if ((s = D.alloc((size_t)n * sizeof(double)))) return s;
  if ((s = RK.alloc(sizeof(int)))) return s;
  // G = A^T A
  if ((s = gemm_f64(ctx, st, A_dev, 1, n, A_dev, n, 1, nullptr, G.as<double>(), n, n, m))) return s;
  if ((s = sym_eig_f64(ctx, st, G.as<double>(), V.as<double>(), n))) return s;
  SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                 k_inv_eigs<<<1, 256, 0, st>>>(G.as<double>(), n, rcond, D.as<double>(),
                                               RK.as<int>()));
  // W = V diag(d) V^T into G's storage, then R = W A^T
  if ((s = gemm_f64(ctx, st, V.as<double>(), n, 1, V.as<double>(), 1, n, D.as<double>(),
                    G.as<double>(), n, n, n)))
    return s;
  if ((s = gemm_f64(ctx, st, G.as<double>(), n, 1, A_dev, 1, n, nullptr, R_dev, n, m, n))) return s;
  if (R32_dev) {
    SPECULA_LAUNCH(ctx, SPECULA_K_CALIB, st,
                   k_f64_to_f32<<<1216, 256, 0, st>>>(R_dev, R32_dev, (size_t)n * m));
  }
  int hr = 0;
  SPECULA_CK(cudaMemcpyAsync(&hr, RK.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPECULA_CK(cudaStreamSynchronize(st));
  *rank = hr;
  return SPECULA_OK;
}
