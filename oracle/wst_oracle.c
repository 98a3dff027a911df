/*
 * FP64 oracle of the w-stacking imager (Gheller, Taffoni & Goz, arXiv:2301.06061).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct CPU
 * statement of what the GPU path computes.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Everything is double precision.  FP32 inputs (u, v, w, visibilities, weights)
 * are promoted exactly.  The file is compiled with -ffp-contract=off so that the
 * coordinate arithmetic below rounds exactly as written.
 *
 * Method (paper section 2):
 *   Eq. 1  V(u,v,w) = sum over sky of I/n * exp(-2 pi i (u l + v m + w (n-1)))
 *   Eq. 2  w-stacking inversion: per w-plane 2D inverse Fourier transform of the
 *          gridded visibilities, multiplied by exp(+2 pi i w (n-1)), summed over w.
 *   Eq. 3  convolutional gridding: grid(u_i, v_j, w_k) = sum_m V_m G(...)
 *          with a Gaussian kernel of 7 cells support; visibilities go to the
 *          closest w-plane (no convolution along w).
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - grid coordinate x = N/2 + u*FoV (cells), tap start i0 = ceil(x - W/2),
 *     W consecutive cells i0..i0+W-1 weighted by G(i - x);
 *   - a visibility whose footprint leaves [0,N) on either axis is dropped;
 *   - planes are cell-centred: k = clamp(floor((w - w_min) * (N_w/(w_max - w_min))),
 *     0, N_w-1), plane centre w_k = w_min + (k + 1/2) dw, dw = (w_max - w_min)/N_w;
 *   - image pixel (a, b) sits at l = (a - N/2) FoV/N, m = (b - N/2) FoV/N,
 *     stored row-major with row index b (m) and column index a (l);
 *   - the output is the unnormalised dirty image
 *       D(a,b) = sum_k e^{2 pi i w_k t(l,m)} F_k(a,b) / (Ghat(nu_a) Ghat(nu_b)),
 *     t = n - 1 = -(l^2+m^2)/(1+sqrt(1-l^2-m^2)), nu_a = (a - N/2)/N, and
 *     D = 0 where l^2 + m^2 >= 1;
 *   - Ghat(nu) = integral over [-W/2, W/2] of G(x) cos(2 pi nu x) dx.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WO_PI 3.14159265358979323846264338327950288

enum { WO_GAUSS = 0, WO_ES = 1, WO_TABLE = 2 };

typedef struct {
  int32_t n;          /* image side (cells = pixels per axis)                  */
  double fov;         /* field of view, radians                                */
  int32_t n_w;        /* number of w-planes                                    */
  double w_min;       /* plane range, already resolved by the caller           */
  double w_max;
  int32_t support;    /* W, kernel support in cells                            */
  int32_t kernel;     /* WO_GAUSS, WO_ES or WO_TABLE                           */
  double kparam;      /* Gaussian sigma in cells, or the ES beta               */
  const double *ktable; /* WO_TABLE: samples of G on [-W/2, W/2], uniform      */
  int32_t ktable_len;
} wo_config;

/* ------------------------------------------------------------------------- */
/* Convolution kernel G (Eq. 3)                                               */
/* ------------------------------------------------------------------------- */

double wo_kernel_eval(const wo_config *c, double x) {
  const double half = 0.5 * c->support;
  if (x < -half || x > half) return 0.0;
  if (c->kernel == WO_GAUSS) {
    const double s = c->kparam;
    return exp(-(x * x) / (2.0 * s * s));
  }
  if (c->kernel == WO_ES) {
    /* exponential of semicircle, exp(beta (sqrt(1 - (2x/W)^2) - 1)) */
    const double z = 2.0 * x / c->support;
    return exp(c->kparam * (sqrt(1.0 - z * z) - 1.0));
  }
  /* piecewise-linear interpolation of a uniform table on [-W/2, W/2] */
  const int L = c->ktable_len;
  const double pos = (x + half) * (double)(L - 1) / (double)c->support;
  int i = (int)floor(pos);
  if (i < 0) i = 0;
  if (i > L - 2) i = L - 2;
  const double f = pos - (double)i;
  return (1.0 - f) * c->ktable[i] + f * c->ktable[i + 1];
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(WO_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    /* recompute derivative at the converged node */
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void wo_gauss_legendre(int n, double *x, double *w) { gauss_legendre(n, x, w); }

/*
 * Ghat(nu) = int_{-W/2}^{W/2} G(x) cos(2 pi nu x) dx, composite Gauss-Legendre:
 * the support is cut into segments (64 per cell for analytic kernels, one per
 * table interval for tabulated kernels, so that every kink of the piecewise
 * linear table is a segment end) with 16 nodes per segment.
 */
void wo_kernel_ft(const wo_config *c, int64_t n_nu, const double *nu, double *out) {
  const int NG = 16;
  double gx[16], gw[16];
  gauss_legendre(NG, gx, gw);
  const double half = 0.5 * c->support;
  const int nseg = (c->kernel == WO_TABLE) ? (c->ktable_len - 1) : 64 * c->support;
  const double h = (double)c->support / nseg;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_nu; ++i) {
    double acc = 0.0;
    for (int s = 0; s < nseg; ++s) {
      const double a = -half + s * h;
      const double mid = a + 0.5 * h;
      double part = 0.0;
      for (int g = 0; g < NG; ++g) {
        const double x = mid + 0.5 * h * gx[g];
        part += gw[g] * wo_kernel_eval(c, x) * cos(2.0 * WO_PI * nu[i] * x);
      }
      acc += 0.5 * h * part;
    }
    out[i] = acc;
  }
}

/* ------------------------------------------------------------------------- */
/* Visibility placement (Eq. 3 discretisation, nearest w-plane)               */
/* ------------------------------------------------------------------------- */

/* status codes written per visibility by wo_locate */
enum { WO_KEPT = 0, WO_DROPPED = 1, WO_NONFINITE = 2 };

static double plane_width(const wo_config *c) { return (c->w_max - c->w_min) / c->n_w; }

static int locate_one(const wo_config *c, float uf, float vf, float wf, int32_t *k, int32_t *i0,
                      int32_t *j0, double *x, double *y) {
  if (!isfinite(uf) || !isfinite(vf) || !isfinite(wf)) return WO_NONFINITE;
  const double half_n = 0.5 * c->n;
  const double half_w = 0.5 * c->support;
  const double xx = half_n + (double)uf * c->fov;
  const double yy = half_n + (double)vf * c->fov;
  const double ci = ceil(xx - half_w);
  const double cj = ceil(yy - half_w);
  if (ci < 0.0 || cj < 0.0 || ci + c->support > c->n || cj + c->support > c->n) return WO_DROPPED;
  /* plane scale N_w / (w_max - w_min): one rounded product per visibility */
  const double range = c->w_max - c->w_min;
  int32_t kk = 0;
  if (range > 0.0) {
    const double scale = (double)c->n_w / range;
    const double q = floor(((double)wf - c->w_min) * scale);
    if (q < 0.0)
      kk = 0;
    else if (q > c->n_w - 1)
      kk = c->n_w - 1;
    else
      kk = (int32_t)q;
  }
  *k = kk;
  *i0 = (int32_t)ci;
  *j0 = (int32_t)cj;
  *x = xx;
  *y = yy;
  return WO_KEPT;
}

static int vis_finite(const float *vis, const float *weight, int64_t j) {
  if (!isfinite(vis[2 * j]) || !isfinite(vis[2 * j + 1])) return 0;
  if (weight && !isfinite(weight[j])) return 0;
  return 1;
}

/* Per visibility: plane k, tap starts (i0, j0) and status; k = i0 = j0 = -1 when
 * not kept.  Returns the number of kept visibilities. */
int64_t wo_locate(const wo_config *c, int64_t n_vis, const float *u, const float *v, const float *w,
                  const float *vis, const float *weight, int32_t *k_out, int32_t *i0_out,
                  int32_t *j0_out, int32_t *status_out) {
  int64_t kept = 0;
  for (int64_t j = 0; j < n_vis; ++j) {
    int32_t k = -1, i0 = -1, j0 = -1;
    double x, y;
    int st = locate_one(c, u[j], v[j], w[j], &k, &i0, &j0, &x, &y);
    /* a non-finite input of any kind is counted as such, before the footprint test */
    if (!vis_finite(vis, weight, j)) st = WO_NONFINITE;
    if (st != WO_KEPT) k = i0 = j0 = -1;
    else ++kept;
    if (k_out) k_out[j] = k;
    if (i0_out) i0_out[j] = i0;
    if (j0_out) j0_out[j] = j0;
    if (status_out) status_out[j] = st;
  }
  return kept;
}

/* Eq. 3: grid planes [k0, k1) into out[(k - k0) * N*N + q*N + p] (row q = v axis). */
void wo_grid(const wo_config *c, int64_t n_vis, const float *u, const float *v, const float *w,
             const float *vis, const float *weight, int32_t k0, int32_t k1, double complex *out) {
  const int64_t N = c->n;
  const int W = c->support;
  memset(out, 0, sizeof(double complex) * (size_t)(k1 - k0) * N * N);
  for (int64_t j = 0; j < n_vis; ++j) {
    int32_t k, i0, j0;
    double x, y;
    if (locate_one(c, u[j], v[j], w[j], &k, &i0, &j0, &x, &y) != WO_KEPT) continue;
    if (!vis_finite(vis, weight, j)) continue;
    if (k < k0 || k >= k1) continue;
    const double om = weight ? (double)weight[j] : 1.0;
    const double complex V = om * ((double)vis[2 * j] + I * (double)vis[2 * j + 1]);
    double complex *g = out + (int64_t)(k - k0) * N * N;
    for (int b = 0; b < W; ++b) {
      const double gy = wo_kernel_eval(c, (double)(j0 + b) - y);
      for (int a = 0; a < W; ++a) {
        const double gxv = wo_kernel_eval(c, (double)(i0 + a) - x);
        g[(int64_t)(j0 + b) * N + (i0 + a)] += V * gxv * gy;
      }
    }
  }
}

/* ------------------------------------------------------------------------- */
/* FFT: textbook iterative radix-2 Cooley-Tukey, double precision             */
/* ------------------------------------------------------------------------- */

/* In-place length-n (power of two) DFT  X[k] = sum_j x[j] exp(sign 2 pi i j k / n). */
void wo_fft1d(double complex *x, int64_t n, int sign) {
  /* bit-reversal permutation */
  for (int64_t i = 1, j = 0; i < n; ++i) {
    int64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double complex t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  for (int64_t len = 2; len <= n; len <<= 1) {
    const int64_t h = len >> 1;
    for (int64_t m = 0; m < h; ++m) {
      const double ang = sign * 2.0 * WO_PI * (double)m / (double)len;
      const double complex tw = cos(ang) + I * sin(ang);
      for (int64_t s = 0; s < n; s += len) {
        const double complex a = x[s + m];
        const double complex b = x[s + m + h] * tw;
        x[s + m] = a + b;
        x[s + m + h] = a - b;
      }
    }
  }
}

/*
 * Centred unnormalised 2D transform of an N x N array (row index q, column p):
 *   F[b,a] = sum_{q,p} g[q,p] exp(sign 2 pi i ((p-N/2)(a-N/2) + (q-N/2)(b-N/2)) / N)
 * computed as (-1)^(p+q) pre-multiplication, row and column FFTs, and (-1)^(a+b)
 * post-multiplication (valid for N divisible by 4).
 */
void wo_fft2_centered(double complex *g, int64_t N, int sign) {
  for (int64_t q = 0; q < N; ++q)
    for (int64_t p = 0; p < N; ++p)
      if ((p + q) & 1) g[q * N + p] = -g[q * N + p];
#pragma omp parallel
  {
    double complex *line = (double complex *)malloc(sizeof(double complex) * N);
#pragma omp for schedule(static)
    for (int64_t q = 0; q < N; ++q) wo_fft1d(g + q * N, N, sign);
#pragma omp for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
      for (int64_t q = 0; q < N; ++q) line[q] = g[q * N + p];
      wo_fft1d(line, N, sign);
      for (int64_t q = 0; q < N; ++q) g[q * N + p] = line[q];
    }
    free(line);
  }
  for (int64_t b = 0; b < N; ++b)
    for (int64_t a = 0; a < N; ++a)
      if ((a + b) & 1) g[b * N + a] = -g[b * N + a];
}

/* ------------------------------------------------------------------------- */
/* Phase screen and plane accumulation (Eq. 2)                                */
/* ------------------------------------------------------------------------- */

/* t = n - 1 = sqrt(1 - l^2 - m^2) - 1, written without cancellation; NAN outside the sphere */
static double n_minus_one(double l, double m) {
  const double r2 = l * l + m * m;
  if (r2 >= 1.0) return NAN;
  return -r2 / (1.0 + sqrt(1.0 - r2));
}

double wo_n_minus_one(double l, double m) { return n_minus_one(l, m); }

static double complex cis_cycles(double phi) {
  /* exp(2 pi i phi), argument reduced modulo one cycle first */
  const double r = phi - floor(phi + 0.5);
  return cos(2.0 * WO_PI * r) + I * sin(2.0 * WO_PI * r);
}

static double plane_centre(const wo_config *c, int k) { return c->w_min + (k + 0.5) * plane_width(c); }

double wo_plane_centre(const wo_config *c, int k) { return plane_centre(c, k); }

/* per-axis correction 1/Ghat(nu_a), nu_a = (a - N/2)/N */
static double *correction_table(const wo_config *c) {
  const int64_t N = c->n;
  double *nu = (double *)malloc(sizeof(double) * N);
  double *gh = (double *)malloc(sizeof(double) * N);
  for (int64_t a = 0; a < N; ++a) nu[a] = (double)(a - N / 2) / (double)N;
  wo_kernel_ft(c, N, nu, gh);
  for (int64_t a = 0; a < N; ++a) gh[a] = 1.0 / gh[a];
  free(nu);
  return gh;
}

/*
 * The full w-stacking image (paper section 2, Eq. 2-3): for each plane, grid,
 * centred 2D transform with the positive exponent, multiply by the plane's
 * phase screen and add into the image; finally divide by Ghat(nu_a) Ghat(nu_b).
 * apply_correction = 0 returns the uncorrected sum U instead.
 */
void wo_image(const wo_config *c, int64_t n_vis, const float *u, const float *v, const float *w,
              const float *vis, const float *weight, int apply_correction, double complex *image) {
  const int64_t N = c->n;
  const double dl = c->fov / (double)N;
  double complex *plane = (double complex *)malloc(sizeof(double complex) * N * N);
  memset(image, 0, sizeof(double complex) * N * N);
  for (int k = 0; k < c->n_w; ++k) {
    wo_grid(c, n_vis, u, v, w, vis, weight, k, k + 1, plane);
    wo_fft2_centered(plane, N, +1);
    const double wk = plane_centre(c, k);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < N; ++b) {
      const double m = (double)(b - N / 2) * dl;
      for (int64_t a = 0; a < N; ++a) {
        const double l = (double)(a - N / 2) * dl;
        const double t = n_minus_one(l, m);
        if (isnan(t)) continue;
        image[b * N + a] += cis_cycles(wk * t) * plane[b * N + a];
      }
    }
  }
  free(plane);
  if (apply_correction) {
    double *corr = correction_table(c);
    for (int64_t b = 0; b < N; ++b)
      for (int64_t a = 0; a < N; ++a) image[b * N + a] *= corr[a] * corr[b];
    free(corr);
  }
}

/*
 * The same w-stacking image evaluated directly at chosen pixels, without planes
 * or FFTs: the gridding sum and the plane transform commute, so
 *   D(a,b) = C_a C_b sum_j w_j V_j S_{k_j}(a,b) Kx_j(a) Ky_j(b),
 *   Kx_j(a) = sum_{s<W} G(i0_j + s - x_j) exp(2 pi i (i0_j + s - N/2)(a - N/2)/N).
 * Used where the planes do not fit (16384^2) and as a cross-check of wo_image.
 */
void wo_image_pixels(const wo_config *c, int64_t n_vis, const float *u, const float *v,
                     const float *w, const float *vis, const float *weight, int apply_correction,
                     int64_t n_pix, const int32_t *pa, const int32_t *pb, double complex *out) {
  const int64_t N = c->n;
  const int W = c->support;
  const double dl = c->fov / (double)N;
  /* exp(2 pi i m / N) for m in [0, N) */
  double complex *cis = (double complex *)malloc(sizeof(double complex) * N);
  for (int64_t m = 0; m < N; ++m) cis[m] = cexp(2.0 * WO_PI * I * (double)m / (double)N);
  double *ghat = NULL;
  if (apply_correction) {
    double *nu = (double *)malloc(sizeof(double) * 2 * n_pix);
    ghat = (double *)malloc(sizeof(double) * 2 * n_pix);
    for (int64_t i = 0; i < n_pix; ++i) {
      nu[2 * i] = (double)(pa[i] - N / 2) / (double)N;
      nu[2 * i + 1] = (double)(pb[i] - N / 2) / (double)N;
    }
    wo_kernel_ft(c, 2 * n_pix, nu, ghat);
    free(nu);
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n_pix; ++i) {
    const int64_t a = pa[i], b = pb[i];
    const double l = (double)(a - N / 2) * dl, m = (double)(b - N / 2) * dl;
    const double t = n_minus_one(l, m);
    if (isnan(t)) {
      out[i] = 0.0;
      continue;
    }
    double complex *screen = (double complex *)malloc(sizeof(double complex) * c->n_w);
    for (int k = 0; k < c->n_w; ++k) screen[k] = cis_cycles(plane_centre(c, k) * t);
    double complex acc = 0.0;
    for (int64_t j = 0; j < n_vis; ++j) {
      int32_t k, i0, j0;
      double x, y;
      if (locate_one(c, u[j], v[j], w[j], &k, &i0, &j0, &x, &y) != WO_KEPT) continue;
      if (!vis_finite(vis, weight, j)) continue;
      const double om = weight ? (double)weight[j] : 1.0;
      double complex kx = 0.0, ky = 0.0;
      for (int s = 0; s < W; ++s) {
        int64_t mx = ((int64_t)(i0 + s - N / 2) * (a - N / 2)) % N;
        if (mx < 0) mx += N;
        int64_t my = ((int64_t)(j0 + s - N / 2) * (b - N / 2)) % N;
        if (my < 0) my += N;
        kx += wo_kernel_eval(c, (double)(i0 + s) - x) * cis[mx];
        ky += wo_kernel_eval(c, (double)(j0 + s) - y) * cis[my];
      }
      const double complex V = om * ((double)vis[2 * j] + I * (double)vis[2 * j + 1]);
      acc += V * screen[k] * kx * ky;
    }
    free(screen);
    if (apply_correction) acc /= ghat[2 * i] * ghat[2 * i + 1];
    out[i] = acc;
  }
  free(cis);
  free(ghat);
}

/*
 * Direct Fourier transform (the exact dirty image the method approximates):
 *   D(l,m) = sum_j w_j V_j exp(+2 pi i (u_j l + v_j m + w_j (n - 1)))
 * for pixels (a, b) of an N x N image with spacing FoV/N.  No w-binning, no kernel.
 */
void wo_dft_pixels(int64_t n_vis, const float *u, const float *v, const float *w, const float *vis,
                   const float *weight, int32_t n, double fov, int64_t n_pix, const int32_t *pa,
                   const int32_t *pb, double complex *out) {
  const double dl = fov / (double)n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n_pix; ++i) {
    const double l = (double)(pa[i] - n / 2) * dl, m = (double)(pb[i] - n / 2) * dl;
    const double t = n_minus_one(l, m);
    if (isnan(t)) {
      out[i] = 0.0;
      continue;
    }
    double complex acc = 0.0;
    for (int64_t j = 0; j < n_vis; ++j) {
      if (!isfinite(u[j]) || !isfinite(v[j]) || !isfinite(w[j])) continue;
      if (!vis_finite(vis, weight, j)) continue;
      const double om = weight ? (double)weight[j] : 1.0;
      const double phi = (double)u[j] * l + (double)v[j] * m + (double)w[j] * t;
      acc += om * ((double)vis[2 * j] + I * (double)vis[2 * j + 1]) * cis_cycles(phi);
    }
    out[i] = acc;
  }
}

/* Forward measurement (Eq. 1) of a point-source sky, used only by tests:
 *   V_j = sum_s S_s exp(-2 pi i (u_j l_s + v_j m_s + w_j (n_s - 1))). */
void wo_predict_points(int64_t n_vis, const float *u, const float *v, const float *w, int64_t n_src,
                       const double *l, const double *m, const double *flux, double complex *out) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n_vis; ++j) {
    double complex acc = 0.0;
    for (int64_t s = 0; s < n_src; ++s) {
      const double t = n_minus_one(l[s], m[s]);
      const double phi = (double)u[j] * l[s] + (double)v[j] * m[s] + (double)w[j] * t;
      acc += flux[s] * cis_cycles(-phi);
    }
    out[j] = acc;
  }
}

/* ------------------------------------------------------------------------- */
/* Adjoint (the conjugate transpose of wo_image, step by step in reverse)     */
/* ------------------------------------------------------------------------- */

/*
 * dvis_j = w_j sum_{taps} G(i0+s-x_j) G(j0+r-y_j) gh_{k_j}[j0+r, i0+s],
 * gh_k = centred 2D transform with the negative exponent of
 *        conj(screen_k) * C_a C_b * dimage        (C omitted if apply_correction = 0).
 * Dropped and non-finite visibilities receive 0.
 */
void wo_degrid(const wo_config *c, int64_t n_vis, const float *u, const float *v, const float *w,
               const float *vis, const float *weight, int apply_correction,
               const double complex *dimage, double complex *dvis) {
  const int64_t N = c->n;
  const int W = c->support;
  const double dl = c->fov / (double)N;
  double *corr = apply_correction ? correction_table(c) : NULL;
  double complex *plane = (double complex *)malloc(sizeof(double complex) * N * N);
  for (int64_t j = 0; j < n_vis; ++j) dvis[j] = 0.0;
  for (int k = 0; k < c->n_w; ++k) {
    const double wk = plane_centre(c, k);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < N; ++b) {
      const double m = (double)(b - N / 2) * dl;
      for (int64_t a = 0; a < N; ++a) {
        const double l = (double)(a - N / 2) * dl;
        const double t = n_minus_one(l, m);
        double complex val = 0.0;
        if (!isnan(t)) {
          val = conj(cis_cycles(wk * t)) * dimage[b * N + a];
          if (corr) val *= corr[a] * corr[b];
        }
        plane[b * N + a] = val;
      }
    }
    wo_fft2_centered(plane, N, -1);
    for (int64_t j = 0; j < n_vis; ++j) {
      int32_t kk, i0, j0;
      double x, y;
      if (locate_one(c, u[j], v[j], w[j], &kk, &i0, &j0, &x, &y) != WO_KEPT) continue;
      if (!vis_finite(vis, weight, j)) continue;
      if (kk != k) continue;
      const double om = weight ? (double)weight[j] : 1.0;
      double complex acc = 0.0;
      for (int r = 0; r < W; ++r) {
        const double gy = wo_kernel_eval(c, (double)(j0 + r) - y);
        for (int s = 0; s < W; ++s) {
          const double gxv = wo_kernel_eval(c, (double)(i0 + s) - x);
          acc += gxv * gy * plane[(int64_t)(j0 + r) * N + (i0 + s)];
        }
      }
      dvis[j] = om * acc;
    }
  }
  free(plane);
  free(corr);
}

/*
 * Gradient of a real loss with respect to the samples of a tabulated kernel,
 * through the uncorrected image U (the grid correction is differentiated by the
 * caller).  With gh_k the adjoint grid of dU (as in wo_degrid, no correction)
 * and c_{rs} = Re(conj(gh_k[j0+r, i0+s]) * w_j V_j) for each tap, every tap adds
 *   c_{rs} * G_y(r) * dG_x(s)/dtable  +  c_{rs} * G_x(s) * dG_y(r)/dtable,
 * where dG/dtable is the linear-interpolation weight of the two bracketing samples.
 * The result is the derivative d Re<dU, U> / d table, i.e. the chain rule for a real
 * loss whose gradient with respect to U (conjugate-Wirtinger convention) is dU.
 */
void wo_kernel_grad(const wo_config *c, int64_t n_vis, const float *u, const float *v,
                    const float *w, const float *vis, const float *weight,
                    const double complex *dimage, double *dtable) {
  const int64_t N = c->n;
  const int W = c->support;
  const int L = c->ktable_len;
  const double half = 0.5 * W;
  const double dl = c->fov / (double)N;
  double complex *plane = (double complex *)malloc(sizeof(double complex) * N * N);
  for (int i = 0; i < L; ++i) dtable[i] = 0.0;
  for (int k = 0; k < c->n_w; ++k) {
    const double wk = plane_centre(c, k);
    for (int64_t b = 0; b < N; ++b) {
      const double m = (double)(b - N / 2) * dl;
      for (int64_t a = 0; a < N; ++a) {
        const double l = (double)(a - N / 2) * dl;
        const double t = n_minus_one(l, m);
        plane[b * N + a] = isnan(t) ? 0.0 : conj(cis_cycles(wk * t)) * dimage[b * N + a];
      }
    }
    wo_fft2_centered(plane, N, -1);
    for (int64_t j = 0; j < n_vis; ++j) {
      int32_t kk, i0, j0;
      double x, y;
      if (locate_one(c, u[j], v[j], w[j], &kk, &i0, &j0, &x, &y) != WO_KEPT) continue;
      if (!vis_finite(vis, weight, j)) continue;
      if (kk != k) continue;
      const double om = weight ? (double)weight[j] : 1.0;
      const double complex V = om * ((double)vis[2 * j] + I * (double)vis[2 * j + 1]);
      for (int r = 0; r < W; ++r) {
        const double ty = (double)(j0 + r) - y;
        const double gy = wo_kernel_eval(c, ty);
        for (int s = 0; s < W; ++s) {
          const double tx = (double)(i0 + s) - x;
          const double gxv = wo_kernel_eval(c, tx);
          const double cr = creal(conj(plane[(int64_t)(j0 + r) * N + (i0 + s)]) * V);
          /* x factor */
          {
            const double pos = (tx + half) * (double)(L - 1) / (double)W;
            int i = (int)floor(pos);
            if (i < 0) i = 0;
            if (i > L - 2) i = L - 2;
            const double f = pos - i;
            dtable[i] += cr * gy * (1.0 - f);
            dtable[i + 1] += cr * gy * f;
          }
          /* y factor */
          {
            const double pos = (ty + half) * (double)(L - 1) / (double)W;
            int i = (int)floor(pos);
            if (i < 0) i = 0;
            if (i > L - 2) i = L - 2;
            const double f = pos - i;
            dtable[i] += cr * gxv * (1.0 - f);
            dtable[i + 1] += cr * gxv * f;
          }
        }
      }
    }
  }
  free(plane);
}

int wo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
