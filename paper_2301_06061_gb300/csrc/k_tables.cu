// Plan tables built on the device at plan creation: FFT twiddles, the grid
// correction 1/Ghat(nu) and the l^2 terms of the phase screen (section 2, Eq. 2-3).
#include <math.h>

#include "wst_internal.cuh"

namespace wst {

KernelParams kernel_params(const wst_plan_s *p) {
  KernelParams k;
  k.kind = p->cfg.kernel;
  k.support = p->W;
  k.half = 0.5f * (float)p->W;
  double s = p->cfg.kparam;
  k.inv2s2 = (k.kind == WST_KERNEL_GAUSS) ? (float)(1.0 / (2.0 * s * s)) : 0.0f;
  k.l2c = (k.kind == WST_KERNEL_GAUSS) ? (float)(1.4426950408889634 / (2.0 * s * s)) : 0.0f;
  k.beta = (k.kind == WST_KERNEL_ES) ? (float)s : 0.0f;
  k.two_over_w = 2.0f / (float)p->W;
  k.table = p->ktable;
  k.table_len = p->cfg.ktable_len;
  k.table_scale = (k.kind == WST_KERNEL_TABLE) ? (float)((double)(p->cfg.ktable_len - 1) / p->W) : 0.0f;
  k.tap_table = p->ktap;
  k.per_cell = p->ktap ? (p->cfg.ktable_len - 1) / p->W : 0;
  return k;
}

// Tap-major copy of a kernel table with L - 1 = W pc samples: entry [i][a] holds the two
// samples that bracket tap a at sub-cell position i / pc, so the W taps of one
// visibility (all at the same sub-cell offset) are one contiguous run of W pairs.
__global__ void k_tap_table(const float *t, float2 *tap, int W, int pc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= W * pc) return;
  const int i = idx / W, a = idx % W;
  tap[idx] = make_float2(t[a * pc + i], t[a * pc + i + 1]);
}

cudaError_t build_tap_table(wst_plan_s *p) {
  if (!p->ktap) return cudaSuccess;
  const int pc = (p->cfg.ktable_len - 1) / p->W;
  k_tap_table<<<(p->W * pc + 255) / 256, 256, 0, p->stream>>>(p->ktable, p->ktap, p->W, pc);
  p->launches += 1;
  return cudaGetLastError();
}

// half-wave table exp(+2 pi i m / N), m < N/2, rounded once from FP64
__global__ void k_twiddles(float2 *tw, int n) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n / 2) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  tw[m] = make_float2((float)c, (float)s);
}

// l_a^2 with l_a = (a - N/2) * fov/N, as float-float and FP64
__global__ void k_l2(float2 *l2ff, double *l2d, int n, double dl) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  double l = (double)(a - n / 2) * dl;
  double l2 = l * l;
  l2ff[a] = ff_split(l2);
  l2d[a] = l2;
}

__device__ double kernel_eval_d(int kind, double x, double half, double param, const float *tab,
                                int tlen, int W) {
  if (x < -half || x > half) return 0.0;
  if (kind == WST_KERNEL_GAUSS) return exp(-(x * x) / (2.0 * param * param));
  if (kind == WST_KERNEL_ES) {
    double z = 2.0 * x / W;
    return exp(param * (sqrt(fmax(0.0, 1.0 - z * z)) - 1.0));
  }
  double pos = (x + half) * (double)(tlen - 1) / (double)W;
  int i = (int)floor(pos);
  i = max(0, min(i, tlen - 2));
  double f = pos - (double)i;
  return (1.0 - f) * (double)tab[i] + f * (double)tab[i + 1];
}

// 1/Ghat(nu_a), Ghat(nu) = int_{-W/2}^{W/2} G(x) cos(2 pi nu x) dx by composite Simpson in
// FP64: 256 panels per cell for analytic kernels; for a table, one panel per table
// interval so the piecewise-linear kinks fall on panel ends.  One block per nu_a.
__global__ void k_correction(float *corr, int n, int kind, int W, double param, const float *tab,
                             int tlen) {
  int a = blockIdx.x;
  double nu = (double)(a - n / 2) / (double)n;
  double half = 0.5 * W;
  int panels = (kind == WST_KERNEL_TABLE) ? (tlen - 1) : 256 * W;
  double h = (double)W / panels;
  double acc = 0.0;
  for (int s = threadIdx.x; s < panels; s += blockDim.x) {
    double x0 = -half + s * h;
    double xm = x0 + 0.5 * h;
    double x1 = x0 + h;
    // Simpson's rule on [x0, x1] (for a table the kinks sit exactly on x0 and x1)
    double f0 = kernel_eval_d(kind, x0, half, param, tab, tlen, W) * cospi(2.0 * nu * x0);
    double fm = kernel_eval_d(kind, xm, half, param, tab, tlen, W) * cospi(2.0 * nu * xm);
    double f1 = kernel_eval_d(kind, x1, half, param, tab, tlen, W) * cospi(2.0 * nu * x1);
    acc += (h / 6.0) * (f0 + 4.0 * fm + f1);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) corr[a] = (float)(1.0 / red[0]);
}

cudaError_t build_tables(wst_plan_s *p) {
  const int n = p->n;
  k_twiddles<<<(n + 255) / 256, 256, 0, p->stream>>>(p->tw, n);
  k_l2<<<(n + 255) / 256, 256, 0, p->stream>>>(p->l2ff, p->l2d, n, p->cfg.fov / (double)n);
  p->launches += 2;
  return cudaGetLastError();
}

cudaError_t build_correction(wst_plan_s *p) {
  k_correction<<<p->n, 256, 0, p->stream>>>(p->corr, p->n, p->cfg.kernel, p->W, p->cfg.kparam,
                                             p->ktable, p->cfg.ktable_len);
  p->launches += 1;
  return cudaGetLastError();
}

// Plane range per image: either the configured one, or the min/max of the finite w
// found by the sort's reduction (stored as order-preserving integers).
__device__ __forceinline__ float ordered_to_float(uint32_t o) {
  uint32_t b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(b);
}

__global__ void k_plane_centres(double *wrange, float4 *wrange_ff, float2 *wcentre, double *wcentre_d, float2 *dwff,
                                const uint32_t *wminmax, int batch, int n_w, double cfg_lo,
                                double cfg_hi, int from_data) {
  int img = blockIdx.x * blockDim.x + threadIdx.x;
  if (img >= batch) return;
  double lo = cfg_lo, hi = cfg_hi;
  if (from_data) {
    uint32_t omin = wminmax[2 * img], omax = wminmax[2 * img + 1];
    if (omin == 0xFFFFFFFFu) {  // no finite w in this image
      lo = hi = 0.0;
    } else {
      lo = (double)ordered_to_float(omin);
      hi = (double)ordered_to_float(omax);
    }
  }
  double scale = (hi > lo) ? (double)n_w / (hi - lo) : 0.0;
  double dw = (hi - lo) / (double)n_w;
  wrange[4 * img + 0] = lo;
  wrange[4 * img + 1] = scale;
  wrange[4 * img + 2] = dw;
  wrange[4 * img + 3] = hi;
  dwff[img] = ff_split(dw);
  const float2 lo_ff = ff_split(lo), sc_ff = ff_split(scale);
  wrange_ff[img] = make_float4(lo_ff.x, lo_ff.y, sc_ff.x, sc_ff.y);
  for (int k = 0; k < n_w; ++k) {
    double wk = lo + ((double)k + 0.5) * dw;
    wcentre[img * n_w + k] = ff_split(wk);
    wcentre_d[img * n_w + k] = wk;
  }
}

cudaError_t build_plane_centres(wst_plan_s *p) {
  const bool from_data = p->cfg.w_min == p->cfg.w_max;
  k_plane_centres<<<(p->batch + 63) / 64, 64, 0, p->stream>>>(
      p->wrange, p->wrange_ff, p->wcentre, p->wcentre_d, p->dwff, p->W_.wminmax, p->batch, p->n_w, p->cfg.w_min,
      p->cfg.w_max, from_data ? 1 : 0);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace wst
