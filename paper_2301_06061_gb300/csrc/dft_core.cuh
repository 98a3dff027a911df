// Direct transform core shared by k_dft (k_dft.cu) and k_dft_partials (wst_noalloc.cu):
// the exact dirty image at a few pixels (the conjugate of Eq. 1 summed over the
// visibilities), phases formed in float-float (u l + v m + w (n-1) with l, m, n-1 carried
// as float-float) and reduced modulo one cycle before an FP32 sincospi, so a phase of
// thousands of cycles keeps about 1e-9 cycle accuracy.
#pragma once

#include "wst_internal.cuh"

namespace wst {

constexpr int kDftPix = 8;  // pixels per CTA (every thread evaluates all of them)
constexpr int kDftThreads = 256;

struct PixelLMN {
  ff l, m, t;
  bool valid;
};

__device__ __forceinline__ ff ff_from_double(double d) {
  float2 s = ff_split(d);
  return {s.x, s.y};
}

// phi = u l + v m + w t with exact float products (two_prod) and float-float sums
__device__ __forceinline__ ff phase_ff(float u, float v, float w, const ff &l, const ff &m, const ff &t) {
  ff a = ff_mul({u, 0.0f}, l);
  ff b = ff_mul({v, 0.0f}, m);
  ff c = ff_mul({w, 0.0f}, t);
  return ff_add(ff_add(a, b), c);
}

// The CTA's share of out_i = sum_j w_j V_j exp(2 pi i (u_j l_i + v_j m_i + w_j (n_i - 1)))
// for the kDftPix pixels pix0 .. pix0 + kDftPix - 1 (those below n_pix): the visibilities
// j = blockIdx.x * kDftThreads + threadIdx.x + k * gridDim.x * kDftThreads, skipping any
// with a non-finite coordinate, value or weight.  Pixels outside the unit sphere get 0.
// Thread i < kDftPix returns the CTA's sum for pixel pix0 + i (summed in a fixed order:
// a warp butterfly, then the warps in index order); other threads return 0.  Every
// thread of the CTA must call it (it synchronises the CTA).
__device__ __forceinline__ float2 dft_cta_partial(int64_t n_vis, const float *__restrict__ u,
                                                  const float *__restrict__ v, const float *__restrict__ w,
                                                  const float2 *__restrict__ vis, const float *__restrict__ weight,
                                                  int n, double dl, int64_t n_pix, const int32_t *__restrict__ pa,
                                                  const int32_t *__restrict__ pb, int64_t pix0) {
  PixelLMN px[kDftPix];
#pragma unroll
  for (int i = 0; i < kDftPix; ++i) {
    const int64_t q = pix0 + i;
    px[i].valid = false;
    px[i].l = px[i].m = px[i].t = {0.0f, 0.0f};
    if (q < n_pix) {
      const double l = (double)(pa[q] - n / 2) * dl, m = (double)(pb[q] - n / 2) * dl;
      const double r2 = l * l + m * m;
      if (r2 < 1.0) {
        px[i].valid = true;
        px[i].l = ff_from_double(l);
        px[i].m = ff_from_double(m);
        px[i].t = ff_from_double(-r2 / (1.0 + sqrt(1.0 - r2)));
      }
    }
  }
  float2 acc[kDftPix];
#pragma unroll
  for (int i = 0; i < kDftPix; ++i) acc[i] = make_float2(0.0f, 0.0f);
  for (int64_t j = (int64_t)blockIdx.x * kDftThreads + threadIdx.x; j < n_vis;
       j += (int64_t)gridDim.x * kDftThreads) {
    const float uf = u[j], vf = v[j], wf = w[j];
    float2 val = vis[j];
    const float wt = weight ? weight[j] : 1.0f;
    if (!(isfinite(uf) && isfinite(vf) && isfinite(wf) && isfinite(val.x) && isfinite(val.y) && isfinite(wt)))
      continue;
    val = make_float2(val.x * wt, val.y * wt);
#pragma unroll
    for (int i = 0; i < kDftPix; ++i) {
      if (!px[i].valid) continue;
      const float2 e = cis_cycles_ff(phase_ff(uf, vf, wf, px[i].l, px[i].m, px[i].t));
      const float2 y = cmul(val, e);
      acc[i].x += y.x;
      acc[i].y += y.y;
    }
  }
  __shared__ float2 red[kDftThreads / 32][kDftPix];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kDftPix; ++i) {
    float x = acc[i].x, y = acc[i].y;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
    }
    if (lane == 0) red[wid][i] = make_float2(x, y);
  }
  __syncthreads();
  float2 s = make_float2(0.0f, 0.0f);
  if (threadIdx.x < kDftPix)
    for (int k = 0; k < kDftThreads / 32; ++k) s = make_float2(s.x + red[k][threadIdx.x].x, s.y + red[k][threadIdx.x].y);
  return s;
}

}  // namespace wst
