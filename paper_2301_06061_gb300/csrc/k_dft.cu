// Direct transforms: the exact dirty image at chosen pixels (the conjugate of Eq. 1,
// summed over visibilities) and Eq. 1 itself for a point-source sky.  Phases are
// formed in float-float (u l + v m + w (n-1) with l, m, n-1 carried as float-float)
// and reduced modulo one cycle before an FP32 sincospi, so a phase of thousands of
// cycles keeps about 1e-9 cycle accuracy.
#include "dft_core.cuh"

namespace wst {

__global__ void __launch_bounds__(kDftThreads)
k_dft(int64_t n_vis, const float *__restrict__ u, const float *__restrict__ v, const float *__restrict__ w,
      const float2 *__restrict__ vis, const float *__restrict__ weight, int n, double dl, int64_t n_pix,
      const int32_t *__restrict__ pa, const int32_t *__restrict__ pb, float2 *__restrict__ out) {
  const int64_t pix0 = (int64_t)blockIdx.y * kDftPix;
  const float2 s = dft_cta_partial(n_vis, u, v, w, vis, weight, n, dl, n_pix, pa, pb, pix0);
  if (threadIdx.x < kDftPix && pix0 + threadIdx.x < n_pix) {
    atomicAdd(&out[pix0 + threadIdx.x].x, s.x);
    atomicAdd(&out[pix0 + threadIdx.x].y, s.y);
  }
}

cudaError_t dft_pixels(int64_t n_vis, const float *u, const float *v, const float *w, const float2 *vis,
                       const float *weight, int n, double fov, int64_t n_pix, const int32_t *pa,
                       const int32_t *pb, float2 *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float2) * n_pix, s);
  if (e != cudaSuccess || n_pix == 0) return e;
  const int64_t pix_blocks = (n_pix + kDftPix - 1) / kDftPix;
  int64_t vis_blocks = (n_vis + kDftThreads - 1) / kDftThreads;
  // about 4 CTAs per SM in total, at least one visibility block per pixel group
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t target = ((int64_t)sms * 4 + pix_blocks - 1) / pix_blocks;
  if (vis_blocks > target) vis_blocks = target;
  if (vis_blocks < 1) vis_blocks = 1;
  for (int64_t y0 = 0; y0 < pix_blocks; y0 += 65535) {
    const int64_t ny = (pix_blocks - y0 < 65535) ? pix_blocks - y0 : 65535;
    dim3 grd((unsigned)vis_blocks, (unsigned)ny);
    k_dft<<<grd, kDftThreads, 0, s>>>(n_vis, u, v, w, vis, weight, n, fov / (double)n,
                                      n_pix - y0 * kDftPix, pa + y0 * kDftPix, pb + y0 * kDftPix,
                                      out + y0 * kDftPix);
  }
  return cudaGetLastError();
}

constexpr int kSrcTile = 256;

__global__ void __launch_bounds__(256)
k_predict(int64_t n_vis, const float *__restrict__ u, const float *__restrict__ v, const float *__restrict__ w,
          int64_t n_src, const double *__restrict__ l, const double *__restrict__ m,
          const double *__restrict__ flux, float2 *__restrict__ out) {
  __shared__ ff sl[kSrcTile], sm_[kSrcTile], st[kSrcTile];
  __shared__ float sf[kSrcTile];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = j < n_vis;
  const float uf = in ? u[j] : 0.0f, vf = in ? v[j] : 0.0f, wf = in ? w[j] : 0.0f;
  float2 acc = make_float2(0.0f, 0.0f);
  for (int64_t s0 = 0; s0 < n_src; s0 += kSrcTile) {
    __syncthreads();
    for (int i = threadIdx.x; i < kSrcTile && s0 + i < n_src; i += blockDim.x) {
      const double ls = l[s0 + i], ms = m[s0 + i];
      const double r2 = ls * ls + ms * ms;
      sl[i] = ff_from_double(ls);
      sm_[i] = ff_from_double(ms);
      st[i] = ff_from_double(r2 < 1.0 ? -r2 / (1.0 + sqrt(1.0 - r2)) : 0.0);
      sf[i] = (float)flux[s0 + i];
    }
    __syncthreads();
    const int cnt = (int)((n_src - s0) < kSrcTile ? (n_src - s0) : kSrcTile);
    if (in)
      for (int i = 0; i < cnt; ++i) {
        const float2 e = cis_cycles_ff(ff_neg(phase_ff(uf, vf, wf, sl[i], sm_[i], st[i])));
        acc.x = fmaf(sf[i], e.x, acc.x);
        acc.y = fmaf(sf[i], e.y, acc.y);
      }
  }
  if (in) out[j] = acc;
}

cudaError_t predict_points(int64_t n_vis, const float *u, const float *v, const float *w, int64_t n_src,
                           const double *l, const double *m, const double *flux, float2 *out,
                           cudaStream_t s) {
  if (n_vis == 0) return cudaSuccess;
  k_predict<<<(unsigned)((n_vis + 255) / 256), 256, 0, s>>>(n_vis, u, v, w, n_src, l, m, flux, out);
  return cudaGetLastError();
}

}  // namespace wst
