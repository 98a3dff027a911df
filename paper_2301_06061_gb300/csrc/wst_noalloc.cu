// wst_dft_noalloc: the direct transform of wst_dft for callers that may not allocate
// device memory.  Its scratch (per visibility-block partial sums) is a fixed-size
// file-scope __device__ array instead of memory from cudaMalloc or a workspace, and
// the sum over blocks is done by a second pass in a fixed order, so the output is
// written with plain stores (no output clearing, no atomics).
#include <mutex>

#include "wst_internal.cuh"

namespace {

constexpr int kNaPix = 8;        // pixels per thread
constexpr int kNaThreads = 256;
constexpr int kNaVisBlocks = 64; // visibility blocks, i.e. partial sums per pixel
constexpr int kNaMaxDevices = 64;
static_assert(WST_DFT_NOALLOC_MAX_PIX % kNaPix == 0, "pixel groups");

// partial sums [visibility block][pixel]; 64 x 4096 x 8 B = 2 MiB on every device
// that loads the library, held until the process exits
__device__ __align__(256) float2 g_dft_partials[kNaVisBlocks * WST_DFT_NOALLOC_MAX_PIX];

std::mutex g_setup_mutex;
float2 *g_partials_addr[kNaMaxDevices] = {};

using wst::ff;

__device__ __forceinline__ ff na_ff(double d) {
  float2 s = wst::ff_split(d);
  return {s.x, s.y};
}

// pass 1: block (b, g) sums visibilities b, b + 64 blocks, ... for the 8 pixels of group g
// and stores one partial per pixel; every slot pass 2 reads is written here first.
__global__ void __launch_bounds__(kNaThreads)
k_dft_partials(int64_t n_vis, const float *__restrict__ u, const float *__restrict__ v,
               const float *__restrict__ w, const float2 *__restrict__ vis,
               const float *__restrict__ weight, int n, double dl, int64_t n_pix,
               const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
               float2 *__restrict__ partials) {
  const int64_t pix0 = (int64_t)blockIdx.y * kNaPix;
  ff l[kNaPix], m[kNaPix], t[kNaPix];
  bool valid[kNaPix];
#pragma unroll
  for (int i = 0; i < kNaPix; ++i) {
    const int64_t q = pix0 + i;
    valid[i] = false;
    l[i] = m[i] = t[i] = {0.0f, 0.0f};
    if (q < n_pix) {
      const double lx = (double)(pa[q] - n / 2) * dl, my = (double)(pb[q] - n / 2) * dl;
      const double r2 = lx * lx + my * my;
      if (r2 < 1.0) {
        valid[i] = true;
        l[i] = na_ff(lx);
        m[i] = na_ff(my);
        t[i] = na_ff(-r2 / (1.0 + sqrt(1.0 - r2)));
      }
    }
  }
  float2 acc[kNaPix];
#pragma unroll
  for (int i = 0; i < kNaPix; ++i) acc[i] = make_float2(0.0f, 0.0f);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_vis;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float uf = u[j], vf = v[j], wf = w[j];
    float2 val = vis[j];
    const float wt = weight ? weight[j] : 1.0f;
    if (!(isfinite(uf) && isfinite(vf) && isfinite(wf) && isfinite(val.x) && isfinite(val.y) && isfinite(wt)))
      continue;
    val = make_float2(val.x * wt, val.y * wt);
#pragma unroll
    for (int i = 0; i < kNaPix; ++i) {
      if (!valid[i]) continue;
      ff ph = wst::ff_add(wst::ff_add(wst::ff_mul({uf, 0.0f}, l[i]), wst::ff_mul({vf, 0.0f}, m[i])),
                          wst::ff_mul({wf, 0.0f}, t[i]));
      const float2 e = wst::cis_cycles_ff(ph);
      const float2 y = wst::cmul(val, e);
      acc[i].x += y.x;
      acc[i].y += y.y;
    }
  }
  __shared__ float2 red[kNaThreads / 32][kNaPix];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kNaPix; ++i) {
    float x = acc[i].x, y = acc[i].y;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
    }
    if (lane == 0) red[wid][i] = make_float2(x, y);
  }
  __syncthreads();
  if (threadIdx.x < kNaPix && pix0 + threadIdx.x < n_pix) {
    float2 s = make_float2(0.0f, 0.0f);
    for (int k = 0; k < kNaThreads / 32; ++k) s = make_float2(s.x + red[k][threadIdx.x].x, s.y + red[k][threadIdx.x].y);
    partials[(int64_t)blockIdx.x * n_pix + pix0 + threadIdx.x] = s;
  }
}

// pass 2: out[pixel] = sum over the visibility blocks, in block order
__global__ void k_dft_reduce(const float2 *__restrict__ partials, int blocks, int64_t n_pix,
                             float2 *__restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_pix) return;
  float2 s = make_float2(0.0f, 0.0f);
  for (int b = 0; b < blocks; ++b) {
    const float2 x = partials[(int64_t)b * n_pix + q];
    s.x += x.x;
    s.y += x.y;
  }
  out[q] = s;
}

// Per-device set-up: the device address of g_dft_partials.  In host code the symbol
// names a host-side stand-in, so its address must come from the runtime, with the
// device current.  Done once per device, on that device's first call.
wst_status partials_address(float2 **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WST_ERR_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return WST_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_dft_partials) != cudaSuccess || !ptr) return WST_ERR_CUDA;
    g_partials_addr[dev] = (float2 *)ptr;
  }
  *out = g_partials_addr[dev];
  return WST_OK;
}

}  // namespace

extern "C" wst_status wst_dft_noalloc(int64_t n_vis, const float *u, const float *v, const float *w,
                                      const void *vis, const float *weight, int32_t n, double fov,
                                      int64_t n_pix, const int32_t *pa, const int32_t *pb, void *out,
                                      void *cuda_stream) {
  if (n_vis < 0 || n_pix < 0 || n < 2 || !(fov > 0.0)) return WST_ERR_INVALID_ARG;
  if (n_pix > WST_DFT_NOALLOC_MAX_PIX) return WST_ERR_UNSUPPORTED;
  if (n_pix > 0 && (!pa || !pb || !out)) return WST_ERR_INVALID_ARG;
  if (n_vis > 0 && (!u || !v || !w || !vis)) return WST_ERR_INVALID_ARG;
  if (n_pix == 0) return WST_OK;
  float2 *partials = nullptr;
  wst_status st = partials_address(&partials);
  if (st != WST_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  dim3 grd(kNaVisBlocks, (unsigned)((n_pix + kNaPix - 1) / kNaPix));
  k_dft_partials<<<grd, kNaThreads, 0, s>>>(n_vis, u, v, w, (const float2 *)vis, weight, n, fov / (double)n,
                                             n_pix, pa, pb, partials);
  k_dft_reduce<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(partials, kNaVisBlocks, n_pix, (float2 *)out);
  return cudaGetLastError() == cudaSuccess ? WST_OK : WST_ERR_CUDA;
}
