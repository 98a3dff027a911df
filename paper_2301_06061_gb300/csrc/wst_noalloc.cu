// wst_dft_noalloc: the direct transform of wst_dft for callers that may not allocate
// device memory.  Its scratch (per visibility-block partial sums) is a fixed-size
// file-scope __device__ array instead of memory from cudaMalloc or a workspace, and
// the sum over blocks is done by a second pass in a fixed order, so the output is
// written with plain stores (no output clearing, no atomics).  The per-block sum is the
// same device code as k_dft's (dft_core.cuh).
#include <cuda.h>  // driver types only (entry points are fetched at run time; no libcuda link)

#include <mutex>

#include "dft_core.cuh"

namespace {

constexpr int kNaVisBlocks = 64;  // visibility blocks, i.e. partial sums per pixel
constexpr int kNaCacheSlots = 64; // contexts whose scratch address is remembered
static_assert(WST_DFT_NOALLOC_MAX_PIX % wst::kDftPix == 0, "pixel groups");

// partial sums [visibility block][pixel]; 64 x 4096 x 8 B = 2 MiB on every device
// that loads the library, held until the process exits
__device__ __align__(256) float2 g_dft_partials[kNaVisBlocks * WST_DFT_NOALLOC_MAX_PIX];

// pass 1: block (b, g) sums visibilities b, b + 64 blocks, ... for the 8 pixels of group g
// and stores one partial per pixel; every slot pass 2 reads is written here first (also
// when n_vis is 0: the partials are then zeros).
__global__ void __launch_bounds__(wst::kDftThreads)
k_dft_partials(int64_t n_vis, const float *__restrict__ u, const float *__restrict__ v,
               const float *__restrict__ w, const float2 *__restrict__ vis,
               const float *__restrict__ weight, int n, double dl, int64_t n_pix,
               const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
               float2 *__restrict__ partials) {
  const int64_t pix0 = (int64_t)blockIdx.y * wst::kDftPix;
  const float2 s = wst::dft_cta_partial(n_vis, u, v, w, vis, weight, n, dl, n_pix, pa, pb, pix0);
  if (threadIdx.x < wst::kDftPix && pix0 + threadIdx.x < n_pix)
    partials[(int64_t)blockIdx.x * n_pix + pix0 + threadIdx.x] = s;
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

// The device address of g_dft_partials.  In host code the symbol names a host-side
// stand-in, so the address must come from cudaGetSymbolAddress.  That address belongs
// to a CUDA context (a device's primary context, a context the caller created with the
// driver API, a primary context re-created after cudaDeviceReset), so it is remembered
// per context, under the driver's unique context id: the first call in each context
// looks it up with that context current; later calls in it only read the table.
using GetCurrentFn = CUresult (*)(CUcontext *);
using GetIdFn = CUresult (*)(CUcontext, unsigned long long *);

struct AddrCache {
  std::mutex mu;
  bool resolved = false;
  GetCurrentFn get_current = nullptr;
  GetIdFn get_id = nullptr;
  unsigned long long id[kNaCacheSlots] = {};
  float2 *addr[kNaCacheSlots] = {};
  int used = 0, next = 0;
};
AddrCache g_cache;

wst_status symbol_address(float2 **out) {
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_dft_partials) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return WST_ERR_CUDA;
  }
  *out = (float2 *)ptr;
  return WST_OK;
}

wst_status partials_address(float2 **out) {
  std::lock_guard<std::mutex> lock(g_cache.mu);
  if (!g_cache.resolved) {
    g_cache.resolved = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_cache.get_current = (GetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_cache.get_id = (GetIdFn)f;
    cudaGetLastError();
  }
  // without the driver's context id the address is looked up on every call
  if (!g_cache.get_current || !g_cache.get_id) return symbol_address(out);
  CUcontext ctx = nullptr;
  if (g_cache.get_current(&ctx) != CUDA_SUCCESS) return WST_ERR_CUDA;
  if (!ctx) {
    // no context is current yet: the runtime's lookup creates the device's primary
    // context and makes it current
    wst_status st = symbol_address(out);
    if (st != WST_OK) return st;
    if (g_cache.get_current(&ctx) != CUDA_SUCCESS || !ctx) return WST_ERR_CUDA;
  }
  unsigned long long cid = 0;
  if (g_cache.get_id(ctx, &cid) != CUDA_SUCCESS) return WST_ERR_CUDA;
  for (int i = 0; i < g_cache.used; ++i)
    if (g_cache.id[i] == cid) {
      *out = g_cache.addr[i];
      return WST_OK;
    }
  wst_status st = symbol_address(out);
  if (st != WST_OK) return st;
  const int slot = g_cache.used < kNaCacheSlots ? g_cache.used++ : (g_cache.next++ % kNaCacheSlots);
  g_cache.id[slot] = cid;
  g_cache.addr[slot] = *out;
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
  dim3 grd(kNaVisBlocks, (unsigned)((n_pix + wst::kDftPix - 1) / wst::kDftPix));
  k_dft_partials<<<grd, wst::kDftThreads, 0, s>>>(n_vis, u, v, w, (const float2 *)vis, weight, n,
                                                  fov / (double)n, n_pix, pa, pb, partials);
  k_dft_reduce<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(partials, kNaVisBlocks, n_pix, (float2 *)out);
  return cudaGetLastError() == cudaSuccess ? WST_OK : WST_ERR_CUDA;
}
