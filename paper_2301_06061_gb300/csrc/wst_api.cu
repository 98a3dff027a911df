// C ABI of libwst (declared in include/wst.h): plan life cycle, workspace carving,
// argument validation and the orchestration of the K-S / K-G / K-F / K-P kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "wst_internal.cuh"

using namespace wst;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

wst_status fail(wst_plan_s *p, wst_status s, const char *msg) {
  if (p) p->last_error = msg;
  return s;
}

wst_status cuda_fail(wst_plan_s *p, cudaError_t e, const char *where) {
  if (p) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    p->last_error = buf;
  }
  return WST_ERR_CUDA;
}

#define WST_CUDA(p, call, where)                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, where); \
  } while (0)

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

struct Layout {
  size_t keyinfo_planes, records, offsets, cursor, scan_tmp, counters, wminmax, occ, binmag, rowbound, comp, total;
};

Layout layout_for(const wst_plan_s *p, int64_t n_vis) {
  Layout L;
  size_t off = 0;
  const size_t plane_bytes = (size_t)p->chunk * p->n * p->n * sizeof(float2);
  const size_t keyinfo_bytes = (size_t)n_vis * (sizeof(uint4) + sizeof(float4));  // keys + value stash
  L.keyinfo_planes = off;
  off += align_up(plane_bytes > keyinfo_bytes ? plane_bytes : keyinfo_bytes);
  L.records = off;
  off += align_up((size_t)n_vis * sizeof(Record));
  L.offsets = off;
  off += align_up((size_t)(p->n_buckets + 1) * sizeof(uint32_t));
  L.cursor = off;
  off += align_up((size_t)(p->n_buckets + 1) * sizeof(uint32_t));
  L.scan_tmp = off;
  off += align_up((size_t)scan_tmp_words(p->n_buckets + 1) * sizeof(uint32_t));
  L.counters = off;
  off += align_up(CNT_SLOTS * sizeof(unsigned long long));
  L.wminmax = off;
  off += align_up((size_t)2 * p->batch * sizeof(uint32_t));
  L.occ = off;
  off += align_up((size_t)p->n_planes * p->n);
  L.binmag = off;
  if (p->n >= kFixedMinN) off += align_up((size_t)(p->n_buckets / kColBlocks) * bins_per_row(p->n) * sizeof(float));
  L.rowbound = off;
  if (p->n >= kFixedMinN) off += align_up((size_t)(p->n_buckets / kColBlocks) * sizeof(float2));
  L.comp = off;
  if (p->chunk < p->n_planes) off += align_up((size_t)p->batch * p->n_img * p->n_img * sizeof(float2));
  L.total = off;
  return L;
}

// batch offsets to the device without a host synchronisation (passed as kernel args)
struct OffsetsArg {
  int64_t v[64];
};
__global__ void k_set_offsets(int64_t *dst, OffsetsArg a, int count) {
  int i = threadIdx.x;
  if (i < count) dst[i] = a.v[i];
}

void destroy_tables(wst_plan_s *p) {
  cudaFree(p->tw);
  cudaFree(p->corr);
  cudaFree(p->l2ff);
  cudaFree(p->l2d);
  cudaFree(p->ktable);
  cudaFree(p->ktap);
  cudaFree(p->wrange);
  cudaFree(p->wrange_ff);
  cudaFree(p->wcentre);
  cudaFree(p->wcentre_d);
  cudaFree(p->dwff);
  cudaFree(p->batch_off);
  for (auto *l : {&p->ev_sort, &p->ev_img})
    for (auto e : l->ev) cudaEventDestroy(e);
}

// stage ids of the timing event pairs
enum { ST_SORT = 0, ST_GRID = 1, ST_ROWS = 2, ST_COLS_A = 3, ST_COLS_B = 4 };

cudaError_t time_begin(wst_plan_s *p, wst_plan_s::EventList &l, int stage) {
  if (!p->timing) return cudaSuccess;
  const size_t need = 2 * (size_t)(l.used + 1);
  while (l.ev.size() < need) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    l.ev.push_back(e);
  }
  if (l.stage.size() < (size_t)l.used + 1) l.stage.resize(l.used + 1);
  l.stage[l.used] = stage;
  return cudaEventRecord(l.ev[2 * l.used], p->stream);
}

cudaError_t time_end(wst_plan_s *p, wst_plan_s::EventList &l) {
  if (!p->timing) return cudaSuccess;
  cudaError_t r = cudaEventRecord(l.ev[2 * l.used + 1], p->stream);
  ++l.used;
  return r;
}

}  // namespace

extern "C" {

const char *wst_version(void) { return "0.1.0"; }

const char *wst_status_string(wst_status s) {
  switch (s) {
    case WST_OK: return "ok";
    case WST_ERR_INVALID_ARG: return "invalid argument";
    case WST_ERR_OOM: return "out of memory / workspace too small";
    case WST_ERR_CUDA: return "CUDA error";
    case WST_ERR_TIMEOUT: return "device wait timed out";
    case WST_ERR_UNSUPPORTED: return "unsupported";
    case WST_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

wst_status wst_plan_create(const wst_config *cfg, void *cuda_stream, wst_plan *out) {
  if (!out) return WST_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return WST_ERR_INVALID_ARG;
  if (cfg->oversample < 0 || cfg->oversample > 2) return WST_ERR_UNSUPPORTED;
  if (cfg->grid_n < 0 || (cfg->grid_n > 0 && cfg->oversample == 2)) return WST_ERR_INVALID_ARG;
  // the plan works on the grid: M cells of N/(M fov) wavelengths (the image's pixel
  // size), and images are the central N x N of the grid's transform
  int m = 0;
  if (cfg->grid_n > 0) {
    if (!is_pow2(cfg->grid_n) || cfg->grid_n < 64 || cfg->grid_n > 16384) return WST_ERR_UNSUPPORTED;
    if (cfg->n < 64 || cfg->n > cfg->grid_n || (cfg->n & 1)) return WST_ERR_UNSUPPORTED;
    m = cfg->grid_n;
  } else {
    if (!is_pow2(cfg->n) || cfg->n < 64) return WST_ERR_UNSUPPORTED;
    m = cfg->n * (cfg->oversample == 2 ? 2 : 1);
    if (m > 16384) return WST_ERR_UNSUPPORTED;
  }
  wst_config c = *cfg;
  c.n = m;
  c.fov = cfg->fov * (double)m / (double)cfg->n;  // (fov M) / N: one rounding
  c.oversample = m == cfg->n ? 1 : 2;
  c.grid_n = m;
  if (!(c.fov > 0.0) || !isfinite(c.fov)) return WST_ERR_INVALID_ARG;
  if (c.n_w < 1 || c.n_w > 4096) return WST_ERR_INVALID_ARG;
  if (!isfinite(c.w_min) || !isfinite(c.w_max) || c.w_min > c.w_max) return WST_ERR_INVALID_ARG;
  if (c.support < 2 || c.support > kMaxSupport) return WST_ERR_UNSUPPORTED;
  if (c.kernel == WST_KERNEL_GAUSS || c.kernel == WST_KERNEL_ES) {
    if (!(c.kparam > 0.0) || !isfinite(c.kparam)) return WST_ERR_INVALID_ARG;
  } else if (c.kernel == WST_KERNEL_TABLE) {
    if (c.ktable_len < 2 || c.ktable_len > 65536) return WST_ERR_INVALID_ARG;
  } else {
    return WST_ERR_INVALID_ARG;
  }
  if (c.batch < 1 || c.batch > 4096 || c.planes_per_chunk < 0) return WST_ERR_INVALID_ARG;
  if (c.flags & ~(WST_FLAG_KAHAN | WST_FLAG_FP64_SCREEN | WST_FLAG_TIMING | WST_FLAG_WFOLD))
    return WST_ERR_INVALID_ARG;
  const int64_t n_buckets = (int64_t)c.batch * c.n_w * c.n * kColBlocks;
  if (n_buckets + 1 >= (int64_t)0xFFFFFFFFu) return WST_ERR_UNSUPPORTED;

  wst_plan_s *p = new wst_plan_s();
  p->cfg = c;
  p->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&p->device);
  p->n = c.n;
  p->n_img = cfg->n;
  p->crop = (c.n - cfg->n) / 2;
  p->log2n = ilog2(c.n);
  p->W = c.support;
  p->n_w = c.n_w;
  p->batch = c.batch;
  p->n_planes = c.batch * c.n_w;
  p->chunk = c.planes_per_chunk > 0 ? (c.planes_per_chunk < p->n_planes ? c.planes_per_chunk : p->n_planes)
                                    : p->n_planes;
  if (p->chunk > 65535) p->chunk = 65535;  // planes of a chunk index a grid dimension
  p->fb = 1 << (p->log2n / 2);
  p->fa = c.n / p->fb;
  p->n_buckets = n_buckets;
  p->timing = (c.flags & WST_FLAG_TIMING) != 0;

  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, count)                                                  \
  if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), sizeof(*(ptr)) * (size_t)(count));
  ALLOC(p->tw, c.n);
  ALLOC(p->corr, c.n);
  ALLOC(p->l2ff, c.n);
  ALLOC(p->l2d, c.n);
  ALLOC(p->wrange, 4 * c.batch);
  ALLOC(p->wrange_ff, c.batch);
  ALLOC(p->wcentre, p->n_planes);
  ALLOC(p->wcentre_d, p->n_planes);
  ALLOC(p->dwff, c.batch);
  ALLOC(p->batch_off, c.batch + 1);
  if (c.kernel == WST_KERNEL_TABLE) ALLOC(p->ktable, c.ktable_len);
  if (c.kernel == WST_KERNEL_TABLE && (c.ktable_len - 1) % c.support == 0) ALLOC(p->ktap, c.ktable_len - 1);
#undef ALLOC
  if (e != cudaSuccess) {
    destroy_tables(p);
    delete p;
    return e == cudaErrorMemoryAllocation ? WST_ERR_OOM : WST_ERR_CUDA;
  }
  e = build_tables(p);
  if (e == cudaSuccess && c.kernel != WST_KERNEL_TABLE) e = build_correction(p);
  if (e != cudaSuccess) {
    destroy_tables(p);
    delete p;
    return WST_ERR_CUDA;
  }
  *out = p;
  return WST_OK;
}

void wst_plan_destroy(wst_plan p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  destroy_tables(p);
  delete p;
}

wst_status wst_plan_set_stream(wst_plan p, void *cuda_stream) {
  if (!p) return WST_ERR_INVALID_ARG;
  p->stream = (cudaStream_t)cuda_stream;
  return WST_OK;
}

wst_status wst_plan_set_wait_limit(wst_plan p, uint64_t wait_ns) {
  if (!p) return WST_ERR_INVALID_ARG;
  if (wait_ns > 60000000000ull) return fail(p, WST_ERR_INVALID_ARG, "wait limit above 60 s");
  p->wait_ns = wait_ns;
  return WST_OK;
}

wst_status wst_plan_workspace_bytes(wst_plan p, int64_t n_vis, size_t *bytes) {
  if (!p || !bytes || n_vis < 0 || n_vis >= (int64_t)0xFFFFFFFFu) return WST_ERR_INVALID_ARG;
  *bytes = layout_for(p, n_vis).total;
  return WST_OK;
}

wst_status wst_plan_set_workspace(wst_plan p, void *ptr, size_t bytes) {
  if (!p) return WST_ERR_INVALID_ARG;
  if (!ptr || ((uintptr_t)ptr % kAlign) != 0) return fail(p, WST_ERR_INVALID_ARG, "workspace pointer NULL or not 256-byte aligned");
  p->ws = (char *)ptr;
  p->ws_bytes = bytes;
  p->vis_set = false;
  return WST_OK;
}

wst_status wst_plan_set_kernel_table(wst_plan p, const float *table_dev) {
  if (!p) return WST_ERR_INVALID_ARG;
  if (p->cfg.kernel != WST_KERNEL_TABLE) return fail(p, WST_ERR_STATE, "plan kernel is not a table");
  if (p->cfg.flags & WST_FLAG_WFOLD) return fail(p, WST_ERR_UNSUPPORTED, "no kernel gradient with WST_FLAG_WFOLD");
  if (!table_dev) return fail(p, WST_ERR_INVALID_ARG, "table pointer is NULL");
  WST_CUDA(p, cudaMemcpyAsync(p->ktable, table_dev, sizeof(float) * p->cfg.ktable_len,
                              cudaMemcpyDeviceToDevice, p->stream), "table copy");
  WST_CUDA(p, build_correction(p), "correction table");
  WST_CUDA(p, build_tap_table(p), "tap table");
  p->table_set = true;
  return WST_OK;
}

// The address the kernels use for a caller's array, or NULL if the device cannot reach
// it: device or managed memory as is; page-locked host memory through its mapping into
// the device's address space (on GB300 the accesses cross NVLink-C2C: the kernels read
// the inputs and write the image in place, no separate copy); pageable host memory only
// where the device reports cudaDevAttrPageableMemoryAccess.
static const void *device_view(const wst_plan_s *p, const void *ptr, bool *is_host = nullptr) {
  if (!ptr) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (is_host) *is_host = a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ptr;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  int pageable = 0;
  if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, p->device) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return pageable ? ptr : nullptr;
}

// The part of wst_plan_set_vis and wst_plan_set_vis_rows after their coordinate
// arguments are checked: values, weights, batch offsets, workspace, then the sort.
static wst_status set_vis_common(wst_plan_s *p, int64_t n_vis, const VisCoords &coords, const void *vis,
                                 const float *weight, const int64_t *batch_offsets) {
  bool host_vis = false;
  if (n_vis > 0) {
    const void *dvis = device_view(p, vis, &host_vis), *dwt = weight ? device_view(p, weight) : nullptr;
    if (!dvis || (weight && !dwt))
      return fail(p, WST_ERR_INVALID_ARG, "visibility arrays must be device or page-locked host memory");
    vis = dvis;
    weight = (const float *)dwt;
  }
  if (p->batch > 1 && !batch_offsets) return fail(p, WST_ERR_INVALID_ARG, "batch offsets required");
  std::vector<int64_t> off(p->batch + 1);
  if (batch_offsets) {
    for (int i = 0; i <= p->batch; ++i) off[i] = batch_offsets[i];
    if (off[0] != 0 || off[p->batch] != n_vis) return fail(p, WST_ERR_INVALID_ARG, "batch offsets must run from 0 to n_vis");
    for (int i = 0; i < p->batch; ++i)
      if (off[i + 1] < off[i]) return fail(p, WST_ERR_INVALID_ARG, "batch offsets must be non-decreasing");
  } else {
    off[0] = 0;
    off[1] = n_vis;
  }
  if (p->cfg.kernel == WST_KERNEL_TABLE && !p->table_set) return fail(p, WST_ERR_STATE, "kernel table not set");
  if (!p->ws) return fail(p, WST_ERR_OOM, "no workspace set");
  const Layout L = layout_for(p, n_vis);
  if (L.total > p->ws_bytes) return fail(p, WST_ERR_OOM, "workspace too small for n_vis");
  Workspace &W = p->W_;
  W.keyinfo = (uint4 *)(p->ws + L.keyinfo_planes);
  W.stash = (float4 *)(W.keyinfo + n_vis);
  W.planes = (float2 *)(p->ws + L.keyinfo_planes);
  W.records = (Record *)(p->ws + L.records);
  W.offsets = (uint32_t *)(p->ws + L.offsets);
  W.cursor = (uint32_t *)(p->ws + L.cursor);
  W.scan_tmp = (uint32_t *)(p->ws + L.scan_tmp);
  W.counters = (unsigned long long *)(p->ws + L.counters);
  W.wminmax = (uint32_t *)(p->ws + L.wminmax);
  W.occ = (uint8_t *)(p->ws + L.occ);
  W.binmag = (float *)(p->ws + L.binmag);
  W.rowbound = (float2 *)(p->ws + L.rowbound);
  W.comp = (p->chunk < p->n_planes) ? (float2 *)(p->ws + L.comp) : nullptr;
  W.bytes = L.total;
  p->launches = 0;
  for (int i0 = 0; i0 <= p->batch; i0 += 64) {
    ++p->launches;
    OffsetsArg a;
    const int cnt = (p->batch + 1 - i0) < 64 ? (p->batch + 1 - i0) : 64;
    for (int i = 0; i < cnt; ++i) a.v[i] = off[i0 + i];
    k_set_offsets<<<1, 64, 0, p->stream>>>(p->batch_off + i0, a, cnt);
  }
  WST_CUDA(p, cudaGetLastError(), "batch offsets");
  p->n_vis = n_vis;
  p->has_weight = weight != nullptr;
  WST_CUDA(p, time_begin(p, p->ev_sort, ST_SORT), "event");
  WST_CUDA(p, sort_visibilities(p, coords, (const float2 *)vis, weight, host_vis), "sort");
  WST_CUDA(p, time_end(p, p->ev_sort), "event");
  p->launches_sort = p->launches;
  p->vis_set = true;
  return WST_OK;
}

wst_status wst_plan_set_vis(wst_plan p, int64_t n_vis, const float *u, const float *v, const float *w,
                            const void *vis, const float *weight, const int64_t *batch_offsets) {
  if (!p) return WST_ERR_INVALID_ARG;
  p->vis_set = false;
  if (n_vis < 0 || n_vis >= (int64_t)0xFFFFFFFFu) return fail(p, WST_ERR_INVALID_ARG, "n_vis out of range");
  if (n_vis > 0 && (!u || !v || !w || !vis)) return fail(p, WST_ERR_INVALID_ARG, "NULL visibility array");
  VisCoords c;
  if (n_vis > 0) {
    c.u = (const float *)device_view(p, u);
    c.v = (const float *)device_view(p, v);
    c.w = (const float *)device_view(p, w);
    if (!c.u || !c.v || !c.w)
      return fail(p, WST_ERR_INVALID_ARG, "visibility arrays must be device or page-locked host memory");
  }
  return set_vis_common(p, n_vis, c, vis, weight, batch_offsets);
}

wst_status wst_plan_set_vis_rows(wst_plan p, int64_t n_vis, const double *uvw_m, int64_t n_rows,
                                 const double *chan_scale, int32_t n_chan, const void *vis, const float *weight,
                                 const int64_t *batch_offsets) {
  if (!p) return WST_ERR_INVALID_ARG;
  p->vis_set = false;
  if (n_vis < 0 || n_vis >= (int64_t)0xFFFFFFFFu) return fail(p, WST_ERR_INVALID_ARG, "n_vis out of range");
  if (n_chan < 1 || n_rows < 0) return fail(p, WST_ERR_INVALID_ARG, "n_chan must be >= 1 and n_rows >= 0");
  if (n_vis > 0 && (n_vis - 1) / n_chan >= n_rows)
    return fail(p, WST_ERR_INVALID_ARG, "n_vis exceeds n_rows * n_chan");
  if (n_vis > 0 && (!uvw_m || !chan_scale || !vis)) return fail(p, WST_ERR_INVALID_ARG, "NULL visibility array");
  VisCoords c;
  c.n_chan = (uint32_t)n_chan;
  if (n_vis > 0) {
    c.rows = (const double *)device_view(p, uvw_m);
    c.scale = (const double *)device_view(p, chan_scale);
    if (!c.rows || !c.scale)
      return fail(p, WST_ERR_INVALID_ARG, "row and channel arrays must be device or page-locked host memory");
  }
  return set_vis_common(p, n_vis, c, vis, weight, batch_offsets);
}

static wst_status check_ready(wst_plan_s *p) {
  if (!p) return WST_ERR_INVALID_ARG;
  if (!p->vis_set) return fail(p, WST_ERR_STATE, "no visibilities set");
  return WST_OK;
}

wst_status wst_grid(wst_plan p, int32_t b, int32_t e, void *out) {
  wst_status st = check_ready(p);
  if (st) return st;
  if (b < 0 || e > p->n_planes || b > e || (!out && e > b)) return fail(p, WST_ERR_INVALID_ARG, "plane range or output");
  WST_CUDA(p, grid_rows(p, b, e, (float2 *)out, false), "grid");
  return WST_OK;
}

wst_status wst_fft_correct(wst_plan p, int32_t b, int32_t e, void *grid_inout, void *image_inout) {
  wst_status st = check_ready(p);
  if (st) return st;
  if (b < 0 || e > p->n_planes || b > e) return fail(p, WST_ERR_INVALID_ARG, "plane range");
  if (e == b) return WST_OK;
  if (!grid_inout || !image_inout) return fail(p, WST_ERR_INVALID_ARG, "NULL buffer");
  float2 *g = (float2 *)grid_inout;
  WST_CUDA(p, fft_rows(p, g, e - b, +1, true, false), "rows");
  WST_CUDA(p, fft_cols_a(p, g, e - b, +1, false, nullptr), "cols A");
  WST_CUDA(p, fft_cols_b_accumulate(p, g, b, e, (float2 *)image_inout, nullptr,
                                    (p->cfg.flags & WST_FLAG_KAHAN) != 0, false, true),
           "cols B");
  return WST_OK;
}

wst_status wst_correct(wst_plan p, void *image) {
  if (!p) return WST_ERR_INVALID_ARG;
  if (!image) return fail(p, WST_ERR_INVALID_ARG, "NULL image");
  if (p->cfg.kernel == WST_KERNEL_TABLE && !p->table_set) return fail(p, WST_ERR_STATE, "kernel table not set");
  WST_CUDA(p, correct_image(p, (float2 *)image), "correct");
  return WST_OK;
}

// The plane sum over global planes [b, e) of every image they touch, chunk by chunk;
// images that no plane of the range belongs to are set to zero.
static wst_status image_range(wst_plan_s *p, int b, int e, void *image_out, uint32_t flags) {
  wst_status st = check_ready(p);
  if (st) return st;
  if (!image_out) return fail(p, WST_ERR_INVALID_ARG, "NULL image");
  if (flags & ~WST_NO_CORRECTION) return fail(p, WST_ERR_INVALID_ARG, "unknown flags");
  if (b < 0 || e > p->n_planes || b > e) return fail(p, WST_ERR_INVALID_ARG, "plane range");
  const bool correct = !(flags & WST_NO_CORRECTION);
  const bool kahan = (p->cfg.flags & WST_FLAG_KAHAN) != 0;
  float2 *img = (float2 *)device_view(p, image_out);
  if (!img) return fail(p, WST_ERR_INVALID_ARG, "image must be device or page-locked host memory");
  const size_t img_bytes = sizeof(float2) * (size_t)p->n_img * p->n_img;
  // images outside the range hold no plane of it: zero
  const int i0 = b < e ? b / p->n_w : p->batch, i1 = b < e ? (e - 1) / p->n_w + 1 : p->batch;
  if (i0 > 0) WST_CUDA(p, cudaMemsetAsync(img, 0, img_bytes * i0, p->stream), "memset");
  if (i1 < p->batch) WST_CUDA(p, cudaMemsetAsync(img + (size_t)i1 * p->n_img * p->n_img, 0,
                                                 img_bytes * (p->batch - i1), p->stream), "memset");
  float2 *planes = p->W_.planes;
  p->n_chunks = 0;
  p->launches = 0;
  WST_CUDA(p, cudaMemsetAsync(p->W_.counters + CNT_ROWS, 0, sizeof(unsigned long long), p->stream), "memset");
  for (int p0 = b; p0 < e; p0 += p->chunk) {
    const int p1 = (p0 + p->chunk < e) ? p0 + p->chunk : e;
    WST_CUDA(p, time_begin(p, p->ev_img, ST_GRID), "event");
    WST_CUDA(p, grid_rows(p, p0, p1, planes, true), "grid + rows");
    WST_CUDA(p, time_end(p, p->ev_img), "event");
    WST_CUDA(p, time_begin(p, p->ev_img, ST_COLS_A), "event");
    WST_CUDA(p, fft_cols_a(p, planes, p1 - p0, +1, false, p->W_.occ), "cols A");
    WST_CUDA(p, time_end(p, p->ev_img), "event");
    WST_CUDA(p, time_begin(p, p->ev_img, ST_COLS_B), "event");
    WST_CUDA(p, fft_cols_b_accumulate(p, planes, p0, p1, img, p->W_.comp, kahan, correct, false, p0 == b, p1 == e),
             "cols B");
    WST_CUDA(p, time_end(p, p->ev_img), "event");
    ++p->n_chunks;
  }
  p->launches_image = p->launches;
  return WST_OK;
}

wst_status wst_image(wst_plan p, void *image_out, uint32_t flags) {
  if (!p) return WST_ERR_INVALID_ARG;
  return image_range(p, 0, p->n_planes, image_out, flags);
}

wst_status wst_image_range(wst_plan p, int32_t plane_begin, int32_t plane_end, void *image_out, uint32_t flags) {
  if (!p) return WST_ERR_INVALID_ARG;
  return image_range(p, plane_begin, plane_end, image_out, flags);
}

wst_status wst_degrid(wst_plan p, const void *dimage, void *dvis, uint32_t flags) {
  wst_status st = check_ready(p);
  if (st) return st;
  if (!dimage || (!dvis && p->n_vis > 0)) return fail(p, WST_ERR_INVALID_ARG, "NULL buffer");
  if (flags & ~WST_NO_CORRECTION) return fail(p, WST_ERR_INVALID_ARG, "unknown flags");
  if (p->cfg.flags & WST_FLAG_WFOLD) return fail(p, WST_ERR_UNSUPPORTED, "no adjoint with WST_FLAG_WFOLD");
  const bool correct = !(flags & WST_NO_CORRECTION);
  if (p->n_vis > 0) WST_CUDA(p, cudaMemsetAsync(dvis, 0, sizeof(float2) * p->n_vis, p->stream), "memset");
  float2 *planes = p->W_.planes;
  for (int p0 = 0; p0 < p->n_planes; p0 += p->chunk) {
    const int p1 = (p0 + p->chunk < p->n_planes) ? p0 + p->chunk : p->n_planes;
    WST_CUDA(p, fft_cols_bh_from_image(p, (const float2 *)dimage, p0, p1, planes, correct), "cols B^H");
    WST_CUDA(p, fft_cols_a(p, planes, p1 - p0, -1, true, nullptr), "cols A^H");
    WST_CUDA(p, rows_adjoint(p, p0, p1, planes, (float2 *)dvis, nullptr), "rows^H + degrid");
  }
  return WST_OK;
}

wst_status wst_kernel_grad(wst_plan p, const void *dimage, float *dtable, uint32_t flags) {
  wst_status st = check_ready(p);
  if (st) return st;
  if (p->cfg.kernel != WST_KERNEL_TABLE) return fail(p, WST_ERR_STATE, "plan kernel is not a table");
  if (!(flags & WST_NO_CORRECTION)) return fail(p, WST_ERR_UNSUPPORTED, "kernel gradient needs WST_NO_CORRECTION");
  if (p->cfg.ktable_len > 16384) return fail(p, WST_ERR_UNSUPPORTED, "table longer than 16384 samples");
  if (!dimage || !dtable) return fail(p, WST_ERR_INVALID_ARG, "NULL buffer");
  WST_CUDA(p, cudaMemsetAsync(dtable, 0, sizeof(float) * p->cfg.ktable_len, p->stream), "memset");
  float2 *planes = p->W_.planes;
  for (int p0 = 0; p0 < p->n_planes; p0 += p->chunk) {
    const int p1 = (p0 + p->chunk < p->n_planes) ? p0 + p->chunk : p->n_planes;
    WST_CUDA(p, fft_cols_bh_from_image(p, (const float2 *)dimage, p0, p1, planes, false), "cols B^H");
    WST_CUDA(p, fft_cols_a(p, planes, p1 - p0, -1, true, nullptr), "cols A^H");
    WST_CUDA(p, rows_adjoint(p, p0, p1, planes, nullptr, dtable), "rows^H + kernel gradient");
  }
  return WST_OK;
}

wst_status wst_vis_cells(wst_plan p, int32_t *plane, int32_t *i0, int32_t *j0) {
  wst_status st = check_ready(p);
  if (st) return st;
  if (p->n_vis > 0 && (!plane || !i0 || !j0)) return fail(p, WST_ERR_INVALID_ARG, "NULL buffer");
  if (p->n_vis == 0) return WST_OK;
  WST_CUDA(p, vis_cells(p, plane, i0, j0, p->n_vis), "vis cells");
  return WST_OK;
}

wst_status wst_get_stats(wst_plan p, wst_stats *out) {
  if (!p || !out) return WST_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  WST_CUDA(p, cudaStreamSynchronize(p->stream), "synchronize");
  out->n_vis = p->n_vis;
  out->n_chunks = p->n_chunks;
  if (p->vis_set) {
    unsigned long long cnt[CNT_SLOTS];
    WST_CUDA(p, cudaMemcpy(cnt, p->W_.counters, sizeof(cnt), cudaMemcpyDeviceToHost), "counters");
    out->n_kept = (int64_t)cnt[CNT_KEPT];
    out->n_dropped = (int64_t)cnt[CNT_DROPPED];
    out->n_nonfinite = (int64_t)cnt[CNT_NONFINITE];
    out->device_error = (int32_t)cnt[CNT_ERROR];
    out->n_rows_gridded = (int64_t)cnt[CNT_ROWS];
    double wr[4];
    WST_CUDA(p, cudaMemcpy(wr, p->wrange, sizeof(wr), cudaMemcpyDeviceToHost), "w range");
    out->w_min = wr[0];
    out->w_max = wr[3];
  }
  if (p->timing) {  // sums since the previous wst_get_stats, then the lists restart
    float *dst[5] = {&out->ms_sort, &out->ms_grid, &out->ms_rows, &out->ms_cols_a, &out->ms_cols_b};
    for (auto *l : {&p->ev_sort, &p->ev_img}) {
      for (int i = 0; i < l->used; ++i) {
        float ms = 0.0f;
        WST_CUDA(p, cudaEventElapsedTime(&ms, l->ev[2 * i], l->ev[2 * i + 1]), "event time");
        *dst[l->stage[i]] += ms;
      }
      l->used = 0;
    }
    out->ms_total = out->ms_grid + out->ms_rows + out->ms_cols_a + out->ms_cols_b;
  }
  out->n_launches = p->launches_sort + p->launches_image;
  return out->device_error ? WST_ERR_TIMEOUT : WST_OK;
}

const char *wst_last_error(wst_plan p) { return p ? p->last_error.c_str() : ""; }

wst_status wst_dft(int64_t n_vis, const float *u, const float *v, const float *w, const void *vis,
                   const float *weight, int32_t n, double fov, int64_t n_pix, const int32_t *pa,
                   const int32_t *pb, void *out, void *stream) {
  if (n_vis < 0 || n_pix < 0 || n < 2 || !(fov > 0.0)) return WST_ERR_INVALID_ARG;
  if (n_pix > 0 && (!pa || !pb || !out)) return WST_ERR_INVALID_ARG;
  if (n_vis > 0 && (!u || !v || !w || !vis)) return WST_ERR_INVALID_ARG;
  cudaError_t e = dft_pixels(n_vis, u, v, w, (const float2 *)vis, weight, n, fov, n_pix, pa, pb,
                             (float2 *)out, (cudaStream_t)stream);
  return e == cudaSuccess ? WST_OK : WST_ERR_CUDA;
}

wst_status wst_predict_points(int64_t n_vis, const float *u, const float *v, const float *w, int64_t n_src,
                              const double *l, const double *m, const double *flux, void *out,
                              void *stream) {
  if (n_vis < 0 || n_src < 0) return WST_ERR_INVALID_ARG;
  if (n_vis > 0 && (!u || !v || !w || !out)) return WST_ERR_INVALID_ARG;
  if (n_src > 0 && (!l || !m || !flux)) return WST_ERR_INVALID_ARG;
  cudaError_t e = predict_points(n_vis, u, v, w, n_src, l, m, flux, (float2 *)out, (cudaStream_t)stream);
  return e == cudaSuccess ? WST_OK : WST_ERR_CUDA;
}

}  // extern "C"
