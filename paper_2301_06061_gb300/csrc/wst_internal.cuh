// Internal declarations shared by the libwst translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wst.h"

namespace wst {

constexpr int kMaxSupport = 16;  // W <= 16
constexpr int kColBlocks = 1;    // sub-buckets per row (by tap-start column; a row's sub-buckets
                                 // are contiguous).  More than one spreads the histogram atomics
                                 // but enlarges the offsets table and the scan: slower at 16384^2.
constexpr uint32_t kDropKey = 0xFFFFFFFFu;
// Column bins of the fixed-point gridder's bound: for every row bucket (image, plane, j0)
// the sort sums max(|Re|, |Im|) of the weighted values whose W taps reach each bin of
// kBinCols columns.
constexpr int kBinCols = 64, kBinShift = 6;
constexpr int kFixedMinN = 8192;  // image sizes whose rows use fixed-point accumulation
__host__ __device__ constexpr int bins_per_row(int n) { return n >= kBinCols ? n / kBinCols : 1; }

// counters[] slots in the workspace
// CNT_ROWS: non-empty (plane, row) items the imaging path gridded since wst_image began
enum { CNT_KEPT = 0, CNT_DROPPED = 1, CNT_NONFINITE = 2, CNT_ERROR = 3, CNT_WORK = 4, CNT_ROWS = 5, CNT_SLOTS = 8 };

// 32-byte sorted record of a visibility filed under (image, plane, row j0).  The head
// (16 bytes, all the gridder reads): tap start i0 (14 bits, N <= 16384) and the sub-cell
// offsets g_x, g_y in [0,1) quantised to 24 bits, packed as  xpack = i0 << 18 | g_x >> 6,
// ypack = (g_x & 63) << 24 | g_y;  then the weighted value.  The tail: the caller's
// index and weight (adjoint).  One record fills one 32-byte DRAM sector, so the scatter
// into sorted order writes whole sectors (no read-modify-write of partial sectors).
struct __align__(16) RecHead {
  uint32_t xpack;
  uint32_t ypack;
  float vre;
  float vim;
};
struct __align__(32) Record {
  RecHead h;
  uint32_t index;  // caller's visibility index
  float weight;    // caller's weight (1 without weights)
  uint32_t pad[2];
};

__device__ __forceinline__ RecHead rec_head(const Record *rec, uint32_t s) {
  const uint4 q = __ldg(reinterpret_cast<const uint4 *>(rec + s));
  RecHead h;
  h.xpack = q.x;
  h.ypack = q.y;
  h.vre = __uint_as_float(q.z);
  h.vim = __uint_as_float(q.w);
  return h;
}
__host__ __device__ __forceinline__ int rec_i0(const RecHead &r) { return (int)(r.xpack >> 18); }
__device__ __forceinline__ float rec_gx(const RecHead &r) {
  return (float)(((r.xpack & 0x3FFFFu) << 6) | (r.ypack >> 24)) * (1.0f / 16777216.0f);
}
__device__ __forceinline__ float rec_gy(const RecHead &r) {
  return (float)(r.ypack & 0xFFFFFFu) * (1.0f / 16777216.0f);
}

struct KernelParams {
  int kind;        // WST_KERNEL_*
  int support;     // W
  float half;      // W/2
  float inv2s2;    // GAUSS: 1/(2 sigma^2)
  float l2c;       // GAUSS: log2(e)/(2 sigma^2), so that G(x) = 2^(-x^2 l2c)
  float beta;      // ES
  float two_over_w;
  const float *table;  // TABLE: device samples
  int table_len;
  float table_scale;   // (L-1)/W
  const float2 *tap_table;  // TABLE with L - 1 = W * per_cell: [per_cell][W] pairs (T[a pc + i], T[a pc + i + 1])
  int per_cell;
};

struct Workspace {
  uint4 *keyinfo;      // per visibility: key, 0, xpack, ypack (aliases the plane buffer)
  float4 *stash;       // per visibility: value, weight, after keyinfo (host inputs only)
  Record *records;     // sorted records
  uint32_t *offsets;   // bucket offsets [n_buckets + 1]
  uint32_t *cursor;    // scatter cursors (a copy of the offsets, advanced by the scatter)
  uint32_t *scan_tmp;  // scan partial sums
  unsigned long long *counters;  // CNT_* slots
  uint32_t *wminmax;   // per image: ordered-int min and max of finite w
  uint8_t *occ;        // per (plane of the chunk, row): 1 if any visibility reaches the row
  float *binmag;       // per (row bucket, column bin): magnitude sum (fixed-point bound)
  float2 *rowbound;    // per grid row: (largest bin sum, total of the bin sums) over its W buckets
  float2 *planes;      // chunk of planes
  float2 *comp;        // Kahan compensation image [batch][N*N]
  size_t bytes;
};

}  // namespace wst

struct wst_plan_s {
  wst_config cfg;
  cudaStream_t stream = nullptr;
  int device = 0;
  // geometry
  int n = 0, log2n = 0, W = 0, n_w = 0, batch = 1, n_planes = 0, chunk = 0;
  // oversampled grid: the kernels work on the grid (n, cfg.fov of the grid); the image
  // is the central n_img x n_img of it, starting at grid index crop
  int n_img = 0, crop = 0;
  int fa = 0, fb = 0;  // four-step column split N = fa * fb (fa contiguous block rows)
  int64_t n_buckets = 0;
  // owned device tables
  float2 *tw = nullptr;      // exp(+2 pi i m / N), m < N
  float *corr = nullptr;     // 1 / Ghat(nu_a)
  float2 *l2ff = nullptr;    // l_a^2 as float-float
  double *l2d = nullptr;     // l_a^2 in FP64 (WST_FLAG_FP64_SCREEN)
  float *ktable = nullptr;   // TABLE kernel samples
  float2 *ktap = nullptr;    // TABLE samples in tap-major pairs (see KernelParams::tap_table)
  double *wrange = nullptr;  // per image: w_lo, scale = n_w/(w_hi-w_lo), dw, w_hi
  float4 *wrange_ff = nullptr;  // per image: w_lo and scale as float-float pairs
  float2 *wcentre = nullptr; // per global plane: centre w_k as float-float
  double *wcentre_d = nullptr;  // per global plane: centre w_k (FP64)
  float2 *dwff = nullptr;    // per image: plane spacing dw as float-float
  bool table_set = false;
  // limit of the device-side waits for data (the row kernel's bulk copies), nanoseconds;
  // 0 = expire at once (failure-path testing, wst_plan_set_wait_limit)
  unsigned long long wait_ns = 2000000000ull;
  // workspace
  char *ws = nullptr;
  size_t ws_bytes = 0;
  wst::Workspace W_;
  int64_t n_vis = 0;
  bool vis_set = false;
  bool has_weight = false;
  int64_t *batch_off = nullptr;  // device copy of batch offsets [batch+1]
  // timing: CUDA events recorded around each stage launch (WST_FLAG_TIMING)
  struct EventList {
    std::vector<cudaEvent_t> ev;  // pairs (2i, 2i+1)
    std::vector<int> stage;       // stage id of pair i
    int used = 0;
  };
  bool timing = false;
  EventList ev_sort, ev_img;
  int n_chunks = 0;
  int64_t launches_sort = 0, launches_image = 0;
  int64_t launches = 0;       // incremented by every launcher
  std::string last_error;
};

namespace wst {

// ------------------------------------------------------------------------------------
// error-free float transforms and float-float ("double-single") arithmetic
// (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2)
// ------------------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return quick_two_sum(p.hi, e);
}
__host__ __device__ __forceinline__ float2 ff_split(double d) {
  float hi = (float)d;
  float lo = (float)(d - (double)hi);
  return make_float2(hi, lo);
}

// n - 1 = sqrt(1 - l^2 - m^2) - 1 in float-float; valid = l^2 + m^2 < 1.  Only the
// absolute error of n - 1 reaches the phase w (n - 1), so the root is taken without a
// division: s0 = x rsqrt(x) (relative error ~2^-22), then one Newton step
// s = s0 + (x - s0^2) rsqrt(x) / 2 with the residual formed exactly (two_prod), which
// leaves a relative error near 2^-44; s - 1 is then an error-free float-float sum.
__device__ __forceinline__ ff n_minus_one_ff(float2 l2, float2 m2, bool &valid) {
  ff r2 = ff_add({l2.x, l2.y}, {m2.x, m2.y});
  valid = r2.hi < 1.0f;
  if (!valid) return {0.0f, 0.0f};
  const ff x = ff_add({1.0f, 0.0f}, ff_neg(r2));  // x.hi >= 2^-24 > 0
  const float rs = rsqrtf(x.hi);
  const float s0 = __fmul_rn(x.hi, rs);
  const ff p = two_prod(s0, s0);
  const float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
  const ff s = quick_two_sum(s0, __fmul_rn(res, __fmul_rn(0.5f, rs)));
  return ff_add(s, {-1.0f, 0.0f});
}

// exp(2 pi i phi) for a float-float phase in cycles: reduce modulo one cycle exactly
// in the high word, then FP32 sincospi of the small remainder.
__device__ __forceinline__ float2 cis_cycles_ff(ff phi) {
  float n = rintf(phi.hi);
  float r = __fadd_rn(__fsub_rn(phi.hi, n), phi.lo);
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, s);
}
__device__ __forceinline__ float2 cis_cycles_d(double phi) {
  double r = phi - rint(phi);
  float s, c;
  sincospif(2.0f * (float)r, &s, &c);
  return make_float2(c, s);
}

// ------------------------------------------------------------------------------------
// convolution kernel G (section 2, Eq. 3)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float kernel_eval(const KernelParams &k, float x) {
  if (x < -k.half || x > k.half) return 0.0f;
  if (k.kind == WST_KERNEL_GAUSS) return expf(-x * x * k.inv2s2);
  if (k.kind == WST_KERNEL_ES) {
    float z = x * k.two_over_w;
    return expf(k.beta * (sqrtf(fmaxf(0.0f, 1.0f - z * z)) - 1.0f));
  }
  float pos = (x + k.half) * k.table_scale;
  int i = (int)floorf(pos);
  i = max(0, min(i, k.table_len - 2));
  float f = pos - (float)i;
  return fmaf(f, __ldg(k.table + i + 1) - __ldg(k.table + i), __ldg(k.table + i));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

}  // namespace wst

// ------------------------------------------------------------------------------------
// host-side launchers (defined in the k_*.cu files)
// ------------------------------------------------------------------------------------
namespace wst {

KernelParams kernel_params(const wst_plan_s *p);
cudaError_t build_tap_table(wst_plan_s *p);

// k_tables.cu
cudaError_t build_tables(wst_plan_s *p);
cudaError_t build_correction(wst_plan_s *p);
cudaError_t build_plane_centres(wst_plan_s *p);

// Where the sort reads the (u, v, w) of visibility j: per-visibility FP32 arrays, or
// (rows != nullptr) a row of FP64 metres times a channel's nu / c, the product in FP64
// rounded once to FP32, for visibility j = row * n_chan + channel.
struct VisCoords {
  const float *u = nullptr, *v = nullptr, *w = nullptr;
  const double *rows = nullptr;   // [n_rows][3] u, v, w in metres
  const double *scale = nullptr;  // [n_chan] nu / c
  uint32_t n_chan = 1;
};
template <bool ROWS>
__device__ __forceinline__ void coords_uvw(const VisCoords &c, int64_t j, float &u, float &v, float &w) {
  if constexpr (ROWS) {
    const uint32_t r = (uint32_t)j / c.n_chan, ch = (uint32_t)j - r * c.n_chan;  // j < 2^32
    const double s = c.scale[ch];
    const double *m = c.rows + 3 * (size_t)r;
    u = __double2float_rn(__dmul_rn(m[0], s));
    v = __double2float_rn(__dmul_rn(m[1], s));
    w = __double2float_rn(__dmul_rn(m[2], s));
  } else {
    u = c.u[j];
    v = c.v[j];
    w = c.w[j];
  }
}
template <bool ROWS>
__device__ __forceinline__ float coords_w(const VisCoords &c, int64_t j) {
  if constexpr (ROWS) {
    const uint32_t r = (uint32_t)j / c.n_chan, ch = (uint32_t)j - r * c.n_chan;
    return __double2float_rn(__dmul_rn(c.rows[3 * (size_t)r + 2], c.scale[ch]));
  }
  return c.w[j];
}

// k_sort.cu
cudaError_t sort_visibilities(wst_plan_s *p, const VisCoords &coords, const float2 *vis, const float *weight,
                              bool host_inputs);
cudaError_t vis_cells(wst_plan_s *p, int32_t *plane, int32_t *i0, int32_t *j0, int64_t n_bound);
int64_t scan_tmp_words(int64_t n);

// k_rowgrid.cu
cudaError_t grid_rows(wst_plan_s *p, int p0, int p1, float2 *out, bool fft);
cudaError_t rows_adjoint(wst_plan_s *p, int p0, int p1, const float2 *planes, float2 *dvis, float *dtab);

// k_fft.cu
cudaError_t fft_rows(wst_plan_s *p, float2 *planes, int nplanes, int dir, bool presign,
                     bool postsign);
// occ (nullable): per (plane of the call, row) 0 if the row is known to be zero
cudaError_t fft_cols_a(wst_plan_s *p, float2 *planes, int nplanes, int dir, bool twiddle_first,
                       const uint8_t *occ);
// forward: accumulate planes [p0,p1) (stored at planes[0..]) into image (+comp); range_start
// (range_end): p0 (p1) is the start (end) of the requested plane range, so the images the
// call touches start (finish) their sums in it
cudaError_t fft_cols_b_accumulate(wst_plan_s *p, const float2 *planes, int p0, int p1,
                                  float2 *image, float2 *comp, bool kahan, bool correct,
                                  bool staged_add, bool range_start = false, bool range_end = false);
// adjoint: planes [p0,p1) from the image tile: sign * conj(screen) * corr * dimage, DFT(-1)
cudaError_t fft_cols_bh_from_image(wst_plan_s *p, const float2 *dimage, int p0, int p1,
                                   float2 *planes, bool correct);
cudaError_t correct_image(wst_plan_s *p, float2 *image);

// k_dft.cu
cudaError_t dft_pixels(int64_t n_vis, const float *u, const float *v, const float *w,
                       const float2 *vis, const float *weight, int n, double fov, int64_t n_pix,
                       const int32_t *pa, const int32_t *pb, float2 *out, cudaStream_t s);
cudaError_t predict_points(int64_t n_vis, const float *u, const float *v, const float *w,
                           int64_t n_src, const double *l, const double *m, const double *flux,
                           float2 *out, cudaStream_t s);

}  // namespace wst
