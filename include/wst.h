/*
 * wst.h -- C ABI of libwst, a GB300 (sm_103a) w-stacking imager.
 *
 * Method: Gheller, Taffoni & Goz, "High Performance W-stacking for Imaging Radio
 * Astronomy Data: a Parallel and Accelerated Solution", arXiv:2301.06061.
 *   section 2, Eq. 1   measurement equation (what a visibility is)
 *   section 2, Eq. 2   w-stacking inversion: per w-plane 2D Fourier transform,
 *                      phase correction exp(2 pi i w (n - 1)), sum over planes
 *   section 2, Eq. 3   convolutional gridding with a Gaussian kernel of 7 cells
 *   section 2 / 3.2    pipeline: gridding -> FFT per w-plane -> phase shift and
 *                      reduction of the w-planes into the final image
 *
 * Conventions used by every entry point
 *   - N x N image, N a power of two in [64, 16384]; field of view FoV radians;
 *     pixel (a, b) sits at l = (a - N/2) FoV/N, m = (b - N/2) FoV/N; images are
 *     complex64 (interleaved re, im), row-major with row index b (m axis).
 *   - Grid cell (p, q) holds u = (p - N/2)/FoV, v = (q - N/2)/FoV wavelengths;
 *     planes are complex64, row-major with row index q (v axis).
 *   - A visibility at x = N/2 + u FoV (computed in FP64) touches the W cells
 *     i0 = ceil(x - W/2) ... i0 + W - 1 with weight G(i - x) (same along v).
 *     A visibility whose footprint leaves [0, N) on either axis is dropped and
 *     counted; one with a non-finite u, v, w, value or weight is counted apart
 *     (as non-finite, whatever its footprint).
 *   - Planes are cell-centred on [w_min, w_max]: k = clamp(floor((w - w_min) *
 *     (N_w / (w_max - w_min))), 0, N_w - 1), centre w_k = w_min + (k + 1/2) dw.
 *   - The image is the unnormalised dirty image
 *       D(a,b) = sum_k e^{+2 pi i w_k (n-1)} F_k(a,b) / (Ghat(nu_a) Ghat(nu_b)),
 *     F_k the centred 2D transform of plane k with the positive exponent,
 *     n - 1 = -(l^2+m^2)/(1+sqrt(1-l^2-m^2)), nu_a = (a - N/2)/N, Ghat the
 *     Fourier transform of the truncated kernel; D = 0 where l^2 + m^2 >= 1.
 *
 * Memory and errors
 *   - Every data pointer is a DEVICE pointer owned by the caller unless stated;
 *     it is borrowed for the duration of the stream work the call enqueues.
 *   - All work is enqueued on the plan's CUDA stream; calls return once it is
 *     enqueued.  Argument errors are reported synchronously.  Device-side
 *     conditions (e.g. a bounded wait running out) set a device error word that
 *     wst_get_stats reads (it synchronises the stream).
 *   - No entry point traps, aborts or exits; nothing throws across the ABI.
 *   - Scratch memory ("workspace") is caller-provided device memory
 *     (wst_plan_workspace_bytes / wst_plan_set_workspace).  The plan itself owns
 *     only small tables (twiddles, grid-correction, screen terms) it allocates
 *     with cudaMalloc at creation.
 */
#ifndef WST_H
#define WST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum wst_status {
  WST_OK = 0,
  WST_ERR_INVALID_ARG = 1, /* a pointer, size or configuration value is invalid   */
  WST_ERR_OOM = 2,         /* a table allocation failed or the workspace is short  */
  WST_ERR_CUDA = 3,        /* a CUDA runtime call failed (see wst_last_error)      */
  WST_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out                   */
  WST_ERR_UNSUPPORTED = 5, /* valid but outside what this library implements       */
  WST_ERR_STATE = 6        /* call out of order (e.g. no visibilities set)         */
} wst_status;

/* Convolution kernels G (section 2, Eq. 3). */
enum {
  WST_KERNEL_GAUSS = 0, /* exp(-x^2 / (2 sigma^2)), |x| <= W/2; kparam = sigma (cells) */
  WST_KERNEL_ES = 1,    /* exp(beta (sqrt(1 - (2x/W)^2) - 1));  kparam = beta        */
  WST_KERNEL_TABLE = 2  /* piecewise-linear samples on [-W/2, W/2], ktable_len of them */
};

/* wst_config.flags */
#define WST_FLAG_KAHAN 0x1u       /* compensated (Kahan) accumulation of the planes   */
#define WST_FLAG_FP64_SCREEN 0x2u /* phase argument in native FP64, not float-float   */
#define WST_FLAG_TIMING 0x4u      /* record per-stage CUDA-event times in wst_image   */
/* WST_FLAG_WFOLD: every visibility with w < 0 is replaced by its Hermitian mirror
 * (u, v, w, V) -> (-u, -v, -w, conj V) before placement, so the planes only span
 * [min |w|, max |w|] (half the usual range: half the plane spacing at the same N_w).
 * A mirrored visibility contributes the complex conjugate of its original term to
 * Eq. 2, so Re(image) is the dirty image of the original visibilities and Im(image)
 * is not.  Not in the paper (a known variant of w-stacking).  wst_degrid and
 * wst_kernel_grad return WST_ERR_UNSUPPORTED with it (the map is only real-linear). */
#define WST_FLAG_WFOLD 0x8u

/* per-call flags of wst_image / wst_correct / wst_degrid / wst_kernel_grad */
#define WST_NO_CORRECTION 0x1u /* omit the 1/(Ghat(nu_a) Ghat(nu_b)) grid correction */

typedef struct wst_config {
  int32_t n;                /* image side N: a power of two, 64..16384; with grid_n   */
                            /* set, any even N with 64 <= N <= grid_n                  */
  double fov;               /* field of view in radians (> 0)                          */
  int32_t n_w;              /* w-planes per image, 1..4096                             */
  double w_min, w_max;      /* plane range (wavelengths); equal => min/max of the data */
  int32_t support;          /* kernel support W in cells, 2..16                        */
  int32_t kernel;           /* WST_KERNEL_*                                            */
  double kparam;            /* sigma (GAUSS) or beta (ES); unused for TABLE            */
  int32_t ktable_len;       /* TABLE: number of samples, 2..65536                      */
  uint32_t flags;           /* WST_FLAG_*                                              */
  int32_t planes_per_chunk; /* planes held in the workspace at once; 0 = all           */
  int32_t batch;            /* independent images sharing this geometry, >= 1          */
  int32_t oversample;       /* 0 or 1: grid = image (the paper's design); 2: a grid of  */
                            /* 2N cells of 1/(2 fov) wavelengths, the same pixels, the */
                            /* image the central N x N (2N <= 16384)                   */
  int32_t grid_n;           /* 0: the grid side M follows from oversample; otherwise M  */
                            /* itself, a power of two, N <= M <= 16384 (oversample 0 or */
                            /* 1): M cells of N/(M fov) wavelengths, the image the      */
                            /* central N x N of the M x M transform, oversampling       */
                            /* factor M/N (1.25 for N = 3276, M = 4096)                 */
} wst_config;

typedef struct wst_stats {
  int64_t n_vis;       /* visibilities passed to wst_plan_set_vis                      */
  int64_t n_kept;      /* visibilities gridded                                         */
  int64_t n_dropped;   /* footprint outside the grid                                   */
  int64_t n_nonfinite; /* non-finite u, v, w, value or weight                          */
  double w_min, w_max; /* plane range of image 0                                       */
  /* WST_FLAG_TIMING: CUDA-event times (ms) per stage, summed over every
   * wst_plan_set_vis (sort) and wst_image call since the previous wst_get_stats;
   * ms_total = grid + rows + cols_a + cols_b */
  float ms_sort, ms_grid, ms_rows, ms_cols_a, ms_cols_b, ms_total;
  int32_t device_error; /* 0, or a WST_ERR_* raised on the device                       */
  int32_t n_chunks;     /* plane chunks used by the last wst_image                      */
  int64_t n_launches;   /* kernels launched by the last set_vis + wst_image             */
  int64_t n_rows_gridded; /* (plane, row) grid rows the last wst_image / wst_image_range  */
                          /* gridded and transformed: the rows some visibility reaches; */
                          /* the others are known zero and never written or read       */
} wst_stats;

typedef struct wst_plan_s *wst_plan;

/* Library version string, e.g. "0.1.0". */
const char *wst_version(void);

/* Static description of a status code. */
const char *wst_status_string(wst_status s);

/*
 * Create a plan for one imaging geometry (section 2: the mesh N_u x N_v x N_w and
 * the kernel of Eq. 3).  `cuda_stream` is a cudaStream_t (NULL = legacy default
 * stream).  Builds, on the device, the FFT twiddles, the grid-correction table
 * 1/Ghat(nu) (composite Simpson quadrature in FP64) and the l^2 terms of the phase
 * screen.  For WST_KERNEL_TABLE the correction is built by wst_plan_set_kernel_table.
 * Errors: INVALID_ARG (bad config), UNSUPPORTED, OOM, CUDA.  *out is NULL on error.
 */
wst_status wst_plan_create(const wst_config *cfg, void *cuda_stream, wst_plan *out);

/* Release the plan's tables.  Waits for the plan's stream. NULL is a no-op. */
void wst_plan_destroy(wst_plan plan);

/* Change the stream subsequent calls enqueue on. */
wst_status wst_plan_set_stream(wst_plan plan, void *cuda_stream);

/*
 * Time limit, in nanoseconds, of the plan's device-side waits for data: the row FFT of
 * a 16384-point grid (wst_fft_correct) waits on each row's bulk copy into shared
 * memory.  Default 2e9 (2 s); at most 6e10.  On expiry the kernel sets the device error
 * word to WST_ERR_TIMEOUT (read by wst_get_stats), waits -- with the default limit,
 * whatever this setting -- for the copy it has in flight, and returns; the plan stays
 * usable (the word is cleared by the next wst_plan_set_vis).  0 makes every such wait
 * expire at once without looking: it exercises that failure path on purpose (tests of
 * the caller's error handling).  Not in the paper.  Errors: INVALID_ARG.
 */
wst_status wst_plan_set_wait_limit(wst_plan plan, uint64_t wait_ns);

/*
 * Bytes of device workspace needed for `n_vis` visibilities (sort buffers,
 * bucket offsets, one chunk of planes, compensation image).  Host-only call.
 */
wst_status wst_plan_workspace_bytes(wst_plan plan, int64_t n_vis, size_t *bytes);

/*
 * Hand the plan a caller-owned device buffer of `bytes` bytes (256-byte aligned).
 * It must stay valid while the plan uses it.  Errors: INVALID_ARG (NULL, misaligned).
 */
wst_status wst_plan_set_workspace(wst_plan plan, void *device_ptr, size_t bytes);

/*
 * WST_KERNEL_TABLE only: copy `ktable_len` FP32 samples (device pointer) of G on
 * [-W/2, W/2] into the plan and rebuild 1/Ghat on the device (Simpson's rule on
 * every table interval in FP64, so that the interpolation kinks are panel ends).
 */
wst_status wst_plan_set_kernel_table(wst_plan plan, const float *table_dev);

/*
 * Bind visibilities and bucket-sort them (device) by (image, plane, row of the first tap).
 * u, v, w: FP32 [n_vis] wavelengths; vis: complex64 [n_vis]; weight: FP32 [n_vis]
 * or NULL (natural weights 1).  The arrays may be device memory or page-locked host
 * memory (cudaHostAlloc / cudaHostRegister): the sort kernels then read them in place
 * through the host mapping (on GB300 over NVLink-C2C), with no separate copy; pageable
 * host memory only where the device reports cudaDevAttrPageableMemoryAccess.  batch_offsets: HOST int64 [batch + 1], image i
 * owns visibilities [off[i], off[i+1]) (NULL allowed when batch == 1).  The
 * plane range is taken from the config or, if w_min == w_max, from the min/max
 * of the finite w of each image.  The inputs are read during this call's stream
 * work only (values are copied into the sorted records).  Errors: INVALID_ARG,
 * OOM (workspace missing or too small), CUDA.
 */
wst_status wst_plan_set_vis(wst_plan plan, int64_t n_vis, const float *u, const float *v,
                            const float *w, const void *vis, const float *weight,
                            const int64_t *batch_offsets);

/*
 * wst_plan_set_vis for visibilities laid out by row and channel, as an interferometer
 * records them (one row = one baseline at one time; the LOFAR datasets of section 4
 * are of this shape, sub-bands split into channels): visibility i belongs to row
 * r = i / n_chan and channel c = i % n_chan,
 * and its coordinates in wavelengths are
 *     (u, v, w)_i = fl32(uvw_m[3 r + k] * chan_scale[c]),  k = 0, 1, 2,
 * the product of the row's baseline coordinates in metres and the channel's nu / c,
 * formed in FP64 and rounded once to FP32.  The result is exactly that of
 * wst_plan_set_vis with those u, v, w; the inputs shrink from 20 to 8 bytes per
 * visibility plus 24 per row (plus 4 per visibility with weights).
 * uvw_m: FP64 [n_rows x 3]; chan_scale: FP64 [n_chan]; vis, weight, batch_offsets as
 * for wst_plan_set_vis (index i).  n_vis <= n_rows * n_chan (the last row may be
 * partial).  Every array may be device memory or page-locked host memory (read in
 * place).  Errors: INVALID_ARG (n_chan < 1, n_rows too small, NULL or unreachable
 * arrays), OOM, CUDA.
 */
wst_status wst_plan_set_vis_rows(wst_plan plan, int64_t n_vis, const double *uvw_m, int64_t n_rows,
                                 const double *chan_scale, int32_t n_chan, const void *vis,
                                 const float *weight, const int64_t *batch_offsets);

/*
 * Eq. 3: grid planes [plane_begin, plane_end) (global plane index image*N_w + k)
 * into grid_out, complex64 [(plane_end - plane_begin) x M x M], natural layout, M the
 * grid side (N; 2N with oversample = 2; grid_n when set).
 */
wst_status wst_grid(wst_plan plan, int32_t plane_begin, int32_t plane_end, void *grid_out);

/*
 * Eq. 2 for planes [plane_begin, plane_end): transform each plane of grid_inout
 * (layout of wst_grid; overwritten) with the centred positive-exponent 2D FFT,
 * multiply by the plane's phase screen and ADD the central N x N into image_inout,
 * complex64 [batch x N x N].  No grid correction (see wst_correct).
 */
wst_status wst_fft_correct(wst_plan plan, int32_t plane_begin, int32_t plane_end, void *grid_inout,
                           void *image_inout);

/* Multiply image_inout [batch x N x N] by 1/(Ghat(nu_a) Ghat(nu_b)). */
wst_status wst_correct(wst_plan plan, void *image_inout);

/*
 * The whole hot path (Eq. 2-3): grid, FFT, phase screen and plane sum for every
 * plane of every image, then the grid correction (unless WST_NO_CORRECTION).
 * image_out: complex64 [batch x N x N], overwritten; device memory or page-locked
 * host memory, which the last column pass then writes in place (on GB300 over
 * NVLink-C2C) with no separate copy.  Planes are processed in
 * chunks of planes_per_chunk held in the workspace; with WST_FLAG_KAHAN the
 * plane sum is compensated on chip within a chunk and across chunks.
 */
wst_status wst_image(wst_plan plan, void *image_out, uint32_t flags);

/*
 * wst_image restricted to the global planes [plane_begin, plane_end) (plane index
 * image * N_w + k): image_out[i] = the grid-corrected (unless WST_NO_CORRECTION) sum of
 * Eq. 2 over the planes of image i in the range, zero for images with no plane in it.
 * The paper divides the mesh among MPI tasks and reduces their partial results into
 * the image (section 3.1, the slab decomposition, and section 3.2, the reduce of each
 * slab); here each process (one GPU) images a range of w-planes and the caller sums the
 * partial images (one all-reduce): Eq. 2 is a sum over planes and the grid correction
 * is linear, so the partial images of ranges that partition [0, batch * N_w) add up to
 * wst_image.  Layout, memory and chunking as wst_image.  Errors: INVALID_ARG (range).
 */
wst_status wst_image_range(wst_plan plan, int32_t plane_begin, int32_t plane_end, void *image_out,
                           uint32_t flags);

/*
 * Adjoint of wst_image (degridding; the paper lists it as future work in its
 * conclusions): dvis_j = w_j sum_taps G G g_k[q,p], g_k the centred 2D transform
 * with the negative exponent of conj(screen_k) * C_a C_b * dimage.
 * WST_ERR_UNSUPPORTED with WST_FLAG_WFOLD.  With an oversampled grid (M > N)
 * the image enters the grid zero-padded around its central N x N, the adjoint of the
 * forward crop.  dimage: complex64 [batch x N x N]; dvis_out: complex64 [n_vis] in the
 * caller's order (0 for dropped and non-finite visibilities).
 */
wst_status wst_degrid(wst_plan plan, const void *dimage, void *dvis_out, uint32_t flags);

/*
 * WST_KERNEL_TABLE only: gradient of Re<dimage, U> with respect to the kernel
 * samples, U the image without grid correction (WST_NO_CORRECTION must be set:
 * the correction's dependence on the table is left to the caller).  The kernel G of
 * Eq. 3 is the imager's free choice (section 2 uses a Gaussian of 7 cells; the
 * conclusions name better convolution kernels as future work): this gradient lets a
 * caller fit the table.  On an oversampled grid dimage enters zero-padded, as in
 * wst_degrid.  dtable_out: FP32 [ktable_len], overwritten.
 */
wst_status wst_kernel_grad(wst_plan plan, const void *dimage, float *dtable_out, uint32_t flags);

/*
 * Per visibility, in the caller's order, the plane k (within its image) and
 * tap starts i0 (u axis) and j0 (v axis) assigned by the sort, or -1 for a
 * dropped or non-finite one.  int32 device arrays [n_vis].
 */
wst_status wst_vis_cells(wst_plan plan, int32_t *plane_out, int32_t *i0_out, int32_t *j0_out);

/* Counters, plane range and timings.  Synchronises the plan's stream. */
wst_status wst_get_stats(wst_plan plan, wst_stats *out);

/* Message of the last error on this plan ("" if none).  Valid until the next call. */
const char *wst_last_error(wst_plan plan);

/*
 * Direct transform (the exact dirty image; conjugate of Eq. 1) at n_pix pixels:
 *   out_i = sum_j w_j V_j exp(2 pi i (u_j l + v_j m + w_j (n - 1))),
 * l, m from (pa_i, pb_i) on an N x N grid of spacing fov/N.  Phase arguments are
 * formed and reduced modulo one cycle in float-float (about 44 bits), the sum in
 * FP32 with per-block partial sums.  pa, pb: int32 device [n_pix]; out: complex64.
 */
wst_status wst_dft(int64_t n_vis, const float *u, const float *v, const float *w, const void *vis,
                   const float *weight, int32_t n, double fov, int64_t n_pix, const int32_t *pa,
                   const int32_t *pb, void *out, void *cuda_stream);

/*
 * Eq. 1 for a point-source sky: V_j = sum_s S_s exp(-2 pi i (u_j l_s + v_j m_s +
 * w_j (n_s - 1))).  l, m, flux: FP64 device [n_src]; out: complex64 [n_vis].
 */
wst_status wst_predict_points(int64_t n_vis, const float *u, const float *v, const float *w,
                              int64_t n_src, const double *l, const double *m, const double *flux,
                              void *out, void *cuda_stream);

/*
 * Largest n_pix accepted by wst_dft_noalloc (size of its built-in scratch).
 */
#define WST_DFT_NOALLOC_MAX_PIX 4096

/*
 * wst_dft without any device allocation.  (The paper has no counterpart: this is
 * an interface for a class of callers, not part of the method.)
 *
 * Who needs it: code that must not call cudaMalloc, cudaFree or an allocating
 * library routine -- a real-time pipeline (e.g. a correlator back end) that
 * forbids allocation after start-up because cudaMalloc/cudaFree can block and
 * synchronise the device; a component inside an application whose memory pool has
 * reserved the whole device, so a fresh allocation would fail or fragment it; or a
 * plug-in that must keep the host application's device footprint fixed.  Such a
 * caller passes inputs and outputs it already owns; this call brings its own
 * scratch.
 *
 * Same arguments and result as wst_dft (out_i = sum_j w_j V_j exp(2 pi i (u_j l +
 * v_j m + w_j (n-1))), float-float phases), but the partial sums live in a fixed
 * 2 MiB array compiled into the library (one per GPU that loads it, kept until the
 * process exits), reduced by a second pass in a fixed order, so repeated calls give
 * identical bits and `out` needs no clearing.
 *
 * Limits and rules:
 *   - n_pix <= WST_DFT_NOALLOC_MAX_PIX, else WST_ERR_UNSUPPORTED and nothing runs.
 *   - The array's device address belongs to a CUDA context (a device's primary
 *     context, a context the caller made current with the driver API, the primary
 *     context re-created after cudaDeviceReset).  The first call in each context
 *     looks it up (cudaGetSymbolAddress, with that context current) and remembers
 *     it under the driver's unique context id; later calls in that context reuse
 *     it.  Make that first call before any stream capture.
 *   - Every call on a device shares the one array: calls whose GPU work overlaps
 *     (other streams, other host threads) race and corrupt each other's sums.
 *     Serialise them, e.g. on one stream.
 *   - Each call writes every scratch slot it later reads; nothing carries over.
 */
wst_status wst_dft_noalloc(int64_t n_vis, const float *u, const float *v, const float *w,
                           const void *vis, const float *weight, int32_t n, double fov,
                           int64_t n_pix, const int32_t *pa, const int32_t *pb, void *out,
                           void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* WST_H */
