// K-S: device bucket sort of visibilities by (image, w-plane, row of the first tap).
//
// Placement follows section 2 / Eq. 3: a visibility at x = N/2 + u FoV touches the W
// cells i0 = ceil(x - W/2) ... i0 + W - 1 and goes to the closest w-plane.  x, the tap
// start and the plane index are computed in FP64 with explicitly rounded operations
// (no contraction), so they are the same numbers a plain double-precision program
// gets.  The sub-cell offsets g = i0 - (x - W/2) in [0,1) are quantised to 24 bits.
//
// Buckets replace the paper's per-slab linked lists (section 3.2): both hand the
// gridder the visibilities of one region of the mesh contiguously.  Here the region
// is one row j0 of one plane, so grid row q of a plane reads the W contiguous buckets
// j0 = q - W + 1 ... q as one range.
#include "wst_internal.cuh"

namespace wst {

__device__ __forceinline__ uint32_t float_to_ordered(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ bool finite2(float2 a) { return isfinite(a.x) && isfinite(a.y); }

// per image min / max of the finite w (order-preserving integer encoding)
// (fold: of |w|, the w of the mirrored visibilities)
template <bool ROWS>
__global__ void k_wrange(VisCoords coords, const int64_t *boff, uint32_t *wminmax, bool fold) {
  const int img = blockIdx.y;
  const int64_t b0 = boff[img], b1 = boff[img + 1];
  uint32_t mn = 0xFFFFFFFFu, mx = 0u;
  for (int64_t j = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b1;
       j += (int64_t)gridDim.x * blockDim.x) {
    float x = coords_w<ROWS>(coords, j);
    if (fold) x = fabsf(x);
    if (isfinite(x)) {
      uint32_t o = float_to_ordered(x);
      mn = min(mn, o);
      mx = max(mx, o);
    }
  }
  for (int s = 16; s > 0; s >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, s));
    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, s));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mn != 0xFFFFFFFFu) atomicMin(&wminmax[2 * img], mn);
    if (mx != 0u) atomicMax(&wminmax[2 * img + 1], mx);
  }
}

struct SortGeom {
  int n, W, n_w;
  double half_n, half_w, fov;
  float fov_hi, fov_lo;    // fov as a float-float pair
  float half_nf, half_wf;  // N/2 and W/2 (exact in FP32)
};

// The placement decisions (tap start ceil(x - W/2), plane floor((w - w_lo) scale)) are
// those of the FP64 expressions below.  They are taken from float-float values (about
// 46 significant bits, no FP64 instruction) whenever the float-float value is farther
// from the decision boundary than its error bound allows, and from the FP64 expressions
// otherwise (a few visibilities in 10^7).

// FP64 reference placement of one visibility (the rare path)
struct Placement {
  int ci, cj, k;
  uint32_t fx, fy;
  bool dropped;
};

__device__ __noinline__ Placement place_fp64(float uf, float vf, float wf, const SortGeom g, double w_lo,
                                             double scale) {
  Placement P;
  int &ci_out = P.ci, &cj_out = P.cj, &k_out = P.k;
  bool &dropped = P.dropped;
  uint32_t &fx = P.fx, &fy = P.fy;
  const double x = __dadd_rn(g.half_n, __dmul_rn((double)uf, g.fov));
  const double y = __dadd_rn(g.half_n, __dmul_rn((double)vf, g.fov));
  const double hx = __dsub_rn(x, g.half_w), hy = __dsub_rn(y, g.half_w);
  const double ci = ceil(hx), cj = ceil(hy);
  dropped = ci < 0.0 || cj < 0.0 || ci + g.W > g.n || cj + g.W > g.n;
  ci_out = cj_out = k_out = 0;
  fx = fy = 0u;
  if (dropped) return P;
  if (scale > 0.0) {
    const double q = floor(__dmul_rn(__dsub_rn((double)wf, w_lo), scale));
    k_out = q < 0.0 ? 0 : (q > g.n_w - 1 ? g.n_w - 1 : (int)q);
  }
  ci_out = (int)ci;
  cj_out = (int)cj;
  // exact offsets in [0, 1), quantised to 2^-24 (round to nearest, kept below 1)
  const double gx = __dsub_rn(ci, hx), gy = __dsub_rn(cj, hy);
  fx = (uint32_t)min(__double2uint_rn(gx * 16777216.0), 16777215u);
  fy = (uint32_t)min(__double2uint_rn(gy * 16777216.0), 16777215u);
  return P;
}

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// hx = half_n + u fov - half_w as hi + lo (|error| below 2^-46 (|u fov| + n))
__device__ __forceinline__ void tap_arg_ff(float uf, const SortGeom &g, float &hi, float &lo) {
  const float ph = __fmul_rn(uf, g.fov_hi);
  const float pe = __fmaf_rn(uf, g.fov_hi, -ph);  // u fov_hi - ph, exactly
  const float pl = __fmaf_rn(uf, g.fov_lo, pe);
  float sh, se, th, te;
  two_sum_f(g.half_nf, ph, sh, se);
  two_sum_f(sh, -g.half_wf, th, te);
  hi = th;
  lo = __fadd_rn(__fadd_rn(se, te), pl);
}

// c + floor/ceil decision of hi + lo against the integers around floor(hi):
// returns e0 = (hi + lo) - floor(hi) and e1 = floor(hi) + 1 - (hi + lo); the
// one near zero is accurate because its leading part is exact
__device__ __forceinline__ void frac_ff(float hi, float lo, float &fl, float &e0, float &e1) {
  fl = floorf(hi);
  const float fr = __fsub_rn(hi, fl);  // exact
  e0 = __fadd_rn(fr, lo);
  e1 = __fsub_rn(__fsub_rn(1.0f, fr), lo);
}

// pass 1: placement, bucket key, histogram rank (warp-aggregated atomics); ROWS: the
// coordinates come from rows and channels (one instance each, so that the plain one
// keeps its registers)
template <bool ROWS>
__global__ void __launch_bounds__(256, 5) k_keys(VisCoords coords, const float2 *__restrict__ vis,
                       const float *__restrict__ weight, const int64_t *__restrict__ boff,
                       const double *__restrict__ wrange, const float4 *__restrict__ wrange_ff, SortGeom g,
                       uint32_t *offsets, uint4 *keyinfo, unsigned long long *counters,
                       float4 *__restrict__ stash, bool fold) {
  const int img = blockIdx.y;
  const int64_t b0 = boff[img], b1 = boff[img + 1];
  const float4 wff = wrange_ff[img];  // w_lo (hi, lo), scale (hi, lo)
  const bool scale_pos = wrange[4 * img + 1] > 0.0;
  const int64_t span = b1 - b0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float nf = (float)g.n, wn = (float)g.W;
  // uniform trip count across the warp so that the warp-level votes are safe
  const int64_t start = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  uint32_t n_kept = 0, n_dropped = 0, n_nonfinite = 0;
  for (int64_t base = start; base < span; base += stride) {
    const int64_t jj = base + (threadIdx.x & 31);
    const bool in = jj < span;
    const int64_t j = b0 + jj;
    bool nonfinite = false, dropped = false, kept = false;
    uint32_t key = kDropKey, xpack = 0, ypack = 0, mirrored = 0;
    if (in) {
      float uf, vf, wf;
      coords_uvw<ROWS>(coords, j, uf, vf, wf);
      if (fold && wf < 0.0f) {  // Hermitian mirror (exact sign flips); the scatter conjugates V
        uf = -uf;
        vf = -vf;
        wf = -wf;
        mirrored = 1;
      }
      const float2 val = vis[j];
      const float wt = weight ? weight[j] : 1.0f;
      if (stash) stash[j] = make_float4(val.x, val.y, wt, 0.0f);  // value and weight for the scatter
      if (!(isfinite(uf) && isfinite(vf) && isfinite(wf) && finite2(val) && isfinite(wt))) {
        nonfinite = true;
      } else {
        float xh, xl, yh, yl;
        tap_arg_ff(uf, g, xh, xl);
        tap_arg_ff(vf, g, yh, yl);
        float flx, ex0, ex1, fly, ey0, ey1;
        frac_ff(xh, xl, flx, ex0, ex1);
        frac_ff(yh, yl, fly, ey0, ey1);
        // tap start = ceil(hx): fl if hx <= fl, fl + 1 if fl < hx <= fl + 1, else fl + 2
        const float cxf = flx + (ex0 <= 0.0f ? 0.0f : (ex1 < 0.0f ? 2.0f : 1.0f));
        const float cyf = fly + (ey0 <= 0.0f ? 0.0f : (ey1 < 0.0f ? 2.0f : 1.0f));
        const float epsx = (fabsf(xh) + nf) * 0x1p-40f, epsy = (fabsf(yh) + nf) * 0x1p-40f;
        bool sure = fminf(fabsf(ex0), fabsf(ex1)) > epsx && fminf(fabsf(ey0), fabsf(ey1)) > epsy;
        // far outside the mesh the decision cannot change: dropped either way
        const bool out = xh < -4.0f || yh < -4.0f || xh > nf + 4.0f || yh > nf + 4.0f;
        int ci = 0, cj = 0, k = 0;
        uint32_t fx = 0, fy = 0;
        if (out) {
          dropped = true;
          sure = true;
        } else {
          ci = (int)cxf;
          cj = (int)cyf;
          dropped = cxf < 0.0f || cyf < 0.0f || cxf + wn > nf || cyf + wn > nf;
          if (!dropped && scale_pos && !(wff.z > 0.0f)) sure = false;  // scale below FP32 range
          if (!dropped && scale_pos && wff.z > 0.0f) {
            // plane = floor((w - w_lo) scale), clamped
            float dh, de;
            two_sum_f(wf, -wff.x, dh, de);
            const float dl = __fsub_rn(de, wff.y);
            const float qh = __fmul_rn(dh, wff.z);
            const float ql = __fadd_rn(__fmaf_rn(dh, wff.z, -qh), __fmaf_rn(dh, wff.w, __fmul_rn(dl, wff.z)));
            if (qh < -2.0f) k = 0;
            else if (qh > (float)g.n_w + 2.0f) k = g.n_w - 1;
            else {
              float flq, eq0, eq1;
              frac_ff(qh, ql, flq, eq0, eq1);
              // floor(q): fl if fl <= q < fl + 1, fl - 1 if q < fl, fl + 1 if q >= fl + 1
              const float kq = flq + (eq0 < 0.0f ? -1.0f : (eq1 <= 0.0f ? 1.0f : 0.0f));
              const float epsq = (fabsf(wf) * wff.z + fabsf(qh) + 1.0f) * 0x1p-38f;
              sure = sure && fminf(fabsf(eq0), fabsf(eq1)) > epsq;
              k = kq < 0.0f ? 0 : (kq > (float)(g.n_w - 1) ? g.n_w - 1 : (int)kq);
            }
          }
          if (!dropped) {
            // offsets g = c - hx in [0, 1): the difference c - hi is exact
            const float gx = __fsub_rn(__fsub_rn(cxf, xh), xl), gy = __fsub_rn(__fsub_rn(cyf, yh), yl);
            fx = min(__float2uint_rn(fmaxf(gx, 0.0f) * 16777216.0f), 16777215u);
            fy = min(__float2uint_rn(fmaxf(gy, 0.0f) * 16777216.0f), 16777215u);
          }
        }
        if (!sure) {
          const Placement P = place_fp64(uf, vf, wf, g, wrange[4 * img + 0], wrange[4 * img + 1]);
          ci = P.ci;
          cj = P.cj;
          k = P.k;
          dropped = P.dropped;
          fx = P.fx;
          fy = P.fy;
        }
        if (!dropped) {
          key = (uint32_t)((((int64_t)img * g.n_w + k) * g.n + cj) * kColBlocks + (int64_t)ci * kColBlocks / g.n);
          xpack = ((uint32_t)ci << 18) | (fx >> 6);
          ypack = ((fx & 63u) << 24) | fy;
          kept = true;
        }
      }
    }
    // warp-aggregated histogram: one reduction (no return value) per distinct key in the warp
    const unsigned active = __ballot_sync(0xFFFFFFFFu, kept);
    if (kept) {
      const unsigned peers = __match_any_sync(active, key);
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&offsets[key], (uint32_t)__popc(peers));
    }
    if (in) keyinfo[j] = make_uint4(key, mirrored, xpack, ypack);
    n_kept += kept;
    n_dropped += dropped;
    n_nonfinite += nonfinite;
  }
  // the warp's counts, one reduction each
  n_kept = __reduce_add_sync(0xFFFFFFFFu, n_kept);
  n_dropped = __reduce_add_sync(0xFFFFFFFFu, n_dropped);
  n_nonfinite = __reduce_add_sync(0xFFFFFFFFu, n_nonfinite);
  if ((threadIdx.x & 31) == 0) {
    if (n_kept) atomicAdd(&counters[CNT_KEPT], (unsigned long long)n_kept);
    if (n_dropped) atomicAdd(&counters[CNT_DROPPED], (unsigned long long)n_dropped);
    if (n_nonfinite) atomicAdd(&counters[CNT_NONFINITE], (unsigned long long)n_nonfinite);
  }
}

// ---------------------------------------------------------------------------------
// exclusive scan of uint32 counts, in place, multi-level (4096 items per block)
// ---------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *total) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = x;
  for (int s = 1; s < 32; s <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
    if (lane >= s) incl += y;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t ws = warp_sums[lane];
    uint32_t wi = ws;
    for (int s = 1; s < 32; s <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, s);
      if (lane >= s) wi += y;
    }
    warp_sums[lane] = wi - ws;  // exclusive warp offsets
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint32_t r = warp_sums[wid] + incl - x;
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const uint32_t *data, int64_t n, uint32_t *block_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += data[base + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  __shared__ uint32_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = ws[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = t;
  }
}

__global__ void k_scan_apply(uint32_t *data, int64_t n, const uint32_t *block_offsets) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? data[base + i] : 0u;
    s += v[i];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, &total) + (block_offsets ? block_offsets[blockIdx.x] : 0u);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) data[base + i] = run;
    run += v[i];
  }
}

static int64_t scan_blocks(int64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

int64_t scan_tmp_words(int64_t n) {
  int64_t words = 0;
  while (n > 1) {
    n = scan_blocks(n);
    words += n + 64;
  }
  return words + 64;
}

static cudaError_t scan_exclusive(uint32_t *data, int64_t n, uint32_t *tmp, cudaStream_t s,
                                  int64_t &launches) {
  const int64_t nb = scan_blocks(n);
  if (nb <= 1) {
    k_scan_apply<<<1, kScanThreads, 0, s>>>(data, n, nullptr);
    launches += 1;
    return cudaGetLastError();
  }
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, tmp);
  cudaError_t e = scan_exclusive(tmp, nb, tmp + nb + 64, s, launches);
  if (e != cudaSuccess) return e;
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, tmp);
  launches += 2;
  return cudaGetLastError();
}

// pass 2: scatter records to their sorted position.  A visibility's position is its
// bucket's cursor, advanced by a warp-aggregated atomic (one per distinct key in the
// warp); kScatterIlp visibilities are in flight per thread, their loads and atomics
// issued before any result is used.  The order inside a bucket is not specified.
// For the gridder's fixed-point bound, max(|Re|, |Im|) of each weighted value is added to
// the column bins its W taps reach (one or two) of its row bucket.
constexpr int kScatterIlp = 4;

// x added to bin[id] for every valid lane, with one global atomic per run of adjacent
// lanes that share the bin (consecutive channels of one baseline often do): a segmented
// inclusive scan over the warp leaves each run's sum in its last lane.  Every lane of the
// warp calls it; invalid lanes take ids no bin has, so they start runs of their own.
__device__ __forceinline__ void add_bin_runs(float *__restrict__ bin, uint64_t id, float x, bool valid) {
  constexpr unsigned kFull = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  if (!valid) {
    id = ~0ull - (uint64_t)lane;
    x = 0.0f;
  }
  const uint64_t prev = __shfl_up_sync(kFull, id, 1), next = __shfl_down_sync(kFull, id, 1);
  const bool tail = lane == 31 || next != id;
  int start = (lane == 0 || prev != id) ? lane : 0;  // the run's first lane, by a max-scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) start = max(start, __shfl_up_sync(kFull, start, o));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(kFull, x, o);
    if (lane - o >= start) x += y;
  }
  if (valid && tail) atomicAdd(bin + id, x);
}

__global__ void k_scatter(const float2 *__restrict__ vis, const float *__restrict__ weight,
                          const uint4 *__restrict__ keyinfo, uint32_t *__restrict__ cursor, int64_t n_vis,
                          Record *__restrict__ records, float *__restrict__ binmag, int nb, int W,
                          const float4 *__restrict__ stash) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  // uniform trip count across the warp (warp-level votes below)
  const int64_t start = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  for (int64_t w0 = start; w0 < n_vis; w0 += stride * kScatterIlp) {
    uint4 ki[kScatterIlp];
#pragma unroll
    for (int h = 0; h < kScatterIlp; ++h) {
      const int64_t j = w0 + h * stride + lane;
      ki[h] = j < n_vis ? keyinfo[j] : make_uint4(kDropKey, 0u, 0u, 0u);
    }
    uint32_t base[kScatterIlp], peers[kScatterIlp];
#pragma unroll
    for (int h = 0; h < kScatterIlp; ++h) {
      const bool kept = ki[h].x != kDropKey;
      const unsigned active = __ballot_sync(0xFFFFFFFFu, kept);
      peers[h] = kept ? __match_any_sync(active, ki[h].x) : 0u;
      base[h] = (kept && lane == __ffs(peers[h]) - 1) ? atomicAdd(&cursor[ki[h].x], (uint32_t)__popc(peers[h])) : 0u;
    }
    float2 val[kScatterIlp];
    float wt[kScatterIlp];
#pragma unroll
    for (int h = 0; h < kScatterIlp; ++h) {
      const int64_t j = w0 + h * stride + lane;
      if (ki[h].x != kDropKey) {
        if (stash) {
          const float4 vw = stash[j];
          val[h] = make_float2(vw.x, vw.y);
          wt[h] = vw.z;
        } else {
          val[h] = vis[j];
          wt[h] = weight ? weight[j] : 1.0f;
        }
      }
    }
#pragma unroll
    for (int h = 0; h < kScatterIlp; ++h) {
      const bool kept = ki[h].x != kDropKey;
      const uint32_t b = __shfl_sync(0xFFFFFFFFu, base[h], kept ? __ffs(peers[h]) - 1 : lane);
      float vre = 0.0f, vim = 0.0f;
      if (kept) {
        vre = val[h].x * wt[h];
        vim = (ki[h].y ? -val[h].y : val[h].y) * wt[h];  // mirrored: conj
      }
      if (binmag) {  // the whole warp: the first bin by runs, the second (rare) directly
        const float mag = fmaxf(fabsf(vre), fabsf(vim));
        const int i0 = (int)(ki[h].z >> 18);
        const int bl = min(i0 >> kBinShift, nb - 1), bh = min((i0 + W - 1) >> kBinShift, nb - 1);
        const uint64_t row0 = (uint64_t)(ki[h].x / kColBlocks) * (uint64_t)nb;
        add_bin_runs(binmag, row0 + (uint64_t)bl, mag, kept);
        if (kept && bh != bl) atomicAdd(binmag + row0 + bh, mag);
      }
      if (!kept) continue;
      const uint32_t pos = b + __popc(peers[h] & ((1u << lane) - 1u));
      uint4 *dst = reinterpret_cast<uint4 *>(records + pos);
      dst[0] = make_uint4(ki[h].z, ki[h].w, __float_as_uint(vre), __float_as_uint(vim));
      dst[1] = make_uint4((uint32_t)(w0 + h * stride + lane), __float_as_uint(wt[h]), 0u, 0u);
    }
  }
}

// Per grid row q of every (image, plane): over the column bins b, the largest and the
// total of M_b = sum of bin b of the buckets j0 = q - W + 1 ... q (one warp per row; rows
// no visibility reaches get zeros).  The fused row kernel takes its fixed-point quantum
// from them.
__global__ void k_row_bounds(const float *__restrict__ binmag, const uint32_t *__restrict__ offsets,
                             int64_t n_rows, int n, int nb, int W, float2 *__restrict__ rowbound) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_rows; r += warps) {
    const int q = (int)(r % n);
    const int d_lo = min(q, W - 1);
    float mmax = 0.0f, mtot = 0.0f;
    if (offsets[(r - d_lo) * kColBlocks] != offsets[(r + 1) * kColBlocks]) {
      for (int b = lane; b < nb; b += 32) {
        float m = 0.0f;
        for (int d = 0; d <= d_lo; ++d) m += binmag[(size_t)(r - d) * nb + b];
        mmax = fmaxf(mmax, m);
        mtot += m;
      }
      for (int o = 16; o > 0; o >>= 1) {
        mmax = fmaxf(mmax, __shfl_xor_sync(0xFFFFFFFFu, mmax, o));
        mtot += __shfl_xor_sync(0xFFFFFFFFu, mtot, o);
      }
    }
    if (lane == 0) rowbound[r] = make_float2(mmax, mtot);
  }
}

static unsigned grid_for(int64_t n, int threads, int max_blocks) {
  int64_t b = (n + threads - 1) / threads;
  if (b > max_blocks) b = max_blocks;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t sort_visibilities(wst_plan_s *p, const VisCoords &coords, const float2 *vis, const float *weight,
                              bool host_inputs) {
  // inputs in host memory are read once: the placement pass leaves value and weight in
  // device memory for the scatter
  float4 *stash = host_inputs ? p->W_.stash : nullptr;
  cudaStream_t s = p->stream;
  Workspace &ws = p->W_;
  const int64_t nb1 = p->n_buckets + 1;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.counters, 0, sizeof(unsigned long long) * CNT_SLOTS, s))) return e;
  if ((e = cudaMemsetAsync(ws.offsets, 0, sizeof(uint32_t) * nb1, s))) return e;
  // w range of each image (only consulted when the config leaves it to the data)
  if ((e = cudaMemsetAsync(ws.wminmax, 0, sizeof(uint32_t) * 2 * p->batch, s))) return e;
  for (int i = 0; i < p->batch; ++i) {  // min slots start at all-ones
    if ((e = cudaMemsetAsync(ws.wminmax + 2 * i, 0xFF, sizeof(uint32_t), s))) return e;
  }
  const int64_t avg = p->n_vis / p->batch + 1;
  dim3 grd(grid_for(avg, 256, 4096), p->batch);
  const bool fold = (p->cfg.flags & WST_FLAG_WFOLD) != 0;
  if (p->cfg.w_min == p->cfg.w_max) {
    if (coords.rows) k_wrange<true><<<grd, 256, 0, s>>>(coords, p->batch_off, ws.wminmax, fold);
    else k_wrange<false><<<grd, 256, 0, s>>>(coords, p->batch_off, ws.wminmax, fold);
    p->launches += 1;
  }
  if ((e = build_plane_centres(p))) return e;
  SortGeom g;
  g.n = p->n;
  g.W = p->W;
  g.n_w = p->n_w;
  g.half_n = 0.5 * p->n;
  g.half_w = 0.5 * p->W;
  g.fov = p->cfg.fov;
  g.fov_hi = (float)g.fov;
  g.fov_lo = (float)(g.fov - (double)g.fov_hi);
  g.half_nf = (float)g.half_n;
  g.half_wf = (float)g.half_w;
  if (coords.rows)
    k_keys<true><<<grd, 256, 0, s>>>(coords, vis, weight, p->batch_off, p->wrange, p->wrange_ff, g, ws.offsets,
                                     ws.keyinfo, ws.counters, stash, fold);
  else
    k_keys<false><<<grd, 256, 0, s>>>(coords, vis, weight, p->batch_off, p->wrange, p->wrange_ff, g, ws.offsets,
                                      ws.keyinfo, ws.counters, stash, fold);
  p->launches += 1;
  if ((e = cudaGetLastError())) return e;
  if ((e = scan_exclusive(ws.offsets, nb1, ws.scan_tmp, s, p->launches))) return e;
  if ((e = cudaMemcpyAsync(ws.cursor, ws.offsets, sizeof(uint32_t) * nb1, cudaMemcpyDeviceToDevice, s))) return e;
  const int nb = bins_per_row(p->n);
  float *binmag = p->n >= kFixedMinN ? ws.binmag : nullptr;  // only long rows use the bound
  if (binmag && (e = cudaMemsetAsync(binmag, 0, sizeof(float) * (size_t)(p->n_buckets / kColBlocks) * nb, s)))
    return e;
  k_scatter<<<grid_for(p->n_vis, 256, 152 * 16), 256, 0, s>>>(vis, weight, ws.keyinfo, ws.cursor, p->n_vis,
                                                              ws.records, binmag, nb, p->W, stash);
  p->launches += 1;
  if (binmag) {
    const int64_t n_rows = p->n_buckets / kColBlocks;
    k_row_bounds<<<grid_for(n_rows * 32, 256, 152 * 8), 256, 0, s>>>(binmag, ws.offsets, n_rows, p->n, nb, p->W,
                                                                     ws.rowbound);
    p->launches += 1;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// per-visibility placement read back from the sorted records (inspection call)
// ---------------------------------------------------------------------------------
__global__ void k_vis_cells(const Record *rec, const uint32_t *offsets,
                            int64_t n_buckets, int64_t n_bound, int n, int n_w,
                            int32_t *plane, int32_t *i0, int32_t *j0) {
  const int64_t n_kept = offsets[n_buckets];  // records beyond it are not written
  const int64_t n_iter = n_kept < n_bound ? n_kept : n_bound;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_iter;
       s += (int64_t)gridDim.x * blockDim.x) {
    // bucket = last b with offsets[b] <= s
    int64_t lo = 0, hi = n_buckets;  // offsets[lo] <= s < offsets[hi]
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (offsets[mid] <= (uint32_t)s) lo = mid; else hi = mid;
    }
    const uint32_t j = rec[s].index;
    const int64_t row_bucket = lo / kColBlocks;
    plane[j] = (int)((row_bucket / n) % n_w);
    j0[j] = (int)(row_bucket % n);
    i0[j] = rec_i0(rec[s].h);
  }
}

cudaError_t vis_cells(wst_plan_s *p, int32_t *plane, int32_t *i0, int32_t *j0, int64_t n_bound) {
  cudaStream_t s = p->stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(plane, 0xFF, sizeof(int32_t) * p->n_vis, s))) return e;
  if ((e = cudaMemsetAsync(i0, 0xFF, sizeof(int32_t) * p->n_vis, s))) return e;
  if ((e = cudaMemsetAsync(j0, 0xFF, sizeof(int32_t) * p->n_vis, s))) return e;
  if (n_bound > 0)
    k_vis_cells<<<grid_for(n_bound, 256, 152 * 16), 256, 0, s>>>(
        p->W_.records, p->W_.offsets, p->n_buckets, n_bound, p->n, p->n_w, plane,
        i0, j0);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace wst
