// K-G gridding (section 2, Eq. 3), K-D degridding (its adjoint) and K-KG (gradient
// with respect to a tabulated kernel).
//
// Gridding is "owner computes": one CTA per (plane, 64x64 tile) accumulates, in shared
// memory, every tap that lands in its tile -- from its own bucket and from the spill
// classes of its left, upper and upper-left neighbours -- and then writes the whole
// tile with plain coalesced 16-byte stores.  Every plane cell is written exactly once,
// zeros included, so no memset and no global atomics are needed.  The paper's kernel
// instead lets one thread per visibility atomically add into global memory.
//
// A warp handles one visibility at a time: lanes 0..W-1 evaluate the u-profile
// G(a - W/2 + g_x), lanes 16..16+W-1 the v-profile, and each lane then owns taps
// t = lane + 32 i of the W x W footprint (a = t mod W, b = t div W).  The tile is
// stored planar (re, im) with row stride T + W, which is W mod 32, so the 32 taps a
// warp adds per step hit 32 different banks.
#include "wst_internal.cuh"

namespace wst {

constexpr int kGridThreads = 256;
constexpr int kWarps = kGridThreads / 32;

__device__ __forceinline__ void bucket_ranges(const uint32_t *off, int64_t plane_tiles_base,
                                              int tiles, int tx, int ty, uint32_t beg[4],
                                              uint32_t end[4], int dx[4], int dy[4]) {
  const int64_t b = ((plane_tiles_base + ty) * tiles + tx) * kClasses;
  beg[0] = off[b];
  end[0] = off[b + 4];
  dx[0] = 0;
  dy[0] = 0;
  beg[1] = end[1] = beg[2] = end[2] = beg[3] = end[3] = 0;
  dx[1] = -kTile, dy[1] = 0;
  dx[2] = 0, dy[2] = -kTile;
  dx[3] = -kTile, dy[3] = -kTile;
  if (tx > 0) {  // left neighbour: classes 1 (x only) and 2 (x and y)
    const int64_t bl = b - kClasses;
    beg[1] = off[bl + 1];
    end[1] = off[bl + 3];
  }
  if (ty > 0) {  // upper neighbour: classes 2 and 3
    const int64_t bu = b - (int64_t)tiles * kClasses;
    beg[2] = off[bu + 2];
    end[2] = off[bu + 4];
  }
  if (tx > 0 && ty > 0) {  // upper-left: class 2
    const int64_t bul = b - (int64_t)tiles * kClasses - kClasses;
    beg[3] = off[bul + 2];
    end[3] = off[bul + 3];
  }
}

__device__ __forceinline__ float frac24(uint32_t pack) {
  return (float)(pack & 0xFFFFFFu) * (1.0f / 16777216.0f);
}

// grid plane chunk [p0, p0 + gridDim-planes): blockIdx.x = tile, blockIdx.y = plane offset.
// W is a template parameter so that the tap map t -> (t mod W, t div W) is hoisted out of
// the per-visibility loop.
template <int W>
__global__ void __launch_bounds__(kGridThreads)
k_grid_tiles(const Record *__restrict__ rec, const uint32_t *__restrict__ off, int p0, int tiles,
             int n, KernelParams kp, float2 *__restrict__ out, int checker) {
  extern __shared__ float smem[];
  constexpr int S = kTile + W;  // row stride (floats), == W mod 32
  float *sre = smem;
  float *sim = smem + kTile * S;
  const int tx = blockIdx.x % tiles, ty = blockIdx.x / tiles;
  const int pl = blockIdx.y;
  const int P = p0 + pl;
  uint32_t beg[4], end[4];
  int dx[4], dy[4];
  bucket_ranges(off, (int64_t)P * tiles, tiles, tx, ty, beg, end, dx, dy);
  float2 *dst_plane = out + (size_t)pl * n * n;
  if (end[0] == beg[0] && end[1] == beg[1] && end[2] == beg[2] && end[3] == beg[3]) {
    // no visibility reaches this tile (most of them): write its zeros and leave
    float4 *dst = reinterpret_cast<float4 *>(dst_plane);
    const int half_t = kTile / 2;
    for (int e = threadIdx.x; e < kTile * half_t; e += kGridThreads) {
      const int row = e / half_t, c2 = (e % half_t) * 2;
      dst[((size_t)(ty * kTile + row) * n + tx * kTile + c2) >> 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    return;
  }
  for (int i = threadIdx.x; i < kTile * S; i += kGridThreads) {
    sre[i] = 0.0f;
    sim[i] = 0.0f;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int WW = W * W;
  constexpr int ROUNDS = (WW + 31) / 32;
  // this lane's taps: t = lane + 32 it -> column a, row b of the footprint
  int ta[ROUNDS], tb[ROUNDS];
  bool tv[ROUNDS];
#pragma unroll
  for (int it = 0; it < ROUNDS; ++it) {
    const int t = lane + 32 * it;
    tv[it] = t < WW;
    ta[it] = tv[it] ? t % W : 0;
    tb[it] = tv[it] ? t / W : 0;
  }
  const int tap = lane & 15;
  const float targ0 = (float)tap - 0.5f * (float)W;
#pragma unroll 1
  for (int rg = 0; rg < 4; ++rg) {
    const uint32_t b0 = beg[rg], cnt = end[rg] - beg[rg];
    // each warp takes batches of 32 records: one coalesced load, then broadcast by shuffles
#pragma unroll 1
    for (uint32_t base = (uint32_t)wid * 32; base < cnt; base += kWarps * 32) {
      Record mine = {0u, 0u, 0.0f, 0.0f};
      if (base + lane < cnt) mine = rec[b0 + base + lane];
      const int nb = min(32, (int)(cnt - base));
#pragma unroll 1
      for (int r = 0; r < nb; ++r) {
        const uint32_t xp = __shfl_sync(0xFFFFFFFFu, mine.xpack, r);
        const uint32_t yp = __shfl_sync(0xFFFFFFFFu, mine.ypack, r);
        const float vre = __shfl_sync(0xFFFFFFFFu, mine.vre, r);
        const float vim = __shfl_sync(0xFFFFFFFFu, mine.vim, r);
        const int cx = (int)(xp >> kFracBits) + dx[rg];
        const int cy = (int)(yp >> kFracBits) + dy[rg];
        // lanes 0..15 -> u-profile tap `lane`, lanes 16..31 -> v-profile tap `lane - 16`
        const float g = (lane < 16) ? frac24(xp) : frac24(yp);
        const float prof = (tap < W) ? kernel_eval(kp, targ0 + g) : 0.0f;
#pragma unroll
        for (int it = 0; it < ROUNDS; ++it) {
          const float ga = __shfl_sync(0xFFFFFFFFu, prof, ta[it]);
          const float gb = __shfl_sync(0xFFFFFFFFu, prof, 16 + tb[it]);
          const int px = cx + ta[it], py = cy + tb[it];
          if (tv[it] && (unsigned)px < (unsigned)kTile && (unsigned)py < (unsigned)kTile) {
            const float wgt = ga * gb;
            atomicAdd(&sre[py * S + px], vre * wgt);
            atomicAdd(&sim[py * S + px], vim * wgt);
          }
        }
      }
    }
  }
  __syncthreads();
  // flush: one cell per thread and step (consecutive columns: conflict-free shared reads,
  // coalesced 8-byte stores); optional (-1)^(p+q) centring sign
  for (int e = threadIdx.x; e < kTile * kTile; e += kGridThreads) {
    const int row = e / kTile, col = e % kTile;
    const int q = ty * kTile + row, p = tx * kTile + col;
    const float sg = (checker && ((p + q) & 1)) ? -1.0f : 1.0f;
    dst_plane[(size_t)q * n + p] = make_float2(sg * sre[row * S + col], sg * sim[row * S + col]);
  }
}

template <int W>
static void launch_grid(wst_plan_s *p, int p0, int np, float2 *out, bool checker) {
  const size_t smem = sizeof(float) * 2 * kTile * (kTile + W);
  dim3 grd(p->tiles * p->tiles, np);
  k_grid_tiles<W><<<grd, kGridThreads, smem, p->stream>>>(p->W_.records, p->W_.offsets, p0, p->tiles, p->n,
                                                          kernel_params(p), out, checker ? 1 : 0);
}

cudaError_t grid_planes(wst_plan_s *p, int p0, int p1, float2 *out, bool checker) {
  const int np = p1 - p0;
  if (np <= 0) return cudaSuccess;
  switch (p->W) {
#define WST_GRID_CASE(w) \
  case w: launch_grid<w>(p, p0, np, out, checker); break;
    WST_GRID_CASE(2) WST_GRID_CASE(3) WST_GRID_CASE(4) WST_GRID_CASE(5) WST_GRID_CASE(6) WST_GRID_CASE(7)
    WST_GRID_CASE(8) WST_GRID_CASE(9) WST_GRID_CASE(10) WST_GRID_CASE(11) WST_GRID_CASE(12)
    WST_GRID_CASE(13) WST_GRID_CASE(14) WST_GRID_CASE(15) WST_GRID_CASE(16)
#undef WST_GRID_CASE
    default: return cudaErrorInvalidValue;
  }
  p->launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// K-D: degridding, the adjoint of the gridding sum.  One CTA per (plane, tile) loads
// the tile plus its (W-1)-cell halo into shared memory and interpolates every record
// filed under the tile (all spill classes): dvis = w * sum_taps G_a G_b plane[q, p].
// ---------------------------------------------------------------------------------
template <bool GRAD>
__global__ void __launch_bounds__(kGridThreads)
k_degrid_tiles(const Record *__restrict__ rec, const uint32_t *__restrict__ off,
               const uint32_t *__restrict__ perm, const float *__restrict__ rweight, int p0,
               int tiles, int n, KernelParams kp, const float2 *__restrict__ planes,
               float2 *__restrict__ dvis, float *__restrict__ dtab) {
  extern __shared__ float smem[];
  const int W = kp.support;
  const int H = kTile + W - 1;  // tile + halo
  float2 *tile = reinterpret_cast<float2 *>(smem);
  float *ptab = smem + 2 * H * H;  // GRAD: partial table
  const int tx = blockIdx.x % tiles, ty = blockIdx.x / tiles;
  const int pl = blockIdx.y;
  const int P = p0 + pl;
  const int64_t b = (((int64_t)P * tiles + ty) * tiles + tx) * kClasses;
  const uint32_t r0 = off[b], r1 = off[b + kClasses];
  if (r0 == r1) return;  // uniform across the block
  const float2 *src = planes + (size_t)pl * n * n;
  for (int i = threadIdx.x; i < H * H; i += kGridThreads) {
    const int row = i / H, col = i % H;
    const int q = ty * kTile + row, p = tx * kTile + col;
    tile[i] = (q < n && p < n) ? src[(size_t)q * n + p] : make_float2(0.0f, 0.0f);
  }
  if (GRAD)
    for (int i = threadIdx.x; i < kp.table_len; i += kGridThreads) ptab[i] = 0.0f;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int WW = W * W;
  const int rounds = (WW + 31) >> 5;
  const uint32_t cnt = r1 - r0;
#pragma unroll 1
  for (uint32_t base = (uint32_t)wid * 32; base < cnt; base += kWarps * 32) {
    Record mine = {0u, 0u, 0.0f, 0.0f};
    if (base + lane < cnt) mine = rec[r0 + base + lane];
    const int nb = min(32, (int)(cnt - base));
#pragma unroll 1
    for (int r = 0; r < nb; ++r) {
      const uint32_t xp = __shfl_sync(0xFFFFFFFFu, mine.xpack, r);
      const uint32_t yp = __shfl_sync(0xFFFFFFFFu, mine.ypack, r);
      const int cx = (int)(xp >> kFracBits), cy = (int)(yp >> kFracBits);
      const int tap = lane & 15;
      const float g = (lane < 16) ? frac24(xp) : frac24(yp);
      const float targ = (float)tap - kp.half + g;
      const float prof = (tap < W) ? kernel_eval(kp, targ) : 0.0f;
      float sre = 0.0f, sim = 0.0f;
      if (!GRAD) {
#pragma unroll 1
        for (int it = 0; it < rounds; ++it) {
          const int t = lane + 32 * it;
          const bool valid = t < WW;
          const int a = valid ? t % W : 0;
          const int bb = valid ? t / W : 0;
          const float ga = __shfl_sync(0xFFFFFFFFu, prof, a);
          const float gb = __shfl_sync(0xFFFFFFFFu, prof, 16 + bb);
          if (valid) {
            const float2 c = tile[(cy + bb) * H + cx + a];
            const float wgt = ga * gb;
            sre = fmaf(wgt, c.x, sre);
            sim = fmaf(wgt, c.y, sim);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          sre += __shfl_xor_sync(0xFFFFFFFFu, sre, o);
          sim += __shfl_xor_sync(0xFFFFFFFFu, sim, o);
        }
        if (lane == 0) {
          const uint32_t s = r0 + base + r;
          const float wt = rweight ? rweight[s] : 1.0f;
          dvis[perm[s]] = make_float2(wt * sre, wt * sim);
        }
      } else {
        // c_ab = Re(conj(gh[q,p]) * (w V)); the u-profile tap a collects sum_b c_ab G_b and
        // the v-profile tap b collects sum_a c_ab G_a; both are scattered into the
        // table samples bracketing the tap's argument with linear-interpolation weights.
        const float vre = __shfl_sync(0xFFFFFFFFu, mine.vre, r);
        const float vim = __shfl_sync(0xFFFFFFFFu, mine.vim, r);
        float acc = 0.0f;  // lane tap < W: accumulated profile derivative weight
        for (int bb = 0; bb < W; ++bb) {
          const float gb = __shfl_sync(0xFFFFFFFFu, prof, 16 + bb);
          for (int a = 0; a < W; ++a) {
            const float ga = __shfl_sync(0xFFFFFFFFu, prof, a);
            const float2 c = tile[(cy + bb) * H + cx + a];
            const float cr = c.x * vre + c.y * vim;
            // lane a (u-profile) gets cr * gb, lane 16 + bb (v-profile) gets cr * ga
            if (lane == a) acc = fmaf(cr, gb, acc);
            if (lane == 16 + bb) acc = fmaf(cr, ga, acc);
          }
        }
        if (tap < W) {
          float pos = (targ + kp.half) * kp.table_scale;
          int i = (int)floorf(pos);
          i = max(0, min(i, kp.table_len - 2));
          const float f = pos - (float)i;
          atomicAdd(&ptab[i], acc * (1.0f - f));
          atomicAdd(&ptab[i + 1], acc * f);
        }
      }
    }
  }
  if (GRAD) {
    __syncthreads();
    for (int i = threadIdx.x; i < kp.table_len; i += kGridThreads)
      if (ptab[i] != 0.0f) atomicAdd(&dtab[i], ptab[i]);
  }
}

cudaError_t degrid_planes(wst_plan_s *p, int p0, int p1, const float2 *planes, float2 *dvis) {
  const int np = p1 - p0;
  if (np <= 0) return cudaSuccess;
  const int H = kTile + p->W - 1;
  const size_t smem = sizeof(float2) * H * H;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_degrid_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         160 * 1024);
    attr = true;
  }
  dim3 grd(p->tiles * p->tiles, np);
  k_degrid_tiles<false><<<grd, kGridThreads, smem, p->stream>>>(
      p->W_.records, p->W_.offsets, p->W_.perm, p->has_weight ? p->W_.rweight : nullptr, p0,
      p->tiles, p->n, kernel_params(p), planes, dvis, nullptr);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t kernel_grad_planes(wst_plan_s *p, int p0, int p1, const float2 *planes, float *dtab) {
  const int np = p1 - p0;
  if (np <= 0) return cudaSuccess;
  const int H = kTile + p->W - 1;
  const size_t smem = sizeof(float2) * H * H + sizeof(float) * p->cfg.ktable_len;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_degrid_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr = true;
  }
  dim3 grd(p->tiles * p->tiles, np);
  k_degrid_tiles<true><<<grd, kGridThreads, smem, p->stream>>>(
      p->W_.records, p->W_.offsets, p->W_.perm, nullptr, p0, p->tiles, p->n, kernel_params(p),
      planes, nullptr, dtab);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace wst
