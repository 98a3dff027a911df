// Row-wise gridding fused with the row FFT (K-G + K-F rows), and its adjoint fused with
// degridding (K-D) or with the tabulated-kernel gradient (K-KG).
//
// Forward, per (plane, row q) work item: the visibilities whose W-row footprint covers
// row q are the contiguous buckets j0 = q - W + 1 ... q (k_sort.cu).  If there are
// none the row is zero: the item writes zeros and is done (no gridding, no FFT, no read
// of a plane).  Otherwise the row is accumulated in shared memory -- each thread takes
// visibilities, weights its W taps by G(a - W/2 + g_x) G(d - W/2 + g_y), d = q - j0,
// and adds them with shared-memory atomics (section 2, Eq. 3) -- then transformed in
// place (centring sign (-1)^(p+q) folded into the first stage) and written once.  The
// paper's gridder instead adds every tap of every visibility to the mesh in global
// memory, and the FFT reads the mesh back.
//
// Adjoint, per item: the row of the adjoint plane is transformed with the negative
// exponent (sign (-1)^(p+q) after the last stage), kept in shared memory, and every
// visibility whose footprint covers the row reads its W taps from it: degridding adds
// w G_y(d) sum_a G_x(a) row[i0 + a] to dvis; the kernel gradient scatters the tap
// products into a shared partial table.  Rows nobody reads are skipped.
//
// Items are handed out by a device counter to persistent CTAs (one row or, for short
// rows, RowCfg::RPC rows per CTA step).
//
// Fixed-point accumulation.  Shared-memory integer atomics sustain about three times
// the rate of float ones on this GPU.  The sort leaves, per row bucket and bin of 64
// columns, the sum of max(|Re|, |Im|) of the weighted values whose taps reach the bin;
// for row q, M_b = the sum of bin b over the buckets j0 = q - W + 1 ... q bounds every
// cell of bin b by M_b G^2 (G the largest |kernel value|); the sort's last pass
// (k_row_bounds) leaves max_b M_b and sum_b M_b per row.  With B = max_b M_b G^2 the
// row is accumulated in int32 units of delta = B / 2^34: each tap is rounded to a
// multiple of delta (error <= delta/2).  B is a sum of magnitudes, far above the cells
// of a dense bin (random phases add up like a square root), which is what makes the
// fine quantum usable; but a cell or a single tap can exceed 2^31 delta = B/8 (a
// dominant visibility, a coherent pile-up), so every integer atomic returns the old
// value and the kernel checks for a wrapped partial sum or a saturated conversion: if
// any occurred in the row, the row is zeroed and accumulated again with float atomics.
// Rows whose busiest bin holds fewer than 64 mean contributions take delta = B / 2^30,
// which cannot overflow (sparse rows would otherwise overflow often; their cells are
// few-term sums, for which the coarser quantum is precise enough).
// Rows whose busiest bin holds more than kFixedBinCap times the row's mean magnitude
// per visibility-row (the bins count a visibility-row once per bin it reaches,
// 1 + (W - 1)/64 bins on average) go straight to float atomics.  On the benchmark
// workload the image error against the FP64 oracle equals that of all-float
// accumulation.  Images narrower than kFixedMinN (8192) keep float atomics throughout.
#include "fft_core.cuh"

namespace wst {

template <int N>
__device__ __forceinline__ void zero_row(float2 *srow, int jt) {
  float4 *p = reinterpret_cast<float4 *>(srow);
  for (int i = jt; i < N / 2; i += RowCfg<N>::TPR) p[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// The W x-taps G(a - W/2 + g_x), a = 0 .. W-1.  For the Gaussian, three exponentials
// instead of W: with t = g_x - W/2, G(t + a + 1) / G(t + a) = R q^a, R = exp(-(2t + 1) c),
// q = exp(-2c), c = 1/(2 sigma^2); each exponential is a power of two, exp(-y c) =
// 2^(-y c log2 e), with c log2 e rounded once from FP64 (the FP32 argument carries the
// same rounding as with exp).
template <int WT>
__device__ __forceinline__ void x_taps(const KernelParams &kp, float gx, float q, float (&g)[WT]) {
  if (kp.kind == WST_KERNEL_GAUSS) {
    const float t = gx - kp.half;
    float ga = exp2f(-t * t * kp.l2c);
    float ra = exp2f(-(2.0f * t + 1.0f) * kp.l2c);
#pragma unroll
    for (int a = 0; a < WT; ++a) {
      g[a] = ga;
      ga *= ra;
      ra *= q;
    }
  } else if (kp.tap_table) {
    // tabulated kernel: all W taps share the sub-cell position, so their bracketing
    // samples are one contiguous run of W pairs (tap-major table)
    const float pos = gx * (float)kp.per_cell;
    const int i = min((int)pos, kp.per_cell - 1);
    const float f = pos - (float)i;
    const float2 *run = kp.tap_table + (size_t)i * WT;
    if constexpr (WT % 2 == 0) {  // 16-byte aligned: two taps per load
      const float4 *run4 = reinterpret_cast<const float4 *>(run);
#pragma unroll
      for (int a = 0; a < WT / 2; ++a) {
        const float4 t = __ldg(run4 + a);
        g[2 * a] = fmaf(f, t.y - t.x, t.x);
        g[2 * a + 1] = fmaf(f, t.w - t.z, t.z);
      }
    } else {
#pragma unroll
      for (int a = 0; a < WT; ++a) {
        const float2 t = __ldg(run + a);
        g[a] = fmaf(f, t.y - t.x, t.x);
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < WT; ++a) g[a] = kernel_eval(kp, (float)a - kp.half + gx);
  }
}

constexpr int kFixedBinCap = 8192;
// Short rows (N < kFixedMinN) carry few visibility-rows each: the bound's extra barriers
// cost more than the float atomics they would save, so they keep float accumulation.
template <int N>
constexpr bool kFixedRows = N >= kFixedMinN;

// one tap into the planar row: float atomics, or (FIXED) the tap already in units of the
// row's quantum (the record's value was scaled by 1/delta once), converted and added as
// an integer atomic; ovf turns negative if the cell's partial sum wrapped around (the
// returned old value and the new sum have signs no in-range sum can give).  Saturated
// conversions are excluded per record (grid_row), not per tap.
template <bool FIXED>
__device__ __forceinline__ void add_tap(float *sre, float *sim, int c, float re, float im, int &ovf) {
  if constexpr (FIXED) {
    const int xr = __float2int_rn(re), xi = __float2int_rn(im);
    const int o1 = atomicAdd(reinterpret_cast<int *>(sre) + c, xr);
    const int o2 = atomicAdd(reinterpret_cast<int *>(sim) + c, xi);
    const int s1 = o1 + xr, s2 = o2 + xi;
    ovf |= ((o1 ^ s1) & (xr ^ s1)) | ((o2 ^ s2) & (xi ^ s2));
  } else {
    atomicAdd(&sre[c], re);
    atomicAdd(&sim[c], im);
  }
}

// Accumulate the visibilities of rows j0 = q - d_lo ... q into the row, stored planar
// (re[0..N), im[0..N)).  Their sub-buckets are contiguous in the sorted records, so the
// range bnd[0] .. bnd[d_lo + 1] is split evenly over the row's threads, one visibility
// per thread (two in flight); bnd[i] is where row j0 = q - d_lo + i starts.  WT > 0
// fixes the support at compile time.
__device__ __forceinline__ void cp_async16_rg(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// The previous row's transformed values, written out while this row is gridded: two
// groups of four of a thread's outputs while the row's offsets load, then four per
// record it grids, the rest when its gridding ends, so that a row's 128 KB leave the SM
// spread over the next row's gridding instead of in one burst at the end of its
// transform.
template <int N>
struct PendingRow {
  static constexpr int EPT = RowCfg<N>::EPT, TPR = RowCfg<N>::TPR, CH = 4, NCH = EPT / CH;
  static constexpr int NST = num_stages(N, EPT), RL = stage_radix(N, EPT, NST - 1);
  float2 v[EPT];
  float2 *orow;
  int next;  // next group of CH outputs to write; NCH: nothing pending
  // one group, chosen by a chain of branches whose stores are separate asm statements
  // (a merged store would index v at run time and move it out of registers)
  template <int C>
  __device__ __forceinline__ void write_group(int jt) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int e = C * CH + k;  // output e = b RL + r of the last stage
      float2 *a = orow + out_index<N, EPT, TPR, NST - 1>(jt, e / RL, e % RL);
      asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(v[e].x), "f"(v[e].y) : "memory");
    }
  }
  template <int C = 0>
  __device__ __forceinline__ void write_chain(int jt) {
    if constexpr (C < NCH) {
      if (next == C) write_group<C>(jt);
      else write_chain<C + 1>(jt);
    }
  }
  __device__ __forceinline__ void write_one(int jt) {
    if (next >= NCH) return;
    write_chain(jt);
    ++next;
  }
  __device__ __forceinline__ void write_all(int jt) {
#pragma unroll
    for (int c = 0; c < NCH; ++c)
      if (c >= next) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
          const int e = c * CH + k;
          __stcs(&orow[out_index<N, EPT, TPR, NST - 1>(jt, e / RL, e % RL)], v[e]);
        }
      }
    next = NCH;
  }
};
struct NoPending {
  __device__ __forceinline__ void write_one(int) {}
  __device__ __forceinline__ void write_all(int) {}
};

// With FIXED, qscale = 1/delta and gmax the largest |kernel value|: a record whose scaled
// value times gmax comes within 0.2% of 2^31 (a margin for the rounding of the taps)
// could saturate a conversion, and sends the row to float atomics like a wrapped sum.
template <int N, int WT, bool FIXED, class PEND>
__device__ __forceinline__ int grid_row(float *sre, float *sim, const Record *__restrict__ rec,
                                        const uint32_t *bnd, int d_lo, const KernelParams &kp, int jt,
                                        float qscale, float gmax, RecHead *stg, int stg_stride, PEND &pd) {
  constexpr int TPR = RowCfg<N>::TPR;
  int ovf = 0;
  const uint32_t s_end = bnd[d_lo + 1];
  if constexpr (WT > 0) {
    const float q = exp2f(-2.0f * kp.l2c);
    // this thread's record heads are copied into its own three shared slots two records
    // ahead (cp.async), so two loads are in flight while a record is gridded
    const uint32_t slot0 = (uint32_t)__cvta_generic_to_shared(stg);
    const uint32_t sstep = (uint32_t)(stg_stride * sizeof(RecHead));
    uint32_t s = bnd[0] + jt;
    if (s < s_end) cp_async16_rg(slot0, rec + s);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (s + TPR < s_end) cp_async16_rg(slot0 + sstep, rec + s + TPR);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int i = 0;  // the thread's records come in increasing order, so do their buckets
    int cur = 0, nxt = 2;  // slot of this record, slot of the one two ahead
    for (; s < s_end; s += TPR) {
      if (s + 2 * TPR < s_end) cp_async16_rg(slot0 + nxt * sstep, rec + s + 2 * TPR);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 2;" ::: "memory");
      const RecHead r = stg[cur * stg_stride];
      cur = cur == 2 ? 0 : cur + 1;
      nxt = nxt == 2 ? 0 : nxt + 1;
      while (i < d_lo && bnd[i + 1] <= s) ++i;  // the last row starting at or before the record
      // the record's row offset keeps y in [-W/2, W/2): no range test
      const float y = (float)(d_lo - i) - kp.half + rec_gy(r);
      const float gy = kp.kind == WST_KERNEL_GAUSS ? exp2f(-y * y * kp.l2c) : kernel_eval(kp, y);
      float g[WT];
      x_taps<WT>(kp, rec_gx(r), q, g);
      const int i0 = rec_i0(r);
      const float gq = FIXED ? gy * qscale : gy;
      const float vre = r.vre * gq, vim = r.vim * gq;
      if (FIXED && fmaxf(fabsf(vre), fabsf(vim)) * gmax >= 0x1.ffp30f) ovf = -1;
#pragma unroll
      for (int a = 0; a < WT; ++a) add_tap<FIXED>(sre, sim, i0 + a, vre * g[a], vim * g[a], ovf);
      pd.write_one(jt);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else {
    const int W = kp.support;
    for (uint32_t s = bnd[0] + jt; s < s_end; s += TPR) {
      int i = d_lo;
      while (s < bnd[i]) --i;
      const RecHead r = rec_head(rec, s);
      const float gy = kernel_eval(kp, (float)(d_lo - i) - kp.half + rec_gy(r));
      const float gx = rec_gx(r);
      const int i0 = rec_i0(r);
      const float gq = FIXED ? gy * qscale : gy;
      const float vre = r.vre * gq, vim = r.vim * gq;
      if (FIXED && fmaxf(fabsf(vre), fabsf(vim)) * gmax >= 0x1.ffp30f) ovf = -1;
      for (int a = 0; a < W; ++a) {
        const float g = kernel_eval(kp, (float)a - kp.half + gx);
        add_tap<FIXED>(sre, sim, i0 + a, vre * g, vim * g, ovf);
      }
      pd.write_one(jt);
    }
  }
  return ovf;
}

// One non-empty row q of a plane: accumulate, transform (FFT) and write it (with a
// PendingRow, during the next row's gridding: pd holds the row before this one on entry
// and this row on return).  Every thread of the row group calls it; it ends with the row
// buffer free again.
template <int N, bool FFT, int WT, class PEND>
__device__ __forceinline__ void grid_one_row(float2 *srow, uint32_t *bnd, const Record *__restrict__ rec,
                                             const uint32_t *__restrict__ off, int64_t b0, int q, bool nonempty,
                                             const KernelParams &kp, float2 *__restrict__ orow,
                                             const float2 *twt, int jt, const float2 *__restrict__ rowbound,
                                             float gmax, RecHead *stg, int stg_stride, PEND &pd) {
  using C = RowCfg<N>;
  constexpr int EPT = C::EPT, TPR = C::TPR;
  constexpr int NST = num_stages(N, EPT);
  constexpr int R0 = stage_radix(N, EPT, 0);
  constexpr int RL = stage_radix(N, EPT, NST - 1);
  auto smi = [](int i) { return i + i / EPT; };
  const int W = WT > 0 ? WT : kp.support;
  float *sre = reinterpret_cast<float *>(srow), *sim = sre + N;  // planar accumulation
  const int d_lo = min(q, W - 1);
  // the row's largest bin sum and total of the bin sums (k_row_bounds), broadcast
  float2 mb = make_float2(0.0f, 0.0f);
  if (nonempty) {
    for (int i = jt; i <= d_lo + 1; i += TPR) bnd[i] = off[(b0 + q - d_lo + i) * kColBlocks];
    if constexpr (kFixedRows<N>) mb = __ldg(rowbound + b0 + q);
  }
  // two groups of the previous row's outputs go out while the offsets load (more, or one
  // more after the first record heads are requested, measured slower)
  pd.write_one(jt);
  pd.write_one(jt);
  zero_row<N>(srow, jt);
  __syncthreads();
  // the same decision and quantum in every thread of the row
  const uint32_t cnt = nonempty ? bnd[d_lo + 1] - bnd[0] : 0u;
  const float mmax = mb.x, mtot = mb.y;
  const float bound = mmax * (gmax * gmax);
  // n_eff: the busiest bin's magnitude in units of the row's mean per visibility-row
  const float n_eff = mmax * (float)cnt * (1.0f + (float)(W - 1) / (float)kBinCols) / fmaxf(mtot, 0x1p-126f);
  const bool fixed = kFixedRows<N> && nonempty && cnt < (1u << 30) && bound >= 0x1p-90f && bound <= 0x1p+100f &&
                     n_eff <= (float)kFixedBinCap;
  // a bin of fewer than ~64 mean contributions may hold a single tap above B/8: such rows
  // take delta = B / 2^30, with which no tap or partial sum can leave the int32 range
  const float unit = n_eff >= 64.0f ? 0x1p-34f : 0x1p-30f;
  bool fx = fixed;
  int ovf = 0;
  if (nonempty) {
    if (fixed)
      ovf = grid_row<N, WT, true>(sre, sim, rec, bnd, d_lo, kp, jt, 1.0f / (bound * unit), gmax, stg, stg_stride, pd);
    else grid_row<N, WT, false>(sre, sim, rec, bnd, d_lo, kp, jt, 1.0f, gmax, stg, stg_stride, pd);
  }
  bool redo = false;  // a tap or a partial sum left the int32 range: accumulate in float
  if constexpr (kFixedRows<N>) redo = __syncthreads_or(ovf < 0);
  else __syncthreads();
  if (redo) {
    zero_row<N>(srow, jt);
    __syncthreads();
    if (nonempty) grid_row<N, WT, false>(sre, sim, rec, bnd, d_lo, kp, jt, 1.0f, gmax, stg, stg_stride, pd);
    fx = false;
    __syncthreads();
  }
  pd.write_all(jt);  // the previous row is out before this one's transform takes its place
  const float delta = fx ? bound * unit : 1.0f;
  const int *ire = reinterpret_cast<const int *>(sre), *iim = reinterpret_cast<const int *>(sim);
  if constexpr (FFT) {
    float2 v[EPT];
    if (fx) {
#pragma unroll
      for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int idx = in_index<N, EPT, TPR, 0>(jt, b, r);
          const float sg = ((idx + q) & 1) ? -delta : delta;  // centring sign and quantum
          v[b * R0 + r] = make_float2(sg * __int2float_rn(ire[idx]), sg * __int2float_rn(iim[idx]));
        }
    } else {
#pragma unroll
      for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int idx = in_index<N, EPT, TPR, 0>(jt, b, r);
          const float sg = ((idx + q) & 1) ? -1.0f : 1.0f;  // centring sign
          v[b * R0 + r] = make_float2(sg * sre[idx], sg * sim[idx]);
        }
    }
    __syncthreads();  // natural-order reads done before the padded writes
    const TableTw<N, EPT, TPR, 1> twp{twt, jt};
    stage_compute_f<N, EPT, TPR, 0, 1>(v, jt, twp);
    middle_stages_f<N, EPT, TPR, 1, 1>(v, jt, srow, smi, twp);
    stage_compute_f<N, EPT, TPR, NST - 1, 1>(v, jt, twp);
    if constexpr (std::is_same_v<PEND, PendingRow<N>>) {
      // kept for the next row's gridding (assigned on every path, so that the old values
      // are dead after their last write)
#pragma unroll
      for (int e = 0; e < EPT; ++e) pd.v[e] = v[e];
      pd.orow = orow;
      pd.next = (orow && nonempty) ? 0 : PEND::NCH;
    } else if (orow && nonempty) {
#pragma unroll
      for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r)  // streaming stores: keep the L2 for the records
          __stcs(&orow[out_index<N, EPT, TPR, NST - 1>(jt, b, r)], v[b * RL + r]);
    }
  } else {
    if (orow) {
      if (fx)
        for (int i = jt; i < N; i += TPR)
          orow[i] = make_float2(delta * __int2float_rn(ire[i]), delta * __int2float_rn(iim[i]));
      else
        for (int i = jt; i < N; i += TPR) orow[i] = make_float2(sre[i], sim[i]);
    }
  }
  __syncthreads();  // the row buffer is reused by the next row
}

// rows handed out per counter fetch (one row per CTA step); warp 0 scans a batch, one
// lane per row.  Eight rows keep the end of the kernel's row stream balanced.
constexpr int kRowBatch = 8;

template <int N, bool FFT, int WT>
__global__ void __launch_bounds__(RowCfg<N>::THREADS)
k_grid_rows(const Record *__restrict__ rec, const uint32_t *__restrict__ off, int p0, int np,
            KernelParams kp, float2 *__restrict__ out, uint8_t *__restrict__ occ,
            unsigned long long *__restrict__ counter, Tw tw, const float2 *__restrict__ rowbound,
            unsigned long long *__restrict__ rows_done) {
  using C = RowCfg<N>;
  constexpr int TPR = C::TPR, RPC = C::RPC;
  extern __shared__ __align__(16) float2 sm_rows[];
  __shared__ long long s_item;
  __shared__ uint32_t s_bnd[RPC][kMaxSupport + 2];
  __shared__ uint32_t s_gmax;  // largest |kernel value| (FP32 bits)
  const int rl = threadIdx.x / TPR, jt = threadIdx.x % TPR;
  float2 *srow = sm_rows + rl * C::PADL;
  float2 *twt = sm_rows + RPC * C::PADL;  // twiddle tables (visible after the first barrier)
  // three record-head slots per thread after the tables
  RecHead *stg = reinterpret_cast<RecHead *>(twt + (FFT ? line_table_size<N, C::EPT, TPR>() : 0)) + threadIdx.x;
  const int stg_stride = C::THREADS;
  if constexpr (FFT) fill_line_tables<N, C::EPT, TPR>(twt, tw);
  // G^2 of the fixed-point bound (G = 1 for the Gaussian and the ES kernel, the largest
  // |sample| of a table: linear interpolation stays below it)
  if (threadIdx.x == 0) s_gmax = __float_as_uint(1.0f);
  if (kp.kind == WST_KERNEL_TABLE) {
    __syncthreads();
    float gm = 0.0f;
    for (int i = threadIdx.x; i < kp.table_len; i += blockDim.x) gm = fmaxf(gm, fabsf(__ldg(kp.table + i)));
    if (threadIdx.x == 0) s_gmax = 0u;
    __syncthreads();
    atomicMax(&s_gmax, __float_as_uint(gm));
  }
  __syncthreads();
  const float gmax = __uint_as_float(s_gmax);
  const long long total = (long long)np * N;
  const int W = WT > 0 ? WT : kp.support;
  auto row_empty = [&](long long item) {
    const int64_t b0 = (int64_t)(p0 + item / N) * N;
    const int q = (int)(item % N);
    return off[(b0 + max(0, q - W + 1)) * kColBlocks] == off[(b0 + q + 1) * kColBlocks];
  };
  if constexpr (RPC == 1) {
    // batches of kRowBatch rows: warp 0 finds the non-empty ones (and fills occ), the
    // CTA then grids and transforms only those; the next batch is fetched meanwhile
    __shared__ int s_list[kRowBatch], s_cnt;
    unsigned long long next = 0;
    // the transforming path writes each row during the next row's gridding
    std::conditional_t<FFT, PendingRow<N>, NoPending> pd;
    if constexpr (FFT) {
      pd.next = PendingRow<N>::NCH;
      pd.orow = nullptr;
    }
    if (threadIdx.x == 0) next = atomicAdd(counter, (unsigned long long)kRowBatch);
    while (true) {
      if (threadIdx.x == 0) {
        s_item = (long long)next;
        next = atomicAdd(counter, (unsigned long long)kRowBatch);
      }
      __syncthreads();
      const long long base = s_item;
      if (base >= total) break;
      if (threadIdx.x < 32) {
        const long long item = base + threadIdx.x;
        const bool valid = (int)threadIdx.x < kRowBatch && item < total;
        const bool nonempty = valid && !row_empty(item);
        if (valid) occ[item] = nonempty ? 1 : 0;
        // plain gridding hands the planes to the caller: it also lists the empty rows,
        // which get zeros; the column pass reads only occupied rows of transformed planes
        const bool listed = FFT ? nonempty : valid;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, listed);
        if (listed) s_list[__popc(m & ((1u << threadIdx.x) - 1u))] = threadIdx.x * 2 + (nonempty ? 1 : 0);
        if (threadIdx.x == 0) s_cnt = __popc(m);
        if (rows_done) {  // the occupied rows of the batch, for the caller's statistics
          const unsigned occupied = __ballot_sync(0xFFFFFFFFu, nonempty);
          if (threadIdx.x == 0 && occupied) atomicAdd(rows_done, (unsigned long long)__popc(occupied));
        }
      }
      __syncthreads();
      const int cnt = s_cnt;
      for (int k = 0; k < cnt; ++k) {
        const int e = s_list[k];
        const long long item = base + (e >> 1);
        const int pl = (int)(item / N), q = (int)(item % N);
        grid_one_row<N, FFT, WT>(srow, s_bnd[0], rec, off, (int64_t)(p0 + pl) * N, q, e & 1, kp,
                                 out + ((int64_t)pl * N + q) * N, twt, jt, rowbound, gmax, stg, stg_stride, pd);
      }
    }
    pd.write_all(jt);  // the CTA's last row
  } else {
    while (true) {
      if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, (unsigned long long)RPC);
      __syncthreads();
      const long long base = s_item;
      __syncthreads();
      if (base >= total) break;
      const long long item = base + rl;
      const bool valid = item < total;
      const int pl = valid ? (int)(item / N) : 0;
      const int q = valid ? (int)(item % N) : 0;
      const bool empty = !valid || row_empty(item);
      if (valid && jt == 0) occ[item] = empty ? 0 : 1;
      if (rows_done && valid && jt == 0 && !empty) atomicAdd(rows_done, 1ull);
      float2 *orow = valid && (!FFT || !empty) ? out + ((int64_t)pl * N + q) * N : nullptr;
      NoPending none;
      grid_one_row<N, FFT, WT>(srow, s_bnd[rl], rec, off, (int64_t)(p0 + pl) * N, q, !empty, kp, orow, twt, jt,
                               rowbound, gmax, stg, stg_stride, none);
    }
  }
}

// -------------------------------------------------------------------------------------
// adjoint: row FFT^H of the adjoint plane + degridding / kernel gradient
// -------------------------------------------------------------------------------------
template <int N, bool KGRAD>
__global__ void __launch_bounds__(RowCfg<N>::THREADS)
k_rows_adjoint(const float2 *__restrict__ planes, const Record *__restrict__ rec,
               const uint32_t *__restrict__ off, int p0, int np, KernelParams kp,
               float2 *__restrict__ dvis, float *__restrict__ dtab,
               unsigned long long *__restrict__ counter, Tw tw) {
  using C = RowCfg<N>;
  constexpr int EPT = C::EPT, TPR = C::TPR, RPC = C::RPC;
  constexpr int NST = num_stages(N, EPT);
  constexpr int R0 = stage_radix(N, EPT, 0);
  constexpr int RL = stage_radix(N, EPT, NST - 1);
  extern __shared__ __align__(16) float2 sm_rows[];
  __shared__ long long s_item;
  float2 *twt = sm_rows + RPC * C::PADL;  // twiddle tables (visible after the first barrier)
  fill_line_tables<N, C::EPT, TPR>(twt, tw);
  float *ptab = reinterpret_cast<float *>(twt + line_table_size<N, C::EPT, C::TPR>());  // KGRAD partial table
  const int rl = threadIdx.x / TPR, jt = threadIdx.x % TPR;
  float2 *srow = sm_rows + rl * C::PADL;
  auto smi = [](int i) { return i + i / EPT; };
  const long long total = (long long)np * N;
  const int W = kp.support;
  if (KGRAD) {
    for (int i = threadIdx.x; i < kp.table_len; i += blockDim.x) ptab[i] = 0.0f;
  }
  while (true) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, (unsigned long long)RPC);
    __syncthreads();
    const long long base = s_item;
    __syncthreads();
    if (base >= total) break;
    const long long item = base + rl;
    const bool valid = item < total;
    const int pl = valid ? (int)(item / N) : 0;
    const int q = valid ? (int)(item % N) : 0;
    const int64_t b0 = (int64_t)(p0 + pl) * N;
    const bool empty = !valid || off[(b0 + max(0, q - W + 1)) * kColBlocks] == off[(b0 + q + 1) * kColBlocks];
    if constexpr (RPC == 1) {
      if (empty) continue;  // nobody reads this row
    }
    const float2 *grow = planes + ((int64_t)pl * N + q) * N;
    float2 v[EPT];
#pragma unroll
    for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
      for (int r = 0; r < R0; ++r) v[b * R0 + r] = grow[in_index<N, EPT, TPR, 0>(jt, b, r)];
    const TableTw<N, EPT, TPR, -1> twp{twt, jt};
    stage_compute_f<N, EPT, TPR, 0, -1>(v, jt, twp);
    middle_stages_f<N, EPT, TPR, 1, -1>(v, jt, srow, smi, twp);
    stage_compute_f<N, EPT, TPR, NST - 1, -1>(v, jt, twp);
    __syncthreads();  // every padded read done before the natural-order writes
#pragma unroll
    for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int idx = out_index<N, EPT, TPR, NST - 1>(jt, b, r);
        float2 x = v[b * RL + r];
        if ((idx + q) & 1) x = make_float2(-x.x, -x.y);
        srow[idx] = x;
      }
    __syncthreads();
    if (valid && !empty) {
      for (int d = 0; d < W && q - d >= 0; ++d) {
        const uint32_t s0 = off[(b0 + q - d) * kColBlocks], s1 = off[(b0 + q - d + 1) * kColBlocks];
        const float ty = (float)d - kp.half;
        for (uint32_t s = s0 + jt; s < s1; s += TPR) {
          const RecHead rc = rec_head(rec, s);
          const float targ_y = ty + rec_gy(rc);
          const float gy = kernel_eval(kp, targ_y);
          const float gx0 = rec_gx(rc);
          const float2 *cell = srow + rec_i0(rc);
          if (!KGRAD) {
            float are = 0.0f, aim = 0.0f;
            for (int a = 0; a < W; ++a) {
              const float g = kernel_eval(kp, (float)a - kp.half + gx0);
              are = fmaf(g, cell[a].x, are);
              aim = fmaf(g, cell[a].y, aim);
            }
            const uint2 tail = __ldg(reinterpret_cast<const uint2 *>(rec + s) + 2);  // index, weight
            const float wt = __uint_as_float(tail.y) * gy;
            const uint32_t j = tail.x;
            atomicAdd(&dvis[j].x, wt * are);
            atomicAdd(&dvis[j].y, wt * aim);
          } else {
            // c_a = Re(conj(gh[q, i0 + a]) (w V)); x-profile tap a gets c_a G_y(d), the
            // y-profile tap d gets sum_a c_a G_x(a); each is split over the two table
            // samples bracketing the tap's argument
            float sum_cx = 0.0f;
            for (int a = 0; a < W; ++a) {
              const float targ = (float)a - kp.half + gx0;
              const float2 c = cell[a];
              const float cr = c.x * rc.vre + c.y * rc.vim;
              sum_cx = fmaf(cr, kernel_eval(kp, targ), sum_cx);
              const float pos = (targ + kp.half) * kp.table_scale;
              int i = (int)floorf(pos);
              i = max(0, min(i, kp.table_len - 2));
              const float f = pos - (float)i;
              atomicAdd(&ptab[i], cr * gy * (1.0f - f));
              atomicAdd(&ptab[i + 1], cr * gy * f);
            }
            const float pos = (targ_y + kp.half) * kp.table_scale;
            int i = (int)floorf(pos);
            i = max(0, min(i, kp.table_len - 2));
            const float f = pos - (float)i;
            atomicAdd(&ptab[i], sum_cx * (1.0f - f));
            atomicAdd(&ptab[i + 1], sum_cx * f);
          }
        }
      }
    }
    __syncthreads();
  }
  if (KGRAD) {
    __syncthreads();
    for (int i = threadIdx.x; i < kp.table_len; i += blockDim.x)
      if (ptab[i] != 0.0f) atomicAdd(&dtab[i], ptab[i]);
  }
}

// -------------------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------------------
static Tw tw_half(const wst_plan_s *p) {
  Tw t;
  t.t = p->tw;
  t.hmask = (p->n >> 1) - 1;
  t.hbit = p->n >> 1;
  return t;
}

template <class K>
static cudaError_t persistent_grid(wst_plan_s *p, K kern, int threads, size_t smem, int &grid) {
  // always raised to the request: the 48 KB default counts the kernel's static shared
  // memory too, so a dynamic request just under 48 KB can already exceed it
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) return e;
  grid = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

template <int N, bool FFT>
static cudaError_t launch_grid_rows(wst_plan_s *p, int p0, int np, float2 *out) {
  using C = RowCfg<N>;
  // the imaging path has the common supports unrolled
  auto kern = !FFT ? k_grid_rows<N, FFT, 0>
              : p->cfg.support == 7 ? k_grid_rows<N, FFT, 7>
              : p->cfg.support == 8 ? k_grid_rows<N, FFT, 8> : k_grid_rows<N, FFT, 0>;
  const size_t smem = sizeof(float2) * (C::RPC * C::PADL + (FFT ? line_table_size<N, C::EPT, C::TPR>() : 0)) +
                      3 * C::THREADS * sizeof(RecHead);
  int grid = 0;
  cudaError_t e = persistent_grid(p, kern, C::THREADS, smem, grid);
  if (e != cudaSuccess) return e;
  unsigned long long *counter = p->W_.counters + CNT_WORK;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return e;
  kern<<<grid, C::THREADS, smem, p->stream>>>(p->W_.records, p->W_.offsets, p0, np, kernel_params(p), out,
                                             p->W_.occ, counter, tw_half(p), p->W_.rowbound,
                                             FFT ? p->W_.counters + CNT_ROWS : nullptr);
  return cudaGetLastError();
}

template <int N, bool KGRAD>
static cudaError_t launch_rows_adjoint(wst_plan_s *p, int p0, int np, const float2 *planes, float2 *dvis,
                                       float *dtab) {
  using C = RowCfg<N>;
  auto kern = k_rows_adjoint<N, KGRAD>;
  const size_t smem = sizeof(float2) * (C::RPC * C::PADL + line_table_size<N, C::EPT, C::TPR>()) +
                      (KGRAD ? sizeof(float) * p->cfg.ktable_len : 0);
  int grid = 0;
  cudaError_t e = persistent_grid(p, kern, C::THREADS, smem, grid);
  if (e != cudaSuccess) return e;
  unsigned long long *counter = p->W_.counters + CNT_WORK;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return e;
  kern<<<grid, C::THREADS, smem, p->stream>>>(planes, p->W_.records, p->W_.offsets, p0, np, kernel_params(p),
                                             dvis, dtab, counter, tw_half(p));
  return cudaGetLastError();
}

#define WST_N_SWITCH(n, CALL)         \
  switch (n) {                        \
    case 64: return CALL(64);         \
    case 128: return CALL(128);       \
    case 256: return CALL(256);       \
    case 512: return CALL(512);       \
    case 1024: return CALL(1024);     \
    case 2048: return CALL(2048);     \
    case 4096: return CALL(4096);     \
    case 8192: return CALL(8192);     \
    case 16384: return CALL(16384);   \
  }                                   \
  return cudaErrorInvalidValue;

cudaError_t grid_rows(wst_plan_s *p, int p0, int p1, float2 *out, bool fft) {
  const int np = p1 - p0;
  if (np <= 0) return cudaSuccess;
  p->launches += 1;
  if (fft) {
#define CALL_F(n) launch_grid_rows<n, true>(p, p0, np, out)
    WST_N_SWITCH(p->n, CALL_F)
#undef CALL_F
  } else {
#define CALL_G(n) launch_grid_rows<n, false>(p, p0, np, out)
    WST_N_SWITCH(p->n, CALL_G)
#undef CALL_G
  }
}

cudaError_t rows_adjoint(wst_plan_s *p, int p0, int p1, const float2 *planes, float2 *dvis, float *dtab) {
  const int np = p1 - p0;
  if (np <= 0) return cudaSuccess;
  p->launches += 1;
  if (dtab) {
#define CALL_K(n) launch_rows_adjoint<n, true>(p, p0, np, planes, nullptr, dtab)
    WST_N_SWITCH(p->n, CALL_K)
#undef CALL_K
  } else {
#define CALL_D(n) launch_rows_adjoint<n, false>(p, p0, np, planes, dvis, nullptr)
    WST_N_SWITCH(p->n, CALL_D)
#undef CALL_D
  }
}

}  // namespace wst
