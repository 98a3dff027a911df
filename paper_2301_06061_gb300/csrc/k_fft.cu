// K-F: per-plane centred 2D FFT (section 2, Eq. 2: the inner (u,v) integral; the paper
// calls FFTW on the CPU for it, section 3.2), and K-P: the w-correction phase screen
// and the reduction of the w-planes into the image, fused into the last FFT pass.
//
// Layout of the transform of an N x N plane (N = A * B, A >= B):
//   pass R  : row FFTs of length N, one row (or several short rows) per CTA, whole row
//             in shared memory, Stockham radix-16 stages with register butterflies.
//   pass CA : four-step column stage A: for each a < A the length-B DFT over the rows
//             a + A*b, then the twiddle w_N^{a c}; in place.  16-column bands.
//   pass CB : four-step column stage B: for each c < B the length-A DFT over the
//             contiguous rows A*c + a, giving output rows c + B*d.  Forward direction:
//             the result never goes back to memory -- each CTA multiplies it by the
//             centring sign, the phase screen of every plane of the chunk and adds it
//             (Kahan-compensated) into the image tile it owns.
// The centring (-1)^(p+q) is applied by the gridder's store (or the row pass for the
// staged API) and (-1)^(a+b) in the CB epilogue.  The adjoint runs the conjugate
// transposes in reverse order: CB^H (image tile -> plane rows, conjugate screen,
// correction and sign fused), CA^H (twiddle first), row pass with the (-1)^(p+q) sign.
//
// Twiddles come from one table exp(+2 pi i m/N) rounded once from FP64; every
// sub-length L divides N, so w_L^m = tw[m N/L].
#include <cuda.h>  // CUtensorMap and the tensor-map encoder's types (the encoder is fetched at run time)

#include <mutex>

#include "fft_core.cuh"

namespace wst {

template <int N, int DIR, bool PRESIGN, bool POSTSIGN>
__global__ void __launch_bounds__(RowCfg<N>::THREADS)
k_rows(float2 *__restrict__ planes, Tw tw) {
  using C = RowCfg<N>;
  constexpr int EPT = C::EPT, TPR = C::TPR;
  constexpr int NST = num_stages(N, EPT);
  extern __shared__ float2 sm_rows[];
  const int rl = threadIdx.x / TPR, jt = threadIdx.x % TPR;
  const int q = blockIdx.x * C::RPC + rl;
  float2 *row = planes + ((size_t)blockIdx.y * N + q) * N;
  float2 *srow = sm_rows + rl * C::PADL;
  auto smi = [](int i) { return i + i / EPT; };
  float2 v[EPT];
  constexpr int R0 = stage_radix(N, EPT, 0);
#pragma unroll
  for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int idx = in_index<N, EPT, TPR, 0>(jt, b, r);
      float2 x = row[idx];
      if (PRESIGN && ((idx + q) & 1)) x = make_float2(-x.x, -x.y);
      v[b * R0 + r] = x;
    }
  stage_compute<N, EPT, TPR, 0, DIR>(v, jt, tw, 1);
  if constexpr (NST > 1) {
    middle_stages<N, EPT, TPR, 1, DIR>(v, jt, srow, smi, tw, 1);
    stage_compute<N, EPT, TPR, NST - 1, DIR>(v, jt, tw, 1);
  }
  constexpr int RL = stage_radix(N, EPT, NST - 1);
#pragma unroll
  for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int idx = out_index<N, EPT, TPR, NST - 1>(jt, b, r);
      float2 x = v[b * RL + r];
      if (POSTSIGN && ((idx + q) & 1)) x = make_float2(-x.x, -x.y);
      row[idx] = x;
    }
}

// ---------------------------------------------------------------------------------
// pass R for long rows (N >= kRowsTmaMin): a whole padded row fills most of an SM's
// shared memory, so one CTA per SM loops over rows.  As soon as the last stage has read
// its inputs out of shared memory, one thread starts TMA bulk copies of the CTA's next
// row into the freed buffer (mbarrier with transaction count), so the load of row r+1
// overlaps the last stage and the stores of row r.  Stage 0 reads the row in natural
// (unpadded) order; later stages use the padded layout.  Every wait is bounded: on
// timeout the CTA records WST_ERR_TIMEOUT in the device error word and returns.
// ---------------------------------------------------------------------------------
constexpr int kRowsTmaMin = 16384;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done != 0;
}

// Wait for the phase with a time limit; a zero limit expires at once without looking
// (the plan's failure-path test setting, wst_plan_set_wait_limit).  The clock is read
// only once the first look finds the phase incomplete (the limit counts from there).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase, unsigned long long limit_ns) {
  if (limit_ns == 0) return false;
  if (mbar_try_wait(mbar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(mbar, phase)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

template <int BYTES>
__device__ __forceinline__ void tma_load_row(uint32_t dst_smem, const float2 *src, uint32_t mbar) {
  constexpr int kPiece = 32768;
  constexpr int kPieces = BYTES / kPiece;
  static_assert(BYTES % kPiece == 0, "row size");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(BYTES) : "memory");
#pragma unroll
  for (int i = 0; i < kPieces; ++i) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_smem + i * kPiece),
        "l"(reinterpret_cast<const char *>(src) + (size_t)i * kPiece), "r"(kPiece), "r"(mbar)
        : "memory");
  }
}

template <int N, int DIR, bool PRESIGN, bool POSTSIGN>
__global__ void __launch_bounds__(RowCfg<N>::THREADS, 1)
k_rows_tma(float2 *__restrict__ planes, int64_t total_rows, Tw tw, unsigned long long *err,
           unsigned long long wait_ns) {
  using C = RowCfg<N>;
  static_assert(C::RPC == 1, "one row per CTA");
  constexpr int EPT = C::EPT, TPR = C::TPR;
  constexpr int NST = num_stages(N, EPT);
  constexpr int R0 = stage_radix(N, EPT, 0);
  constexpr int RL = stage_radix(N, EPT, NST - 1);
  extern __shared__ __align__(128) float2 sm_rows[];
  __shared__ __align__(8) unsigned long long mbar_storage;
  const int jt = threadIdx.x;
  auto smi = [](int i) { return i + i / EPT; };
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm_rows);
  const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&mbar_storage);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  int64_t row = blockIdx.x;
  uint32_t phase = 0;
  if (threadIdx.x == 0 && row < total_rows) tma_load_row<N * 8>(sbase, planes + row * N, mbar);
  for (; row < total_rows; row += gridDim.x) {
    // one warp polls the barrier; the others wait at the CTA barrier without issuing
    bool ok = true;
    if (threadIdx.x < 32) ok = mbar_wait_bounded(mbar, phase, wait_ns);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, (unsigned long long)WST_ERR_TIMEOUT);
        // let the copy in flight into our buffer land before the CTA exits: bounded, with
        // the full limit whatever the plan's setting
        mbar_wait_bounded(mbar, phase, kWaitLimitNs);
      }
      __syncthreads();
      return;
    }
    phase ^= 1u;
    const int q = (int)(row % N);
    float2 *grow = planes + row * N;
    float2 v[EPT];
#pragma unroll
    for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int idx = in_index<N, EPT, TPR, 0>(jt, b, r);
        float2 x = sm_rows[idx];  // natural order, as copied
        if (PRESIGN && ((idx + q) & 1)) x = make_float2(-x.x, -x.y);
        v[b * R0 + r] = x;
      }
    __syncthreads();  // natural-order reads done before the padded writes
    stage_compute<N, EPT, TPR, 0, DIR>(v, jt, tw, 1);
    middle_stages<N, EPT, TPR, 1, DIR>(v, jt, sm_rows, smi, tw, 1);
    __syncthreads();  // every read of this row is done: the buffer is free
    if (threadIdx.x == 0 && row + gridDim.x < total_rows) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tma_load_row<N * 8>(sbase, planes + (row + gridDim.x) * N, mbar);
    }
    stage_compute<N, EPT, TPR, NST - 1, DIR>(v, jt, tw, 1);
#pragma unroll
    for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int idx = out_index<N, EPT, TPR, NST - 1>(jt, b, r);
        float2 x = v[b * RL + r];
        if (POSTSIGN && ((idx + q) & 1)) x = make_float2(-x.x, -x.y);
        grow[idx] = x;
      }
  }
}

// ---------------------------------------------------------------------------------
// pass CA: four-step column stage A, length-LB lines over rows a + A*i, 16-col bands
// ---------------------------------------------------------------------------------
constexpr int kCB = 16;  // columns per band (128 bytes per row segment)

template <int L, int CB = kCB>
struct ColCfg {
  static constexpr int EPT = L >= 8 ? 8 : L;
  static constexpr int TPL = L / EPT;
  static constexpr int THREADS = TPL * CB;
  static constexpr int PADW = CB + 1;  // smem row stride (float2)
};

template <int LB, int DIR, bool TW_FIRST>
__global__ void __launch_bounds__(ColCfg<LB>::THREADS)
k_cols_a(float2 *__restrict__ planes, Tw tw, int n, const uint8_t *__restrict__ occ) {
  using C = ColCfg<LB>;
  constexpr int EPT = C::EPT, TPL = C::TPL;
  constexpr int NST = num_stages(LB, EPT);
  __shared__ float2 sm[LB * C::PADW];
  const int A = n / LB;
  const int col = threadIdx.x % kCB, jt = threadIdx.x / kCB;
  const int a = blockIdx.y;
  const int kp = blockIdx.x * kCB + col;
  float2 *base = planes + (size_t)blockIdx.z * n * n + kp;
  const size_t rstride = (size_t)A * n;  // line element i -> row a + A*i
  base += (size_t)a * n;
  auto smi = [col](int i) { return i * C::PADW + col; };
  float2 v[EPT];
  constexpr int R0 = stage_radix(LB, EPT, 0);
#pragma unroll
  for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int i = in_index<LB, EPT, TPL, 0>(jt, b, r);
      // rows the gridder left empty are zero: do not read them
      float2 x = (occ && !occ[(size_t)blockIdx.z * n + a + A * i]) ? make_float2(0.0f, 0.0f)
                                                                     : base[(size_t)i * rstride];
      if (TW_FIRST) x = cmul(x, twiddle(tw, a * i, DIR));
      v[b * R0 + r] = x;
    }
  stage_compute<LB, EPT, TPL, 0, DIR>(v, jt, tw, A);
  if constexpr (NST > 1) {
    middle_stages<LB, EPT, TPL, 1, DIR>(v, jt, sm, smi, tw, A);
    stage_compute<LB, EPT, TPL, NST - 1, DIR>(v, jt, tw, A);
  }
  constexpr int RL = stage_radix(LB, EPT, NST - 1);
#pragma unroll
  for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int c = out_index<LB, EPT, TPL, NST - 1>(jt, b, r);
      float2 x = v[b * RL + r];
      if (!TW_FIRST) x = cmul(x, twiddle(tw, a * c, DIR));
      base[(size_t)c * rstride] = x;
    }
}

// 16-byte asynchronous global -> shared copies (sm_80+ LDGSTS), grouped per plane
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Pass CA, persistent: each CTA walks tiles (plane, a, 32-column band: 256-byte row
// segments) in band-fastest order; tiles are copied into a ring of three shared slots
// with cp.async, two tiles ahead (rows the gridder left empty are zero-filled instead of
// read, their flags loaded ahead).  16 elements per thread (LB = 32, 64, 128: radix 16,
// then LB/16 with the stage twiddles in registers); the exchange between the two
// register stages is made in place in the tile's slot (three barriers per tile), which
// keeps two CTAs per SM with the deeper ring.  A warp covers 32 columns at one line
// position: shared-memory accesses are conflict-free without padding and twiddles are
// warp-uniform.  The factors w_N^{a c} of a tile come from a shared table filled with the
// tile (three in rotation), each factor evaluated by sincospi.
template <int LB, int DIR, bool TW_FIRST>
__global__ void __launch_bounds__(LB / 16 * 32, 512 / (LB / 16 * 32))
k_cols_a16(float2 *__restrict__ planes, Tw tw, int n, const uint8_t *__restrict__ occ, int nplanes) {
  constexpr int CB = 32, EPT = 16, TPL = LB / EPT, THREADS = TPL * CB;
  constexpr int R1 = LB / 16;  // radix of the second stage
  static_assert(num_stages(LB, EPT) == 2 && stage_radix(LB, EPT, 1) == R1, "two stages");
  constexpr int PIECES = LB * (CB / 2);     // 16-byte pieces per tile
  constexpr int PPT = PIECES / THREADS;     // pieces per thread (8)
  static_assert(PIECES % THREADS == 0, "pieces");
  __shared__ __align__(16) float2 stage[3][LB * CB];
  __shared__ float2 s_tw[3][LB];    // w_N^{DIR a c}, c < LB, of the tiles in flight
  const int A = n / LB;
  const int lg_bands = 31 - __clz(n / CB), lg_A = 31 - __clz(A);
  const int total = nplanes << (lg_bands + lg_A);
  const int col = threadIdx.x % CB, jt = threadIdx.x / CB;
  float2 twr[total_tw_count<LB, EPT>()];
  all_twiddles<LB, EPT, TPL, DIR>(twr, jt, tw, A);
  const size_t rstride = (size_t)A * n;  // line element i -> row a + A*i
  // the occupancy bytes of a tile's rows, loaded a tile ahead and kept raw until issue()
  // tests them: turning them into booleans at once made every warp wait for the loads
  auto load_flags = [&](int t, uint32_t (&f)[PPT]) {
    const int a = (t >> lg_bands) & (A - 1), z = t >> (lg_bands + lg_A);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int i = (threadIdx.x + k * THREADS) / (CB / 2);
      f[k] = (t >= total || !occ) ? 1u : (uint32_t)occ[(size_t)z * n + a + A * i];
    }
  };
  auto issue = [&](int t, float2 *buf, const uint32_t (&f)[PPT]) {
    const int band = t & ((1 << lg_bands) - 1);
    const int a = (t >> lg_bands) & (A - 1), z = t >> (lg_bands + lg_A);
    const float2 *src = planes + (size_t)z * n * n + (size_t)a * n + band * CB;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int c = threadIdx.x + k * THREADS;
      const int i = c / (CB / 2), part = c % (CB / 2);
      if (f[k])
        cp_async16(sbuf + (uint32_t)(i * CB + 2 * part) * 8u, src + i * rstride + 2 * part);
      else
        reinterpret_cast<float4 *>(buf)[(i * CB + 2 * part) / 2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  };
  // evaluated, not loaded: a table load here stalled the filling warps for an L2 round
  // trip on every tile, and the CTA's other warps then waited for them at the next barrier
  const float two_over_n = 2.0f / (float)n;
  auto fill_tw = [&](int t, float2 *dst) {
    const int a = (t >> lg_bands) & (A - 1);
    if (threadIdx.x < LB) dst[threadIdx.x] = twiddle_direct((a * (int)threadIdx.x) & (n - 1), two_over_n, DIR);
  };
  int t = blockIdx.x;
  uint32_t f0[PPT], f1[PPT];
  const int G = gridDim.x;
  // tiles it and it + 1 in flight before the loop; tile it + 2 is issued after the first
  // barrier of tile it, into the slot of tile it - 1
  load_flags(t, f0);
  if (t < total) { issue(t, stage[0], f0); fill_tw(t, s_tw[0]); }
  cp_async_commit();
  load_flags(t + G, f0);
  if (t + G < total) { issue(t + G, stage[1], f0); fill_tw(t + G, s_tw[1]); }
  cp_async_commit();
  load_flags(t + 2 * G, f1);
  for (int it = 0; t < total; ++it, t += G) {
    const int band = t & ((1 << lg_bands) - 1);
    const int a = (t >> lg_bands) & (A - 1), z = t >> (lg_bands + lg_A);
    const float2 *tws = s_tw[it % 3];
    cp_async_wait<1>();
    __syncthreads();  // tile it landed; every thread is done with tile it - 1
    if (t + 2 * G < total) {
      issue(t + 2 * G, stage[(it + 2) % 3], f1);
      fill_tw(t + 2 * G, s_tw[(it + 2) % 3]);
    }
    cp_async_commit();
    load_flags(t + 3 * G, f1);
    float2 *buf = stage[it % 3];
    float2 v[EPT];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = jt + r * TPL;
      float2 x = buf[i * CB + col];
      if (TW_FIRST) x = cmul(x, tws[i]);
      v[r] = x;
    }
    dft<16, DIR>(v);
    __syncthreads();  // every stage-0 read of the slot done before the exchange in place
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[(16 * jt + r) * CB + col] = v[r];
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 16 / R1; ++b)
#pragma unroll
      for (int r = 0; r < R1; ++r) v[b * R1 + r] = buf[(jt + b * TPL + 16 * r) * CB + col];
    stage_compute_pre<LB, EPT, 1, DIR>(v, twr);
    float2 *dst = planes + (size_t)z * n * n + (size_t)a * n + band * CB + col;
#pragma unroll
    for (int b = 0; b < 16 / R1; ++b)
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int c = jt + b * TPL + 16 * r;
        float2 x = v[b * R1 + r];
        if (!TW_FIRST) x = cmul(x, tws[c]);
        __stcs(&dst[(size_t)c * rstride], x);
      }
  }
  cp_async_wait<0>();
}

// mbarrier and TMA helpers of the TMA-fed kernels
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void tma_load_tile3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                                uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

// ---------------------------------------------------------------------------------
// phase screen helpers (K-P)
//
// The screen of plane k at pixel (a, b) is e^{2 pi i w_k t}, t = n - 1, with w_k = w_0 +
// k dw inside an image.  It is evaluated exactly (float-float argument, reduced modulo
// one cycle) at an anchor plane, and advanced to the next plane by one complex multiply
// with the pixel's step e^{2 pi i dw t}, itself evaluated exactly at the anchor.  Anchors
// are the first plane of an image in a chunk and every kAnchor-th plane after it, so
// the rounding of the recurrence never compounds over more than kAnchor - 1 products.
// ---------------------------------------------------------------------------------
constexpr int kAnchor = 16;

struct ScreenCtx {
  const float2 *l2ff;      // l_a^2 float-float
  const double *l2d;       // l_a^2 FP64
  const float2 *wc;        // plane centres float-float (global plane index)
  const double *wcd;       // plane centres FP64
  const float2 *dwff;      // plane spacing per image, float-float
  const double *wrange;    // per image: w_lo, scale, dw, w_hi
  const float *corr;       // 1/Ghat
};

// exact screen of plane P at pixel (kp, kq) times `scale`, and (STEP) the per-plane step
template <bool FP64S, bool STEP = true>
__device__ __forceinline__ void screen_anchor(const ScreenCtx &sc, int kp, int kq, int P, int img, float scale,
                                              float2 &scr, float2 &stp) {
  scr = make_float2(0.0f, 0.0f);
  if (STEP) stp = make_float2(0.0f, 0.0f);
  if constexpr (FP64S) {
    const double r2 = sc.l2d[kp] + sc.l2d[kq];
    if (!(r2 < 1.0)) return;
    const double t = -r2 / (1.0 + sqrt(1.0 - r2));
    scr = cis_cycles_d(sc.wcd[P] * t);
    if (STEP) stp = cis_cycles_d(sc.wrange[4 * img + 2] * t);
  } else {
    bool valid;
    const ff t = n_minus_one_ff(sc.l2ff[kp], sc.l2ff[kq], valid);
    if (!valid) return;
    const float2 w = sc.wc[P];
    scr = cis_cycles_ff(ff_mul({w.x, w.y}, t));
    if (STEP) {
      const float2 dw = sc.dwff[img];
      stp = cis_cycles_ff(ff_mul({dw.x, dw.y}, t));
    }
  }
  scr.x *= scale;
  scr.y *= scale;
}

__device__ __forceinline__ void kahan_add(float2 &s, float2 &c, float2 y) {
  const float yx = __fsub_rn(y.x, c.x), yy = __fsub_rn(y.y, c.y);
  const float tx = __fadd_rn(s.x, yx), ty = __fadd_rn(s.y, yy);
  c.x = __fsub_rn(__fsub_rn(tx, s.x), yx);
  c.y = __fsub_rn(__fsub_rn(ty, s.y), yy);
  s.x = tx;
  s.y = ty;
}

// float-float screen of the plane at w from a cached t = n - 1 (t.x is NaN outside the
// unit sphere), and (STEP) the step for the plane spacing dw
template <bool STEP>
__device__ __forceinline__ void screen_from_t(float2 t2, float2 w, float2 dw, float scale, float2 &scr,
                                              float2 &stp) {
  scr = make_float2(0.0f, 0.0f);
  if (STEP) stp = make_float2(0.0f, 0.0f);
  if (isnan(t2.x)) return;
  const ff t = {t2.x, t2.y};
  scr = cis_cycles_ff(ff_mul({w.x, w.y}, t));
  if (STEP) stp = cis_cycles_ff(ff_mul({dw.x, dw.y}, t));
  scr.x *= scale;
  scr.y *= scale;
}

// epilogue modes.  ACC_RANGE_START / ACC_RANGE_END: the call's first (last) plane starts
// (ends) the requested plane range, so every image the chunk touches starts (finishes)
// its sum here even if its first (last) plane lies outside the range.
enum { ACC_CORRECT = 4, ACC_KAHAN = 8, ACC_STAGED = 16, ACC_RANGE_START = 32, ACC_RANGE_END = 64 };

// ---------------------------------------------------------------------------------
// pass CB (forward) + K-P: length-LA DFT over rows A*c + a, then the centring sign and
// the screen, and the (Kahan-compensated) sum over the chunk's planes of each image.
// ---------------------------------------------------------------------------------
// The tile of plane P (rows A c .. A c + A - 1, 16 columns) is copied into one of two
// shared staging buffers while the previous plane is transformed, so the strided loads
// of the tile never stall the FFT.
template <int LA>
__device__ __forceinline__ void stage_tile_async(float2 *buf, const float2 *plane, int n, int row0, int col0) {
  constexpr int CHUNKS = LA * (kCB * 8 / 16);  // 16-byte pieces per tile
  const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
  for (int i = threadIdx.x; i < CHUNKS; i += ColCfg<LA>::THREADS) {
    const int row = i / (kCB / 2), part = i % (kCB / 2);
    cp_async16(sbuf + (uint32_t)(row * kCB + 2 * part) * 8u, plane + (size_t)(row0 + row) * n + col0 + 2 * part);
  }
}

// Tile copy for THREADS threads (16-byte pieces, LA rows of kCB columns).
template <int LA, int THREADS>
__device__ __forceinline__ void stage_tile_async16(float2 *buf, const float2 *plane, int n, int row0, int col0) {
  constexpr int CHUNKS = LA * (kCB / 2);
  static_assert(CHUNKS % THREADS == 0, "pieces");
  const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll
  for (int k = 0; k < CHUNKS / THREADS; ++k) {
    const int i = threadIdx.x + k * THREADS;
    const int row = i / (kCB / 2), part = i % (kCB / 2);
    cp_async16(sbuf + (uint32_t)(row * kCB + 2 * part) * 8u, plane + (size_t)(row0 + row) * n + col0 + 2 * part);
  }
}

// Write one pixel's plane sum (s, compensation cmp) of a chunk: merged with the running
// (sum, compensation) of earlier chunks unless the image's first plane is in this chunk,
// and finished (compensation folded in, grid correction f applied) if its last plane is.
__device__ __forceinline__ void flush_pixel(float2 *im, float2 *cp, size_t o, float2 sum, float2 cmp,
                                            bool first_any, bool last_any, int flags, float f) {
  if (flags & ACC_STAGED) {
    im[o] = cadd(im[o], csub(sum, cmp));
    return;
  }
  if (!first_any) {
    float2 acc_s = im[o];
    float2 acc_c = cp ? cp[o] : make_float2(0.0f, 0.0f);
    kahan_add(acc_s, acc_c, sum);
    kahan_add(acc_s, acc_c, make_float2(-cmp.x, -cmp.y));
    sum = acc_s;
    cmp = acc_c;
  }
  if (last_any) {
    float2 out = csub(sum, cmp);
    if (flags & ACC_CORRECT) out = make_float2(out.x * f, out.y * f);
    im[o] = out;
  } else {
    im[o] = sum;
    if (cp) cp[o] = cmp;
  }
}

template <int LA, bool FP64S, bool CROP>
__global__ void __launch_bounds__(ColCfg<LA>::THREADS, ColCfg<LA>::THREADS >= 32 ? 512 / ColCfg<LA>::THREADS : 1)
k_cols_b_acc(const float2 *__restrict__ planes, int p0, int p1, int n_w, Tw tw,
             int n, ScreenCtx sc, float2 *__restrict__ image, float2 *__restrict__ comp, int flags,
             int n_img_arg, int crop_arg) {
  // an image smaller than the grid (CROP) is its central n_img x n_img from grid index
  // crop; otherwise both are compile-time facts, which keeps the registers of the
  // plain kernel free for the transform
  const int n_img = CROP ? n_img_arg : n, crop = CROP ? crop_arg : 0;
  using C = ColCfg<LA>;
  constexpr int EPT = C::EPT, TPL = C::TPL;
  constexpr int NST = num_stages(LA, EPT);
  constexpr int RL = stage_radix(LA, EPT, NST - 1);
  constexpr int R0 = stage_radix(LA, EPT, 0);
  __shared__ float2 sm[LA * C::PADW];
  __shared__ __align__(16) float2 stage_buf[2][LA * kCB];
  __shared__ float2 s_step[EPT][C::THREADS];  // per-plane screen step of each output (thread-private)
  __shared__ float2 s_nm1[FP64S ? 1 : EPT][C::THREADS];  // n - 1 of each output, float-float
  const int B = n / LA;
  const int col = threadIdx.x % kCB, jt = threadIdx.x / kCB;
  const int c = blockIdx.y;
  // only the bands that hold image columns (from the band of column crop: the image's
  // side need not be a multiple of the band, nor crop of its width)
  const int col0 = (crop / kCB + (int)blockIdx.x) * kCB;
  const int kp = col0 + col;
  auto smi = [col](int i) { return i * C::PADW + col; };
  const bool kahan = flags & ACC_KAHAN;
  const size_t plane_elems = (size_t)n * n;
  // the same length-LA transform runs once per plane: its twiddles stay in registers
  float2 twr[total_tw_count<LA, EPT>() > 0 ? total_tw_count<LA, EPT>() : 1];
  all_twiddles<LA, EPT, TPL, 1>(twr, jt, tw, B);
  stage_tile_async<LA>(stage_buf[0], planes, n, LA * c, col0);
  cp_async_commit();
  int P = p0;
  while (P < p1) {
    const int img = P / n_w;
    const int pstart = P;
    const int pend = min(p1, (img + 1) * n_w);
    float2 s[EPT], cc[EPT], scr[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) s[e] = cc[e] = make_float2(0.0f, 0.0f);
    for (; P < pend; ++P) {
      // prefetch the next plane's tile, then wait for this plane's
      if (P + 1 < p1) stage_tile_async<LA>(stage_buf[(P + 1 - p0) & 1], planes + (size_t)(P + 1 - p0) * plane_elems, n,
                                           LA * c, col0);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      if ((P - pstart) % kAnchor == 0) {
        // the step e^{2 pi i dw t} is one number per pixel and image: evaluated once
#pragma unroll
        for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const int kq = c + B * out_index<LA, EPT, TPL, NST - 1>(jt, b, r);
            const float sg = ((kq + kp) & 1) ? -1.0f : 1.0f;
            float2 &st = s_step[b * RL + r][threadIdx.x];
            if constexpr (FP64S) {
              if (P == pstart) screen_anchor<true, true>(sc, kp, kq, P, img, sg, scr[b * RL + r], st);
              else screen_anchor<true, false>(sc, kp, kq, P, img, sg, scr[b * RL + r], st);
            } else {
              // n - 1 depends on the pixel only: evaluated at the image's first plane
              float2 &t2 = s_nm1[b * RL + r][threadIdx.x];
              if (P == pstart) {
                bool valid;
                const ff t = n_minus_one_ff(sc.l2ff[kp], sc.l2ff[kq], valid);
                t2 = valid ? make_float2(t.hi, t.lo) : make_float2(__int_as_float(0x7fc00000), 0.0f);
                screen_from_t<true>(t2, sc.wc[P], sc.dwff[img], sg, scr[b * RL + r], st);
              } else {
                screen_from_t<false>(t2, sc.wc[P], sc.dwff[img], sg, scr[b * RL + r], st);
              }
            }
          }
      }
      const float2 *tile = stage_buf[(P - p0) & 1];
      float2 v[EPT];
#pragma unroll
      for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) v[b * R0 + r] = tile[in_index<LA, EPT, TPL, 0>(jt, b, r) * kCB + col];
      stage_compute_pre<LA, EPT, 0, 1>(v, twr);
      if constexpr (NST > 1) {
        middle_stages_pre<LA, EPT, TPL, 1, 1>(v, jt, sm, smi, twr);
        stage_compute_pre<LA, EPT, NST - 1, 1>(v, twr);
      }
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float2 y = cmul(v[e], scr[e]);
        if (kahan) kahan_add(s[e], cc[e], y);
        else s[e] = cadd(s[e], y);
        scr[e] = cmul(scr[e], s_step[e][threadIdx.x]);
      }
      __syncthreads();  // staging buffer and shared memory reused by the next planes
    }
    // flush this image's tile: its sum starts in this chunk if its first plane is at
    // or after p0, and is complete if its last plane is before p1
    const bool first_any = img * n_w >= p0 || (flags & ACC_RANGE_START);
    const bool last_any = (img + 1) * n_w <= p1 || (flags & ACC_RANGE_END);
    float2 *im = image + (size_t)img * n_img * n_img;
    float2 *cp = comp ? comp + (size_t)img * n_img * n_img : nullptr;
#pragma unroll
    for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int e = b * RL + r;
        const int kq = c + B * out_index<LA, EPT, TPL, NST - 1>(jt, b, r);
        if (CROP && (kq < crop || kq >= crop + n_img || kp < crop || kp >= crop + n_img))
          continue;  // a grid row or column outside the image
        const float f = (flags & ACC_CORRECT) ? sc.corr[kp] * sc.corr[kq] : 1.0f;
        flush_pixel(im, cp, (size_t)(kq - crop) * n_img + (kp - crop), s[e], cc[e], first_any, last_any, flags, f);
      }
  }
}

// Pass CB + K-P with 16 elements per thread for LA = 64, 128 (radix 16, then LA/16):
// one exchange per plane, made in place in the plane's staging buffer (each half-warp
// covers the 16 columns at one line position), so a plane costs four barriers for 16
// outputs per thread.  Screen, Kahan sum and flush as in k_cols_b_acc.
template <int LA, bool FP64S, bool CROP>
__global__ void __launch_bounds__(LA / 16 * kCB, LA == 128 ? 3 : 6)
k_cols_b16(const float2 *__restrict__ planes, int p0, int p1, int n_w, Tw tw,
           int n, ScreenCtx sc, float2 *__restrict__ image, float2 *__restrict__ comp, int flags,
           int n_img_arg, int crop_arg) {
  const int n_img = CROP ? n_img_arg : n, crop = CROP ? crop_arg : 0;  // as in k_cols_b_acc
  constexpr int EPT = 16, TPL = LA / EPT, THREADS = TPL * kCB, R1 = LA / 16;
  static_assert(num_stages(LA, EPT) == 2 && stage_radix(LA, EPT, 1) == R1, "two stages");
  __shared__ __align__(16) float2 stage_buf[2][LA * kCB];
  static_assert(EPT * THREADS <= LA * kCB, "anchor screens fit a staging buffer");
  __shared__ float2 s_step[EPT][THREADS];                  // per-plane screen step of each output
  __shared__ float2 s_nm1[FP64S ? 1 : EPT][THREADS];       // n - 1 of each output, float-float
  const int B = n / LA;
  const int col = threadIdx.x % kCB, jt = threadIdx.x / kCB;
  const int c = blockIdx.y;
  // only the bands that hold image columns (from the band of column crop: the image's
  // side need not be a multiple of the band, nor crop of its width)
  const int col0 = (crop / kCB + (int)blockIdx.x) * kCB;
  const int kp = col0 + col;
  const bool kahan = flags & ACC_KAHAN;
  const size_t plane_elems = (size_t)n * n;
  // stage-1 twiddles (one list per line position jt, read as half-warp broadcasts)
  constexpr int NTW = total_tw_count<LA, EPT>();
  __shared__ float2 s_tw1[NTW][TPL];
  if (threadIdx.x < TPL) {
    float2 twr[NTW];
    all_twiddles<LA, EPT, TPL, 1>(twr, threadIdx.x, tw, B);
#pragma unroll
    for (int i = 0; i < NTW; ++i) s_tw1[i][threadIdx.x] = twr[i];
  }
  // output e = b R1 + r of this thread is line element jt + b TPL + 16 r, image row c + B (that)
  auto out_row = [&](int b, int r) { return c + B * (jt + b * TPL + 16 * r); };
  stage_tile_async16<LA, THREADS>(stage_buf[0], planes, n, LA * c, col0);
  cp_async_commit();
  int P = p0;
  while (P < p1) {
    const int img = P / n_w;
    const int pstart = P;
    const int pend = min(p1, (img + 1) * n_w);
    float2 s[EPT], cc[EPT], scr[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) s[e] = cc[e] = make_float2(0.0f, 0.0f);
    for (; P < pend; ++P) {
      if ((P - pstart) % kAnchor == 0) {
        // anchors: a rolled loop keeps the float-float screen evaluation of one output
        // live at a time; the results pass through the free staging buffer (the one the
        // next plane's tile goes to), before that copy is issued
        float2 *s_anchor = stage_buf[(P + 1 - p0) & 1];
        const float2 wP = FP64S ? make_float2(0.0f, 0.0f) : sc.wc[P];
        const float2 dwI = FP64S ? make_float2(0.0f, 0.0f) : sc.dwff[img];
#pragma unroll 1
        for (int e = 0; e < EPT; ++e) {
          const int kq = out_row(e / R1, e % R1);
          const float sg = ((kq + kp) & 1) ? -1.0f : 1.0f;
          float2 &st = s_step[e][threadIdx.x];
          float2 a;
          if constexpr (FP64S) {
            if (P == pstart) screen_anchor<true, true>(sc, kp, kq, P, img, sg, a, st);
            else screen_anchor<true, false>(sc, kp, kq, P, img, sg, a, st);
          } else {
            float2 &t2 = s_nm1[e][threadIdx.x];
            if (P == pstart) {
              bool valid;
              const ff t = n_minus_one_ff(sc.l2ff[kp], sc.l2ff[kq], valid);
              t2 = valid ? make_float2(t.hi, t.lo) : make_float2(__int_as_float(0x7fc00000), 0.0f);
              screen_from_t<true>(t2, wP, dwI, sg, a, st);
            } else {
              screen_from_t<false>(t2, wP, dwI, sg, a, st);
            }
          }
          s_anchor[e * THREADS + threadIdx.x] = a;
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e) scr[e] = s_anchor[e * THREADS + threadIdx.x];
        __syncthreads();  // every read of the staging buffer done before the copy into it
      }
      if (P + 1 < p1)
        stage_tile_async16<LA, THREADS>(stage_buf[(P + 1 - p0) & 1], planes + (size_t)(P + 1 - p0) * plane_elems, n,
                                        LA * c, col0);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      float2 *tile = stage_buf[(P - p0) & 1];
      float2 v[EPT];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = tile[(jt + r * TPL) * kCB + col];
      dft<16, 1>(v);
      __syncthreads();  // every stage-0 load of the tile done before the in-place exchange
#pragma unroll
      for (int r = 0; r < 16; ++r) tile[(16 * jt + r) * kCB + col] = v[r];
      __syncthreads();
#pragma unroll
      for (int b = 0; b < EPT / R1; ++b)
#pragma unroll
        for (int r = 0; r < R1; ++r) v[b * R1 + r] = tile[(jt + b * TPL + 16 * r) * kCB + col];
#pragma unroll
      for (int b = 0; b < EPT / R1; ++b) {
#pragma unroll
        for (int r = 1; r < R1; ++r) v[b * R1 + r] = cmul(v[b * R1 + r], s_tw1[b * (R1 - 1) + r - 1][jt]);
        dft<R1, 1>(&v[b * R1]);
      }
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float2 y = cmul(v[e], scr[e]);
        if (kahan) kahan_add(s[e], cc[e], y);
        else s[e] = cadd(s[e], y);
        scr[e] = cmul(scr[e], s_step[e][threadIdx.x]);
      }
      __syncthreads();  // staging buffer reused by the next planes
    }
    const bool first_any = img * n_w >= p0 || (flags & ACC_RANGE_START);
    const bool last_any = (img + 1) * n_w <= p1 || (flags & ACC_RANGE_END);
    float2 *im = image + (size_t)img * n_img * n_img;
    float2 *cp = comp ? comp + (size_t)img * n_img * n_img : nullptr;
#pragma unroll
    for (int b = 0; b < EPT / R1; ++b)
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int e = b * R1 + r;
        const int kq = out_row(b, r);
        if (CROP && (kq < crop || kq >= crop + n_img || kp < crop || kp >= crop + n_img))
          continue;  // a grid row or column outside the image
        const float f = (flags & ACC_CORRECT) ? sc.corr[kp] * sc.corr[kq] : 1.0f;
        flush_pixel(im, cp, (size_t)(kq - crop) * n_img + (kp - crop), s[e], cc[e], first_any, last_any, flags, f);
      }
  }
}

// ---------------------------------------------------------------------------------
// Pass CB + K-P with TMA tile loads and a blocked Horner plane sum (LA = 64, 128).
//
// Tiles (LA rows x 16 columns of a plane, 128-byte row segments) are copied by the
// tensor engine: one thread issues cp.async.bulk.tensor for a plane's tile into a ring of
// three shared slots, each with an mbarrier that counts the copy's bytes; the ring runs
// two planes ahead.  Every wait on a slot is bounded (wait_ns; on expiry the CTA records
// WST_ERR_TIMEOUT, lets its copies in flight land and returns).  The transform is that of
// k_cols_b16 (radix 16, in-place exchange in the slot, then LA/16), with two CTA barriers
// per plane: one after the stage-0 reads (the slot of the previous plane is then free
// and is refilled), one after the exchange.
//
// Plane sum (Eq. 2).  Within an image the screen of plane P at a pixel is
// screen_P = screen_L s^(P - L) for any plane L, s = e^{2 pi i dw (n-1)} the pixel's step.
// The planes are taken in anchor blocks of up to kAnchor; over a block with last plane L
//   sum_P v_P screen_P = screen_L sum_P v_P conj(s)^(L - P),
// evaluated by Horner's rule as the planes arrive, acc <- acc conj(s) + v_P (one complex
// multiply-add per output and plane; |s| = 1).  At the block's last plane acc is
// multiplied by the exact screen of that plane (float-float argument) and added, Kahan-
// compensated, to the image's running sum; the next block starts from zero.  The
// rounding of a block therefore stays within one block (as the recurrence of k_cols_b16
// stays within kAnchor - 1 steps), and the blocks are summed with compensation.
// ---------------------------------------------------------------------------------
constexpr int kColsBRing = 3;

template <int LA, bool FP64S, bool CROP>
__global__ void __launch_bounds__(LA / 16 * kCB, LA == 128 ? 3 : 6)
k_cols_b_tma(const __grid_constant__ CUtensorMap tmap, int p0, int p1, int n_w, Tw tw, int n, ScreenCtx sc,
             float2 *__restrict__ image, float2 *__restrict__ comp, int flags, int n_img_arg, int crop_arg,
             unsigned long long *__restrict__ err, unsigned long long wait_ns, int first_lo, int last_hi) {
  // an image starts its sum in this call if its first plane is at or after first_lo (p0,
  // or below every plane when the call starts the requested range) and finishes it if its
  // last plane is before last_hi (p1, or above every plane when the call ends the range)
  const int n_img = CROP ? n_img_arg : n, crop = CROP ? crop_arg : 0;  // as in k_cols_b_acc
  constexpr int EPT = 16, TPL = LA / EPT, THREADS = TPL * kCB, R1 = LA / 16;
  static_assert(num_stages(LA, EPT) == 2 && stage_radix(LA, EPT, 1) == R1, "two stages");
  constexpr uint32_t kTileBytes = LA * kCB * sizeof(float2);
  static_assert(EPT * THREADS <= LA * kCB, "anchor screens fit a slot");
  __shared__ __align__(128) float2 ring[kColsBRing][LA * kCB];
  __shared__ float2 s_cstep[EPT][THREADS];  // conj of each output's per-plane screen step
  constexpr int NTW = total_tw_count<LA, EPT>();
  __shared__ float2 s_tw1[NTW][TPL];
  __shared__ __align__(8) unsigned long long s_mbar[kColsBRing];
  // l^2 (float-float) and the grid correction 1/Ghat of the tile's LA grid rows c + B m
  // and of its kCB columns, read once: every screen evaluation of the tile takes its
  // n - 1 arguments from here, and the flush its correction factors
  __shared__ float2 s_l2q[LA];
  __shared__ float2 s_l2p[kCB];
  __shared__ float s_corq[LA], s_corp[kCB];
  const int B = n / LA;
  const int col = threadIdx.x % kCB, jt = threadIdx.x / kCB;
  const int c = blockIdx.y;
  // only the bands that hold image columns (from the band of column crop: the image's
  // side need not be a multiple of the band, nor crop of its width)
  const int col0 = (crop / kCB + (int)blockIdx.x) * kCB;
  const int kp = col0 + col;
  const bool kahan = flags & ACC_KAHAN;
  const uint32_t mbar0 = (uint32_t)__cvta_generic_to_shared(&s_mbar[0]);
  const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(&ring[0][0]);
  if (threadIdx.x < TPL) {
    float2 twr[NTW];
    all_twiddles<LA, EPT, TPL, 1>(twr, threadIdx.x, tw, B);
#pragma unroll
    for (int i = 0; i < NTW; ++i) s_tw1[i][threadIdx.x] = twr[i];
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kColsBRing; ++i) mbar_init(mbar0 + 8u * i, 1u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (!FP64S) {
    for (int i = threadIdx.x; i < LA; i += THREADS) s_l2q[i] = sc.l2ff[c + B * i];
    if (threadIdx.x < kCB) s_l2p[threadIdx.x] = sc.l2ff[col0 + threadIdx.x];
  }
  if (flags & ACC_CORRECT) {
    for (int i = threadIdx.x; i < LA; i += THREADS) s_corq[i] = sc.corr[c + B * i];
    if (threadIdx.x < kCB) s_corp[threadIdx.x] = sc.corr[col0 + threadIdx.x];
  }
  __syncthreads();
  const int nplanes = p1 - p0;
  int issued = 0;  // thread 0: planes (indices within the call) whose tile copy is issued
  auto issue = [&](int q) {
    const int slot = q % kColsBRing;
    tma_load_tile3d(ring0 + (uint32_t)slot * kTileBytes, &tmap, 2 * col0, LA * c, q, mbar0 + 8u * slot, kTileBytes);
  };
  if (threadIdx.x == 0)
    for (; issued < kColsBRing && issued < nplanes; ++issued) issue(issued);
  // output e = b R1 + r of this thread is line element jt + b TPL + 16 r, image row c + B (that)
  auto out_line = [&](int e) { return jt + (e / R1) * TPL + 16 * (e % R1); };
  auto out_row = [&](int e) { return c + B * out_line(e); };
  int P = p0;
  bool failed = false;
  while (P < p1 && !failed) {
    const int img = P / n_w;
    const int pstart = P;
    const int pend = min(p1, (img + 1) * n_w);
    // the per-plane step of each output for this image (exact), conjugated.  The screen
    // evaluations are long dependent chains (n - 1, float-float product, sincospi): four
    // outputs at a time give the scheduler independent work without keeping all sixteen
    // live; the results reach the unrolled plane loop through thread-private shared slots
    {
      const float2 dwI = FP64S ? make_float2(0.0f, 0.0f) : sc.dwff[img];
#pragma unroll 4
      for (int e = 0; e < EPT; ++e) {
        const int kq = out_row(e);
        float2 a, st;
        if constexpr (FP64S) {
          screen_anchor<true, true>(sc, kp, kq, P, img, 1.0f, a, st);
        } else {
          bool valid;
          const ff t = n_minus_one_ff(s_l2p[col], s_l2q[out_line(e)], valid);
          st = valid ? cis_cycles_ff(ff_mul({dwI.x, dwI.y}, t)) : make_float2(0.0f, 0.0f);
        }
        s_cstep[e][threadIdx.x] = make_float2(st.x, -st.y);
      }
    }
    float2 S[EPT], Cc[EPT], acc[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) S[e] = Cc[e] = acc[e] = make_float2(0.0f, 0.0f);
    for (; P < pend; ++P) {
      const int q = P - p0;
      const int slot = q % kColsBRing;
      const bool ok = mbar_wait_bounded(mbar0 + 8u * slot, (uint32_t)(q / kColsBRing) & 1u, wait_ns);
      float2 *tile = ring[slot];
      float2 v[EPT];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = tile[(jt + r * TPL) * kCB + col];
      dft<16, 1>(v);
      if (__syncthreads_or(!ok)) {  // every stage-0 read of this slot and all of plane q - 1 done
        failed = true;
        break;
      }
      if (threadIdx.x == 0 && q >= 1 && issued < nplanes) {  // the slot of plane q - 1 is free
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(issued);
        ++issued;
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) tile[(16 * jt + r) * kCB + col] = v[r];
      __syncthreads();
#pragma unroll
      for (int b = 0; b < EPT / R1; ++b)
#pragma unroll
        for (int r = 0; r < R1; ++r) v[b * R1 + r] = tile[(jt + b * TPL + 16 * r) * kCB + col];
#pragma unroll
      for (int b = 0; b < EPT / R1; ++b) {
#pragma unroll
        for (int r = 1; r < R1; ++r) v[b * R1 + r] = cmul(v[b * R1 + r], s_tw1[b * (R1 - 1) + r - 1][jt]);
        dft<R1, 1>(&v[b * R1]);
      }
      // Horner: acc <- acc conj(s) + v
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float2 cs = s_cstep[e][threadIdx.x];
        acc[e] = make_float2(fmaf(acc[e].x, cs.x, fmaf(-acc[e].y, cs.y, v[e].x)),
                             fmaf(acc[e].x, cs.y, fmaf(acc[e].y, cs.x, v[e].y)));
      }
      if ((P - pstart) % kAnchor == kAnchor - 1 || P == pend - 1) {
        // end of an anchor block: the exact screen of plane P (sign included) for each
        // output, through the slot of this plane once every thread is done with it
        __syncthreads();
        float2 *s_anchor = tile;
        const float2 wP = FP64S ? make_float2(0.0f, 0.0f) : sc.wc[P];
#pragma unroll 4
        for (int e = 0; e < EPT; ++e) {
          const int kq = out_row(e);
          const float sg = ((kq + kp) & 1) ? -1.0f : 1.0f;
          float2 a, st;
          if constexpr (FP64S) {
            screen_anchor<true, false>(sc, kp, kq, P, img, sg, a, st);
          } else {
            bool valid;
            const ff t = n_minus_one_ff(s_l2p[col], s_l2q[out_line(e)], valid);
            a = valid ? cis_cycles_ff(ff_mul({wP.x, wP.y}, t)) : make_float2(0.0f, 0.0f);
            a.x *= sg;
            a.y *= sg;
          }
          s_anchor[e * THREADS + threadIdx.x] = a;
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const float2 y = cmul(acc[e], s_anchor[e * THREADS + threadIdx.x]);
          if (kahan) kahan_add(S[e], Cc[e], y);
          else S[e] = cadd(S[e], y);
          acc[e] = make_float2(0.0f, 0.0f);
        }
      }
    }
    if (failed) break;
    const bool first_any = img * n_w >= first_lo;
    const bool last_any = (img + 1) * n_w <= last_hi;
    float2 *im = image + (size_t)img * n_img * n_img;
    float2 *cp = comp ? comp + (size_t)img * n_img * n_img : nullptr;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int kq = out_row(e);
      if (CROP && (kq < crop || kq >= crop + n_img || kp < crop || kp >= crop + n_img))
          continue;  // a grid row or column outside the image
      const float f = (flags & ACC_CORRECT) ? s_corp[col] * s_corq[out_line(e)] : 1.0f;
      flush_pixel(im, cp, (size_t)(kq - crop) * n_img + (kp - crop), S[e], Cc[e], first_any, last_any, flags, f);
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(err, (unsigned long long)WST_ERR_TIMEOUT);
      // every copy issued must land before the CTA exits: bounded, with the full limit
      for (int q = P - p0; q < issued; ++q)
        mbar_wait_bounded(mbar0 + 8u * (q % kColsBRing), (uint32_t)(q / kColsBRing) & 1u, kWaitLimitNs);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// pass CB^H (adjoint): image tile -> planes; sign, correction and conjugate screen fused
// ---------------------------------------------------------------------------------
// An image smaller than the grid (oversampled grid: the image is the central n_img x
// n_img from grid index crop) enters zero-padded: the adjoint of the forward crop.
template <int LA, bool FP64S>
__global__ void __launch_bounds__(ColCfg<LA>::THREADS)
k_cols_bh(const float2 *__restrict__ dimage, int p0, int p1, int n_w, Tw tw,
          int n, ScreenCtx sc, int correct, float2 *__restrict__ planes, int n_img, int crop) {
  using C = ColCfg<LA>;
  constexpr int EPT = C::EPT, TPL = C::TPL;
  constexpr int NST = num_stages(LA, EPT);
  constexpr int RL = stage_radix(LA, EPT, NST - 1);
  constexpr int R0 = stage_radix(LA, EPT, 0);
  __shared__ float2 sm[LA * C::PADW];
  const int B = n / LA;
  const int col = threadIdx.x % kCB, jt = threadIdx.x / kCB;
  const int c = blockIdx.y;
  const int kp = blockIdx.x * kCB + col;
  auto smi = [col](int i) { return i * C::PADW + col; };
  // inputs of the first stage: element d <-> image row kq = c + B d
  float2 dv[EPT], scr[EPT], stp[EPT];
  int img_loaded = -1, pstart = p0;
  for (int P = p0; P < p1; ++P) {
    const int img = P / n_w;
    if (img != img_loaded) {
      const float2 *im = dimage + (size_t)img * n_img * n_img;
      const bool col_in = kp >= crop && kp < crop + n_img;
#pragma unroll
      for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int kq = c + B * in_index<LA, EPT, TPL, 0>(jt, b, r);
          dv[b * R0 + r] = (col_in && kq >= crop && kq < crop + n_img)
                               ? im[(size_t)(kq - crop) * n_img + (kp - crop)]
                               : make_float2(0.0f, 0.0f);
        }
      img_loaded = img;
      pstart = P;
    }
    if ((P - pstart) % kAnchor == 0) {
#pragma unroll
      for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int kq = c + B * in_index<LA, EPT, TPL, 0>(jt, b, r);
          float f = ((kq + kp) & 1) ? -1.0f : 1.0f;
          if (correct) f *= sc.corr[kp] * sc.corr[kq];
          float2 a, st;
          screen_anchor<FP64S>(sc, kp, kq, P, img, f, a, st);
          scr[b * R0 + r] = make_float2(a.x, -a.y);  // conjugate screen
          stp[b * R0 + r] = make_float2(st.x, -st.y);
        }
    }
    float2 v[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      v[e] = cmul(dv[e], scr[e]);
      scr[e] = cmul(scr[e], stp[e]);
    }
    stage_compute<LA, EPT, TPL, 0, -1>(v, jt, tw, B);
    if constexpr (NST > 1) {
      middle_stages<LA, EPT, TPL, 1, -1>(v, jt, sm, smi, tw, B);
      stage_compute<LA, EPT, TPL, NST - 1, -1>(v, jt, tw, B);
    }
    float2 *base = planes + (size_t)(P - p0) * n * n + (size_t)(LA * c) * n + kp;
#pragma unroll
    for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) base[(size_t)out_index<LA, EPT, TPL, NST - 1>(jt, b, r) * n] = v[b * RL + r];
    if constexpr (NST > 1) __syncthreads();
  }
}

// elementwise grid correction
__global__ void k_correct(float2 *image, const float *corr, int n, int crop, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pix = i % ((int64_t)n * n);
    const int a = (int)(pix % n), b = (int)(pix / n);
    const float f = corr[a + crop] * corr[b + crop];  // corr is indexed on the grid
    float2 x = image[i];
    image[i] = make_float2(x.x * f, x.y * f);
  }
}

// ---------------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------------
static Tw tw_of(const wst_plan_s *p) {
  Tw t;
  t.t = p->tw;
  t.hmask = (p->n >> 1) - 1;
  t.hbit = p->n >> 1;
  return t;
}

template <int N, int DIR, bool PRE, bool POST>
static cudaError_t launch_rows(wst_plan_s *p, float2 *planes, int nplanes) {
  using C = RowCfg<N>;
  const size_t smem = sizeof(float2) * C::RPC * C::PADL;
  if constexpr (N >= kRowsTmaMin) {
    auto kern = k_rows_tma<N, DIR, PRE, POST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return e;
    const int64_t rows = (int64_t)nplanes * N;
    const int grid = (int)(rows < sms ? rows : sms);
    kern<<<grid, C::THREADS, smem, p->stream>>>(planes, rows, tw_of(p), p->W_.counters + CNT_ERROR, p->wait_ns);
  } else {
    auto kern = k_rows<N, DIR, PRE, POST>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    dim3 grd(N / C::RPC, nplanes);
    kern<<<grd, C::THREADS, smem, p->stream>>>(planes, tw_of(p));
  }
  return cudaGetLastError();
}

template <int DIR, bool PRE, bool POST>
static cudaError_t rows_dispatch(wst_plan_s *p, float2 *planes, int nplanes) {
  switch (p->n) {
    case 64: return launch_rows<64, DIR, PRE, POST>(p, planes, nplanes);
    case 128: return launch_rows<128, DIR, PRE, POST>(p, planes, nplanes);
    case 256: return launch_rows<256, DIR, PRE, POST>(p, planes, nplanes);
    case 512: return launch_rows<512, DIR, PRE, POST>(p, planes, nplanes);
    case 1024: return launch_rows<1024, DIR, PRE, POST>(p, planes, nplanes);
    case 2048: return launch_rows<2048, DIR, PRE, POST>(p, planes, nplanes);
    case 4096: return launch_rows<4096, DIR, PRE, POST>(p, planes, nplanes);
    case 8192: return launch_rows<8192, DIR, PRE, POST>(p, planes, nplanes);
    case 16384: return launch_rows<16384, DIR, PRE, POST>(p, planes, nplanes);
  }
  return cudaErrorInvalidValue;
}

cudaError_t fft_rows(wst_plan_s *p, float2 *planes, int nplanes, int dir, bool presign, bool postsign) {
  if (nplanes <= 0) return cudaSuccess;
  p->launches += 1;
  if (dir > 0 && !presign && !postsign) return rows_dispatch<1, false, false>(p, planes, nplanes);
  if (dir > 0 && presign && !postsign) return rows_dispatch<1, true, false>(p, planes, nplanes);
  if (dir < 0 && !presign && postsign) return rows_dispatch<-1, false, true>(p, planes, nplanes);
  return cudaErrorInvalidValue;
}

template <int LB, int DIR, bool TWF>
static cudaError_t launch_cols_a(wst_plan_s *p, float2 *planes, int nplanes, const uint8_t *occ) {
  if constexpr (LB >= 32) {  // persistent, staged, 32-column bands, 16 elements per thread
    constexpr int CB = 32, THREADS = LB / 16 * CB;
    auto kern = k_cols_a16<LB, DIR, TWF>;
    int per_sm = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)nplanes * (p->n / LB) * (p->n / CB);
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * sms;
    if (grid > tiles) grid = tiles;
    kern<<<(unsigned)grid, THREADS, 0, p->stream>>>(planes, tw_of(p), p->n, occ, nplanes);
  } else {
    dim3 grd(p->n / kCB, p->n / LB, nplanes);
    k_cols_a<LB, DIR, TWF><<<grd, ColCfg<LB>::THREADS, 0, p->stream>>>(planes, tw_of(p), p->n, occ);
  }
  return cudaGetLastError();
}

template <int DIR, bool TWF>
static cudaError_t cols_a_dispatch(wst_plan_s *p, float2 *planes, int nplanes, const uint8_t *occ) {
  switch (p->fb) {
    case 8: return launch_cols_a<8, DIR, TWF>(p, planes, nplanes, occ);
    case 16: return launch_cols_a<16, DIR, TWF>(p, planes, nplanes, occ);
    case 32: return launch_cols_a<32, DIR, TWF>(p, planes, nplanes, occ);
    case 64: return launch_cols_a<64, DIR, TWF>(p, planes, nplanes, occ);
    case 128: return launch_cols_a<128, DIR, TWF>(p, planes, nplanes, occ);
  }
  return cudaErrorInvalidValue;
}

cudaError_t fft_cols_a(wst_plan_s *p, float2 *planes, int nplanes, int dir, bool twiddle_first,
                       const uint8_t *occ) {
  if (nplanes <= 0) return cudaSuccess;
  p->launches += 1;
  if (dir > 0 && !twiddle_first) return cols_a_dispatch<1, false>(p, planes, nplanes, occ);
  if (dir < 0 && twiddle_first) return cols_a_dispatch<-1, true>(p, planes, nplanes, occ);
  return cudaErrorInvalidValue;
}

static ScreenCtx screen_ctx(wst_plan_s *p) {
  ScreenCtx sc;
  sc.l2ff = p->l2ff;
  sc.l2d = p->l2d;
  sc.wc = p->wcentre;
  sc.wcd = p->wcentre_d;
  sc.dwff = p->dwff;
  sc.wrange = p->wrange;
  sc.corr = p->corr;
  return sc;
}

static bool fp64_screen(const wst_plan_s *p) { return (p->cfg.flags & WST_FLAG_FP64_SCREEN) != 0; }

// cuTensorMapEncodeTiled, fetched from the driver at run time (no link against libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
    cudaGetLastError();
  });
  return fn;
}

// Tensor map of nplanes complex64 n x n planes seen as FP32 [nplanes][n][2n], with a box of
// one tile: kCB complex columns (128 bytes) x `rows` rows x 1 plane.  False if the encoder
// is unavailable or the buffer is not 16-byte aligned (the copies need both).
static bool plane_tile_map(CUtensorMap *m, const float2 *planes, int n, int nplanes, int rows) {
  const EncodeTiledFn enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)planes & 15u) || nplanes < 1) return false;
  const cuuint64_t dims[3] = {2ull * (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nplanes};
  const cuuint64_t strides[2] = {8ull * (cuuint64_t)n, 8ull * (cuuint64_t)n * (cuuint64_t)n};
  const cuuint32_t box[3] = {2u * kCB, (cuuint32_t)rows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(planes), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int LA, bool FP64S, bool CROP>
static void launch_cols_b_variant(wst_plan_s *p, const float2 *planes, int p0, int p1, float2 *image,
                                  float2 *comp, int flags) {
  // the grid's column bands that hold image columns, every row block
  dim3 grd((p->crop + p->n_img + kCB - 1) / kCB - p->crop / kCB, p->n / LA);
  if constexpr (LA == 64 || LA == 128) {
    CUtensorMap map;
    if (plane_tile_map(&map, planes, p->n, p1 - p0, LA))
      k_cols_b_tma<LA, FP64S, CROP><<<grd, LA / 16 * kCB, 0, p->stream>>>(
          map, p0, p1, p->n_w, tw_of(p), p->n, screen_ctx(p), image, comp, flags, p->n_img, p->crop,
          p->W_.counters + CNT_ERROR, p->wait_ns, (flags & ACC_RANGE_START) ? -1 : p0,
          (flags & ACC_RANGE_END) ? 0x7FFFFFFF : p1);
    else
      k_cols_b16<LA, FP64S, CROP><<<grd, LA / 16 * kCB, 0, p->stream>>>(
          planes, p0, p1, p->n_w, tw_of(p), p->n, screen_ctx(p), image, comp, flags, p->n_img, p->crop);
  } else
    k_cols_b_acc<LA, FP64S, CROP><<<grd, ColCfg<LA>::THREADS, 0, p->stream>>>(
        planes, p0, p1, p->n_w, tw_of(p), p->n, screen_ctx(p), image, comp, flags, p->n_img, p->crop);
}

template <int LA>
static cudaError_t launch_cols_b(wst_plan_s *p, const float2 *planes, int p0, int p1, float2 *image,
                                 float2 *comp, int flags) {
  const bool fp64 = fp64_screen(p), crop = p->crop != 0;
  if (fp64 && crop) launch_cols_b_variant<LA, true, true>(p, planes, p0, p1, image, comp, flags);
  else if (fp64) launch_cols_b_variant<LA, true, false>(p, planes, p0, p1, image, comp, flags);
  else if (crop) launch_cols_b_variant<LA, false, true>(p, planes, p0, p1, image, comp, flags);
  else launch_cols_b_variant<LA, false, false>(p, planes, p0, p1, image, comp, flags);
  return cudaGetLastError();
}

cudaError_t fft_cols_b_accumulate(wst_plan_s *p, const float2 *planes, int p0, int p1, float2 *image,
                                  float2 *comp, bool kahan, bool correct, bool staged_add, bool range_start,
                                  bool range_end) {
  if (p1 <= p0) return cudaSuccess;
  p->launches += 1;
  int flags = 0;
  if (range_start) flags |= ACC_RANGE_START;
  if (range_end) flags |= ACC_RANGE_END;
  if (correct) flags |= ACC_CORRECT;
  if (kahan) flags |= ACC_KAHAN;
  if (staged_add) flags |= ACC_STAGED;
  switch (p->fa) {
    case 8: return launch_cols_b<8>(p, planes, p0, p1, image, comp, flags);
    case 16: return launch_cols_b<16>(p, planes, p0, p1, image, comp, flags);
    case 32: return launch_cols_b<32>(p, planes, p0, p1, image, comp, flags);
    case 64: return launch_cols_b<64>(p, planes, p0, p1, image, comp, flags);
    case 128: return launch_cols_b<128>(p, planes, p0, p1, image, comp, flags);
  }
  return cudaErrorInvalidValue;
}

template <int LA>
static cudaError_t launch_cols_bh(wst_plan_s *p, const float2 *dimage, int p0, int p1, float2 *planes,
                                  bool correct) {
  dim3 grd(p->n / kCB, p->n / LA);
  if (fp64_screen(p))
    k_cols_bh<LA, true><<<grd, ColCfg<LA>::THREADS, 0, p->stream>>>(
        dimage, p0, p1, p->n_w, tw_of(p), p->n, screen_ctx(p), correct ? 1 : 0, planes, p->n_img, p->crop);
  else
    k_cols_bh<LA, false><<<grd, ColCfg<LA>::THREADS, 0, p->stream>>>(
        dimage, p0, p1, p->n_w, tw_of(p), p->n, screen_ctx(p), correct ? 1 : 0, planes, p->n_img, p->crop);
  return cudaGetLastError();
}

cudaError_t fft_cols_bh_from_image(wst_plan_s *p, const float2 *dimage, int p0, int p1, float2 *planes,
                                   bool correct) {
  if (p1 <= p0) return cudaSuccess;
  p->launches += 1;
  switch (p->fa) {
    case 8: return launch_cols_bh<8>(p, dimage, p0, p1, planes, correct);
    case 16: return launch_cols_bh<16>(p, dimage, p0, p1, planes, correct);
    case 32: return launch_cols_bh<32>(p, dimage, p0, p1, planes, correct);
    case 64: return launch_cols_bh<64>(p, dimage, p0, p1, planes, correct);
    case 128: return launch_cols_bh<128>(p, dimage, p0, p1, planes, correct);
  }
  return cudaErrorInvalidValue;
}

cudaError_t correct_image(wst_plan_s *p, float2 *image) {
  const int64_t total = (int64_t)p->batch * p->n_img * p->n_img;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_correct<<<(unsigned)blocks, 256, 0, p->stream>>>(image, p->corr, p->n_img, p->crop, total);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace wst
