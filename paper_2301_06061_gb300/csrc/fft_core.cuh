// FFT building blocks shared by the libwst kernels: register DFTs of radix 2..32,
// the Stockham stage schedule, twiddles from a half-wave table, and the shared-memory
// stage driver.  (Included by k_fft.cu and k_rowgrid.cu.)
#pragma once

#include <type_traits>

#include "wst_internal.cuh"

namespace wst {

// ---------------------------------------------------------------------------------
// register DFTs of radix 2, 4, 8, 16 (natural order in and out), sign DIR
// ---------------------------------------------------------------------------------
constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f;  // sin(pi/8)

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {  // a * (DIR * i)
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * exp(DIR * 2 pi i k / 16), k a compile-time constant in [0, 16)
template <int DIR, int K>
__device__ __forceinline__ float2 mul_w16(float2 a) {
  constexpr int k = K & 15;
  if constexpr (k == 0) return a;
  else if constexpr (k == 4) return mul_i<DIR>(a);
  else if constexpr (k == 8) return make_float2(-a.x, -a.y);
  else if constexpr (k == 12) return mul_i<-DIR>(a);
  else {
    // cos / sin of 2 pi k / 16 from the three constants
    constexpr float cs[16] = {1.0f, kC16, kC8, kS16, 0.0f, -kS16, -kC8, -kC16,
                              -1.0f, -kC16, -kC8, -kS16, 0.0f, kS16, kC8, kC16};
    constexpr float c = cs[k];
    constexpr float s = cs[(k + 12) & 15];  // sin(x) = cos(x - pi/2)
    const float sd = DIR > 0 ? s : -s;
    return make_float2(a.x * c - a.y * sd, a.x * sd + a.y * c);
  }
}

template <int DIR>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
  const float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_i<DIR>(csub(b, d));
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, t3);
  d = csub(t1, t3);
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2 *v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    dft4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    o1 = mul_w16<DIR, 2>(o1);
    o2 = mul_w16<DIR, 4>(o2);
    o3 = mul_w16<DIR, 6>(o3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  } else if constexpr (R == 32) {
    // 32 = 2 x 16: X[m] = E[m] + w32^m O[m], X[m + 16] = E[m] - w32^m O[m]
    constexpr float c32[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                              0.83146961230254523708f, 0.70710678118654752440f, 0.55557023301960222474f,
                              0.38268343236508977173f, 0.19509032201612826785f, 0.0f};
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<16, DIR>(e);
    dft<16, DIR>(o);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      // w32^m = cos(pi m/16) + DIR i sin(pi m/16)
      const float c = m <= 8 ? c32[m] : -c32[16 - m];
      const float sn = m <= 8 ? c32[8 - m] : c32[m - 8];
      const float sd = DIR > 0 ? sn : -sn;
      const float2 t = make_float2(o[m].x * c - o[m].y * sd, o[m].x * sd + o[m].y * c);
      v[m] = cadd(e[m], t);
      v[m + 16] = csub(e[m], t);
    }
  } else {
    static_assert(R == 16, "radix");
    // 16 = 4 x 4: inputs r1 + 4 r2, outputs m2 + 4 m1
    float2 y[16];
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) {
      float2 a = v[r1], b = v[r1 + 4], c = v[r1 + 8], d = v[r1 + 12];
      dft4<DIR>(a, b, c, d);
      y[r1 * 4 + 0] = a;
      y[r1 * 4 + 1] = b;
      y[r1 * 4 + 2] = c;
      y[r1 * 4 + 3] = d;
    }
    y[5] = mul_w16<DIR, 1>(y[5]);
    y[6] = mul_w16<DIR, 2>(y[6]);
    y[7] = mul_w16<DIR, 3>(y[7]);
    y[9] = mul_w16<DIR, 2>(y[9]);
    y[10] = mul_w16<DIR, 4>(y[10]);
    y[11] = mul_w16<DIR, 6>(y[11]);
    y[13] = mul_w16<DIR, 3>(y[13]);
    y[14] = mul_w16<DIR, 6>(y[14]);
    y[15] = mul_w16<DIR, 9>(y[15]);
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) {
      float2 a = y[0 * 4 + m2], b = y[1 * 4 + m2], c = y[2 * 4 + m2], d = y[3 * 4 + m2];
      dft4<DIR>(a, b, c, d);
      v[m2 + 0] = a;
      v[m2 + 4] = b;
      v[m2 + 8] = c;
      v[m2 + 12] = d;
    }
  }
}

// ---------------------------------------------------------------------------------
// Stockham stage schedule for a length-L line with EPT elements per thread
// ---------------------------------------------------------------------------------
constexpr int stage_radix(int L, int ept, int s) {
  int rem = L;
  for (int i = 0; i < s; ++i) rem /= (rem < ept ? rem : ept);
  return rem < ept ? rem : ept;
}
constexpr int stage_ns(int L, int ept, int s) {  // product of the radices before stage s
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= stage_radix(L, ept, i);
  return ns;
}
constexpr int num_stages(int L, int ept) {
  int n = 0, rem = L;
  while (rem > 1) {
    rem /= (rem < ept ? rem : ept);
    ++n;
  }
  return n;
}

// exp(dir 2 pi i idx / N) from a half-wave table T[m] = exp(2 pi i m / N), m < N/2
// (64 KB at N = 16384); exp(2 pi i (m + N/2) / N) = -T[m].
struct Tw {
  const float2 *t;
  int hmask;  // N/2 - 1
  int hbit;   // N/2
};

__device__ __forceinline__ float2 twiddle(const Tw &tw, int idx, int dir) {
  float2 w = __ldg(tw.t + (idx & tw.hmask));
  if (idx & tw.hbit) w = make_float2(-w.x, -w.y);
  if (dir < 0) w.y = -w.y;
  return w;
}

// exp(dir 2 pi i idx / N) evaluated on the spot, for a factor that a kernel needs at once
// rather than after a table load: with N a power of two and 0 <= idx < N, idx * (2 / N)
// is exact in FP32, so sincospi sees the exact argument.
__device__ __forceinline__ float2 twiddle_direct(int idx, float two_over_n, int dir) {
  float s, c;
  sincospif((float)idx * two_over_n, &s, &c);
  return make_float2(c, dir > 0 ? s : -s);
}

// Butterfly b of this thread has index j = jt + b * TPL (< L/R); its inputs sit at
// j + r L/R and, after the twiddles w_{NS R}^{(j mod NS) r} and the radix-R DFT, its
// outputs belong at (j / NS) NS R + (j mod NS) + r NS.
template <int L, int EPT, int TPL, int S, int DIR>
__device__ __forceinline__ void stage_compute(float2 (&v)[EPT], int jt, const Tw &tw, int twscale) {
  constexpr int R = stage_radix(L, EPT, S);
  constexpr int NS = stage_ns(L, EPT, S);
#pragma unroll
  for (int b = 0; b < EPT / R; ++b) {
    const int j = jt + b * TPL;
    if constexpr (NS > 1) {
      const int k = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int m = k * r * (L / (NS * R));
        v[b * R + r] = cmul(v[b * R + r], twiddle(tw, m * twscale, DIR));
      }
    }
    dft<R, DIR>(&v[b * R]);
  }
}

// Stage S with the twiddles from a provider: twp(S, b, r, k) is the factor of input r
// of butterfly b (k = j mod NS), S passed as std::integral_constant.
template <int L, int EPT, int TPL, int S, int DIR, class TWP>
__device__ __forceinline__ void stage_compute_f(float2 (&v)[EPT], int jt, const TWP &twp) {
  constexpr int R = stage_radix(L, EPT, S);
  constexpr int NS = stage_ns(L, EPT, S);
#pragma unroll
  for (int b = 0; b < EPT / R; ++b) {
    const int j = jt + b * TPL;
    if constexpr (NS > 1) {
      const int k = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], twp(std::integral_constant<int, S>(), b, r, k));
    }
    dft<R, DIR>(&v[b * R]);
  }
}

// Twiddles of stage S held in registers, for kernels that run the same transform many
// times (one per w-plane): twp[b (R - 1) + r - 1] is the factor of input r of butterfly b.
template <int L, int EPT, int S>
constexpr int stage_tw_count() {
  return stage_ns(L, EPT, S) > 1 ? (EPT / stage_radix(L, EPT, S)) * (stage_radix(L, EPT, S) - 1) : 0;
}
template <int L, int EPT, int S>
constexpr int stage_tw_offset() {  // position of stage S's factors in the concatenated list
  if constexpr (S == 0) return 0;
  else return stage_tw_offset<L, EPT, S - 1>() + stage_tw_count<L, EPT, S - 1>();
}
template <int L, int EPT>
constexpr int total_tw_count() {
  return stage_tw_offset<L, EPT, num_stages(L, EPT)>();
}

template <int L, int EPT, int TPL, int S, int DIR>
__device__ __forceinline__ void stage_twiddles(float2 *twp, int jt, const Tw &tw, int twscale) {
  constexpr int R = stage_radix(L, EPT, S);
  constexpr int NS = stage_ns(L, EPT, S);
  if constexpr (NS > 1) {
#pragma unroll
    for (int b = 0; b < EPT / R; ++b) {
      const int k = (jt + b * TPL) % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) twp[b * (R - 1) + r - 1] = twiddle(tw, k * r * (L / (NS * R)) * twscale, DIR);
    }
  }
}

template <int L, int EPT, int TPL, int DIR, int S = 0>
__device__ __forceinline__ void all_twiddles(float2 *twp, int jt, const Tw &tw, int twscale) {
  if constexpr (S < num_stages(L, EPT)) {
    stage_twiddles<L, EPT, TPL, S, DIR>(twp + stage_tw_offset<L, EPT, S>(), jt, tw, twscale);
    all_twiddles<L, EPT, TPL, DIR, S + 1>(twp, jt, tw, twscale);
  }
}

template <int L, int EPT, int S, int DIR>
__device__ __forceinline__ void stage_compute_pre(float2 (&v)[EPT], const float2 *twp) {
  constexpr int R = stage_radix(L, EPT, S);
  constexpr int NS = stage_ns(L, EPT, S);
#pragma unroll
  for (int b = 0; b < EPT / R; ++b) {
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], twp[stage_tw_offset<L, EPT, S>() + b * (R - 1) + r - 1]);
    }
    dft<R, DIR>(&v[b * R]);
  }
}

template <int L, int EPT, int TPL, int S>
__device__ __forceinline__ int in_index(int jt, int b, int r) {
  constexpr int R = stage_radix(L, EPT, S);
  return jt + b * TPL + r * (L / R);
}
template <int L, int EPT, int TPL, int S>
__device__ __forceinline__ int out_index(int jt, int b, int r) {
  constexpr int R = stage_radix(L, EPT, S);
  constexpr int NS = stage_ns(L, EPT, S);
  const int j = jt + b * TPL;
  return (j / NS) * NS * R + (j % NS) + r * NS;
}

// Run stages 1 .. last-1 through shared memory; `smi` maps a line index to a shared
// memory slot.  On entry v holds the outputs of stage 0 (not yet stored); on return v
// holds the inputs of the last stage, already loaded.
template <int L, int EPT, int TPL, int S, int DIR, class SMI>
__device__ __forceinline__ void middle_stages(float2 (&v)[EPT], int jt, float2 *sm, SMI smi,
                                              const Tw &tw, int twscale) {
  constexpr int NST = num_stages(L, EPT);
  if constexpr (S < NST) {
    // store outputs of stage S-1
    constexpr int RP = stage_radix(L, EPT, S - 1);
#pragma unroll
    for (int b = 0; b < EPT / RP; ++b)
#pragma unroll
      for (int r = 0; r < RP; ++r) sm[smi(out_index<L, EPT, TPL, S - 1>(jt, b, r))] = v[b * RP + r];
    __syncthreads();
    constexpr int R = stage_radix(L, EPT, S);
#pragma unroll
    for (int b = 0; b < EPT / R; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = sm[smi(in_index<L, EPT, TPL, S>(jt, b, r))];
    if constexpr (S + 1 < NST) {
      __syncthreads();  // every load of this stage done before the next stores
      stage_compute<L, EPT, TPL, S, DIR>(v, jt, tw, twscale);
      middle_stages<L, EPT, TPL, S + 1, DIR>(v, jt, sm, smi, tw, twscale);
    }
  }
}

// ---------------------------------------------------------------------------------
// Shared-memory twiddle tables for kernels that transform many lines of length L with
// the same (EPT, TPL) layout.  Stage S >= 1 needs w_L^{k r M}, M = L/(NS R), k = j mod
// NS, j = jt + b TPL.  If NS <= TPL the table is T_S[r - 1][k] (k < NS); otherwise
// k = jt + (b TPL mod NS) and the table is T_S[r - 1][jt] (jt < TPL) times the constant
// w_L^{(b TPL mod NS) r M} = e^{2 pi i b' r / Q}, b' = (b TPL mod NS)/TPL,
// Q = NS R / TPL <= EPT <= 32.  Consecutive threads read consecutive entries (or one
// broadcast entry): no bank conflicts, no sign logic.  Entries hold the positive
// exponent; DIR < 0 conjugates.
// ---------------------------------------------------------------------------------
template <int L, int EPT, int TPL, int S>
constexpr int stage_table_size() {
  if constexpr (S == 0) {
    return 0;
  } else {
    constexpr int R = stage_radix(L, EPT, S), NS = stage_ns(L, EPT, S);
    return (R - 1) * (NS <= TPL ? NS : TPL);
  }
}
template <int L, int EPT, int TPL, int S>
constexpr int stage_table_offset() {
  if constexpr (S == 0) return 0;
  else return stage_table_offset<L, EPT, TPL, S - 1>() + stage_table_size<L, EPT, TPL, S - 1>();
}
template <int L, int EPT, int TPL>
constexpr int line_table_size() {
  return stage_table_offset<L, EPT, TPL, num_stages(L, EPT)>();
}

template <int L, int EPT, int TPL, int S = 1>
__device__ __forceinline__ void fill_line_tables(float2 *T, const Tw &tw) {
  if constexpr (S < num_stages(L, EPT)) {
    constexpr int R = stage_radix(L, EPT, S), NS = stage_ns(L, EPT, S), M = L / (NS * R);
    constexpr int WD = NS <= TPL ? NS : TPL;
    float2 *base = T + stage_table_offset<L, EPT, TPL, S>();
    for (int i = threadIdx.x; i < (R - 1) * WD; i += blockDim.x) base[i] = twiddle(tw, (i % WD) * (i / WD + 1) * M, 1);
    fill_line_tables<L, EPT, TPL, S + 1>(T, tw);
  }
}

// e^{2 pi i e / 32}, e in [0, 32)
__device__ __forceinline__ float2 root32(int e) {
  constexpr float c32[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                            0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                            0.19509032201612826785f, 0.0f};
  const int q = e >> 3, m = e & 7;  // quadrant, position in it
  const float c = c32[m], s = c32[8 - m];
  return q == 0 ? make_float2(c, s) : q == 1 ? make_float2(-s, c) : q == 2 ? make_float2(-c, -s) : make_float2(s, -c);
}

template <int L, int EPT, int TPL, int DIR>
struct TableTw {
  const float2 *T;
  int jt;
  template <int S>
  __device__ __forceinline__ float2 operator()(std::integral_constant<int, S>, int b, int r, int k) const {
    constexpr int R = stage_radix(L, EPT, S), NS = stage_ns(L, EPT, S);
    const float2 *base = T + stage_table_offset<L, EPT, TPL, S>();
    float2 w;
    if constexpr (NS <= TPL) {
      w = base[(r - 1) * NS + k];
    } else {
      constexpr int Q = NS * R / TPL;
      w = base[(r - 1) * TPL + jt];
      const int bq = ((b * TPL) % NS) / TPL;
      const int e = (bq * r * (32 / Q)) & 31;
      if (e != 0) w = cmul(w, root32(e));
    }
    if (DIR < 0) w.y = -w.y;
    return w;
  }
};

// middle_stages with the twiddles from a provider (see stage_compute_f)
template <int L, int EPT, int TPL, int S, int DIR, class SMI, class TWP>
__device__ __forceinline__ void middle_stages_f(float2 (&v)[EPT], int jt, float2 *sm, SMI smi, const TWP &twp) {
  constexpr int NST = num_stages(L, EPT);
  if constexpr (S < NST) {
    constexpr int RP = stage_radix(L, EPT, S - 1);
#pragma unroll
    for (int b = 0; b < EPT / RP; ++b)
#pragma unroll
      for (int r = 0; r < RP; ++r) sm[smi(out_index<L, EPT, TPL, S - 1>(jt, b, r))] = v[b * RP + r];
    __syncthreads();
    constexpr int R = stage_radix(L, EPT, S);
#pragma unroll
    for (int b = 0; b < EPT / R; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = sm[smi(in_index<L, EPT, TPL, S>(jt, b, r))];
    if constexpr (S + 1 < NST) {
      __syncthreads();
      stage_compute_f<L, EPT, TPL, S, DIR>(v, jt, twp);
      middle_stages_f<L, EPT, TPL, S + 1, DIR>(v, jt, sm, smi, twp);
    }
  }
}

// middle_stages with the twiddles from registers (the full list of all_twiddles)
template <int L, int EPT, int TPL, int S, int DIR, class SMI>
__device__ __forceinline__ void middle_stages_pre(float2 (&v)[EPT], int jt, float2 *sm, SMI smi, const float2 *twp) {
  constexpr int NST = num_stages(L, EPT);
  if constexpr (S < NST) {
    constexpr int RP = stage_radix(L, EPT, S - 1);
#pragma unroll
    for (int b = 0; b < EPT / RP; ++b)
#pragma unroll
      for (int r = 0; r < RP; ++r) sm[smi(out_index<L, EPT, TPL, S - 1>(jt, b, r))] = v[b * RP + r];
    __syncthreads();
    constexpr int R = stage_radix(L, EPT, S);
#pragma unroll
    for (int b = 0; b < EPT / R; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = sm[smi(in_index<L, EPT, TPL, S>(jt, b, r))];
    if constexpr (S + 1 < NST) {
      __syncthreads();
      stage_compute_pre<L, EPT, S, DIR>(v, twp);
      middle_stages_pre<L, EPT, TPL, S + 1, DIR>(v, jt, sm, smi, twp);
    }
  }
}

// ---------------------------------------------------------------------------------
// pass R: row FFTs
// ---------------------------------------------------------------------------------
template <int N>
struct RowCfg {
  // 32 elements per thread for the longest rows: radix 32, 32, 16 (two shared-memory
  // round trips); 16 otherwise.  Rows are padded by one element every EPT elements.
  static constexpr int EPT = N >= 16384 ? 32 : (N >= 16 ? 16 : N);
  static constexpr int TPR = N / EPT;
  static constexpr int RPC = TPR >= 256 ? 1 : 256 / TPR;
  static constexpr int THREADS = TPR * RPC;
  static constexpr int PADL = N + N / EPT;
};

}  // namespace wst
