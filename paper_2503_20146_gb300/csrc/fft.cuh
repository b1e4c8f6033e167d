// Register/shared-memory Stockham FFT building blocks for the PWF passes.
//
// Every Filter of Algorithm S2 (F^-1{F{x} W}) is evaluated as a row transform
// and a column transform of a complex64 field. This header holds the pieces
// shared by the row and column kernels:
//   * complex helpers and radix-2/3/4/8/16 DFT butterflies (written from the
//     DFT definition X_k = sum_j x_j exp(s 2 pi i j k / R), s = -1 forward);
//   * a compile-time radix schedule per transform length N (N = 2^a 3^b);
//   * a self-sorting (Stockham) stage runner: stage 0 takes its inputs from
//     registers, middle stages exchange through shared memory, and the last
//     stage leaves its outputs in registers. The inverse transform uses the
//     reversed radix order, so the slot layout at the end of a forward
//     transform equals the one at the start of an inverse transform and vice
//     versa; that is what lets point-wise work run in registers between two
//     transforms of the same pass.
//
// Slot convention: with R the radix of the first (or last) stage, EPT values
// per thread and TPF threads per transform, slot (i, r) of thread t holds
// element  t + i*TPF + r*(N/R),  stored at v[i*R + r].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

// Radix schedule set of this translation unit: 0 (the default, every pass)
// or 1 (the alternative schedules some column shapes are also built with, in
// translation units of their own). Everything schedule-dependent lives in the
// inline namespace named after the set, so both sets link side by side.
#ifndef PWF_SCHED_VARIANT
#define PWF_SCHED_VARIANT 0
#endif
#if PWF_SCHED_VARIANT == 0
#define PWF_KNS sched0
#else
#define PWF_KNS sched1
#endif

namespace pwf {
inline namespace PWF_KNS {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

constexpr int FWD = -1;  // exponent sign of the forward DFT
constexpr int INV = +1;

// (s i) * a, s = DIR
template <int DIR>
__device__ __forceinline__ float2 mul_si(float2 a) {
  if constexpr (DIR == FWD) return make_float2(a.y, -a.x);   // -i a
  else return make_float2(-a.y, a.x);                        // +i a
}

// exp(s 2 pi i m / 16) for the compile-time exponent m
template <int DIR, int M>
__device__ __forceinline__ float2 w16() {
  constexpr int m = M & 15;
  // cos and sin of m*pi/8 for m = 0..15
  constexpr float C[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                           0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                           -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                           0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  constexpr float S[16] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                           1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                           0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                           -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f};
  return make_float2(C[m], DIR == FWD ? -S[m] : S[m]);
}

template <int DIR, int M>
__device__ __forceinline__ float2 twm16(float2 a) {
  constexpr int m = M & 15;
  if constexpr (m == 0) return a;
  else if constexpr (m == 4) return mul_si<DIR>(a);
  else if constexpr (m == 8) return make_float2(-a.x, -a.y);
  else if constexpr (m == 12) return mul_si<-DIR>(a);
  else return cmul(a, w16<DIR, m>());
}

// ---------------------------------------------------------------------------
// radix butterflies (in place on x[0..R))
// ---------------------------------------------------------------------------
template <int DIR>
__device__ __forceinline__ void dft2(float2* x) {
  float2 a = x[0], b = x[1];
  x[0] = cadd(a, b);
  x[1] = csub(a, b);
}

template <int DIR>
__device__ __forceinline__ void dft3(float2* x) {
  constexpr float H = 0.86602540378443865f;  // sqrt(3)/2
  float2 s = cadd(x[1], x[2]);
  float2 d = csub(x[1], x[2]);
  float2 m = make_float2(fmaf(-0.5f, s.x, x[0].x), fmaf(-0.5f, s.y, x[0].y));
  float2 r = mul_si<DIR>(cscale(d, H));
  x[0] = cadd(x[0], s);
  x[1] = cadd(m, r);
  x[2] = csub(m, r);
}

// 4-point DFT on elements x[0], x[S], x[2S], x[3S]
template <int DIR, int S = 1>
__device__ __forceinline__ void dft4s(float2* x) {
  float2 t0 = cadd(x[0], x[2 * S]);
  float2 t1 = csub(x[0], x[2 * S]);
  float2 t2 = cadd(x[S], x[3 * S]);
  float2 t3 = mul_si<DIR>(csub(x[S], x[3 * S]));
  x[0] = cadd(t0, t2);
  x[2 * S] = csub(t0, t2);
  x[S] = cadd(t1, t3);
  x[3 * S] = csub(t1, t3);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* x) { dft4s<DIR, 1>(x); }

// 8-point: radix-2 split into even/odd 4-point DFTs.
template <int DIR>
__device__ __forceinline__ void dft8(float2* x) {
  float2 e[4] = {x[0], x[2], x[4], x[6]};
  float2 o[4] = {x[1], x[3], x[5], x[7]};
  dft4<DIR>(e);
  dft4<DIR>(o);
  o[1] = twm16<DIR, 2>(o[1]);
  o[2] = twm16<DIR, 4>(o[2]);
  o[3] = twm16<DIR, 6>(o[3]);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    x[k] = cadd(e[k], o[k]);
    x[k + 4] = csub(e[k], o[k]);
  }
}

// 16-point: 4 x 4. Inner 4-point DFTs over j = q + 4m (stride 4), twiddle
// W16^(q k1), outer 4-point DFTs over q; output index k1 + 4 k2.
template <int DIR>
__device__ __forceinline__ void dft16(float2* x) {
  float2 y[16];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    float2 a[4] = {x[q], x[q + 4], x[q + 8], x[q + 12]};
    dft4<DIR>(a);
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) y[q * 4 + k1] = a[k1];
  }
  // y[q*4 + k1] *= W16^(q k1)
  y[1 * 4 + 1] = twm16<DIR, 1>(y[5]);
  y[1 * 4 + 2] = twm16<DIR, 2>(y[6]);
  y[1 * 4 + 3] = twm16<DIR, 3>(y[7]);
  y[2 * 4 + 1] = twm16<DIR, 2>(y[9]);
  y[2 * 4 + 2] = twm16<DIR, 4>(y[10]);
  y[2 * 4 + 3] = twm16<DIR, 6>(y[11]);
  y[3 * 4 + 1] = twm16<DIR, 3>(y[13]);
  y[3 * 4 + 2] = twm16<DIR, 6>(y[14]);
  y[3 * 4 + 3] = twm16<DIR, 9>(y[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++) {
    float2 a[4] = {y[k1], y[4 + k1], y[8 + k1], y[12 + k1]};
    dft4<DIR>(a);
#pragma unroll
    for (int k2 = 0; k2 < 4; k2++) x[k1 + 4 * k2] = a[k2];
  }
}

// exp(s 2 pi i m / 32) for the compile-time exponent m
template <int DIR, int M>
__device__ __forceinline__ float2 twm32(float2 a) {
  constexpr int m = M & 31;
  if constexpr ((m & 1) == 0) {
    return twm16<DIR, m / 2>(a);
  } else {
    // cos and sin of m*pi/16 for odd m
    constexpr double PI = 3.14159265358979323846;
    constexpr float c1 = 0.98078528040323043f, s1 = 0.19509032201612825f;  // pi/16
    constexpr float c3 = 0.83146961230254524f, s3 = 0.55557023301960218f;  // 3 pi/16
    constexpr float c5 = 0.55557023301960218f, s5 = 0.83146961230254524f;  // 5 pi/16
    constexpr float c7 = 0.19509032201612825f, s7 = 0.98078528040323043f;  // 7 pi/16
    (void)PI;
    // reduce m to the first quadrant: angle = m pi / 16
    constexpr int q = m / 8, r = m % 8;  // m = 8q + r, r odd
    constexpr float cr = r == 1 ? c1 : r == 3 ? c3 : r == 5 ? c5 : c7;
    constexpr float sr = r == 1 ? s1 : r == 3 ? s3 : r == 5 ? s5 : s7;
    // rotate by q quarter turns
    constexpr float c = q == 0 ? cr : q == 1 ? -sr : q == 2 ? -cr : sr;
    constexpr float sn = q == 0 ? sr : q == 1 ? cr : q == 2 ? -sr : -cr;
    return cmul(a, make_float2(c, DIR == FWD ? -sn : sn));
  }
}

// 32-point: radix-2 split into the 16-point DFTs of the even and odd
// samples, combined with the twiddles W32^k.
template <int DIR>
__device__ __forceinline__ void dft32(float2* x) {
  float2 e[16], o[16];
#pragma unroll
  for (int k = 0; k < 16; k++) {
    e[k] = x[2 * k];
    o[k] = x[2 * k + 1];
  }
  dft16<DIR>(e);
  dft16<DIR>(o);
#pragma unroll
  for (int k = 0; k < 16; k++) {
    float2 w;
    switch (k) {  // resolved at compile time after unrolling
      case 0: w = o[0]; break;
      case 1: w = twm32<DIR, 1>(o[1]); break;
      case 2: w = twm32<DIR, 2>(o[2]); break;
      case 3: w = twm32<DIR, 3>(o[3]); break;
      case 4: w = twm32<DIR, 4>(o[4]); break;
      case 5: w = twm32<DIR, 5>(o[5]); break;
      case 6: w = twm32<DIR, 6>(o[6]); break;
      case 7: w = twm32<DIR, 7>(o[7]); break;
      case 8: w = twm32<DIR, 8>(o[8]); break;
      case 9: w = twm32<DIR, 9>(o[9]); break;
      case 10: w = twm32<DIR, 10>(o[10]); break;
      case 11: w = twm32<DIR, 11>(o[11]); break;
      case 12: w = twm32<DIR, 12>(o[12]); break;
      case 13: w = twm32<DIR, 13>(o[13]); break;
      case 14: w = twm32<DIR, 14>(o[14]); break;
      default: w = twm32<DIR, 15>(o[15]); break;
    }
    x[k] = cadd(e[k], w);
    x[k + 16] = csub(e[k], w);
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* x) {
  if constexpr (R == 2) dft2<DIR>(x);
  else if constexpr (R == 3) dft3<DIR>(x);
  else if constexpr (R == 4) dft4<DIR>(x);
  else if constexpr (R == 8) dft8<DIR>(x);
  else if constexpr (R == 16) dft16<DIR>(x);
  else if constexpr (R == 32) dft32<DIR>(x);
  else static_assert(R == 2, "unsupported radix");
}

// ---------------------------------------------------------------------------
// compile-time radix schedules (forward order; the inverse runs them reversed)
// ---------------------------------------------------------------------------
struct Sched {
  int n, s, r0, r1, r2, r3, r4, r5;
  __host__ __device__ constexpr int r(int i) const {
    return i == 0 ? r0 : i == 1 ? r1 : i == 2 ? r2 : i == 3 ? r3 : i == 4 ? r4 : r5;
  }
};

// The alternative schedules (set 1): the same stages in another order where
// that keeps the values per thread, or smaller radices where it cuts them
// (fewer registers per transform, more warps per SM, shorter dependent chains
// per thread, at the price of more exchanges: 128 = 4.4.4.2 runs one
// transform per warp with four values per thread; 768 and 1536 keep 12 values
// per thread instead of 24).
__host__ __device__ constexpr Sched sched_alt(int n) {
  switch (n) {
    case 128: return {128, 4, 4, 4, 4, 2, 1, 1};
    case 256: return {256, 3, 4, 8, 8, 1, 1, 1};
    case 512: return {512, 3, 8, 8, 8, 1, 1, 1};
    case 768: return {768, 5, 4, 4, 4, 4, 3, 1};
    case 1024: return {1024, 3, 8, 8, 16, 1, 1, 1};
    case 1536: return {1536, 6, 4, 4, 4, 4, 2, 3};
    case 2048: return {2048, 3, 8, 16, 16, 1, 1, 1};
    default: return {0, 0, 1, 1, 1, 1, 1, 1};
  }
}

__host__ __device__ constexpr Sched sched_default(int n) {
  switch (n) {
    case 16: return {16, 1, 16, 1, 1, 1, 1, 1};
    case 32: return {32, 2, 8, 4, 1, 1, 1, 1};
    case 64: return {64, 2, 8, 8, 1, 1, 1, 1};
    case 96: return {96, 3, 8, 4, 3, 1, 1, 1};
    case 128: return {128, 2, 16, 8, 1, 1, 1, 1};
    case 192: return {192, 3, 8, 8, 3, 1, 1, 1};
    case 256: return {256, 2, 16, 16, 1, 1, 1, 1};
    case 384: return {384, 4, 8, 8, 2, 3, 1, 1};
    case 512: return {512, 3, 16, 8, 4, 1, 1, 1};
    case 768: return {768, 4, 8, 8, 4, 3, 1, 1};
    case 1024: return {1024, 3, 16, 8, 8, 1, 1, 1};
    case 1536: return {1536, 4, 8, 8, 8, 3, 1, 1};
    case 2048: return {2048, 3, 16, 16, 8, 1, 1, 1};
    default: return {0, 0, 1, 1, 1, 1, 1, 1};
  }
}

// the schedule of length n in this translation unit's set (set 1 falls back to
// the default for lengths without an alternative)
__host__ __device__ constexpr Sched sched_for(int n) {
#if PWF_SCHED_VARIANT == 1
  return sched_alt(n).s > 0 ? sched_alt(n) : sched_default(n);
#else
  return sched_default(n);
#endif
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// elements per thread: lcm of the radices
__host__ __device__ constexpr int ept_for(int n) {
  Sched s = sched_for(n);
  int e = 1;
  for (int i = 0; i < s.s; i++) e = lcm_c(e, s.r(i));
  return e;
}
__host__ __device__ constexpr int tpf_for(int n) { return n / ept_for(n); }

// radix of stage k of the transform with direction DIR
__host__ __device__ constexpr int stage_radix(int n, int dir, int k) {
  Sched s = sched_for(n);
  return dir == FWD ? s.r(k) : s.r(s.s - 1 - k);
}
// product of the radices before stage k
__host__ __device__ constexpr int stage_ns(int n, int dir, int k) {
  int p = 1;
  for (int i = 0; i < k; i++) p *= stage_radix(n, dir, i);
  return p;
}
// twiddle-table offset of stage k (stage 0 needs none)
__host__ __device__ constexpr int stage_twoff(int n, int dir, int k) {
  int off = 0;
  for (int i = 1; i < k; i++) off += (stage_radix(n, dir, i) - 1) * stage_ns(n, dir, i);
  return off;
}
__host__ __device__ constexpr int twiddle_len(int n, int dir) { return stage_twoff(n, dir, sched_for(n).s); }

// ---------------------------------------------------------------------------
// shared-memory layouts
// ---------------------------------------------------------------------------
// one transform per row; one padding slot per 16 (breaks the stride-R
// bank pattern of the first stage's writes). The TPF threads of one row are
// the only ones that touch it, so a stage barrier covers just them: a named
// barrier (id 1 + row) when they span several warps, a warp barrier when the
// row fits in one warp (NT = threads of the block).
template <int TPF, int NT, bool TWS = false>
struct RowLayout {
  static constexpr bool kTwShared = TWS;  // the twiddle table handed to the transforms is in shared memory
  float2* base;
  int bar;
  __device__ __forceinline__ float2& operator[](int p) const { return base[p + (p >> 4)]; }
  __device__ __forceinline__ void sync() const {
    if constexpr (TPF > 32) {
      asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "n"(TPF) : "memory");
    } else if constexpr (NT >= 32) {
      __syncwarp();
    } else {
      __syncwarp((1u << NT) - 1u);
    }
  }
};
__host__ __device__ constexpr int row_smem_len(int n) { return n + n / 16; }

// C transforms interleaved: element p of column c at row(p)*C + c. With 8 (4)
// columns a row covers half (a quarter) of the banks, and the first stage of a
// transform writes rows b*R0 + r, which for the consecutive b of a warp all
// start on the same bank. One empty row after every 16 (row(p) = p + p/16)
// spreads those rows evenly for R0 = 16 and R0 = 8, while the aligned groups
// of consecutive rows of every other access stay contiguous.
__host__ __device__ constexpr int col_pad_rows(int c) { return (c == 8 || c == 4) ? 1 : 0; }
__host__ __device__ constexpr int col_row(int p, int c) { return col_pad_rows(c) ? p + (p >> 4) : p; }
__host__ __device__ constexpr int col_tile_rows(int n, int c) { return col_pad_rows(c) ? n + n / 16 : n; }
template <int C>
struct ColLayout {
  float2* base;  // already offset by c
  __device__ __forceinline__ float2& operator[](int p) const { return base[col_row(p, C) * C]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// ---------------------------------------------------------------------------
// Stockham stages
// ---------------------------------------------------------------------------
// Twiddle W^(r k) of a radix-R stage (table entry (r - 1) NS + k of the stage
// at offset OFF). Every entry is read from the table, which holds all R - 1
// powers rounded once from double precision. Forming the odd powers as
// products of two power-of-two entries instead saves table reads but doubles
// their rounding error, and that error is the same in every row and column of
// a field: on smooth objects it adds up coherently in the lowest spatial
// frequencies of the modelled intensity. PWF_TWIDDLE_PRODUCTS restores the
// products (for measurement).
// layouts that say so take their twiddle table from shared memory (a plain
// load); every other table is global and read through the read-only path
template <class L, class = void>
struct tw_in_smem {
  static constexpr bool value = false;
};
template <class L>
struct tw_in_smem<L, std::void_t<decltype(L::kTwShared)>> {
  static constexpr bool value = L::kTwShared;
};

template <int R, bool TWS = false>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int off, int ns, int k, int r,
                                          const float2 (&w)[R]) {
#ifdef PWF_TWIDDLE_PRODUCTS
  if ((r & (r - 1)) != 0 && R != 3) {
    const int hi = r >= 16 ? 16 : r >= 8 ? 8 : r >= 4 ? 4 : 2;
    return cmul(w[hi], w[r - hi]);
  }
#else
  (void)w;
#endif
  if constexpr (TWS) return tw[off + (r - 1) * ns + k];
  else return __ldg(&tw[off + (r - 1) * ns + k]);
}

// Runs stages [K, S) of the length-N transform with direction DIR on the slot
// registers v. Before the call, v holds the inputs of stage K in slot order of
// its radix (for K = 0, the transform's input). After it, v holds the outputs
// of the last stage in slot order of the last radix. The layout's barrier
// (sm.sync(): every thread that shares the buffer) is issued before the first
// shared-memory write and after every write phase, so the caller needs no
// barrier around it.
template <int N, int DIR, int K, class L>
__device__ __forceinline__ void fft_stages(float2 (&v)[ept_for(N)], const L& sm, int t,
                                           const float2* __restrict__ tw) {
  constexpr Sched S = sched_for(N);
  constexpr int EPT = ept_for(N);
  constexpr int TPF = tpf_for(N);
  constexpr int R = stage_radix(N, DIR, K);
  constexpr int NS = stage_ns(N, DIR, K);
  constexpr int NB = EPT / R;
  constexpr bool LAST = (K + 1 == S.s);
  static_assert(EPT % R == 0, "radix must divide the per-thread count");

  if constexpr (K > 0) {
    constexpr int OFF = stage_twoff(N, DIR, K);
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = t + i * TPF;
#pragma unroll
      for (int r = 0; r < R; r++) v[i * R + r] = sm[b + r * (N / R)];
    }
    if constexpr (!LAST) sm.sync();  // reads of this stage precede its writes
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = t + i * TPF;
      const int k = b % NS;
      // W^(r k) for r = 1..R-1, each read from the table (computed in double
      // precision, rounded once)
      float2 w[R];
#pragma unroll
      for (int r = 1; r < R; r++) w[r] = twiddle<R, tw_in_smem<L>::value>(tw, OFF, NS, k, r, w);
#pragma unroll
      for (int r = 1; r < R; r++) v[i * R + r] = cmul(v[i * R + r], w[r]);
      dft<R, DIR>(&v[i * R]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NB; i++) dft<R, DIR>(&v[i * R]);
  }

  if constexpr (!LAST) {
    if constexpr (K == 0) sm.sync();  // earlier readers of the buffer are done
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = t + i * TPF;
      const int k = b % NS;
      const int base = (b / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) sm[base + r * NS] = v[i * R + r];
    }
    sm.sync();
    fft_stages<N, DIR, K + 1, L>(v, sm, t, tw);
  }
}

template <int N, int DIR, class L>
__device__ __forceinline__ void fft_run(float2 (&v)[ept_for(N)], const L& sm, int t,
                                        const float2* __restrict__ tw) {
  fft_stages<N, DIR, 0, L>(v, sm, t, tw);
}

// Two interleaved columns per thread (columns c and c + 1 of a ColLayout tile,
// c even): the same stages on two transforms that share every index, twiddle
// and barrier, with one 16-byte shared access per element pair.
template <int C>
struct ColPairLayout {
  float2* base;  // offset by the even column c
  __device__ __forceinline__ float4& operator[](int p) const {
    return *reinterpret_cast<float4*>(base + col_row(p, C) * C);
  }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
// The same without the padding rows: the dense [N][C] tile a TMA box copy
// writes (the first stage's stride-R writes then meet twice the bank
// conflicts of the padded layout; the other accesses stay conflict-free).
template <int C>
struct ColPairLayoutDense {
  float2* base;  // offset by the even column c
  __device__ __forceinline__ float4& operator[](int p) const { return *reinterpret_cast<float4*>(base + p * C); }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// L: a layout whose operator[] gives the float4 of element p of the pair
// (ColPairLayout, or the unpadded ColPairLayoutDense of TMA-filled tiles).
template <int N, int DIR, int K, class L>
__device__ __forceinline__ void fft_stages2(float2 (&v)[ept_for(N)], float2 (&u)[ept_for(N)],
                                            const L& sm, int t, const float2* __restrict__ tw) {
  constexpr Sched S = sched_for(N);
  constexpr int EPT = ept_for(N);
  constexpr int TPF = tpf_for(N);
  constexpr int R = stage_radix(N, DIR, K);
  constexpr int NS = stage_ns(N, DIR, K);
  constexpr int NB = EPT / R;
  constexpr bool LAST = (K + 1 == S.s);

  if constexpr (K > 0) {
    constexpr int OFF = stage_twoff(N, DIR, K);
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = t + i * TPF;
#pragma unroll
      for (int r = 0; r < R; r++) {
        const float4 q = sm[b + r * (N / R)];
        v[i * R + r] = make_float2(q.x, q.y);
        u[i * R + r] = make_float2(q.z, q.w);
      }
    }
    if constexpr (!LAST) sm.sync();
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = t + i * TPF;
      const int k = b % NS;
      float2 w[R];
#pragma unroll
      for (int r = 1; r < R; r++) w[r] = twiddle<R, tw_in_smem<L>::value>(tw, OFF, NS, k, r, w);
#pragma unroll
      for (int r = 1; r < R; r++) {
        v[i * R + r] = cmul(v[i * R + r], w[r]);
        u[i * R + r] = cmul(u[i * R + r], w[r]);
      }
      dft<R, DIR>(&v[i * R]);
      dft<R, DIR>(&u[i * R]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NB; i++) {
      dft<R, DIR>(&v[i * R]);
      dft<R, DIR>(&u[i * R]);
    }
  }

  if constexpr (!LAST) {
    if constexpr (K == 0) sm.sync();
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int b = t + i * TPF;
      const int k = b % NS;
      const int base = (b / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) {
        const float2 a = v[i * R + r], c = u[i * R + r];
        sm[base + r * NS] = make_float4(a.x, a.y, c.x, c.y);
      }
    }
    sm.sync();
    fft_stages2<N, DIR, K + 1, L>(v, u, sm, t, tw);
  }
}

template <int N, int DIR, class L>
__device__ __forceinline__ void fft_run2(float2 (&v)[ept_for(N)], float2 (&u)[ept_for(N)],
                                         const L& sm, int t, const float2* __restrict__ tw) {
  fft_stages2<N, DIR, 0, L>(v, u, sm, t, tw);
}

// radix of the slot layout at the start / end of a transform
template <int N, int DIR>
__host__ __device__ constexpr int first_radix() { return stage_radix(N, DIR, 0); }
template <int N, int DIR>
__host__ __device__ constexpr int last_radix() { return stage_radix(N, DIR, sched_for(N).s - 1); }

// element index of slot j (= i*R + r) for radix R
template <int N, int R>
__device__ __forceinline__ int slot_index(int t, int j) {
  constexpr int TPF = tpf_for(N);
  return t + (j / R) * TPF + (j % R) * (N / R);
}

}  // namespace PWF_KNS
}  // namespace pwf
