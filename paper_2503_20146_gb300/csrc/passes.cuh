// Row and column passes of the fused PWF iteration.
//
// A Filter of Algorithm S2, F^-1{F{x} W}, is split into a row pass (1-D
// transforms along x, contiguous) and a column pass (1-D transforms along y,
// stride nx). Because W is applied on the full 2-D spectrum, one column pass
// does "column FFT -> multiply by W(kx, ky) -> column IFFT" with the product
// in registers; and because a row IFFT of one Filter is followed by the row
// FFT of the next, one row pass does "row IFFT -> the point-wise step of
// Algorithm S1/S2 between the two Filters -> row FFT". Each pass reads and
// writes each field once.
//
// Every pass is in place on its primary buffer: a CTA owns whole rows (row
// pass) or whole columns (column pass) of the field it transforms.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "fft.cuh"
#include "pass_types.h"

namespace pwf {
inline namespace PWF_KNS {

// ---------------------------------------------------------------------------
// launch shapes
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int rows_for(int n) {
  int r = 256 / tpf_for(n);
  return r < 1 ? 1 : (r > 16 ? 16 : r);
}
__host__ __device__ constexpr int row_threads(int n) { return rows_for(n) * tpf_for(n); }
__host__ __device__ constexpr size_t row_smem_bytes(int n) {
  return (size_t)rows_for(n) * row_smem_len(n) * sizeof(float2);
}




// Barrier of the two rows 2y', 2y' + 1 of a row-pass CTA (the packed passes):
// the warp when both fit in one, else named barrier 8 + pair over their
// 2 TPF threads (rows use ids 1..4 only when TPF > 32, so these stay clear).
// With a whole warp or more per row, the packed passes give the pair's one
// transform of the packed row to the even row alone (the odd row hands over
// or takes its half through shared memory); with smaller rows both rows of a
// warp run it, so that every warp-wide barrier sees all its lanes.
template <int N>
__host__ __device__ constexpr bool pk_split_rows() { return tpf_for(N) >= 32; }

template <int N>
__device__ __forceinline__ void pair_sync() {
  constexpr int TPF = tpf_for(N), NT = row_threads(N);
  if constexpr (2 * TPF <= 32) {
    if constexpr (NT >= 32) __syncwarp();
    else __syncwarp((1u << NT) - 1u);
  } else {
    asm volatile("bar.sync %0, %1;\n" ::"r"(8 + (int)(threadIdx.x / (2 * TPF))), "n"(2 * TPF) : "memory");
  }
}

template <int OP>
struct RowT {
  static constexpr bool ifft_in = !(OP == ROW_EXP_FFT || OP == ROW_REAL_FFT || OP == ROW_FFT || OP == ROW_MODE_VG);
  static constexpr bool fft_out = !(OP == ROW_IFFT || OP == ROW_INTENSITY_OUT || OP == ROW_REAL_OUT ||
                                    OP == ROW_GRAD_OUT || OP == ROW_NESTEROV || OP == ROW_MODE_INT);
  static constexpr int nred = (OP == ROW_RESID || OP == ROW_COH_RESID) ? 1
                              : (OP == ROW_NESTEROV_FFT || OP == ROW_NESTEROV) ? 5 : 0;
};

// A projection a pass leaves alone: retired by the stopping rule, or, in
// bounds-checked builds (PWF_BOUNDS_CHECK), outside the plan's batch, which
// also records PWF_ERR_BOUNDS (8) in the status word before any access.
__device__ __forceinline__ bool skip_proj(const PassArgs& a, int proj) {
#ifdef PWF_BOUNDS_CHECK
  if (proj < 0 || proj >= a.B) {
    if (a.kstatus != nullptr) atomicCAS(a.kstatus, 0, 8);
    return true;
  }
#endif
  return a.active != nullptr && a.active[proj] == 0;
}

// Programmatic dependent launch. A pass launched with the programmatic
// stream-serialization attribute is scheduled as soon as the CTAs of the pass
// before it have exited, without waiting for that grid's completion to be
// processed; it waits here until that pass has completed and its writes are
// visible. No pass signals its dependents early: resident CTAs of the next
// pass waiting beside the running one measured slower at 512^2 and above.
// Launched without the attribute, the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch of a pass, with the programmatic attribute when pdl is set.
template <class... P, class... A>
cudaError_t launch_pass(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int pdl, A&&... args) {
  if (!pdl) {
    k<<<grid, block, smem, s>>>(static_cast<A&&>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// exp(z) for complex z. The phase z.y is reduced to [-pi, pi] by Cody and
// Waite's two-constant scheme: C1 = float(2 pi), C2 = float(2 pi - C1), so
// C1 + C2 is 2 pi to within 2^-47, and an FMA per product leaves the reduced
// phase within half an ulp plus k 2^-47 after k turns. On [-pi, pi] the
// hardware sine and cosine are accurate to 2^-21.4 absolute; the modulus uses
// the hardware exponential (a few ulp for |z.x| of order 1).
__device__ __forceinline__ float2 cexpf2(float2 z) {
  constexpr float kInv2Pi = 0.159154943091895336f;
  constexpr float kC1 = 6.28318548202514648f;
  constexpr float kC2 = -1.74845553146951715e-07f;
  const float k = rintf(z.y * kInv2Pi);
  const float r = fmaf(-k, kC2, fmaf(-k, kC1, z.y));
  float s, c;
  __sincosf(r, &s, &c);
  const float m = __expf(z.x);
  return make_float2(m * c, m * s);
}

// exp(z) to about one ulp, for the object field x = exp(psi) that enters the
// forward model and the gradient. The phase is reduced to [-pi, pi] by the same
// two-constant Cody-Waite step as cexpf2 (so that the library sincosf stays on
// its short-argument path), and the library sincosf and expf give the rest.
// The hardware approximations of cexpf2 are 2^-21.4 absolute on the phase and
// a few ulp on the modulus; both errors are smooth functions of psi, so over a
// smooth object they add up coherently in the lowest spatial frequencies of
// the modelled intensity, where the preconditioner of Eq. (11) amplifies them
// by up to N^2. cexpf2 stays where its errors cancel: the correlation sums.
__device__ __forceinline__ float2 cexpf_acc(float2 z) {
  constexpr float kInv2Pi = 0.159154943091895336f;
  constexpr float kC1 = 6.28318548202514648f;
  constexpr float kC2 = -1.74845553146951715e-07f;
  const float k = rintf(z.y * kInv2Pi);
  const float r = fmaf(-k, kC2, fmaf(-k, kC1, z.y));
  float s, c;
  sincosf(r, &s, &c);
  const float m = expf(z.x);
  return make_float2(m * c, m * s);
}

// Block-wide sum of NR thread partials into acc[proj*NACC + first + k] (float64).
template <int NR>
__device__ __forceinline__ void block_reduce_add(const float (&part)[5], double* acc, int first,
                                                 float2* smem_scratch) {
  double* sh = reinterpret_cast<double*>(smem_scratch);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  // blocks of 16 threads (length-16 transforms) fill half a warp
  const int width = blockDim.x < 32 ? (int)blockDim.x : 32;
  const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
  __syncthreads();  // the scratch aliases the FFT buffer
#pragma unroll
  for (int k = 0; k < NR; k++) {
    double s = (double)part[k];
    for (int o = width >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(mask, s, o);
    if (lane == 0) sh[warp * NR + k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NR) {
    double s = 0.0;
    for (int w = 0; w < nwarps; w++) s += sh[w * NR + threadIdx.x];
    atomicAdd(&acc[first + threadIdx.x], s);
  }
}

// ---------------------------------------------------------------------------
// packed real rows
// ---------------------------------------------------------------------------
// The intensity |v|^2 and the residual field G of the IOTF form are real, so
// the row spectrum of row y has X(y, n - kx) = conj X(y, kx). The packed
// passes keep two rows in one complex row, Z(y', kx) = X(2y', kx) + i X(2y' + 1,
// kx) (the row DFT of I(2y') + i I(2y' + 1)), stored on the even row 2y' of the
// field, and the column pass rebuilds
//   X(2y', kx)     = (Z(y', kx) + conj Z(y', n - kx)) / 2,
//   X(2y' + 1, kx) = (Z(y', kx) - conj Z(y', n - kx)) / (2i)
// for kx = 0..n/2 only (the other half is the conjugate). In a packed row, bin
// kx sits at position kx for kx <= n/2 and at n/2 + (n - kx) above, so that
// the bins kx and n - kx of an aligned pair of columns sit in two aligned
// pairs of positions n/2 apart (bins 0 and n/2 pair with each other).
template <int N>
__device__ __forceinline__ int pk_pos(int kx) {
  return kx <= N / 2 ? kx : 3 * N / 2 - kx;
}

// ---------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------
// One row of a row pass: thread t of the TPF threads that own row `row`
// (global row index over the batch) with the row's shared-memory layout sm.
// The thread's partial sums of the pass's reductions are added to part; the
// caller reduces them. Every thread of the row must call this.
template <int N, int OP, class L>
__device__ __forceinline__ void row_body(const PassArgs& a, long long row, int t, const L& sm, float (&part)[5]) {
  constexpr int EPT = ept_for(N);
  constexpr int RS = first_radix<N, FWD>();  // slot radix of real-space data
  constexpr int RK = last_radix<N, FWD>();   // slot radix of spectra
  using T = RowT<OP>;
  const int proj = (int)(row / a.ny);
  const int yrow = (int)(row - (long long)proj * a.ny);
  (void)proj;
  const size_t rb = (size_t)row * N;
  float2 v[EPT];

  // Pull this row's side inputs into L2 while the first transform runs.
  if (t == 0) {
    if constexpr (OP == ROW_MUL_T || OP == ROW_GRADT) l2_prefetch(a.t + (size_t)yrow * N, N * sizeof(float2));
    if constexpr (OP == ROW_GRADT) l2_prefetch(a.u1 + rb, N * sizeof(float2));
    if constexpr (OP == ROW_MODE_INT) {
      if (a.accumulate) l2_prefetch(a.f_out + rb, N * sizeof(float));
    }
    if constexpr (OP == ROW_MUL_V || OP == ROW_MUL_V_PK) l2_prefetch(a.v + rb, N * sizeof(float2));
    if constexpr (OP == ROW_RESID || OP == ROW_COH_RESID || OP == ROW_COH_VJP) l2_prefetch(a.y + rb, N * sizeof(float));
    if constexpr (OP == ROW_GRAD_PACK || OP == ROW_GRAD_OUT) l2_prefetch(a.psi + rb, N * sizeof(float2));
    if constexpr (OP == ROW_NESTEROV_FFT || OP == ROW_NESTEROV) {
      l2_prefetch(a.psi + rb, N * sizeof(float2));
      l2_prefetch(a.phi + rb, N * sizeof(float2));
      l2_prefetch(a.reg + rb, N * sizeof(float));
    }
  }

  // ---- input ----
  if constexpr (OP == ROW_MUL_V_PK) {
    // the inverse transform of packed row y' (stored on the even row) is
    // G(2y') + i G(2y' + 1)
    const bool odd = (yrow & 1) != 0;
    if constexpr (pk_split_rows<N>()) {
      // the even row transforms it and hands Im over to the odd row
      float* own = reinterpret_cast<float*>(sm.base);  // the row buffers as plain float arrays
      const float* other = reinterpret_cast<const float*>(sm.base - row_smem_len(N));
      if (!odd) {
#pragma unroll
        for (int j = 0; j < EPT; j++) v[j] = a.in[rb + pk_pos<N>(slot_index<N, RK>(t, j))];
        fft_run<N, INV>(v, sm, t, a.tw_inv);
      }
      pair_sync<N>();  // the inverse transform's last reads of the even buffer are done
      if (!odd) {
#pragma unroll
        for (int j = 0; j < EPT; j++) own[slot_index<N, RS>(t, j)] = v[j].y;
      }
      pair_sync<N>();
      if (odd) {
#pragma unroll
        for (int j = 0; j < EPT; j++) v[j] = make_float2(other[slot_index<N, RS>(t, j)], 0.f);
      }
      pair_sync<N>();  // the odd row's reads precede the even row's forward transform
    } else {
      // both rows of the pair read and transform it
      const size_t rbe = rb - (size_t)(yrow & 1) * N;
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = a.in[rbe + pk_pos<N>(slot_index<N, RK>(t, j))];
      pair_sync<N>();  // every read of the even row precedes that row's output
      fft_run<N, INV>(v, sm, t, a.tw_inv);
      if (odd) {
#pragma unroll
        for (int j = 0; j < EPT; j++) v[j].x = v[j].y;
      }
    }
  } else if constexpr (T::ifft_in) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[rb + slot_index<N, RK>(t, j)];
    fft_run<N, INV>(v, sm, t, a.tw_inv);
  } else if constexpr (OP == ROW_EXP_FFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cexpf_acc(a.psi[rb + slot_index<N, RS>(t, j)]);
  } else if constexpr (OP == ROW_REAL_FFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = make_float2(a.y[rb + slot_index<N, RS>(t, j)], 0.f);
  } else if constexpr (OP == ROW_MODE_VG) {
    // G (real, passed as y) times the stored detector field of this mode
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      v[j] = cscale(a.v[rb + x], a.y[rb + x]);
    }
  } else {  // ROW_FFT
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[rb + slot_index<N, RS>(t, j)];
  }

  // ---- point-wise step in real space (slots of radix RS) ----
  if constexpr (OP == ROW_IFFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) a.out[rb + slot_index<N, RS>(t, j)] = v[j];
  } else if constexpr (OP == ROW_MUL_T) {
    const size_t tb = (size_t)yrow * N;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      if (a.u1 != nullptr) a.u1[rb + x] = v[j];
      const float2 tt = __ldg(&a.t[tb + x]);
      v[j] = a.conj_t ? cmulc(v[j], tt) : cmul(v[j], tt);
    }
  } else if constexpr (OP == ROW_INTENSITY) {
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      if (a.v != nullptr) a.v[rb + x] = v[j];
      v[j] = make_float2(cabs2(v[j]), 0.f);
    }
  } else if constexpr (OP == ROW_INTENSITY_PK) {
    // I = |v|^2 of this row and of its partner row of the pair (the rows of a
    // CTA come in pairs 2y', 2y' + 1), packed as z = I(2y') + i I(2y' + 1) for
    // one forward transform: the even row's alone where rows span whole warps
    // (the odd row hands its intensities over), else both rows', each storing
    // half of it
    const bool odd = (yrow & 1) != 0;
    float* own = reinterpret_cast<float*>(sm.base);  // the row buffers as plain float arrays
    const float* other = reinterpret_cast<const float*>(sm.base + (odd ? -row_smem_len(N) : row_smem_len(N)));
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      if (a.v != nullptr) a.v[rb + slot_index<N, RS>(t, j)] = v[j];
      v[j].x = cabs2(v[j]);
    }
    pair_sync<N>();  // the inverse transforms' last reads of both buffers are done
    if (odd || !pk_split_rows<N>()) {
#pragma unroll
      for (int j = 0; j < EPT; j++) own[slot_index<N, RS>(t, j)] = v[j].x;
    }
    pair_sync<N>();
    if (!odd || !pk_split_rows<N>()) {
#pragma unroll
      for (int j = 0; j < EPT; j++) {
        const float ip = other[slot_index<N, RS>(t, j)];
        v[j] = odd ? make_float2(ip, v[j].x) : make_float2(v[j].x, ip);
      }
    }
    if constexpr (!pk_split_rows<N>()) pair_sync<N>();  // the partner's reads precede the forward transforms' writes
  } else if constexpr (OP == ROW_MUL_V_PK) {
    // G of this row (moved to .x above)
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cscale(a.v[rb + slot_index<N, RS>(t, j)], v[j].x);
  } else if constexpr (OP == ROW_INTENSITY_OUT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) a.f_out[rb + slot_index<N, RS>(t, j)] = cabs2(v[j]);
  } else if constexpr (OP == ROW_REAL_OUT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) a.f_out[rb + slot_index<N, RS>(t, j)] = v[j].x;
  } else if constexpr (OP == ROW_RESID) {
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const float e = a.y[rb + slot_index<N, RS>(t, j)] - v[j].x;
      part[0] = fmaf(e, e, part[0]);
      v[j] = make_float2(-e, 0.f);
    }
  } else if constexpr (OP == ROW_COH_RESID) {
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const float e = a.y[rb + slot_index<N, RS>(t, j)] - cabs2(v[j]);
      part[0] = fmaf(e, e, part[0]);
      v[j] = cscale(v[j], -e);
    }
  } else if constexpr (OP == ROW_COH_VJP) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cscale(v[j], a.y[rb + slot_index<N, RS>(t, j)]);
  } else if constexpr (OP == ROW_MUL_V) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cscale(a.v[rb + slot_index<N, RS>(t, j)], v[j].x);
  } else if constexpr (OP == ROW_GRAD_OUT) {
    const float s = a.div_maxt2 ? a.gscale / *a.maxt2 : a.gscale;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 xx = cexpf_acc(a.psi[rb + x]);
      a.g_out[rb + x] = cscale(cmulc(v[j], xx), s);
    }
  } else if constexpr (OP == ROW_GRAD_PACK) {
    // g = conj(exp psi) g1 / max|t|^2: Re g out, Im g stays in v for the
    // first row FFT; alpha o psi is formed after it from a second read of psi
    const float s = 1.0f / *a.maxt2;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 g = cscale(cmulc(v[j], cexpf_acc(a.psi[rb + x])), s);
      a.reg[rb + x] = g.x;
      v[j] = make_float2(g.y, 0.f);
    }
  } else if constexpr (OP == ROW_NESTEROV_FFT || OP == ROW_NESTEROV) {
    const float beta = *a.beta;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 p = a.psi[rb + x];
      const float2 fp = a.phi[rb + x];
      const float gr = a.reg[rb + x];
      // total direction: preconditioned g plus the regularizer term = Re g + z
      const float2 g = make_float2(gr + v[j].x, v[j].y);
      const float2 f = make_float2(fmaf(-a.eta, g.x, p.x), fmaf(-a.eta, g.y, p.y));
      const float2 pn = make_float2(fmaf(beta, f.x - fp.x, f.x), fmaf(beta, f.y - fp.y, f.y));
      a.phi[rb + x] = f;
      a.psi_out[rb + x] = pn;
      const float2 xo = cexpf2(p), xn = cexpf_acc(pn);
      const float2 c = cmulc(xn, xo);
      part[0] += c.x;
      part[1] += c.y;
      part[2] += cabs2(xn);
      part[3] += cabs2(xo);
      v[j] = xn;
    }
  } else if constexpr (OP == ROW_GRADT) {
    const float w2 = 2.0f * a.mode_w;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 u = a.u1[rb + x];
      float2 gt = cscale(cmulc(v[j], u), w2);
      if (a.accumulate) gt = cadd(gt, a.gt_scratch[rb + x]);
      a.gt_scratch[rb + x] = gt;
      v[j] = cmulc(v[j], __ldg(&a.t[(size_t)yrow * N + x]));
    }
  } else if constexpr (OP == ROW_MODE_INT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      if (a.v != nullptr) a.v[rb + x] = v[j];
      float fi = a.mode_w * cabs2(v[j]);
      if (a.accumulate) fi += a.f_out[rb + x];
      a.f_out[rb + x] = fi;
    }
  }

  // ---- output ----
  if constexpr (OP == ROW_GRAD_PACK) {
    fft_run<N, FWD>(v, sm, t, a.tw_fwd);
#pragma unroll
    for (int j = 0; j < EPT; j++) a.aux[rb + slot_index<N, RK>(t, j)] = v[j];
    // The second transform runs on an opaque copy of the thread index and
    // buffer pointer: left to itself the compiler shares the two transforms'
    // address arithmetic, keeps it live through the first one and spills.
    int t2;
    float2* b2;
    asm volatile("mov.b32 %0, %1;" : "=r"(t2) : "r"(t));
    asm volatile("mov.b64 %0, %1;" : "=l"(b2) : "l"(sm.base));
    L sm2 = sm;
    sm2.base = b2;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const float2 p = a.psi[rb + slot_index<N, RS>(t2, j)];
      v[j] = make_float2(a.alpha_re * p.x, a.alpha_im * p.y);
    }
    fft_run<N, FWD>(v, sm2, t2, a.tw_fwd);
#pragma unroll
    for (int j = 0; j < EPT; j++) a.out[rb + slot_index<N, RK>(t2, j)] = v[j];
  } else if constexpr (OP == ROW_INTENSITY_PK) {
    const bool odd = (yrow & 1) != 0;
    if constexpr (pk_split_rows<N>()) {
      if (!odd) {  // the even row transforms z and stores the packed row on itself
        fft_run<N, FWD>(v, sm, t, a.tw_fwd);
#pragma unroll
        for (int j = 0; j < EPT; j++) a.out[rb + pk_pos<N>(slot_index<N, RK>(t, j))] = v[j];
      }
    } else {
      fft_run<N, FWD>(v, sm, t, a.tw_fwd);
      const size_t rbe = rb - (odd ? (size_t)N : 0);
#pragma unroll
      for (int j = 0; j < EPT; j++)
        if ((j < EPT / 2) != odd) a.out[rbe + pk_pos<N>(slot_index<N, RK>(t, j))] = v[j];
    }
  } else if constexpr (T::fft_out) {
    fft_run<N, FWD>(v, sm, t, a.tw_fwd);
#pragma unroll
    for (int j = 0; j < EPT; j++) a.out[rb + slot_index<N, RK>(t, j)] = v[j];
  }
}

// Two CTAs per SM where three would make the pass spill: 32 values per
// thread, and the diffuser multiply at 24 (measured at 768^2 and 1536^2: 3.33
// -> 3.06 and 11.9 -> 11.2 ms per iteration of the K = 25 batch; the mode
// intensity pass at 24 lost more with two than it saved, so it keeps three).
__host__ __device__ constexpr int row_min_blocks(int n, int op) {
  return ept_for(n) >= 32 || (ept_for(n) >= 24 && op == ROW_MUL_T) ? 2 : 3;
}

template <int N, int OP>
__global__ void __launch_bounds__(row_threads(N), row_min_blocks(N, OP)) row_kernel(const PassArgs a) {
  pdl_wait();
  constexpr int TPF = tpf_for(N), ROWS = rows_for(N);
  using T = RowT<OP>;
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int rr = tid / TPF, t = tid - rr * TPF;
  const long long row = (long long)blockIdx.x * ROWS + rr + (long long)a.proj0 * a.ny;
  const int proj = (int)(row / a.ny);
  if (skip_proj(a, proj)) return;  // uniform per CTA (ny % ROWS == 0)
  const RowLayout<TPF, ROWS * TPF> sm{smem + rr * row_smem_len(N), 1 + rr};
  float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  row_body<N, OP>(a, row, t, sm, part);

  // ---- reductions ----
  if constexpr (T::nred == 1) {
    block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, smem);
  } else if constexpr (T::nred == 5) {
    block_reduce_add<4>(part, a.acc, proj * NACC + ACC_XR, smem);
  }
}

// ---------------------------------------------------------------------------
// column pass
// ---------------------------------------------------------------------------
// C columns of one projection per tile; thread (t, c) = (tid / C, tid % C)
// holds EPT elements of column c. The arithmetic lives in col_tile(); the two
// kernels differ only in how a tile reaches it: col_kernel reads the first
// stage's inputs straight from global memory (one tile per CTA), and
// col_kernel_pipe is persistent and copies tile k+1 into a second shared
// buffer with cp.async while tile k is transformed.
__host__ __device__ constexpr int col_threads(int n, int c) { return c * tpf_for(n); }
__host__ __device__ constexpr size_t col_smem_bytes(int n, int c) {
  return (size_t)c * col_tile_rows(n, c) * sizeof(float2);
}
__host__ __device__ constexpr size_t colp_smem_bytes(int n, int c) { return 2 * col_smem_bytes(n, c); }
__host__ __device__ constexpr int col_min_blocks(int threads, int ept = 16) {
  return ept >= 32 ? (threads >= 512 ? 1 : 2) : (threads >= 512 ? 1 : threads >= 256 ? 3 : 4);
}
// COL_PRECOND_REG holds two transforms' values per thread: at most two CTAs
// per SM so that they stay in registers
template <int OP>
__host__ __device__ constexpr int col_min_blocks_op(int threads, int ept = 16) {
  return OP == COL_PRECOND_REG && col_min_blocks(threads, ept) > 2 ? 2 : col_min_blocks(threads, ept);
}

// the filter step and the inverse transform of one tile (v holds the forward
// spectrum of the column in slots of the last forward radix)
template <int N, int OP, int S2N, class L>
__device__ __forceinline__ void col_tile_filter(const PassArgs& a, const L& sm, int t, int col,
                                                size_t base, float2 (&v)[ept_for(N)], float2 (&s2)[S2N],
                                                float (&part)[5]) {
  constexpr int EPT = ept_for(N);
  constexpr int RK = last_radix<N, FWD>();
  const size_t ld = (size_t)a.nx;
  if constexpr (OP == COL_Q) {
    const float2 qx = __ldg(&a.qx[col]);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      float2 q = cmul(qx, __ldg(&a.qy[slot_index<N, RK>(t, j)]));
      if (a.conj_q) q = cconj(q);
      v[j] = cscale(cmul(v[j], q), a.scale);
    }
  } else if constexpr (OP == COL_IOTF) {
    const float ixv = __ldg(&a.ix[col]) * a.scale;
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cscale(v[j], ixv * __ldg(&a.iy[slot_index<N, RK>(t, j)]));
  } else if constexpr (OP == COL_RESID_IOTF2) {
    const float ixv = __ldg(&a.ix[col]);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      const float w = ixv * __ldg(&a.iy[ky]);
      const float2 yh = a.yhat[base + (size_t)ky * ld];
      const float2 r = make_float2(fmaf(w, v[j].x, -yh.x), fmaf(w, v[j].y, -yh.y));
      part[0] = fmaf(r.x, r.x, fmaf(r.y, r.y, part[0]));
      v[j] = cscale(r, w * a.scale);
    }
    part[0] *= a.scale;
  } else if constexpr (OP == COL_PRECOND_REG) {
    fft_run<N, FWD>(s2, sm, t, a.tw_fwd);
    const float gx = __ldg(&a.ex[col]);
    const float u2 = __ldg(&a.u2x[col]);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      // Gamma^2 = 1 - STF = 1 - (1 + gx)(1 + gy), gx, gy = STF - 1 of each axis
      // (Eqs. (14)-(15)): both are <= 0, so the three terms do not cancel
      const float gy = __ldg(&a.ey[ky]);
      const float g2 = -fmaf(gx, gy, gx + gy);
      const float r2 = u2 + __ldg(&a.u2y[ky]);
      const float pinv = a.no_precond ? 1.0f : (r2 > 0.f ? 1.0f / r2 : 0.0f);
      // Z = Gamma^2 H + i P^-1 S
      v[j] = make_float2((g2 * v[j].x - pinv * s2[j].y) * a.scale, (g2 * v[j].y + pinv * s2[j].x) * a.scale);
    }
  }
}

// One column of a column pass: thread t of the TPF threads that own column
// `col` of projection `proj`, reading the first stage's inputs straight from
// global memory, with the column's shared-memory layout sm (interleaved with
// other columns or one column alone). Partial sums go to part.
template <int N, int OP, class L>
__device__ __forceinline__ void col_body(const PassArgs& a, int proj, int col, int t, const L& sm,
                                         float (&part)[5]) {
  constexpr int EPT = ept_for(N);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  const size_t base = (size_t)proj * a.ny * a.nx + col;
  const size_t ld = (size_t)a.nx;
  float2 v[EPT];
  float2 s2[(OP == COL_PRECOND_REG) ? EPT : 1];

  if constexpr (OP == COL_IFFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cscale(a.in[base + (size_t)slot_index<N, RK>(t, j) * ld], a.scale);
  } else {
    if constexpr (OP == COL_PRECOND_REG) {
#pragma unroll
      for (int j = 0; j < EPT; j++) s2[j] = a.aux_in[base + (size_t)slot_index<N, RS>(t, j) * ld];
    }
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[base + (size_t)slot_index<N, RS>(t, j) * ld];
    fft_run<N, FWD>(v, sm, t, a.tw_fwd);
    if constexpr (OP == COL_FFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) a.out[base + (size_t)slot_index<N, RK>(t, j) * ld] = v[j];
      return;
    }
    col_tile_filter<N, OP>(a, sm, t, col, base, v, s2, part);
  }
  fft_run<N, INV>(v, sm, t, a.tw_inv);
#pragma unroll
  for (int j = 0; j < EPT; j++) a.out[base + (size_t)slot_index<N, RS>(t, j) * ld] = v[j];
}

template <int N, int OP, int C>
__global__ void __launch_bounds__(col_threads(N, C), col_min_blocks_op<OP>(col_threads(N, C), ept_for(N)))
    col_kernel(const PassArgs a) {
  pdl_wait();
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;
  const int proj = blockIdx.y + a.proj0;
  const int col = blockIdx.x * C + c;
  if (skip_proj(a, proj)) return;
  const ColLayout<C> sm{smem + c};
  float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  col_body<N, OP>(a, proj, col, t, sm, part);
  if constexpr (OP == COL_RESID_IOTF2) block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, smem);
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Persistent, double-buffered: the CTA walks tiles blockIdx.x, +gridDim.x, ...
// The copy of tile k+1 is one cp.async commit group (16-byte chunks); the wait
// for tile k is cp.async.wait_group 1, which returns once that group landed.
template <int N, int OP, int C>
__global__ void __launch_bounds__(col_threads(N, C), col_min_blocks_op<OP>(col_threads(N, C), ept_for(N)))
    col_kernel_pipe(const PassArgs a, int nproj) {
  pdl_wait();
  constexpr int EPT = ept_for(N);
  constexpr int NT = col_threads(N, C);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  constexpr int CHUNKS = N * C / 2;  // 16-byte chunks per tile
  constexpr int TILE = C * col_tile_rows(N, C);
  static_assert(CHUNKS % NT == 0, "tile chunks must divide evenly");
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;
  const int tiles_per_proj = a.nx / C;
  const int ntiles = nproj * tiles_per_proj;
  const size_t ld = (size_t)a.nx;

  auto tile_base = [&](int tile, int& proj, int& col0) -> size_t {
    proj = a.proj0 + tile / tiles_per_proj;
    col0 = (tile % tiles_per_proj) * C;
    return (size_t)proj * a.ny * a.nx + col0;
  };
  auto prefetch = [&](int tile, float2* buf) {
    int proj, col0;
    const size_t b = tile_base(tile, proj, col0);
    if (skip_proj(a, proj)) return;
#pragma unroll
    for (int k = 0; k < CHUNKS / NT; k++) {
      const int q = tid + k * NT;  // chunk q: row q / (C/2), column pair q % (C/2)
      const int row = q / (C / 2), pr = q % (C / 2);
      cp_async16(buf + col_row(row, C) * C + 2 * pr, a.in + b + (size_t)row * ld + 2 * pr);
    }
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, smem);
  cp_async_commit();
  for (int k = 0; tile < ntiles; k++, tile += gridDim.x) {
    float2* cur = smem + (k & 1) * TILE;
    float2* nxt = smem + ((k + 1) & 1) * TILE;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    int proj, col0;
    const size_t base = tile_base(tile, proj, col0) + c;
    const int col = col0 + c;
    if (skip_proj(a, proj)) {
      __syncthreads();
      continue;
    }
    const ColLayout<C> sm{cur + c};
    float2 v[EPT];
    float2 s2[(OP == COL_PRECOND_REG) ? EPT : 1];
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};

    if constexpr (OP == COL_IFFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = cscale(sm[slot_index<N, RK>(t, j)], a.scale);
    } else {
      if constexpr (OP == COL_PRECOND_REG) {
#pragma unroll
        for (int j = 0; j < EPT; j++) s2[j] = a.aux_in[base + (size_t)slot_index<N, RS>(t, j) * ld];
      }
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = sm[slot_index<N, RS>(t, j)];
      fft_run<N, FWD>(v, sm, t, a.tw_fwd);
      if constexpr (OP != COL_FFT) col_tile_filter<N, OP>(a, sm, t, col, base, v, s2, part);
    }
    if constexpr (OP == COL_FFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) a.out[base + (size_t)slot_index<N, RK>(t, j) * ld] = v[j];
    } else {
      fft_run<N, INV>(v, sm, t, a.tw_inv);
#pragma unroll
      for (int j = 0; j < EPT; j++) a.out[base + (size_t)slot_index<N, RS>(t, j) * ld] = v[j];
    }
    if constexpr (OP == COL_RESID_IOTF2) block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, cur);
    __syncthreads();  // cur is refilled by the prefetch of the next-but-one tile
  }
  cp_async_wait<0>();
}

// Transposed tile: the prefetch (8-byte cp.async) stores each of the C columns
// contiguously in shared memory (column stride S, S = 4 mod 16 slots, so the
// row-major copy pattern of a warp - C columns x 32/C rows - falls on every
// bank pair exactly twice), the TPF threads of one column run its transforms
// exactly like a row pass with a barrier of their own, and the results go
// back through shared memory so that the global stores are row-major and
// coalesced. Single-input ops only.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__host__ __device__ constexpr int colt_stride(int n) {
  return row_smem_len(n) + ((4 - row_smem_len(n) % 16) + 16) % 16;
}
__host__ __device__ constexpr size_t colt_smem_bytes(int n, int c) {
  return 2 * (size_t)c * colt_stride(n) * sizeof(float2);
}

// Two columns per thread (the pair c, c + 1): tile staging as col_kernel_pipe,
// then the transforms of both columns share indices, twiddles and barriers and
// move through shared memory 16 bytes at a time. Single-input passes only.
__host__ __device__ constexpr int col2_threads(int n, int c) { return c / 2 * tpf_for(n); }
// two CTAs per SM up to 256 threads, one CTA of 512 (a wide tile, 128 registers a thread)
__host__ __device__ constexpr int col2_min_blocks(int n, int c) { return col2_threads(n, c) > 256 ? 1 : 2; }

template <int N, int OP, class P>
__device__ __forceinline__ void col_pair_filter(const PassArgs& a, int t, int col, size_t base,
                                                float2 (&v)[ept_for(N)], float2 (&u)[ept_for(N)], float (&part)[5]) {
  constexpr int EPT = ept_for(N);
  constexpr int RK = last_radix<N, FWD>();
  const size_t ld = (size_t)a.nx;
  if constexpr (OP == COL_Q) {
    float2 qa = cscale(__ldg(&a.qx[col]), a.scale), qb = cscale(__ldg(&a.qx[col + 1]), a.scale);
    if (a.conj_q) qa = cconj(qa), qb = cconj(qb);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      float2 qy = __ldg(&a.qy[slot_index<N, RK>(t, j)]);
      if (a.conj_q) qy = cconj(qy);
      v[j] = cmul(v[j], cmul(qa, qy));
      u[j] = cmul(u[j], cmul(qb, qy));
    }
  } else if constexpr (OP == COL_IOTF) {
    const float ia = __ldg(&a.ix[col]) * a.scale, ib = __ldg(&a.ix[col + 1]) * a.scale;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const float iy = __ldg(&a.iy[slot_index<N, RK>(t, j)]);
      v[j] = cscale(v[j], ia * iy);
      u[j] = cscale(u[j], ib * iy);
    }
  } else if constexpr (OP == COL_RESID_IOTF2) {
    const float ia = __ldg(&a.ix[col]), ib = __ldg(&a.ix[col + 1]);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      const float iy = __ldg(&a.iy[ky]);
      const float4 yh = *reinterpret_cast<const float4*>(a.yhat + base + (size_t)ky * ld);
      const float wa = ia * iy, wb = ib * iy;
      const float2 ra = make_float2(fmaf(wa, v[j].x, -yh.x), fmaf(wa, v[j].y, -yh.y));
      const float2 rb = make_float2(fmaf(wb, u[j].x, -yh.z), fmaf(wb, u[j].y, -yh.w));
      part[0] = fmaf(ra.x, ra.x, fmaf(ra.y, ra.y, part[0]));
      part[0] = fmaf(rb.x, rb.x, fmaf(rb.y, rb.y, part[0]));
      v[j] = cscale(ra, wa * a.scale);
      u[j] = cscale(rb, wb * a.scale);
    }
    part[0] *= a.scale;
  }
}

// rows of a tensor-map box over a column of n rows (a box dimension is at most 256)
__host__ __device__ constexpr int tma_box_rows(int n) { return n < 256 ? n : 256; }
// L2 prefetch of one box of a 3-D tensor map (a hint: no completion to wait for)
__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap* tm, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(tm), "r"(x), "r"(y), "r"(z)
               : "memory");
}

// NBUF = 2: tile k + 1 is copied while tile k is transformed (one CTA per SM
// at 8 columns); NBUF = 1: one buffer, the copy of the next tile starts after
// the current one is done, and the overlap comes from the second CTA on the SM;
// with a.l2pf, thread 0 then prefetches the next tile into L2 (a few tensor-map
// boxes), so that its copy waits on L2 rather than DRAM.
template <int N, int OP, int C, int NBUF>
__global__ void __launch_bounds__(col2_threads(N, C), col2_min_blocks(N, C))
    col_kernel_pipe2(const __grid_constant__ PassArgs a, int nproj) {
  pdl_wait();
  constexpr int EPT = ept_for(N);
  constexpr int NT = col2_threads(N, C);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  constexpr int CHUNKS = N * C / 2;  // 16-byte chunks per tile
  constexpr int TILE = C * col_tile_rows(N, C);
  static_assert(CHUNKS % NT == 0, "tile chunks must divide evenly");
  static_assert(OP != COL_PRECOND_REG, "single-input passes only");
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int c2 = tid % (C / 2), t = tid / (C / 2);
  const int tiles_per_proj = a.nx / C;
  const int ntiles = nproj * tiles_per_proj;
  const size_t ld = (size_t)a.nx;

  auto tile_base = [&](int tile, int& proj, int& col0) -> size_t {
    proj = a.proj0 + tile / tiles_per_proj;
    col0 = (tile % tiles_per_proj) * C;
    return (size_t)proj * a.ny * a.nx + col0;
  };
  auto prefetch = [&](int tile, float2* buf) {
    int proj, col0;
    const size_t b = tile_base(tile, proj, col0);
    if (skip_proj(a, proj)) return;
#pragma unroll
    for (int k = 0; k < CHUNKS / NT; k++) {
      const int q = tid + k * NT;  // chunk q: row q / (C/2), column pair q % (C/2)
      const int row = q / (C / 2), pr = q % (C / 2);
      cp_async16(buf + col_row(row, C) * C + 2 * pr, a.in + b + (size_t)row * ld + 2 * pr);
    }
  };

  int tile = blockIdx.x;
  if (NBUF == 2 && tile < ntiles) prefetch(tile, smem);
  cp_async_commit();
  for (int k = 0; tile < ntiles; k++, tile += gridDim.x) {
    float2* cur = smem + (NBUF == 2 ? (k & 1) * TILE : 0);
    if constexpr (NBUF == 2) {
      float2* nxt = smem + ((k + 1) & 1) * TILE;
      const int next = tile + gridDim.x;
      if (next < ntiles) prefetch(next, nxt);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      prefetch(tile, cur);
      cp_async_commit();
      cp_async_wait<0>();
      if (a.l2pf && tid == 0) {
        constexpr int PB = tma_box_rows(N);
        const int next = tile + gridDim.x;
        if (next < ntiles) {
          int np, nc;
          (void)tile_base(next, np, nc);
          if (!skip_proj(a, np))
#pragma unroll
            for (int k = 0; k < N / PB; k++) tma_prefetch_l2_3d(&a.tmap, 2 * nc, k * PB, np);
        }
      }
    }
    __syncthreads();

    int proj, col0;
    const size_t base = tile_base(tile, proj, col0) + 2 * c2;
    const int col = col0 + 2 * c2;
    if (skip_proj(a, proj)) {
      __syncthreads();
      continue;
    }
    const ColPairLayout<C> sm{cur + 2 * c2};
    float2 v[EPT], u[EPT];
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};

    if constexpr (OP == COL_IFFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) {
        const float4 q = sm[slot_index<N, RK>(t, j)];
        v[j] = make_float2(q.x * a.scale, q.y * a.scale);
        u[j] = make_float2(q.z * a.scale, q.w * a.scale);
      }
    } else {
#pragma unroll
      for (int j = 0; j < EPT; j++) {
        const float4 q = sm[slot_index<N, RS>(t, j)];
        v[j] = make_float2(q.x, q.y);
        u[j] = make_float2(q.z, q.w);
      }
      fft_run2<N, FWD>(v, u, sm, t, a.tw_fwd);
      if constexpr (OP != COL_FFT) col_pair_filter<N, OP, ColPairLayout<C>>(a, t, col, base, v, u, part);
    }
    if constexpr (OP == COL_FFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++)
        *reinterpret_cast<float4*>(a.out + base + (size_t)slot_index<N, RK>(t, j) * ld) =
            make_float4(v[j].x, v[j].y, u[j].x, u[j].y);
    } else {
      fft_run2<N, INV>(v, u, sm, t, a.tw_inv);
#pragma unroll
      for (int j = 0; j < EPT; j++)
        *reinterpret_cast<float4*>(a.out + base + (size_t)slot_index<N, RS>(t, j) * ld) =
            make_float4(v[j].x, v[j].y, u[j].x, u[j].y);
    }
    if constexpr (OP == COL_RESID_IOTF2) block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, cur);
    __syncthreads();  // cur is refilled by the prefetch of the next-but-one tile
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// packed residual column pass (COL_RESID_PK)
// ---------------------------------------------------------------------------
// COL_RESID_IOTF2 on the packed rows of ROW_INTENSITY_PK: a tile is C packed
// positions [c0, c0 + C) (bins kx = c0..c0 + C - 1) and the C positions nx/2
// apart that hold their mirror bins nx - kx, both halves staged by cp.async
// (16-byte chunks) into one buffer, front rows first. The threads rebuild the
// full-length columns kx, kx + 1 of the row spectrum in place in shared memory
// (every read of the packed halves before any write), transform each column
// pair, form IOTF (IOTF F{I} - F{y}) and the loss (weight 2: the mirror bin
// nx - kx carries the same sum of |.|^2), transform back and write the packed
// residual: the thread holding row 2y' the front pair G(2y') + i G(2y' + 1),
// the one holding 2y' + 1 the mirror pair conj G(2y') + i conj G(2y' + 1)
// (the partner's value comes by shuffle). Bins 0 and nx/2 are their own
// mirrors; the first lane of the first tile leaves them (its first column is
// computed and dropped) to col_kernel_pk_edge, which runs after this kernel.
// Needs the thread holding row y to hold the same slots as the one holding
// y ^ 1, C/2 lanes apart (pk_col_ok).
template <int N>
__host__ __device__ constexpr bool pk_col_ok() {
  return tpf_for(N) % 2 == 0 && (N / first_radix<N, FWD>()) % 2 == 0 && ept_for(N) % 2 == 0;
}

template <int N, int C>
__global__ void __launch_bounds__(col2_threads(N, C), col2_min_blocks(N, C)) col_kernel_pk(const PassArgs a, int nproj) {
  pdl_wait();
  constexpr int EPT = ept_for(N);
  constexpr int TPFC = tpf_for(N);      // threads per column pair
  constexpr int NT = col2_threads(N, C);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  constexpr int H = N / 2;              // packed rows
  constexpr int CHUNKS = H * C / 2;     // 16-byte chunks per half tile
  static_assert(CHUNKS % NT == 0, "half-tile chunks must divide evenly");
  static_assert(pk_col_ok<N>(), "row parity must follow the thread index");
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int c2 = tid % (C / 2), t = tid / (C / 2);
  const int hx = a.nx / 2;
  const int tiles_per_proj = hx / C;
  const int ntiles = nproj * tiles_per_proj;
  const size_t ldp = 2 * (size_t)a.nx;  // packed rows sit on the even rows of the field
  const bool odd = (t & 1) != 0;        // this thread holds the odd rows 2y' + 1
  const ColPairLayout<C> sm{smem + 2 * c2};

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int proj = a.proj0 + tile / tiles_per_proj;
    const int c0 = (tile % tiles_per_proj) * C;
    if (skip_proj(a, proj)) continue;  // uniform over the CTA
    const size_t pbase = (size_t)proj * a.ny * a.nx;
#pragma unroll
    for (int k = 0; k < 2 * CHUNKS / NT; k++) {
      const int q = tid + k * NT;
      const int half = q / CHUNKS, qq = q - half * CHUNKS;
      const int row = qq / (C / 2), pr = qq % (C / 2);
      cp_async16(smem + col_row(half * H + row, C) * C + 2 * pr,
                 a.in + pbase + (size_t)row * ldp + (half ? hx : 0) + c0 + 2 * pr);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    const int kx = c0 + 2 * c2;      // bins kx, kx + 1 (mirrors nx - kx, nx - kx - 1)
    const bool edge = kx == 0;       // bin 0 (and nx/2): col_kernel_pk_edge's
    {
      // X(2y') = (Z + conj Zm) / 2 and X(2y' + 1) = (Z - conj Zm) / (2i) of
      // both columns, from the front (Z) and mirror (Zm) rows y'
      float4 f[EPT / 2], m[EPT / 2];
#pragma unroll
      for (int k = 0; k < EPT / 2; k++) {
        f[k] = sm[t + k * TPFC];
        m[k] = sm[H + t + k * TPFC];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < EPT / 2; k++) {
        const int yp = t + k * TPFC;
        const float4 z = f[k], w = m[k];
        sm[2 * yp] = make_float4(0.5f * (z.x + w.x), 0.5f * (z.y - w.y), 0.5f * (z.z + w.z), 0.5f * (z.w - w.w));
        sm[2 * yp + 1] = make_float4(0.5f * (z.y + w.y), 0.5f * (w.x - z.x), 0.5f * (z.w + w.w), 0.5f * (w.z - z.z));
      }
      __syncthreads();
    }
    float2 v[EPT], u[EPT];
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const float4 q = sm[slot_index<N, RS>(t, j)];
      v[j] = make_float2(q.x, q.y);
      u[j] = make_float2(q.z, q.w);
    }
    fft_run2<N, FWD>(v, u, sm, t, a.tw_fwd);

    const float ia = __ldg(&a.ix[kx]), ib = __ldg(&a.ix[kx + 1]);
    const float wv = edge ? 0.f : 2.f;  // the edge lane's first column is not this kernel's
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      const float iy = __ldg(&a.iy[ky]);
      const float4 yh = *reinterpret_cast<const float4*>(a.yhat + pbase + (size_t)ky * a.nx + kx);
      const float wa = ia * iy, wb = ib * iy;
      const float2 ra = make_float2(fmaf(wa, v[j].x, -yh.x), fmaf(wa, v[j].y, -yh.y));
      const float2 rb = make_float2(fmaf(wb, u[j].x, -yh.z), fmaf(wb, u[j].y, -yh.w));
      part[0] = fmaf(wv * ra.x, ra.x, fmaf(wv * ra.y, ra.y, part[0]));
      part[0] = fmaf(2.f * rb.x, rb.x, fmaf(2.f * rb.y, rb.y, part[0]));
      v[j] = cscale(ra, wa * a.scale);
      u[j] = cscale(rb, wb * a.scale);
    }
    part[0] *= a.scale;
    fft_run2<N, INV>(v, u, sm, t, a.tw_inv);

    // packed output: rows 2y' and 2y' + 1 of a column sit C/2 lanes apart
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const float2 pv = make_float2(__shfl_xor_sync(0xffffffffu, v[j].x, C / 2), __shfl_xor_sync(0xffffffffu, v[j].y, C / 2));
      const float2 pu = make_float2(__shfl_xor_sync(0xffffffffu, u[j].x, C / 2), __shfl_xor_sync(0xffffffffu, u[j].y, C / 2));
      const float2 ve = odd ? pv : v[j], vo = odd ? v[j] : pv;
      const float2 ue = odd ? pu : u[j], uo = odd ? u[j] : pu;
      // front: G(2y') + i G(2y' + 1); mirror: conj G(2y') + i conj G(2y' + 1)
      const float4 o = odd ? make_float4(ve.x + vo.y, vo.x - ve.y, ue.x + uo.y, uo.x - ue.y)
                           : make_float4(ve.x - vo.y, ve.y + vo.x, ue.x - uo.y, ue.y + uo.x);
      float2* dst = a.out + pbase + (size_t)((t >> 1) + (slot_index<N, RS>(0, j) >> 1)) * ldp + (odd ? hx : 0) + kx;
      if (edge)
        dst[1] = make_float2(o.z, o.w);
      else
        *reinterpret_cast<float4*>(dst) = o;
    }
    block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, smem);
    __syncthreads();  // the buffer is refilled by the next tile's copy
  }
  cp_async_wait<0>();
}

// Bins 0 and nx/2 of the packed residual pass, one CTA per projection, after
// col_kernel_pk: both columns of the row spectrum are real (a real row's DC and
// Nyquist bins), so they ride as one complex column W = X0 + i Xh, rebuilt from
// packed positions 0 and nx/2 (X(2y') = Re Z(y'), X(2y' + 1) = Im Z(y')). After
// the forward transform X0^(ky) = (W^(ky) + conj W^(-ky)) / 2 and
// Xh^(ky) = (W^(ky) - conj W^(-ky)) / (2i) (through shared memory); each gets
// its own bin's IOTF and F{y}, the loss (weight 1), and the two residuals go
// back as one column g0 + i gh, whose inverse transform is G0 + i Gh (both
// real), packed again into positions 0 and nx/2.
template <int N>
__global__ void __launch_bounds__(tpf_for(N)) col_kernel_pk_edge(const PassArgs a) {
  pdl_wait();
  constexpr int EPT = ept_for(N), TPF = tpf_for(N);
  constexpr int RS = first_radix<N, FWD>(), RK = last_radix<N, FWD>();
  extern __shared__ float2 smem[];
  const int proj = a.proj0 + blockIdx.x;
  if (skip_proj(a, proj)) return;
  const int t = threadIdx.x;
  const int hx = a.nx / 2;
  const size_t pbase = (size_t)proj * a.ny * a.nx;
  const size_t ldp = 2 * (size_t)a.nx;
  const RowLayout<TPF, TPF> sm{smem, 1};
  float2 v[EPT];
#pragma unroll
  for (int j = 0; j < EPT; j++) {
    const int y = slot_index<N, RS>(t, j);
    const float2 z0 = a.in[pbase + (size_t)(y >> 1) * ldp], zh = a.in[pbase + (size_t)(y >> 1) * ldp + hx];
    v[j] = (y & 1) ? make_float2(z0.y, zh.y) : make_float2(z0.x, zh.x);
  }
  fft_run<N, FWD>(v, sm, t, a.tw_fwd);
  sm.sync();  // the transform's last reads are done
#pragma unroll
  for (int j = 0; j < EPT; j++) sm[slot_index<N, RK>(t, j)] = v[j];
  sm.sync();
  float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  const float i0 = __ldg(&a.ix[0]), ih = __ldg(&a.ix[hx]);
#pragma unroll
  for (int j = 0; j < EPT; j++) {
    const int ky = slot_index<N, RK>(t, j);
    const float2 p = v[j], q = sm[ky == 0 ? 0 : N - ky];
    const float2 x0 = make_float2(0.5f * (p.x + q.x), 0.5f * (p.y - q.y));
    const float2 xh = make_float2(0.5f * (p.y + q.y), 0.5f * (q.x - p.x));
    const float iy = __ldg(&a.iy[ky]);
    const float w0 = i0 * iy, wh = ih * iy;
    const float2 y0 = a.yhat[pbase + (size_t)ky * a.nx], yh = a.yhat[pbase + (size_t)ky * a.nx + hx];
    const float2 r0 = make_float2(fmaf(w0, x0.x, -y0.x), fmaf(w0, x0.y, -y0.y));
    const float2 rh = make_float2(fmaf(wh, xh.x, -yh.x), fmaf(wh, xh.y, -yh.y));
    part[0] = fmaf(r0.x, r0.x, fmaf(r0.y, r0.y, part[0]));
    part[0] = fmaf(rh.x, rh.x, fmaf(rh.y, rh.y, part[0]));
    const float2 g0 = cscale(r0, w0 * a.scale), gh = cscale(rh, wh * a.scale);
    v[j] = make_float2(g0.x - gh.y, g0.y + gh.x);  // g0 + i gh
  }
  part[0] *= a.scale;
  fft_run<N, INV>(v, sm, t, a.tw_inv);  // its first write waits for the reads above
  sm.sync();
#pragma unroll
  for (int j = 0; j < EPT; j++) sm[slot_index<N, RS>(t, j)] = v[j];
  sm.sync();
#pragma unroll
  for (int k = 0; k < EPT / 2; k++) {
    const int yp = t + k * TPF;
    const float2 e = sm[2 * yp], o = sm[2 * yp + 1];
    a.out[pbase + (size_t)yp * ldp] = make_float2(e.x, o.x);
    a.out[pbase + (size_t)yp * ldp + hx] = make_float2(e.y, o.y);
  }
  block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, smem);
}

// ---------------------------------------------------------------------------
// TMA-staged pair kernel
// ---------------------------------------------------------------------------
// As col_kernel_pipe2 with one buffer, but the tile arrives by tensor-memory
// access: one thread issues cp.async.bulk.tensor copies of boxes of C columns
// x min(N, 256) rows into a dense [N][C] tile and arms an mbarrier with the
// tile's byte count; the copy engine completes the barrier. No thread spends
// instructions on address generation or copy chunks, and the other CTA on the
// SM overlaps the copy. The wait is bounded: if the barrier has not completed
// after kTmaWaitCycles, the kernel records PWF_ERR_TIMEOUT in *a.kstatus,
// waits once more (bounded) for the copy in flight and returns.
constexpr long long kTmaWaitCycles = 1ll << 31;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// shared writes of the generic proxy before a TMA write of the same bytes
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_addr(dst)), "l"(tm), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z) : "memory");
}
// thread 0 polls with a cycle bound; returns false (for every thread) if it ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* kstatus, int* s_flag) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (clock64() - t0 > kTmaWaitCycles) {
        ok = 0;
        break;
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  if (*s_flag) {
    while (!mbar_try_wait(bar, parity)) {
    }  // completed: returns at once, and makes the tile visible to this thread
    return true;
  }
  if (threadIdx.x == 0) {
    if (kstatus) atomicExch(kstatus, 7 /* PWF_ERR_TIMEOUT */);
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity) && clock64() - t0 < kTmaWaitCycles) {
    }
  }
  __syncthreads();
  return false;
}
__host__ __device__ constexpr size_t tma_smem_bytes(int n, int c) { return (size_t)n * c * sizeof(float2) + 1024; }

template <int N, int OP, int C>
__global__ void __launch_bounds__(col2_threads(N, C), col2_min_blocks(N, C)) col_kernel_tma2(const __grid_constant__ PassArgs a, int nproj) {
  pdl_wait();
  constexpr int EPT = ept_for(N);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  constexpr int BOX = tma_box_rows(N);
  constexpr unsigned TILE_BYTES = (unsigned)(N * C * sizeof(float2));
  static_assert(N % BOX == 0, "tile rows must be whole boxes");
  static_assert(OP != COL_PRECOND_REG, "single-input passes only");
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar;
  __shared__ int s_flag;
  // TMA destinations on a 1024-byte boundary
  float2* tile = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  const int tid = threadIdx.x;
  const int c2 = tid % (C / 2), t = tid / (C / 2);
  const int tiles_per_proj = a.nx / C;
  const int ntiles = nproj * tiles_per_proj;
  const size_t ld = (size_t)a.nx;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned parity = 0;
  for (int tile_i = blockIdx.x; tile_i < ntiles; tile_i += gridDim.x) {
    const int proj = a.proj0 + tile_i / tiles_per_proj;
    const int col0 = (tile_i % tiles_per_proj) * C;
    if (skip_proj(a, proj)) continue;  // uniform per CTA
    if (tid == 0) {
      fence_proxy_async_shared();  // the previous tile's exchanges precede the copy
      mbar_arrive_expect_tx(&bar, TILE_BYTES);
#pragma unroll
      for (int k = 0; k < N / BOX; k++) tma_load_3d(tile + k * BOX * C, &a.tmap, &bar, 2 * col0, k * BOX, proj);
    }
    if (!mbar_wait_bounded(&bar, parity, a.kstatus, &s_flag)) return;
    parity ^= 1u;

    const size_t base = (size_t)proj * a.ny * a.nx + col0 + 2 * c2;
    const int col = col0 + 2 * c2;
    const ColPairLayoutDense<C> sm{tile + 2 * c2};
    float2 v[EPT], u[EPT];
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if constexpr (OP == COL_IFFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) {
        const float4 q = sm[slot_index<N, RK>(t, j)];
        v[j] = make_float2(q.x * a.scale, q.y * a.scale);
        u[j] = make_float2(q.z * a.scale, q.w * a.scale);
      }
    } else {
#pragma unroll
      for (int j = 0; j < EPT; j++) {
        const float4 q = sm[slot_index<N, RS>(t, j)];
        v[j] = make_float2(q.x, q.y);
        u[j] = make_float2(q.z, q.w);
      }
      fft_run2<N, FWD>(v, u, sm, t, a.tw_fwd);
      if constexpr (OP != COL_FFT) col_pair_filter<N, OP, ColPairLayoutDense<C>>(a, t, col, base, v, u, part);
    }
    if constexpr (OP == COL_FFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++)
        *reinterpret_cast<float4*>(a.out + base + (size_t)slot_index<N, RK>(t, j) * ld) =
            make_float4(v[j].x, v[j].y, u[j].x, u[j].y);
    } else {
      fft_run2<N, INV>(v, u, sm, t, a.tw_inv);
#pragma unroll
      for (int j = 0; j < EPT; j++)
        *reinterpret_cast<float4*>(a.out + base + (size_t)slot_index<N, RS>(t, j) * ld) =
            make_float4(v[j].x, v[j].y, u[j].x, u[j].y);
    }
    if constexpr (OP == COL_RESID_IOTF2) block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, tile);
    __syncthreads();  // every thread is done with the tile before the next copy
  }
}

// The TMA map of a batch of complex64 fields [B][ny][nx] seen as float32
// [B][ny][2 nx]: box = 2C floats (C columns) x min(ny, 256) rows x 1 field.
// Encoded on the host through the driver entry point (no libcuda link).

template <int N, int OP, int C>
__global__ void __launch_bounds__(col_threads(N, C), col_min_blocks(col_threads(N, C), ept_for(N)))
    col_kernel_t(const PassArgs a, int nproj) {
  pdl_wait();
  constexpr int EPT = ept_for(N), TPF = tpf_for(N);
  constexpr int NT = col_threads(N, C);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  constexpr int S = colt_stride(N);
  constexpr int TILE = C * S;
  constexpr int ELEMS = N * C;
  static_assert(ELEMS % NT == 0, "tile elements must divide evenly");
  static_assert(OP != COL_PRECOND_REG, "two-input pass uses the other shapes");
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int c = tid / TPF, t = tid % TPF;      // compute mapping: one column per TPF threads
  const int tiles_per_proj = a.nx / C;
  const int ntiles = nproj * tiles_per_proj;
  const size_t ld = (size_t)a.nx;
  auto at = [](float2* buf, int col, int p) -> float2& { return buf[col * S + p + (p >> 4)]; };

  auto tile_base = [&](int tile, int& proj, int& col0) -> size_t {
    proj = a.proj0 + tile / tiles_per_proj;
    col0 = (tile % tiles_per_proj) * C;
    return (size_t)proj * a.ny * a.nx + col0;
  };
  auto prefetch = [&](int tile, float2* buf) {
    int proj, col0;
    const size_t b = tile_base(tile, proj, col0);
    if (skip_proj(a, proj)) return;
#pragma unroll 8
    for (int k = 0; k < ELEMS / NT; k++) {
      const int q = tid + k * NT;  // row-major over the tile: row q / C, column q % C
      const int row = q / C, cc = q % C;
      cp_async8(&at(buf, cc, row), a.in + b + (size_t)row * ld + cc);
    }
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, smem);
  cp_async_commit();
  for (int k = 0; tile < ntiles; k++, tile += gridDim.x) {
    float2* cur = smem + (k & 1) * TILE;
    float2* nxt = smem + ((k + 1) & 1) * TILE;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    int proj, col0;
    const size_t tb = tile_base(tile, proj, col0);
    if (skip_proj(a, proj)) {
      __syncthreads();
      continue;
    }
    const int col = col0 + c;
    const size_t base = tb + c;
    const RowLayout<TPF, NT> sm{cur + c * S, 1 + c};
    float2 v[EPT];
    float2 s2[1];
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int RO;  // slot radix of the results
    if constexpr (OP == COL_IFFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = cscale(sm[slot_index<N, RK>(t, j)], a.scale);
    } else {
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = sm[slot_index<N, RS>(t, j)];
      fft_run<N, FWD>(v, sm, t, a.tw_fwd);
      if constexpr (OP != COL_FFT) col_tile_filter<N, OP>(a, sm, t, col, base, v, s2, part);
    }
    if constexpr (OP != COL_FFT) fft_run<N, INV>(v, sm, t, a.tw_inv);
    // results back into this column's slots (natural order), then row-major stores
    sm.sync();
    if constexpr (OP == COL_FFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) sm[slot_index<N, RK>(t, j)] = v[j];
    } else {
#pragma unroll
      for (int j = 0; j < EPT; j++) sm[slot_index<N, RS>(t, j)] = v[j];
    }
    (void)RO;
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < ELEMS / NT; kk++) {
      const int q = tid + kk * NT;
      const int row = q / C, cc = q % C;
      a.out[tb + (size_t)row * ld + cc] = at(cur, cc, row);
    }
    if constexpr (OP == COL_RESID_IOTF2) block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, cur);
    __syncthreads();  // cur is refilled by the prefetch of the next-but-one tile
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// column passes of the source-mode variant
// ---------------------------------------------------------------------------
// A mode s(r) = exp(2 pi i (mx x / nx + my y / ny)) shifts the spectrum: with
// X^ = F_y F_row{x}, F_y F_row{x s}(kx, ky) = X^(kx - mx, ky - my). Both passes
// therefore work on 2-D spectra, and the tilt is an index shift:
//   CM_FWD : out column kx = F_y^-1{ Q1 scale X^(kx - mx, . - my) }      (in = X^)
//   CM_BACK: A^(kx - mx, ky - my) (+)= w conj(Q1(kx, ky)) scale F_y{in column kx}(ky)
// (indices mod nx, ny). CM_BACK leaves the accumulated A^ in the column
// spectral domain; one inverse column pass after the last mode replaces the
// per-mode inverse transforms and modulations. Reads and writes go to
// different buffers.

__device__ __forceinline__ int wrap_sub(int k, int m, int n) { return k >= m ? k - m : k - m + n; }

template <int N, int MOP, int C>
__global__ void __launch_bounds__(col_threads(N, C), col_min_blocks(col_threads(N, C), ept_for(N)))
    col_mode_kernel(const PassArgs a) {
  pdl_wait();
  constexpr int EPT = ept_for(N);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;
  const int proj = blockIdx.y + a.proj0;
  const int col = blockIdx.x * C + c;
  if (skip_proj(a, proj)) return;
  const int shifted = ((col - a.mode_mx) % a.nx + a.nx) % a.nx;
  const size_t pb = (size_t)proj * a.ny * a.nx;
  const size_t ld = (size_t)a.nx;
  const ColLayout<C> sm{smem + c};
  const int my = ((a.mode_my % N) + N) % N;
  float2 v[EPT];
  if constexpr (MOP == CM_FWD) {
    const float2 qx = cscale(__ldg(&a.qx[col]), a.scale);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      v[j] = cmul(a.in[pb + shifted + (size_t)wrap_sub(ky, my, N) * ld], cmul(qx, __ldg(&a.qy[ky])));
    }
    fft_run<N, INV>(v, sm, t, a.tw_inv);
#pragma unroll
    for (int j = 0; j < EPT; j++) a.out[pb + col + (size_t)slot_index<N, RS>(t, j) * ld] = v[j];
  } else {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[pb + col + (size_t)slot_index<N, RS>(t, j) * ld];
    fft_run<N, FWD>(v, sm, t, a.tw_fwd);
    const float2 qx = cscale(__ldg(&a.qx[col]), a.scale * a.mode_w);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      float2 r = cmulc(v[j], cmul(qx, __ldg(&a.qy[ky])));
      const size_t o = pb + shifted + (size_t)wrap_sub(ky, my, N) * ld;
      if (a.accumulate) r = cadd(r, a.out[o]);
      a.out[o] = r;
    }
  }
}

// The same passes with the pair of adjacent columns (col, col + 1) per thread
// (shared indices, twiddles and barriers; 16-byte exchanges). Each thread owns
// an aligned pair on the unshifted side (CM_FWD's output, CM_BACK's
// accumulated output); the shifted columns (col -/+ mx, ...) are adjacent but
// not 16-byte aligned for odd mx (and wrap at the edge), so they are read as
// two 8-byte accesses.
template <int N, int MOP, int C>
__global__ void __launch_bounds__(col2_threads(N, C), col2_min_blocks(N, C)) col_mode_kernel2(const PassArgs a) {
  pdl_wait();
  constexpr int EPT = ept_for(N);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int c2 = tid % (C / 2), t = tid / (C / 2);
  const int proj = blockIdx.y + a.proj0;
  const int col = blockIdx.x * C + 2 * c2;  // the thread's aligned pair of columns
  if (skip_proj(a, proj)) return;
  // the other pair: CM_FWD reads columns col - mx, CM_BACK reads col + mx
  // (and writes the aligned pair), so the read-modify-write of the
  // accumulated spectrum stays 16-byte aligned
  const int dm = MOP == CM_FWD ? -a.mode_mx : a.mode_mx;
  const int sh0 = ((col + dm) % a.nx + a.nx) % a.nx;
  const int sh1 = sh0 + 1 < a.nx ? sh0 + 1 : 0;
  const size_t pb = (size_t)proj * a.ny * a.nx;
  const size_t ld = (size_t)a.nx;
  const ColPairLayout<C> sm{smem + 2 * c2};
  const int my = ((a.mode_my % N) + N) % N;
  float2 v[EPT], u[EPT];
  if constexpr (MOP == CM_FWD) {
    // Q1 at the output columns (the mode's own frame)
    const float2 qa = cscale(__ldg(&a.qx[col]), a.scale), qb = cscale(__ldg(&a.qx[col + 1]), a.scale);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      const float2 qy = __ldg(&a.qy[ky]);
      const size_t o = pb + (size_t)wrap_sub(ky, my, N) * ld;
      v[j] = cmul(a.in[o + sh0], cmul(qa, qy));
      u[j] = cmul(a.in[o + sh1], cmul(qb, qy));
    }
    fft_run2<N, INV>(v, u, sm, t, a.tw_inv);
#pragma unroll
    for (int j = 0; j < EPT; j++)
      *reinterpret_cast<float4*>(a.out + pb + col + (size_t)slot_index<N, RS>(t, j) * ld) =
          make_float4(v[j].x, v[j].y, u[j].x, u[j].y);
  } else {
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const size_t o = pb + (size_t)slot_index<N, RS>(t, j) * ld;
      v[j] = a.in[o + sh0];
      u[j] = a.in[o + sh1];
    }
    fft_run2<N, FWD>(v, u, sm, t, a.tw_fwd);
    // Q1 at the input columns (the mode's own frame), weight folded in
    const float ws = a.scale * a.mode_w;
    const float2 qa = cscale(__ldg(&a.qx[sh0]), ws), qb = cscale(__ldg(&a.qx[sh1]), ws);
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int ky = slot_index<N, RK>(t, j);
      const float2 qy = __ldg(&a.qy[ky]);
      const float2 r0 = cmulc(v[j], cmul(qa, qy)), r1 = cmulc(u[j], cmul(qb, qy));
      float4* o = reinterpret_cast<float4*>(a.out + pb + col + (size_t)wrap_sub(ky, my, N) * ld);
      float4 q = make_float4(r0.x, r0.y, r1.x, r1.y);
      if (a.accumulate) {
        const float4 old = *o;
        q = make_float4(q.x + old.x, q.y + old.y, q.z + old.z, q.w + old.w);
      }
      *o = q;
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launch for one transform length
// ---------------------------------------------------------------------------

// number of SMs of the current device (persistent grids)
inline int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  return sms;
}

// Dynamic shared memory above 48 KB needs the attribute set once per kernel
// (done at plan creation, outside any stream capture).
template <int N, int OP>
cudaError_t prep_row() {
  return cudaFuncSetAttribute(row_kernel<N, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem_bytes(N));
}

// row pass over the ny rows of nproj projections starting at a.proj0
template <int N, int OP>
cudaError_t launch_row(const PassArgs& a, int nproj, cudaStream_t s) {
  constexpr int ROWS = rows_for(N);
  const long long nrows = (long long)nproj * a.ny;
  return launch_pass(row_kernel<N, OP>, dim3((unsigned)(nrows / ROWS)), dim3(row_threads(N)), row_smem_bytes(N), s, a.pdl, a);
}

// column-pass shape variants: tile width C, pipelined or not
template <int N, int OP, int C, int PIPE>
struct ColShape {
  static int resident;  // CTAs per SM of the persistent kernels (set by prep)
  static cudaError_t prep() {
    if constexpr (PIPE == 5) {
      constexpr size_t SM = tma_smem_bytes(N, C);
      cudaError_t e = cudaFuncSetAttribute(col_kernel_tma2<N, OP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
      if (e != cudaSuccess) return e;
      int r = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, col_kernel_tma2<N, OP, C>, col2_threads(N, C), SM);
      resident = r > 0 ? r : 1;
      return e;
    } else if constexpr (PIPE == 3 || PIPE == 4) {
      constexpr int NB = PIPE == 3 ? 2 : 1;
      constexpr size_t SM = NB * col_smem_bytes(N, C);
      cudaError_t e = cudaFuncSetAttribute(col_kernel_pipe2<N, OP, C, NB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
      if (e != cudaSuccess) return e;
      int r = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, col_kernel_pipe2<N, OP, C, NB>, col2_threads(N, C), SM);
      resident = r > 0 ? r : 1;
      return e;
    } else if constexpr (PIPE == 2) {
      cudaError_t e = cudaFuncSetAttribute(col_kernel_t<N, OP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)colt_smem_bytes(N, C));
      if (e != cudaSuccess) return e;
      int r = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, col_kernel_t<N, OP, C>, col_threads(N, C),
                                                        colt_smem_bytes(N, C));
      resident = r > 0 ? r : 1;
      return e;
    } else if constexpr (PIPE == 1) {
      cudaError_t e = cudaFuncSetAttribute(col_kernel_pipe<N, OP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)colp_smem_bytes(N, C));
      if (e != cudaSuccess) return e;
      int r = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, col_kernel_pipe<N, OP, C>, col_threads(N, C),
                                                        colp_smem_bytes(N, C));
      resident = r > 0 ? r : 1;
      return e;
    } else {
      return cudaFuncSetAttribute(col_kernel<N, OP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem_bytes(N, C));
    }
  }
  static cudaError_t launch(const PassArgs& a, int nproj, cudaStream_t s) {
    if constexpr (PIPE) {
      const long long ntiles = (long long)nproj * (a.nx / C);
      const long long slots = (long long)device_sms() * resident;
      const int grid = (int)(ntiles < slots ? ntiles : slots);
      if constexpr (PIPE == 5) {
        PassArgs b = a;
        if (!encode_field_tmap(&b.tmap, a.in, a.proj0 + nproj, a.ny, a.nx, C)) return cudaErrorInvalidValue;
        return launch_pass(col_kernel_tma2<N, OP, C>, dim3(grid), dim3(col2_threads(N, C)), tma_smem_bytes(N, C), s, a.pdl, b,
                           nproj);
      } else if constexpr (PIPE == 3)
        return launch_pass(col_kernel_pipe2<N, OP, C, 2>, dim3(grid), dim3(col2_threads(N, C)), colp_smem_bytes(N, C), s,
                           a.pdl, a, nproj);
      else if constexpr (PIPE == 4) {
        PassArgs b = a;  // with a tensor map of the field, the kernel prefetches each next tile into L2
        b.l2pf = encode_field_tmap(&b.tmap, a.in, a.proj0 + nproj, a.ny, a.nx, C) ? 1 : 0;
        return launch_pass(col_kernel_pipe2<N, OP, C, 1>, dim3(grid), dim3(col2_threads(N, C)), col_smem_bytes(N, C), s,
                           a.pdl, b, nproj);
      }
      else if constexpr (PIPE == 2)
        return launch_pass(col_kernel_t<N, OP, C>, dim3(grid), dim3(col_threads(N, C)), colt_smem_bytes(N, C), s, a.pdl, a,
                           nproj);
      else
        return launch_pass(col_kernel_pipe<N, OP, C>, dim3(grid), dim3(col_threads(N, C)), colp_smem_bytes(N, C), s, a.pdl,
                           a, nproj);
    } else {
      dim3 grid((unsigned)(a.nx / C), (unsigned)nproj);
      return launch_pass(col_kernel<N, OP, C>, grid, dim3(col_threads(N, C)), col_smem_bytes(N, C), s, a.pdl, a);
    }
  }
};
template <int N, int OP, int C, int PIPE>
int ColShape<N, OP, C, PIPE>::resident = 1;


// Packed residual shapes (COL_RESID_PK): persistent, one staged buffer, column
// pairs (described like the single-buffered pair shapes, pipe code 4).
template <int N, int C>
struct PkShape {
  static int resident;
  static cudaError_t prep() {
    constexpr size_t SM = col_smem_bytes(N, C);
    cudaError_t e = cudaFuncSetAttribute(col_kernel_pk<N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
    if (e != cudaSuccess) return e;
    int r = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, col_kernel_pk<N, C>, col2_threads(N, C), SM);
    resident = r > 0 ? r : 1;
    return e;
  }
  static cudaError_t launch(const PassArgs& a, int nproj, cudaStream_t s) {
    const long long ntiles = (long long)nproj * (a.nx / 2 / C);
    const long long slots = (long long)device_sms() * resident;
    const int grid = (int)(ntiles < slots ? ntiles : slots);
    cudaError_t e = launch_pass(col_kernel_pk<N, C>, dim3(grid), dim3(col2_threads(N, C)), col_smem_bytes(N, C), s,
                                a.pdl, a, nproj);
    if (e != cudaSuccess) return e;
    // then bins 0 and nx/2 of every projection
    return launch_pass(col_kernel_pk_edge<N>, dim3(nproj), dim3(tpf_for(N)), row_smem_len(N) * sizeof(float2), s, a.pdl,
                       a);
  }
};
template <int N, int C>
int PkShape<N, C>::resident = 1;

// whole warps (the output pairs rows by shuffle), even chunk split; a plan
// takes a shape only where C divides nx/2 (pk_fits)
template <int N, int C>
constexpr bool pk_shape_ok() {
  constexpr int th = col2_threads(N, C);
  return pk_col_ok<N>() && C <= 16 && th >= 32 && th <= 512 && th % 32 == 0 && (N / 2 * C / 2) % th == 0 &&
         col_smem_bytes(N, C) <= 200 * 1024;
}

template <int N, int C>
void add_pk_variant(LengthKernels& k) {
  if constexpr (pk_shape_ok<N, C>()) {
    int& n = k.ncolv[COL_RESID_PK];
    if (n < MAX_COL_VARIANTS)
      k.colv[COL_RESID_PK][n++] = {PkShape<N, C>::launch, PkShape<N, C>::prep, C, 4, PWF_SCHED_VARIANT};
  }
}

// Mode column pass shapes: tile width C, one column per thread or the pair of
// adjacent columns. The first one registered is the default before tuning:
// 8 columns per tile from length 1024 on (4 where 8 would exceed 512
// threads), else 16; the pair kernel where a transform has 16 values per
// thread and at most 64 threads.
__host__ __device__ constexpr int colmode_c(int n) { return n >= 1024 ? (tpf_for(n) * 8 <= 512 ? 8 : 4) : 16; }
__host__ __device__ constexpr bool colmode_pair(int n) { return ept_for(n) == 16 && tpf_for(n) <= 64 && n >= 128; }

template <int N, int MOP, int C, bool PAIR>
constexpr bool mode_shape_ok() {
  constexpr int th = PAIR ? col2_threads(N, C) : col_threads(N, C);
  return th >= 32 && th <= 512 && col_smem_bytes(N, C) <= 200 * 1024 && N % C == 0 &&
         (!PAIR || (C >= 4 && ept_for(N) <= 16));
}

template <int N, int MOP, int C, bool PAIR>
struct ModeShape {
  static cudaError_t prep() {
    if constexpr (PAIR)
      return cudaFuncSetAttribute(col_mode_kernel2<N, MOP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem_bytes(N, C));
    else
      return cudaFuncSetAttribute(col_mode_kernel<N, MOP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem_bytes(N, C));
  }
  static cudaError_t launch(const PassArgs& a, int nproj, cudaStream_t s) {
    dim3 grid((unsigned)(a.nx / C), (unsigned)nproj);
    if constexpr (PAIR)
      return launch_pass(col_mode_kernel2<N, MOP, C>, grid, dim3(col2_threads(N, C)), col_smem_bytes(N, C), s, a.pdl,
                         a);
    else
      return launch_pass(col_mode_kernel<N, MOP, C>, grid, dim3(col_threads(N, C)), col_smem_bytes(N, C), s, a.pdl,
                         a);
  }
};

// pipe code of a mode shape in ColVariant: 0 one column per thread, 6 the pair
constexpr int MODE_PAIR = 6;

template <int N, int MOP, int C, bool PAIR>
void add_mode_variant(LengthKernels& k) {
  if constexpr (mode_shape_ok<N, MOP, C, PAIR>()) {
    int& n = k.ncolmodev[MOP];
    for (int i = 0; i < n; i++)  // once per shape and schedule
      if (k.colmodev[MOP][i].C == C && k.colmodev[MOP][i].pipe == (PAIR ? MODE_PAIR : 0) &&
          k.colmodev[MOP][i].sched == PWF_SCHED_VARIANT)
        return;
    if (n < MAX_MODE_VARIANTS)
      k.colmodev[MOP][n++] = {ModeShape<N, MOP, C, PAIR>::launch, ModeShape<N, MOP, C, PAIR>::prep, C,
                              PAIR ? MODE_PAIR : 0, PWF_SCHED_VARIANT};
  }
}

template <int N, int MOP>
void add_mode_op(LengthKernels& k) {
  add_mode_variant<N, MOP, colmode_pair(N) ? 8 : colmode_c(N), colmode_pair(N)>(k);  // the default first
  add_mode_variant<N, MOP, 16, true>(k);
  add_mode_variant<N, MOP, 8, true>(k);
  add_mode_variant<N, MOP, 4, true>(k);
  add_mode_variant<N, MOP, 16, false>(k);
  add_mode_variant<N, MOP, 8, false>(k);
  add_mode_variant<N, MOP, 4, false>(k);
}

// a shape is offered when its CTA has 16..512 threads and its buffers fit
template <int N, int OP, int C, int PIPE>
constexpr bool col_shape_ok() {
  constexpr bool pair = PIPE == 3 || PIPE == 4 || PIPE == 5;
  constexpr int th = pair ? col2_threads(N, C) : col_threads(N, C);
  constexpr size_t sm = PIPE == 5   ? tma_smem_bytes(N, C)
                       : PIPE == 2 ? colt_smem_bytes(N, C)
                       : (PIPE == 1 || PIPE == 3) ? colp_smem_bytes(N, C)
                                                  : col_smem_bytes(N, C);
  return th >= 16 && th <= 512 && sm <= 200 * 1024 && ((PIPE == 0 || PIPE == 2) || (N * C / 2) % th == 0) &&
         (PIPE != 2 || (OP != COL_PRECOND_REG && (N * C) % th == 0 && C <= 8)) &&
         (!pair || (OP != COL_PRECOND_REG && C >= 4 && th >= 32 && th <= 512));
}

template <int N, int OP, int C, int PIPE>
void add_col_variant(LengthKernels& k) {
  if constexpr (col_shape_ok<N, OP, C, PIPE>()) {
    int& n = k.ncolv[OP];
    if (n < MAX_COL_VARIANTS)
      k.colv[OP][n++] = {ColShape<N, OP, C, PIPE>::launch, ColShape<N, OP, C, PIPE>::prep, C, PIPE, PWF_SCHED_VARIANT};
  }
}

template <int N, int OP>
void add_col_op(LengthKernels& k) {
  // first entry = default before tuning
  add_col_variant<N, OP, (N >= 1024 ? 8 : 16), 1>(k);
  add_col_variant<N, OP, 16, 0>(k);
  add_col_variant<N, OP, 8, 0>(k);
  add_col_variant<N, OP, 4, 0>(k);
  add_col_variant<N, OP, 4, 1>(k);
  if constexpr (N < 1024) add_col_variant<N, OP, 8, 1>(k);
  add_col_variant<N, OP, 8, 2>(k);
  add_col_variant<N, OP, 4, 2>(k);
  add_col_variant<N, OP, 8, 3>(k);
  add_col_variant<N, OP, 8, 4>(k);
  add_col_variant<N, OP, 16, 4>(k);
  add_col_variant<N, OP, 4, 4>(k);
  add_col_variant<N, OP, 8, 5>(k);
  add_col_variant<N, OP, 4, 5>(k);
}

// the radices of this translation unit's schedule of length N into slot `set`
template <int N>
void record_schedule(LengthKernels& k, int set) {
  constexpr Sched S = sched_for(N);
  k.sched_stages[set] = S.s;
  for (int i = 0; i < MAX_SCHED_STAGES; i++) k.sched_radix[set][i] = i < S.s ? S.r(i) : 1;
}

// Column shapes built with this translation unit's schedule set (1: the
// alternative) for every column op, appended after the default set's shapes
// so that the plan-time tuner times both schedules; the shapes that measured
// best with the default schedule.
template <int N>
void add_schedule_shapes(LengthKernels& k) {
  record_schedule<N>(k, PWF_SCHED_VARIANT);
  auto op_shapes = [&](auto op_tag) {
    constexpr int OP = decltype(op_tag)::value;
    add_col_variant<N, OP, 16, 4>(k);
    add_col_variant<N, OP, 8, 4>(k);
    add_col_variant<N, OP, 8, 3>(k);
    add_col_variant<N, OP, 4, 4>(k);
    add_col_variant<N, OP, 8, 1>(k);
    add_col_variant<N, OP, 16, 0>(k);
    add_col_variant<N, OP, 8, 0>(k);
  };
  op_shapes(std::integral_constant<int, COL_Q>{});
  op_shapes(std::integral_constant<int, COL_IOTF>{});
  op_shapes(std::integral_constant<int, COL_RESID_IOTF2>{});
  op_shapes(std::integral_constant<int, COL_PRECOND_REG>{});
  op_shapes(std::integral_constant<int, COL_FFT>{});
  op_shapes(std::integral_constant<int, COL_IFFT>{});
  add_pk_variant<N, 8>(k);  // the packed residual pass
  add_pk_variant<N, 4>(k);
  add_pk_variant<N, 16>(k);
  add_mode_op<N, CM_FWD>(k);  // and the mode column passes
  add_mode_op<N, CM_BACK>(k);
}

template <int N>
LengthKernels make_length_kernels() {
  LengthKernels k{};
  k.n = N;
  record_schedule<N>(k, 0);
#define PWF_ROW(OP)                  \
  k.row[OP] = launch_row<N, OP>;     \
  k.row_prep[OP] = prep_row<N, OP>;
  PWF_ROW(ROW_EXP_FFT) PWF_ROW(ROW_REAL_FFT) PWF_ROW(ROW_FFT) PWF_ROW(ROW_IFFT) PWF_ROW(ROW_MUL_T)
  PWF_ROW(ROW_INTENSITY) PWF_ROW(ROW_INTENSITY_OUT) PWF_ROW(ROW_REAL_OUT) PWF_ROW(ROW_RESID)
  PWF_ROW(ROW_COH_RESID) PWF_ROW(ROW_COH_VJP) PWF_ROW(ROW_MUL_V) PWF_ROW(ROW_GRAD_OUT) PWF_ROW(ROW_GRAD_PACK)
  PWF_ROW(ROW_NESTEROV_FFT) PWF_ROW(ROW_NESTEROV) PWF_ROW(ROW_GRADT) PWF_ROW(ROW_MODE_INT) PWF_ROW(ROW_MODE_VG)
  PWF_ROW(ROW_INTENSITY_PK) PWF_ROW(ROW_MUL_V_PK)
#undef PWF_ROW
  add_col_op<N, COL_Q>(k);
  add_col_op<N, COL_IOTF>(k);
  add_col_op<N, COL_RESID_IOTF2>(k);
  add_col_op<N, COL_PRECOND_REG>(k);
  add_col_op<N, COL_FFT>(k);
  add_col_op<N, COL_IFFT>(k);
  add_pk_variant<N, 8>(k);  // first entry = default before tuning (fits every nx >= 16)
  add_pk_variant<N, 4>(k);
  add_pk_variant<N, 16>(k);
  add_mode_op<N, CM_FWD>(k);
  add_mode_op<N, CM_BACK>(k);
  return k;
}


}  // namespace PWF_KNS
}  // namespace pwf
