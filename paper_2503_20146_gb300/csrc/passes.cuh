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
#include "fft.cuh"

namespace pwf {

// ---------------------------------------------------------------------------
// launch shapes
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int rows_for(int n) {
  int r = 256 / tpf_for(n);
  return r < 1 ? 1 : (r > 16 ? 16 : r);
}
__host__ __device__ constexpr int cols_for(int n) { return n >= 1024 ? 8 : 16; }
__host__ __device__ constexpr int row_threads(int n) { return rows_for(n) * tpf_for(n); }
__host__ __device__ constexpr int col_threads(int n) { return cols_for(n) * tpf_for(n); }
__host__ __device__ constexpr size_t row_smem_bytes(int n) {
  return (size_t)rows_for(n) * row_smem_len(n) * sizeof(float2);
}
__host__ __device__ constexpr size_t col_smem_bytes(int n) {
  return (size_t)cols_for(n) * n * sizeof(float2);
}

// per-projection accumulators (float64)
enum Acc : int { ACC_LOSS = 0, ACC_XR = 1, ACC_XI = 2, ACC_XNEW = 3, ACC_XOLD = 4, NACC = 8 };

// ---------------------------------------------------------------------------
// pass arguments (one struct for every pass; unused fields are null)
// ---------------------------------------------------------------------------
struct PassArgs {
  int B, ny, nx;
  const float2* in;        // primary input (in-place passes: in == out)
  float2* out;             // primary output
  const float2* tw_fwd;    // twiddles of this pass's axis
  const float2* tw_inv;
  // fields
  const float2* psi;       // complex phase psi (read)
  float2* psi_out;         // psi after the Nesterov update
  float2* phi;             // phi_prev in, phi out (Nesterov)
  const float2* t;         // diffuser [ny][nx]
  const float* y;          // measurement
  float2* v;               // detector field v (written by ROW_INTENSITY, read by ROW_MUL_V)
  float2* u1;              // P1{x} (stored for the diffuser gradient)
  float2* aux;             // second output (ROW_GRAD_PACK: F_row{Im g})
  const float2* aux_in;    // second input (COL_PRECOND_REG)
  float* reg;              // Re g
  float* f_out;            // real output (forward model)
  float2* g_out;           // complex output (gradient)
  float2* gt_scratch;      // per-projection diffuser-gradient terms
  const float* maxt2;      // device scalar max |t|^2
  double* acc;             // [B][NACC]
  const int* active;       // [B] convergence flags (null: all active)
  const float* beta;       // device scalar Nesterov coefficient (mu_prev - 1)/mu
  // column-pass filter tables (length nx for *x, ny for *y)
  const float2* qx;
  const float2* qy;
  const float* ix;         // IOTF factors
  const float* iy;
  const float* u2x;        // squared frequency, cycles/pixel
  const float* u2y;
  const float* ex;         // STF exponents pi gamma u^2 xcoh^2
  const float* ey;
  const float2* yhat;      // 2-D spectrum of y
  float scale;             // 1/(nx ny), the inverse-transform normalisation
  float eta;
  float alpha_re, alpha_im;
  float gscale;            // ROW_GRAD_OUT: extra factor
  int conj_q;              // use conj(Q): back-propagation P(-L)
  int conj_t;              // multiply by conj(t)
  int div_maxt2;           // ROW_GRAD_OUT / PACK: divide by max|t|^2
  int no_precond;          // P^-1 := 1
  int proj0;               // first projection of this launch (plain path)
};

enum RowOp : int {
  ROW_EXP_FFT = 0,     // x = exp(psi) -> FFT                           (first pass)
  ROW_REAL_FFT,        // y (real) -> FFT                                (F{y})
  ROW_FFT,             // complex field -> FFT                           (plain)
  ROW_IFFT,            // IFFT -> complex field                          (plain)
  ROW_MUL_T,           // IFFT -> [store u1] -> * t (or conj t) -> FFT
  ROW_INTENSITY,       // IFFT -> v (stored) -> |v|^2 -> FFT
  ROW_INTENSITY_OUT,   // IFFT -> f = |v|^2                              (coherent forward)
  ROW_REAL_OUT,        // IFFT -> f = Re                                 (IOTF forward)
  ROW_RESID,           // IFFT -> f = Re; e = y - f; loss; -e -> FFT
  ROW_COH_RESID,       // IFFT -> v; e = y - |v|^2; loss; v * (-e) -> FFT   (coherent)
  ROW_COH_VJP,         // IFFT -> v; v * grad_f -> FFT                   (coherent VJP)
  ROW_MUL_V,           // IFFT -> G = Re; v * G -> FFT
  ROW_GRAD_OUT,        // IFFT -> g = conj(exp psi) g1 * scale -> g_out
  ROW_GRAD_PACK,       // IFFT -> g; store Re g; FFT(alpha o psi) -> out, FFT(Im g) -> aux
  ROW_NESTEROV_FFT,    // IFFT -> Nesterov update; exp(psi_new) -> FFT
  ROW_NESTEROV,        // IFFT -> Nesterov update
  ROW_GRADT,           // IFFT -> g2; scratch = 2 conj(u1) g2; conj(t) g2 -> FFT
  NUM_ROW_OPS
};

enum ColOp : int {
  COL_Q = 0,           // FFT -> * Q (or conj Q) -> IFFT
  COL_IOTF,            // FFT -> * IOTF -> IFFT
  COL_RESID_IOTF2,     // FFT -> R = IOTF I - Y; loss; * IOTF -> IFFT
  COL_PRECOND_REG,     // FFT(H), FFT(S) -> Gamma^2 H + i P^-1 S -> IFFT
  COL_FFT,             // FFT only
  COL_IFFT,            // IFFT only (scaled)
  NUM_COL_OPS
};

template <int OP>
struct RowT {
  static constexpr bool ifft_in = !(OP == ROW_EXP_FFT || OP == ROW_REAL_FFT || OP == ROW_FFT);
  static constexpr bool fft_out = !(OP == ROW_IFFT || OP == ROW_INTENSITY_OUT || OP == ROW_REAL_OUT ||
                                    OP == ROW_GRAD_OUT || OP == ROW_NESTEROV);
  static constexpr int nred = (OP == ROW_RESID || OP == ROW_COH_RESID) ? 1
                              : (OP == ROW_NESTEROV_FFT || OP == ROW_NESTEROV) ? 5 : 0;
};

__device__ __forceinline__ float2 cexpf2(float2 z) {
  float s, c;
  sincosf(z.y, &s, &c);
  float m = expf(z.x);
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
// row pass
// ---------------------------------------------------------------------------
template <int N, int OP>
__global__ void __launch_bounds__(row_threads(N)) row_kernel(const PassArgs a) {
  constexpr int EPT = ept_for(N), TPF = tpf_for(N), ROWS = rows_for(N);
  constexpr int RS = first_radix<N, FWD>();  // slot radix of real-space data
  constexpr int RK = last_radix<N, FWD>();   // slot radix of spectra
  using T = RowT<OP>;
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int rr = tid / TPF, t = tid - rr * TPF;
  const long long row = (long long)blockIdx.x * ROWS + rr + (long long)a.proj0 * a.ny;
  const int proj = (int)(row / a.ny);
  const int yrow = (int)(row - (long long)proj * a.ny);
  if (a.active != nullptr && a.active[proj] == 0) return;  // uniform per CTA (ny % ROWS == 0)
  const size_t rb = (size_t)row * N;
  const RowLayout sm{smem + rr * row_smem_len(N)};
  float2 v[EPT];
  float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};

  // ---- input ----
  if constexpr (T::ifft_in) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[rb + slot_index<N, RK>(t, j)];
    fft_run<N, INV>(v, sm, t, a.tw_inv);
  } else if constexpr (OP == ROW_EXP_FFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cexpf2(a.psi[rb + slot_index<N, RS>(t, j)]);
  } else if constexpr (OP == ROW_REAL_FFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = make_float2(a.y[rb + slot_index<N, RS>(t, j)], 0.f);
  } else {  // ROW_FFT
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[rb + slot_index<N, RS>(t, j)];
  }

  // ---- point-wise step in real space (slots of radix RS) ----
  float2 w[(OP == ROW_GRAD_PACK) ? EPT : 1];
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
      const float2 xx = cexpf2(a.psi[rb + x]);
      a.g_out[rb + x] = cscale(cmulc(v[j], xx), s);
    }
  } else if constexpr (OP == ROW_GRAD_PACK) {
    const float s = 1.0f / *a.maxt2;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 p = a.psi[rb + x];
      const float2 g = cscale(cmulc(v[j], cexpf2(p)), s);
      a.reg[rb + x] = g.x;
      w[j] = make_float2(g.y, 0.f);
      v[j] = make_float2(a.alpha_re * p.x, a.alpha_im * p.y);
    }
  } else if constexpr (OP == ROW_NESTEROV_FFT || OP == ROW_NESTEROV) {
    const float beta = *a.beta;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 p = a.psi[rb + x];
      const float2 fp = a.phi[rb + x];
      const float gr = a.reg[rb + x];
      // g = Preconditioner(g) + Regularizer(psi) = Re g + z
      const float2 g = make_float2(gr + v[j].x, v[j].y);
      const float2 f = make_float2(fmaf(-a.eta, g.x, p.x), fmaf(-a.eta, g.y, p.y));
      const float2 pn = make_float2(fmaf(beta, f.x - fp.x, f.x), fmaf(beta, f.y - fp.y, f.y));
      a.phi[rb + x] = f;
      a.psi_out[rb + x] = pn;
      const float2 xo = cexpf2(p), xn = cexpf2(pn);
      const float2 c = cmulc(xn, xo);
      part[0] += c.x;
      part[1] += c.y;
      part[2] += cabs2(xn);
      part[3] += cabs2(xo);
      v[j] = xn;
    }
  } else if constexpr (OP == ROW_GRADT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      const int x = slot_index<N, RS>(t, j);
      const float2 u = a.u1[rb + x];
      a.gt_scratch[rb + x] = cscale(cmulc(v[j], u), 2.0f);
      v[j] = cmulc(v[j], __ldg(&a.t[(size_t)yrow * N + x]));
    }
  }

  // ---- output ----
  if constexpr (T::fft_out) {
    fft_run<N, FWD>(v, sm, t, a.tw_fwd);
#pragma unroll
    for (int j = 0; j < EPT; j++) a.out[rb + slot_index<N, RK>(t, j)] = v[j];
    if constexpr (OP == ROW_GRAD_PACK) {
      fft_run<N, FWD>(w, sm, t, a.tw_fwd);
#pragma unroll
      for (int j = 0; j < EPT; j++) a.aux[rb + slot_index<N, RK>(t, j)] = w[j];
    }
  }

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
template <int N, int OP>
__global__ void __launch_bounds__(col_threads(N)) col_kernel(const PassArgs a) {
  constexpr int EPT = ept_for(N), TPF = tpf_for(N), C = cols_for(N);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  extern __shared__ float2 smem[];

  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;
  const int proj = blockIdx.y + a.proj0;
  const int col = blockIdx.x * C + c;
  if (a.active != nullptr && a.active[proj] == 0) return;
  const size_t base = (size_t)proj * a.ny * a.nx + col;
  const size_t ld = (size_t)a.nx;
  const ColLayout<C> sm{smem + c};
  float2 v[EPT];
  float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};

  if constexpr (OP == COL_IFFT) {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[base + (size_t)slot_index<N, RK>(t, j) * ld];
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = cscale(v[j], a.scale);
  } else {
#pragma unroll
    for (int j = 0; j < EPT; j++) v[j] = a.in[base + (size_t)slot_index<N, RS>(t, j) * ld];
    fft_run<N, FWD>(v, sm, t, a.tw_fwd);

    // ---- multiply on the 2-D spectrum (slots of radix RK; ky = slot index) ----
    if constexpr (OP == COL_FFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) a.out[base + (size_t)slot_index<N, RK>(t, j) * ld] = v[j];
      return;
    } else if constexpr (OP == COL_Q) {
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
      float2 s[EPT];
#pragma unroll
      for (int j = 0; j < EPT; j++) s[j] = a.aux_in[base + (size_t)slot_index<N, RS>(t, j) * ld];
      fft_run<N, FWD>(s, sm, t, a.tw_fwd);
      const float exv = __ldg(&a.ex[col]);
      const float u2 = __ldg(&a.u2x[col]);
#pragma unroll
      for (int j = 0; j < EPT; j++) {
        const int ky = slot_index<N, RK>(t, j);
        const float g2 = -expm1f(-(exv + __ldg(&a.ey[ky])));  // Gamma^2 = 1 - STF
        const float r2 = u2 + __ldg(&a.u2y[ky]);
        const float pinv = a.no_precond ? 1.0f : (r2 > 0.f ? 1.0f / r2 : 0.0f);
        // Z = Gamma^2 H + i P^-1 S
        v[j] = make_float2((g2 * v[j].x - pinv * s[j].y) * a.scale, (g2 * v[j].y + pinv * s[j].x) * a.scale);
      }
    }
  }

  fft_run<N, INV>(v, sm, t, a.tw_inv);
#pragma unroll
  for (int j = 0; j < EPT; j++) a.out[base + (size_t)slot_index<N, RS>(t, j) * ld] = v[j];

  if constexpr (OP == COL_RESID_IOTF2) block_reduce_add<1>(part, a.acc, proj * NACC + ACC_LOSS, smem);
}

// ---------------------------------------------------------------------------
// column pass, persistent and software-pipelined
// ---------------------------------------------------------------------------
// One CTA per SM walks over column tiles (proj, c0). While tile k is being
// transformed in one shared-memory buffer, tile k+1 is copied into the other
// with cp.async (16-byte chunks, one commit group per tile); results leave
// from registers with plain stores, which drain while the next tile computes.
// Same arithmetic as col_kernel. Not used for COL_PRECOND_REG (two inputs).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

__host__ __device__ constexpr size_t colp_smem_bytes(int n) { return 2 * col_smem_bytes(n); }
// the double-buffered tile must fit the per-CTA shared memory (227 KB)
__host__ __device__ constexpr bool colp_fits(int n) { return colp_smem_bytes(n) <= 200 * 1024; }

template <int N, int OP>
__global__ void __launch_bounds__(col_threads(N), 1) col_kernel_pipe(const PassArgs a, int nproj) {
  constexpr int EPT = ept_for(N), TPF = tpf_for(N), C = cols_for(N);
  constexpr int NT = col_threads(N);
  constexpr int RS = first_radix<N, FWD>();
  constexpr int RK = last_radix<N, FWD>();
  constexpr int CHUNKS = N * C / 2;  // 16-byte chunks per tile
  static_assert(CHUNKS % NT == 0, "tile chunks must divide evenly");
  static_assert(OP != COL_PRECOND_REG, "two-input pass uses col_kernel");
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
    if (a.active != nullptr && a.active[proj] == 0) return;
#pragma unroll
    for (int k = 0; k < CHUNKS / NT; k++) {
      const int q = tid + k * NT;           // chunk index: row q / (C/2), pair q % (C/2)
      const int row = q / (C / 2), pr = q % (C / 2);
      cp_async16(buf + row * C + 2 * pr, a.in + b + (size_t)row * ld + 2 * pr);
    }
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, smem);
  cp_async_commit();
  for (int k = 0; tile < ntiles; k++, tile += gridDim.x) {
    float2* cur = smem + (k & 1) * (C * N);
    float2* nxt = smem + ((k + 1) & 1) * (C * N);
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    int proj, col0;
    const size_t base = tile_base(tile, proj, col0) + c;
    const int col = col0 + c;
    if (a.active != nullptr && a.active[proj] == 0) {
      __syncthreads();
      continue;
    }
    const ColLayout<C> sm{cur + c};
    float2 v[EPT];
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};

    if constexpr (OP == COL_IFFT) {
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = cscale(sm[slot_index<N, RK>(t, j)], a.scale);
    } else {
#pragma unroll
      for (int j = 0; j < EPT; j++) v[j] = sm[slot_index<N, RS>(t, j)];
      fft_run<N, FWD>(v, sm, t, a.tw_fwd);
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
      }
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

// ---------------------------------------------------------------------------
// host-side launch for one transform length
// ---------------------------------------------------------------------------
using PassFn = cudaError_t (*)(const PassArgs&, int nproj, cudaStream_t);
using PrepFn = cudaError_t (*)();

// Dynamic shared memory above 48 KB needs the attribute set once per kernel
// (done at plan creation, outside any stream capture).
template <int N, int OP>
cudaError_t prep_row() {
  return cudaFuncSetAttribute(row_kernel<N, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem_bytes(N));
}
template <int N, int OP>
cudaError_t prep_col() {
  cudaError_t e = cudaFuncSetAttribute(col_kernel<N, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)col_smem_bytes(N));
  if constexpr (OP != COL_PRECOND_REG && colp_fits(N)) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(col_kernel_pipe<N, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)colp_smem_bytes(N));
  }
  return e;
}

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

// row pass over the ny rows of nproj projections starting at a.proj0
template <int N, int OP>
cudaError_t launch_row(const PassArgs& a, int nproj, cudaStream_t s) {
  constexpr int ROWS = rows_for(N);
  const long long nrows = (long long)nproj * a.ny;
  row_kernel<N, OP><<<(unsigned)(nrows / ROWS), row_threads(N), row_smem_bytes(N), s>>>(a);
  return cudaGetLastError();
}

// column pass over the nx columns of nproj projections starting at a.proj0
template <int N, int OP>
cudaError_t launch_col(const PassArgs& a, int nproj, cudaStream_t s) {
  constexpr int C = cols_for(N);
  const long long ntiles = (long long)nproj * (a.nx / C);
  if constexpr (OP != COL_PRECOND_REG && colp_fits(N)) {
    if (ntiles >= 2 * device_sms()) {
      const int grid = (int)(ntiles < device_sms() ? ntiles : device_sms());
      col_kernel_pipe<N, OP><<<grid, col_threads(N), colp_smem_bytes(N), s>>>(a, nproj);
      return cudaGetLastError();
    }
  }
  dim3 grid((unsigned)(a.nx / C), (unsigned)nproj);
  col_kernel<N, OP><<<grid, col_threads(N), col_smem_bytes(N), s>>>(a);
  return cudaGetLastError();
}

// tables of launchers for one length, filled by the per-length translation units
struct LengthKernels {
  int n;
  PassFn row[NUM_ROW_OPS];
  PassFn col[NUM_COL_OPS];
  PrepFn row_prep[NUM_ROW_OPS];
  PrepFn col_prep[NUM_COL_OPS];
};

template <int N>
LengthKernels make_length_kernels() {
  LengthKernels k{};
  k.n = N;
  k.row[ROW_EXP_FFT] = launch_row<N, ROW_EXP_FFT>;
  k.row_prep[ROW_EXP_FFT] = prep_row<N, ROW_EXP_FFT>;
  k.row[ROW_REAL_FFT] = launch_row<N, ROW_REAL_FFT>;
  k.row_prep[ROW_REAL_FFT] = prep_row<N, ROW_REAL_FFT>;
  k.row[ROW_FFT] = launch_row<N, ROW_FFT>;
  k.row_prep[ROW_FFT] = prep_row<N, ROW_FFT>;
  k.row[ROW_IFFT] = launch_row<N, ROW_IFFT>;
  k.row_prep[ROW_IFFT] = prep_row<N, ROW_IFFT>;
  k.row[ROW_MUL_T] = launch_row<N, ROW_MUL_T>;
  k.row_prep[ROW_MUL_T] = prep_row<N, ROW_MUL_T>;
  k.row[ROW_INTENSITY] = launch_row<N, ROW_INTENSITY>;
  k.row_prep[ROW_INTENSITY] = prep_row<N, ROW_INTENSITY>;
  k.row[ROW_INTENSITY_OUT] = launch_row<N, ROW_INTENSITY_OUT>;
  k.row_prep[ROW_INTENSITY_OUT] = prep_row<N, ROW_INTENSITY_OUT>;
  k.row[ROW_REAL_OUT] = launch_row<N, ROW_REAL_OUT>;
  k.row_prep[ROW_REAL_OUT] = prep_row<N, ROW_REAL_OUT>;
  k.row[ROW_RESID] = launch_row<N, ROW_RESID>;
  k.row_prep[ROW_RESID] = prep_row<N, ROW_RESID>;
  k.row[ROW_COH_RESID] = launch_row<N, ROW_COH_RESID>;
  k.row_prep[ROW_COH_RESID] = prep_row<N, ROW_COH_RESID>;
  k.row[ROW_COH_VJP] = launch_row<N, ROW_COH_VJP>;
  k.row_prep[ROW_COH_VJP] = prep_row<N, ROW_COH_VJP>;
  k.row[ROW_MUL_V] = launch_row<N, ROW_MUL_V>;
  k.row_prep[ROW_MUL_V] = prep_row<N, ROW_MUL_V>;
  k.row[ROW_GRAD_OUT] = launch_row<N, ROW_GRAD_OUT>;
  k.row_prep[ROW_GRAD_OUT] = prep_row<N, ROW_GRAD_OUT>;
  k.row[ROW_GRAD_PACK] = launch_row<N, ROW_GRAD_PACK>;
  k.row_prep[ROW_GRAD_PACK] = prep_row<N, ROW_GRAD_PACK>;
  k.row[ROW_NESTEROV_FFT] = launch_row<N, ROW_NESTEROV_FFT>;
  k.row_prep[ROW_NESTEROV_FFT] = prep_row<N, ROW_NESTEROV_FFT>;
  k.row[ROW_NESTEROV] = launch_row<N, ROW_NESTEROV>;
  k.row_prep[ROW_NESTEROV] = prep_row<N, ROW_NESTEROV>;
  k.row[ROW_GRADT] = launch_row<N, ROW_GRADT>;
  k.row_prep[ROW_GRADT] = prep_row<N, ROW_GRADT>;
  k.col[COL_Q] = launch_col<N, COL_Q>;
  k.col_prep[COL_Q] = prep_col<N, COL_Q>;
  k.col[COL_IOTF] = launch_col<N, COL_IOTF>;
  k.col_prep[COL_IOTF] = prep_col<N, COL_IOTF>;
  k.col[COL_RESID_IOTF2] = launch_col<N, COL_RESID_IOTF2>;
  k.col_prep[COL_RESID_IOTF2] = prep_col<N, COL_RESID_IOTF2>;
  k.col[COL_PRECOND_REG] = launch_col<N, COL_PRECOND_REG>;
  k.col_prep[COL_PRECOND_REG] = prep_col<N, COL_PRECOND_REG>;
  k.col[COL_FFT] = launch_col<N, COL_FFT>;
  k.col_prep[COL_FFT] = prep_col<N, COL_FFT>;
  k.col[COL_IFFT] = launch_col<N, COL_IFFT>;
  k.col_prep[COL_IFFT] = prep_col<N, COL_IFFT>;
  return k;
}

// defined in the per-length translation units
const LengthKernels* kernels_for_length(int n);

}  // namespace pwf
