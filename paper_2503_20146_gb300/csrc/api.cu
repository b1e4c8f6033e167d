// C ABI of the PWF library: plans, filter tables, the pass schedules of
// Algorithms S1/S2, the solver state, CUDA-graph replay of the fused iteration,
// and the unfused per-operation baseline.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include <nvtx3/nvToolsExt.h>
#include <new>
#include <vector>

#include "../../include/pwf.h"
#include "host_tables.h"
#include "persist.cuh"

namespace pwf {
const LengthKernels* length_kernels_16();
const LengthKernels* length_kernels_32();
const LengthKernels* length_kernels_64();
const LengthKernels* length_kernels_96();
const LengthKernels* length_kernels_128();
const LengthKernels* length_kernels_256();
const LengthKernels* length_kernels_512();
const LengthKernels* length_kernels_768();
const LengthKernels* length_kernels_1024();
const LengthKernels* length_kernels_1536();
const LengthKernels* length_kernels_2048();

// TMA map of a batch of complex64 fields [B][ny][nx] as float32 [B][ny][2 nx]
// with boxes of C columns x min(ny, 256) rows (the TMA-staged column shapes).
// The encoder is the driver's, reached through the runtime's entry-point
// query, so the library links only the runtime.
bool encode_field_tmap(CUtensorMap* m, const void* base, int B, int ny, int nx, int C) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  if (!fn || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (nx & 1)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * nx, (cuuint64_t)ny, (cuuint64_t)B};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float2), (cuuint64_t)nx * ny * sizeof(float2)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * C), (cuuint32_t)tma_box_rows(ny), 1u};
  const cuuint32_t estride[3] = {1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

const LengthKernels* kernels_for_length(int n) {
  switch (n) {
    case 16: return length_kernels_16();
    case 32: return length_kernels_32();
    case 64: return length_kernels_64();
    case 96: return length_kernels_96();
    case 128: return length_kernels_128();
    case 256: return length_kernels_256();
    case 512: return length_kernels_512();
    case 768: return length_kernels_768();
    case 1024: return length_kernels_1024();
    case 1536: return length_kernels_1536();
    case 2048: return length_kernels_2048();
    default: return nullptr;
  }
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
// max over the diffuser of |t|^2 (the normalisation of g, Algorithm S2). Values
// are non-negative floats, whose bit patterns order like integers.
__global__ void k_max_abs2(const float2* __restrict__ t, size_t n, float* out) {
  float m = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, cabs2(t[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

// End of one iteration: per-projection loss / correlation / stopping rule,
// accumulator reset, and the Nesterov coefficients of the next iteration.
__global__ void k_finalize(double* acc, int B, int* active, int* iters, double* loss, double* corr,
                           DevIter* it, double corr_tol) {
  pdl_wait();
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  int na = 0, nf = 0;
  for (int p = threadIdx.x; p < B; p += blockDim.x) {
    double* a = acc + (size_t)p * NACC;
    na += finalize_projection(p, a, active, iters, loss, corr, corr_tol, nf);
    for (int k = 0; k < NACC; k++) a[k] = 0.0;
  }
  atomicAdd(&s_active, na);
  if (nf) it->nonfinite = 1;
  __syncthreads();
  if (threadIdx.x == 0) finalize_momentum(it, s_active);
}

__global__ void k_state_reset(DevIter* it, int* active, int* iters, double* loss, double* corr, int B) {
  for (int p = threadIdx.x; p < B; p += blockDim.x) {
    active[p] = 1;
    iters[p] = 0;
    loss[p] = 0.0;
    corr[p] = 0.0;
  }
  if (threadIdx.x == 0) {
    it->mu = 1.0;
    it->beta = 0.0f;
    it->iter = 0;
    it->n_active = B;
    it->nonfinite = 0;
    it->status = PWF_OK;
  }
}

// The device-side loop of pwf_solve: the last node of every iteration sets the
// while-condition of the graph that holds the iteration. ctl[0] is the
// iteration limit and ctl[1] the bodies run so far (both written by the host
// before the launch); the loop ends after ctl[0] bodies whatever the solver
// state holds, or earlier once the stopping rule has retired every projection.
__global__ void k_loop_control(cudaGraphConditionalHandle h, const DevIter* it, int* ctl, double corr_tol) {
  pdl_wait();
  if (threadIdx.x == 0) {
    const int done = ++ctl[1];
    const bool more = done < ctl[0] && (corr_tol <= 0.0 || it->n_active > 0);
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

__global__ void k_gather_loss(const double* acc, double* loss, int B) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < B) loss[p] = acc[(size_t)p * NACC + ACC_LOSS];
}

// grad_t = sum over the batch of the per-projection terms
__global__ void k_batch_sum(const float2* __restrict__ s, float2* __restrict__ out, int B, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    for (int b = 0; b < B; b++) a = cadd(a, s[(size_t)b * n + i]);
    out[i] = a;
  }
}

// t <- t - (eta_t / (2 max|t|^2)) sum_b s_b; s_b = 2 conj(P1{x_b}) P2^H{v_b G_b}
// (the per-projection terms of the diffuser-gradient pass), i.e. a plain step
// along the batch sum of g_t in Algorithm S2's normalisation
__global__ void k_t_update(float2* t, const float2* __restrict__ s, int B, size_t n, float eta_t,
                           const float* __restrict__ maxt2) {
  const float c = eta_t / (2.0f * *maxt2);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    for (int b = 0; b < B; b++) a = cadd(a, s[(size_t)b * n + i]);
    t[i] = make_float2(fmaf(-c, a.x, t[i].x), fmaf(-c, a.y, t[i].y));
  }
}

// ---- unfused per-operation kernels (the plain baseline) ----
enum PlainFilter : int { PF_Q = 0, PF_IOTF = 1, PF_PINV = 2, PF_GAMMA2 = 3, PF_WIENER = 4 };

__global__ void k_exp(const float2* __restrict__ psi, float2* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = cexpf_acc(psi[i]);
}
__global__ void k_filter(float2* X, int ny, int nx, int which, const float2* qx, const float2* qy, int conj,
                         const float* ix, const float* iy, const float* u2x, const float* u2y, const float* ex,
                         const float* ey, int no_precond, float wiener_eps = 0.f) {
  const size_t n = (size_t)ny * nx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nx), ky = (int)(i / nx);
    float2 v = X[i];
    if (which == PF_Q) {
      float2 q = cmul(qx[kx], qy[ky]);
      if (conj) q = cconj(q);
      v = cmul(v, q);
    } else if (which == PF_IOTF) {
      v = cscale(v, ix[kx] * iy[ky]);
    } else if (which == PF_WIENER) {
      const float w = ix[kx] * iy[ky];
      v = cscale(v, w / fmaf(w, w, wiener_eps));
    } else if (which == PF_PINV) {
      const float r2 = u2x[kx] + u2y[ky];
      v = cscale(v, no_precond ? 1.0f : (r2 > 0.f ? 1.0f / r2 : 0.0f));
    } else {
      v = cscale(v, -fmaf(ex[kx], ey[ky], ex[kx] + ey[ky]));  // Gamma^2 = 1 - STF_x STF_y
    }
    X[i] = v;
  }
}
__global__ void k_mul_t(float2* X, const float2* __restrict__ t, size_t n, int conj) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = conj ? cmulc(X[i], t[i]) : cmul(X[i], t[i]);
}
// V = v; X = |v|^2
__global__ void k_abs2_keep(float2* X, float2* V, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = X[i];
    V[i] = v;
    X[i] = make_float2(cabs2(v), 0.f);
  }
}
// X = -(y - Re X), loss += (y - Re X)^2
__global__ void k_resid(float2* X, const float* __restrict__ y, size_t n, double* loss) {
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float e = y[i] - X[i].x;
    s = fmaf(e, e, s);
    X[i] = make_float2(-e, 0.f);
  }
  double d = s;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, d);
}
// X = V * Re X
__global__ void k_mul_v_real(float2* X, const float2* __restrict__ V, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = cscale(V[i], X[i].x);
}
// X = conj(exp psi) X / max|t|^2
__global__ void k_grad(float2* X, const float2* __restrict__ psi, size_t n, const float* maxt2) {
  const float s = 1.0f / *maxt2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = cscale(cmulc(X[i], cexpf_acc(psi[i])), s);
}
// REG = Re X; S = Im X (as a complex field with zero imaginary part)
__global__ void k_split(const float2* __restrict__ X, float* reg, float2* S, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 g = X[i];
    reg[i] = g.x;
    S[i] = make_float2(g.y, 0.f);
  }
}
__global__ void k_copy(const float2* __restrict__ a, float2* b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
// ---- calibration helpers ----
__global__ void k_real_to_complex(const float* __restrict__ I, float2* X, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = make_float2(I[i], 0.f);
}
__global__ void k_abs2_scale(float2* X, size_t n, float s) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = make_float2(cabs2(X[i]) * s, 0.f);
}
__global__ void k_sqrt_clip(float2* X, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = make_float2(sqrtf(fmaxf(X[i].x, 0.f)), 0.f);
}
// out[d] = mean over the other axis of Re X at lag d (axis 1: X[y][d]; axis 0: X[d][x])
__global__ void k_line_mean(const float2* __restrict__ X, int ny, int nx, int axis, double* out) {
  const int lag = blockIdx.x;
  const int n_other = axis == 1 ? ny : nx;
  double s = 0.0;
  for (int k = threadIdx.x; k < n_other; k += blockDim.x)
    s += axis == 1 ? (double)X[(size_t)k * nx + lag].x : (double)X[(size_t)lag * nx + k].x;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    out[lag] = t / n_other;
  }
}
__global__ void k_mean(const float* __restrict__ I, size_t n, double* out) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) s += I[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s / (double)n);
}

// g = (Re g + i Re F^-1{P^-1 F{Im g}}) + (Re a Re rho + i Im a Im rho); Nesterov.
__global__ void k_nesterov_plain(const float* __restrict__ reg, const float2* __restrict__ S,
                                 const float2* __restrict__ H, float2* psi, float2* phi, size_t n, float eta,
                                 float are, float aim, const float* beta_p, double* acc) {
  const float beta = *beta_p;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 rho = H[i];
    const float2 g = make_float2(reg[i] + are * rho.x, S[i].x + aim * rho.y);
    const float2 p = psi[i], fp = phi[i];
    const float2 f = make_float2(p.x - eta * g.x, p.y - eta * g.y);
    const float2 pn = make_float2(f.x + beta * (f.x - fp.x), f.y + beta * (f.y - fp.y));
    phi[i] = f;
    psi[i] = pn;
    const float2 xo = cexpf2(p), xn = cexpf_acc(pn);
    const float2 c = cmulc(xn, xo);
    p0 += c.x;
    p1 += c.y;
    p2 += cabs2(xn);
    p3 += cabs2(xo);
  }
  double d[4] = {p0, p1, p2, p3};
  for (int k = 0; k < 4; k++) {
    for (int o = 16; o > 0; o >>= 1) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[ACC_XR + k], d[k]);
  }
}

// Twiddle table of the length-n transform with forward radices r[0..s) in
// direction D (the inverse runs them reversed), in the layout the stage
// runner reads: stage k >= 1 of radix R after NS points holds W^(q j), q =
// 1..R-1, j < NS, at (sum of (R_i - 1) NS_i over the stages 1..k-1) + (q - 1)
// NS + j; computed in double precision and rounded once.
bool host_twiddles_radices(int n, const int* r, int s, int D, std::vector<float2>& tab) {
  auto radix = [&](int k) { return D == FWD ? r[k] : r[s - 1 - k]; };
  int prod = 1;
  for (int k = 0; k < s; k++) prod *= radix(k);
  if (prod != n) return false;
  size_t len = 0;
  for (int k = 1, ns = radix(0); k < s; ns *= radix(k), k++) len += (size_t)(radix(k) - 1) * ns;
  tab.assign(len > 0 ? len : 1, make_float2(1.f, 0.f));
  size_t off = 0;
  for (int k = 1, ns = radix(0); k < s; ns *= radix(k), k++) {
    const int R = radix(k);
    for (int q = 1; q < R; q++)
      for (int j = 0; j < ns; j++) {
        const long m = ((long)q * j) % ((long)ns * R);
        const double ang = 2.0 * M_PI * (double)m / (double)(ns * R);
        tab[off + (size_t)(q - 1) * ns + j] = make_float2((float)std::cos(ang), (float)(D * std::sin(ang)));
      }
    off += (size_t)(R - 1) * ns;
  }
  return true;
}

// Twiddle table of the length-n transform in direction D, in the layout the
// stage runner reads (stage k >= 1 of radix R after NS points: W^(r j) at
// stage_twoff + (r - 1) NS + j), computed in double precision.
bool host_twiddles(int n, int D, std::vector<float2>& tab) {
  tab.assign(twiddle_len(n, D) > 0 ? twiddle_len(n, D) : 1, make_float2(1.f, 0.f));
  const Sched s = sched_for(n);
  for (int k = 1; k < s.s; k++) {
    const int R = stage_radix(n, D, k), NS = stage_ns(n, D, k), off = stage_twoff(n, D, k);
    for (int r = 1; r < R; r++)
      for (int j = 0; j < NS; j++) {
        const long m = ((long)r * j) % ((long)NS * R);
        const double ang = 2.0 * M_PI * (double)m / (double)(NS * R);
        const size_t idx = (size_t)off + (size_t)(r - 1) * NS + j;
        if (idx >= tab.size()) return false;
        tab[idx] = make_float2((float)std::cos(ang), (float)(D * std::sin(ang)));
      }
  }
  return true;
}

}  // namespace pwf

using namespace pwf;

// ---------------------------------------------------------------------------
// plan and state
// ---------------------------------------------------------------------------
struct AxisTables {
  int n = 0;
  float2* tw_fwd = nullptr;
  float2* tw_inv = nullptr;
  float2* tw_fwd_alt = nullptr;  // twiddles of the alternative radix schedule (column shapes built with it)
  float2* tw_inv_alt = nullptr;
  float2* q1 = nullptr;  // exp(i phi_{L1}) restricted to this axis
  float2* q2 = nullptr;
  float* iotf = nullptr;
  float* u2 = nullptr;   // squared frequency, cycles per pixel
  float* stf = nullptr;  // STF - 1 of this axis, exp(-pi gamma u^2 coh^2) - 1
};

struct Mode {
  int mx, my;
  float w;
};

struct pwf_state {
  int B = 0, ny = 0, nx = 0;
  float2* phi = nullptr;
  int* active = nullptr;
  int* iters = nullptr;
  double* loss = nullptr;
  double* corr = nullptr;
  DevIter* it = nullptr;
};

struct HostPipe;  // solve from host buffers (pwf_solve_host)

struct pwf_plan {
  pwf_plan_desc d{};
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  double* calib = nullptr;               // calibration sums, nx + ny + 1 (allocated on first use)
  const LengthKernels* krow = nullptr;  // length nx
  const LengthKernels* kcol = nullptr;  // length ny
  int colsel[NUM_COL_OPS] = {};  // chosen column-pass shape per op
  float coltime[NUM_COL_OPS][MAX_COL_VARIANTS] = {};  // tuning times (ms per launch)
  int modesel[2] = {0, 0};                              // chosen mode column-pass shape (CM_FWD, CM_BACK)
  float modetime[2][MAX_MODE_VARIANTS] = {};            // their tuning times
  AxisTables ax, ay;
  bool coherent = false;
  // source-mode variant
  std::vector<Mode> modes;   // empty: the paper's IOTF form
  float2* M = nullptr;       // per-mode pass buffer
  float2* ACC = nullptr;     // sum over modes of the back-propagated row spectra
  float* IBUF = nullptr;     // summed intensity, then the residual
  float2* VSTACK = nullptr;  // detector fields of all modes (allocated on first use)
  // workspace
  float2* X = nullptr;
  float2* V = nullptr;
  float2* S = nullptr;
  float* REG = nullptr;
  float2* YH = nullptr;
  double* acc = nullptr;
  float* maxt2 = nullptr;
  int* kstatus = nullptr;    // set by a kernel whose bounded wait ran out (PWF_ERR_TIMEOUT)
  int* loop_ctl = nullptr;   // device-side loop: {iteration limit, bodies run} (written per solve)
  size_t ws_bytes = 0;
  std::vector<void*> allocs;
  // solver
  pwf_state* solve_state = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
  double graph_tol = 0.0;
  double graph_eta_t = -1.0;  // joint diffuser step of the captured graph (< 0: t fixed)
  bool graph_loop = false;    // the graph holds the whole loop (conditional WHILE node)
  float2* GT = nullptr;       // per-projection diffuser-gradient terms (joint refinement)
  pwf_status sticky = PWF_OK;
  char err[256] = "";
  // instrumentation: kernels enqueued, and per-pass event timing
  long long launches = 0;
  long long graph_kernels = 0;  // kernels in the captured iteration graph
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<const char*> prof_names;
  size_t prof_n = 0;
  HostPipe* pipe = nullptr;  // created by the first pwf_solve_host
  // persistent solver (square grids of persist_size; see persist.cuh)
  bool persist = false;          // pwf_solve takes the persistent launch
  int persist_grid = 0;          // CTAs of the cooperative launch
  long long wait_cap = 1ll << 31;  // clock64 cycles one grid barrier may wait
  double* gpart = nullptr;       // [persist_grid][B][NACC]
  unsigned* bar = nullptr;       // grid barrier words
  PersistPhase* phases = nullptr;  // device copy of the iteration's passes
  int* scan_word = nullptr;      // PWF_FLAG_CHECK_FINITE: id of the first pass that wrote a NaN or inf (-1: none)
  std::vector<const char*> scan_names;  // pass names by id
  int cluster = 0;               // cluster-resident variant: CTAs per cluster (0: not used)
  int cluster_sched = 0;         // its radix schedule set (LengthKernels::sched_radix)
  bool cluster_plan = false;     // pwf_solve takes the cluster-resident solver
  DevIter* cit = nullptr;        // [B] per-projection iteration records of that variant
};

namespace {

pwf_status fail(pwf_plan* p, pwf_status s, const char* msg) {
  if (p) {
    std::snprintf(p->err, sizeof(p->err), "%s", msg);
    if (s == PWF_ERR_CUDA && p->sticky == PWF_OK) p->sticky = s;
  }
  return s;
}

pwf_status cuda_fail(pwf_plan* p, cudaError_t e, const char* where) {
  if (p) {
    std::snprintf(p->err, sizeof(p->err), "%s: %s", where, cudaGetErrorString(e));
    if (p->sticky == PWF_OK) p->sticky = PWF_ERR_CUDA;
  }
  return PWF_ERR_CUDA;
}

#define PWF_CUDA(p, call)                                   \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return cuda_fail((p), e__, #call); \
  } while (0)

// pwf_debug_fail_alloc: the allocation that many allocations from now fails
std::atomic<int> g_fail_alloc{-1};

template <class T>
pwf_status dalloc(pwf_plan* p, T** ptr, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  int left = g_fail_alloc.load();
  while (left >= 0 && !g_fail_alloc.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 0) return fail(p, PWF_ERR_NOMEM, "device allocation failed (pwf_debug_fail_alloc)");
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, PWF_ERR_NOMEM, "device allocation failed");
  }
  p->allocs.push_back(q);
  p->ws_bytes += count * sizeof(T);
  *ptr = static_cast<T*>(q);
  return PWF_OK;
}

double fftfreq(int k, int n) { return (double)(k < (n + 1) / 2 ? k : k - n) / (double)n; }  // cycles per sample

// 2 pi L (w - 1/lambda), w = sqrt(lambda^-2 - rho2), in the cancellation-free form
double prop_phase(double rho2, double lambda, double L) {
  const double il = 1.0 / lambda;
  const double w = std::sqrt(il * il - rho2);
  return 2.0 * M_PI * L * (-rho2 / (il + w));
}

pwf_status build_axis(pwf_plan* p, AxisTables& A, int n, double pixel, double coh) {
  A.n = n;
  const pwf_plan_desc& d = p->d;
  // the inverse runs the radices in reverse order, so its table length differs
  std::vector<float2> twf, twi;
  if (!host_twiddles(n, FWD, twf) || !host_twiddles(n, INV, twi))
    return fail(p, PWF_ERR_UNSUPPORTED, "twiddle table layout");
  const int tlf = (int)twf.size(), tli = (int)twi.size();
  std::vector<float2> q1(n), q2(n);
  std::vector<float> io(n), u2(n), st(n);
  for (int k = 0; k < n; k++) {
    const double f = fftfreq(k, n);  // cycles per pixel
    const double u = f / pixel;      // cycles per metre
    const double a1 = prop_phase(u * u, d.wavelength_m, d.L1_m);
    const double a2 = prop_phase(u * u, d.wavelength_m, d.L2_m);
    q1[k] = make_float2((float)std::cos(a1), (float)std::sin(a1));
    q2[k] = make_float2((float)std::cos(a2), (float)std::sin(a2));
    io[k] = (float)std::exp(-0.5 * M_PI * u * u * coh * coh);
    u2[k] = (float)(f * f);
    st[k] = (float)std::expm1(-M_PI * d.gamma * u * u * coh * coh);  // STF of this axis minus 1, Eq. (14)
  }
  pwf_status r;
  if ((r = dalloc(p, &A.tw_fwd, tlf)) || (r = dalloc(p, &A.tw_inv, tli)) || (r = dalloc(p, &A.q1, n)) ||
      (r = dalloc(p, &A.q2, n)) || (r = dalloc(p, &A.iotf, n)) || (r = dalloc(p, &A.u2, n)) ||
      (r = dalloc(p, &A.stf, n)))
    return r;
  PWF_CUDA(p, cudaMemcpy(A.tw_fwd, twf.data(), tlf * sizeof(float2), cudaMemcpyHostToDevice));
  PWF_CUDA(p, cudaMemcpy(A.tw_inv, twi.data(), tli * sizeof(float2), cudaMemcpyHostToDevice));
  if (const LengthKernels* k = kernels_for_length(n); k && k->sched_stages[1] > 0) {
    std::vector<float2> af, ai;
    if (!host_twiddles_radices(n, k->sched_radix[1], k->sched_stages[1], FWD, af) ||
        !host_twiddles_radices(n, k->sched_radix[1], k->sched_stages[1], INV, ai))
      return fail(p, PWF_ERR_UNSUPPORTED, "alternative twiddle table layout");
    if ((r = dalloc(p, &A.tw_fwd_alt, af.size())) || (r = dalloc(p, &A.tw_inv_alt, ai.size()))) return r;
    PWF_CUDA(p, cudaMemcpy(A.tw_fwd_alt, af.data(), af.size() * sizeof(float2), cudaMemcpyHostToDevice));
    PWF_CUDA(p, cudaMemcpy(A.tw_inv_alt, ai.data(), ai.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  PWF_CUDA(p, cudaMemcpy(A.q1, q1.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
  PWF_CUDA(p, cudaMemcpy(A.q2, q2.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
  PWF_CUDA(p, cudaMemcpy(A.iotf, io.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  PWF_CUDA(p, cudaMemcpy(A.u2, u2.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  PWF_CUDA(p, cudaMemcpy(A.stf, st.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  return PWF_OK;
}

int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g > 152 * 16 ? 152 * 16 : (g == 0 ? 1 : g));
}

// passes and end-of-iteration kernels take programmatic dependent launch
int pdl_of(const pwf_plan* p) { return (p->d.flags & PWF_FLAG_NO_PDL) ? 0 : 1; }

PassArgs base_args(pwf_plan* p) {
  PassArgs a{};
  a.B = p->d.batch;
  a.ny = p->d.ny;
  a.nx = p->d.nx;
  a.maxt2 = p->maxt2;
  a.acc = p->acc;
  a.kstatus = p->kstatus;
  a.scale = (float)(1.0 / ((double)p->d.nx * p->d.ny));
  a.eta = (float)p->d.eta;
  const bool no_reg = (p->d.flags & PWF_FLAG_NO_REG) != 0;
  a.alpha_re = no_reg ? 0.f : (float)p->d.alpha_re;
  a.alpha_im = no_reg ? 0.f : (float)p->d.alpha_im;
  a.no_precond = (p->d.flags & PWF_FLAG_NO_PRECOND) ? 1 : 0;
  a.gscale = 1.0f;
  a.mode_w = 1.0f;
  a.proj0 = 0;
  a.pdl = pdl_of(p);
  return a;
}

// projections covered by the passes being enqueued
int nproj_of(const pwf_plan* p) { return p->d.batch; }

const char* const kRowNames[NUM_ROW_OPS] = {
    "row_exp_fft", "row_real_fft", "row_fft", "row_ifft", "row_mul_t", "row_intensity", "row_intensity_out",
    "row_real_out", "row_resid", "row_coh_resid", "row_coh_vjp", "row_mul_v", "row_grad_out", "row_grad_pack",
    "row_nesterov_fft", "row_nesterov", "row_gradt", "row_mode_int", "row_mode_vg", "row_intensity_pk",
    "row_mul_v_pk"};
const char* const kColNames[NUM_COL_OPS] = {"col_q", "col_iotf", "col_resid_iotf2", "col_precond_reg", "col_fft",
                                            "col_ifft", "col_resid_pk"};

// Enqueues one kernel; under pwf_profile_iteration it is bracketed by events.
template <class F>
cudaError_t enqueue(pwf_plan* p, const char* name, F&& launch) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p->prof) {
    if (p->prof_n + 2 > p->ev_pool.size()) {
      for (int k = 0; k < 64; k++) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return cudaErrorMemoryAllocation;
        p->ev_pool.push_back(e);
      }
    }
    e0 = p->ev_pool[p->prof_n];
    e1 = p->ev_pool[p->prof_n + 1];
    cudaEventRecord(e0, p->stream);
  }
  nvtxRangePushA(name);
  cudaError_t e = launch();
  nvtxRangePop();
  p->launches++;
  if (p->prof) {
    cudaEventRecord(e1, p->stream);
    p->prof_names.push_back(name);
    p->prof_n += 2;
  }
  return e;
}

// the tables a row pass on axis x, a column pass on axis y and a propagator
// column pass (Q1 or Q2, conjugated for the back-propagation) read
PassArgs row_args(const pwf_plan* p, PassArgs a) {
  a.tw_fwd = p->ax.tw_fwd;
  a.tw_inv = p->ax.tw_inv;
  return a;
}
PassArgs col_args(const pwf_plan* p, PassArgs a) {
  a.tw_fwd = p->ay.tw_fwd;
  a.tw_inv = p->ay.tw_inv;
  a.qx = nullptr;
  a.ix = p->ax.iotf;
  a.iy = p->ay.iotf;
  a.u2x = p->ax.u2;
  a.u2y = p->ay.u2;
  a.ex = p->ax.stf;
  a.ey = p->ay.stf;
  return a;
}
PassArgs colq_args(const pwf_plan* p, PassArgs a, int which, int conj) {
  a.tw_fwd = p->ay.tw_fwd;
  a.tw_inv = p->ay.tw_inv;
  a.qx = which == 1 ? p->ax.q1 : p->ax.q2;
  a.qy = which == 1 ? p->ay.q1 : p->ay.q2;
  a.conj_q = conj;
  return a;
}

// row pass on axis x, column pass on axis y
// PWF_FLAG_CHECK_FINITE: after every pass a scan of what it wrote; the first
// pass (in stream order) whose output holds a NaN or an infinity leaves its id
__global__ void k_scan_finite(const float* v, size_t n, int id, int* word) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(word, -1, id);
}

cudaError_t scan_output(pwf_plan* p, const char* name, const void* ptr, int proj0, int nproj, int floats_per_px) {
  if (!p->scan_word || !ptr) return cudaSuccess;
  int id = 0;
  while (id < (int)p->scan_names.size() && std::strcmp(p->scan_names[id], name) != 0) id++;
  if (id == (int)p->scan_names.size()) p->scan_names.push_back(name);
  const size_t px = (size_t)p->d.ny * p->d.nx;
  const float* v = static_cast<const float*>(ptr) + (size_t)proj0 * px * floats_per_px;
  const size_t n = (size_t)nproj * px * floats_per_px;
  return enqueue(p, "scan_finite", [&] {
    k_scan_finite<<<grid_for(n), 256, 0, p->stream>>>(v, n, id, p->scan_word);
    return cudaGetLastError();
  });
}

cudaError_t scan_pass(pwf_plan* p, const char* name, const PassArgs& a, int nproj, int op, bool is_row) {
  if (!p->scan_word) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (is_row && (op == ROW_REAL_OUT || op == ROW_INTENSITY_OUT)) return scan_output(p, name, a.f_out, a.proj0, nproj, 1);
  if (is_row && op == ROW_GRAD_OUT) return scan_output(p, name, a.g_out, a.proj0, nproj, 2);
  if ((e = scan_output(p, name, a.out, a.proj0, nproj, 2)) != cudaSuccess) return e;
  if (is_row && (op == ROW_NESTEROV_FFT || op == ROW_NESTEROV)) e = scan_output(p, name, a.psi_out, a.proj0, nproj, 2);
  return e;
}

cudaError_t row(pwf_plan* p, int op, PassArgs a, int nproj) {
  a = row_args(p, a);
  cudaError_t e = enqueue(p, kRowNames[op], [&] { return p->krow->row[op](a, nproj, p->stream); });
  return e != cudaSuccess ? e : scan_pass(p, kRowNames[op], a, nproj, op, true);
}
// the column-axis twiddles of the radix schedule a column shape was built with
PassArgs sched_tables(const pwf_plan* p, PassArgs a, int sched) {
  a.tw_fwd = sched == 1 ? p->ay.tw_fwd_alt : p->ay.tw_fwd;
  a.tw_inv = sched == 1 ? p->ay.tw_inv_alt : p->ay.tw_inv;
  return a;
}

cudaError_t col(pwf_plan* p, int op, PassArgs a, int nproj) {
  a = sched_tables(p, col_args(p, a), p->kcol->colv[op][p->colsel[op]].sched);
  cudaError_t e =
      enqueue(p, kColNames[op], [&] { return p->kcol->colv[op][p->colsel[op]].launch(a, nproj, p->stream); });
  if (op == COL_RESID_PK) p->launches++;  // its second kernel: bins 0 and nx/2
  return e != cudaSuccess ? e : scan_pass(p, kColNames[op], a, nproj, op, false);
}
cudaError_t col_q(pwf_plan* p, PassArgs a, int which, int conj, int nproj) {
  a = sched_tables(p, colq_args(p, a, which, conj), p->kcol->colv[COL_Q][p->colsel[COL_Q]].sched);
  cudaError_t e = enqueue(p, kColNames[COL_Q],
                          [&] { return p->kcol->colv[COL_Q][p->colsel[COL_Q]].launch(a, nproj, p->stream); });
  return e != cudaSuccess ? e : scan_pass(p, kColNames[COL_Q], a, nproj, COL_Q, false);
}

#define LAUNCH(p, expr)                                    \
  do {                                                     \
    cudaError_t e__ = (expr);                              \
    if (e__ != cudaSuccess) return cuda_fail((p), e__, #expr); \
  } while (0)

// Device arrays are read with 16-byte vector loads and 16-byte L2 bulk
// prefetches of whole rows, which need 16-byte aligned bases.
bool a16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }
pwf_status misaligned(pwf_plan* p) { return fail(p, PWF_ERR_INVALID_ARG, "device arrays must be 16-byte aligned"); }

pwf_status compute_maxt2(pwf_plan* p, const float2* t) {
  const size_t n = (size_t)p->d.ny * p->d.nx;
  PWF_CUDA(p, cudaMemsetAsync(p->maxt2, 0, sizeof(float), p->stream));
  k_max_abs2<<<grid_for(n), 256, 0, p->stream>>>(t, n, p->maxt2);
  p->launches++;
  PWF_CUDA(p, cudaGetLastError());
  return PWF_OK;
}

// psi -> X = F_row{exp psi} -> ... -> X = F_row{ P2{t P1{x}} } (row spectrum of v)
pwf_status fused_to_detector(pwf_plan* p, PassArgs a, const float2* psi, const float2* t, float2* u1,
                             bool start_from_psi, int nproj) {
  a.in = p->X;
  a.out = p->X;
  if (start_from_psi) {
    a.psi = psi;
    LAUNCH(p, row(p, ROW_EXP_FFT, a, nproj));
  }
  LAUNCH(p, col_q(p, a, 1, 0, nproj));          // P1: multiply by Q1
  a.t = t;
  a.conj_t = 0;
  a.u1 = u1;
  LAUNCH(p, row(p, ROW_MUL_T, a, nproj));       // t * P1{x}
  a.u1 = nullptr;
  LAUNCH(p, col_q(p, a, 2, 0, nproj));          // P2: multiply by Q2
  return PWF_OK;
}

// X holds the row spectrum of w = v G; back-propagate: P2^H, conj(t), P1^H.
pwf_status fused_backprop(pwf_plan* p, PassArgs a, const float2* t, bool gradt, int nproj,
                          float2* gt_scratch = nullptr) {
  a.in = p->X;
  a.out = p->X;
  a.t = t;
  LAUNCH(p, col_q(p, a, 2, 1, nproj));
  if (gradt) {
    a.u1 = p->S;
    a.gt_scratch = gt_scratch ? gt_scratch : p->YH;
    LAUNCH(p, row(p, ROW_GRADT, a, nproj));
    a.u1 = nullptr;
  } else {
    a.conj_t = 1;
    LAUNCH(p, row(p, ROW_MUL_T, a, nproj));
  }
  LAUNCH(p, col_q(p, a, 1, 1, nproj));
  return PWF_OK;
}

// Tensor Gauss-Hermite modes of a Gaussian source (standard normal rule, k1 =
// 3 or 5 points per axis); node n walks the pattern by sigma n pixels at the
// detector: tilt sigma n p / (lambda (L1 + L2)) cycles/m = that x N p bins.
std::vector<Mode> source_modes(const pwf_plan_desc& d) {
  const int k1 = d.n_modes == 25 ? 5 : 3;
  double nodes[5], weights[5];
  if (k1 == 3) {
    const double r3 = std::sqrt(3.0);
    const double nn[3] = {-r3, 0.0, r3}, ww[3] = {1.0 / 6, 2.0 / 3, 1.0 / 6};
    for (int i = 0; i < 3; i++) nodes[i] = nn[i], weights[i] = ww[i];
  } else {
    const double a = std::sqrt(5.0 - std::sqrt(10.0)), b = std::sqrt(5.0 + std::sqrt(10.0));
    const double wa = (7.0 + 2.0 * std::sqrt(10.0)) / 60.0, wb = (7.0 - 2.0 * std::sqrt(10.0)) / 60.0;
    const double nn[5] = {-b, -a, 0.0, a, b}, ww[5] = {wb, wa, 8.0 / 15, wa, wb};
    for (int i = 0; i < 5; i++) nodes[i] = nn[i], weights[i] = ww[i];
  }
  const double z = d.wavelength_m * (d.L1_m + d.L2_m);
  std::vector<Mode> m;
  for (int iy = 0; iy < k1; iy++)
    for (int ix = 0; ix < k1; ix++) {
      const double sx = d.mode_sigma_px * nodes[ix] * d.pixel_m, sy = d.mode_sigma_px * nodes[iy] * d.pixel_m;
      Mode md;
      md.mx = z > 0 ? (int)std::lrint(sx / z * d.nx * d.pixel_m) : 0;
      md.my = z > 0 ? (int)std::lrint(sy / z * d.ny * d.pixel_m) : 0;
      md.w = (float)(weights[ix] * weights[iy]);
      m.push_back(md);
    }
  return m;
}

// e = y - I; loss += e^2 per projection; I <- -e (= f - y)
__global__ void k_modal_resid(float* I, const float* __restrict__ y, size_t per_proj, double* acc, int proj0) {
  pdl_wait();
  const int proj = blockIdx.y + proj0;
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_proj; i += (size_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)proj * per_proj + i;
    const float e = y[o] - I[o];
    s = fmaf(e, e, s);
    I[o] = -e;
  }
  double d = s;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&acc[(size_t)proj * NACC + ACC_LOSS], d);
}

cudaError_t colmode(pwf_plan* p, int mop, PassArgs a, const Mode& md, int accumulate, int nproj) {
  const ColVariant& sh = p->kcol->colmodev[mop][p->modesel[mop]];
  a = sched_tables(p, a, sh.sched);
  a.qx = p->ax.q1;
  a.qy = p->ay.q1;
  a.mode_mx = md.mx;
  a.mode_my = md.my;
  a.mode_w = md.w;
  a.accumulate = accumulate;
  const char* name = mop == CM_FWD ? "col_mode_fwd" : "col_mode_back";
  cudaError_t e = enqueue(p, name, [&] { return sh.launch(a, nproj, p->stream); });
  return e != cudaSuccess ? e : scan_pass(p, name, a, nproj, -1, false);
}

// X (F_row{x}) -> X^ = F_y F_row{x} in place: the modes read shifted spectra
pwf_status spectrum_for_modes(pwf_plan* p, PassArgs a, int nproj) {
  a.in = p->X;
  a.out = p->X;
  LAUNCH(p, col(p, COL_FFT, a, nproj));
  return PWF_OK;
}

// the spectra CM_BACK accumulated in ACC -> F_y^-1 in place (the scale was
// applied per mode)
pwf_status accumulated_from_spectrum(pwf_plan* p, PassArgs a, int nproj) {
  a.in = p->ACC;
  a.out = p->ACC;
  a.scale = 1.0f;
  LAUNCH(p, col(p, COL_IFFT, a, nproj));
  return PWF_OK;
}

pwf_status ensure_vstack(pwf_plan* p) {
  if (p->VSTACK) return PWF_OK;
  return dalloc(p, &p->VSTACK, p->modes.size() * (size_t)p->d.batch * p->d.ny * p->d.nx);
}

// X holds F_row{exp psi} (turned into its 2-D spectrum in place: X is
// consumed). For every mode: propagate, store v_j (if vstack), and accumulate
// I = sum_j w_j |v_j|^2 into `intensity`.
pwf_status modal_forward(pwf_plan* p, PassArgs a, const float2* t, float* intensity, bool store_v) {
  const size_t n = (size_t)p->d.batch * p->d.ny * p->d.nx;
  if (pwf_status r = spectrum_for_modes(p, a, nproj_of(p))) return r;
  for (size_t j = 0; j < p->modes.size(); j++) {
    const Mode& md = p->modes[j];
    PassArgs b = a;
    b.in = p->X;
    b.out = p->M;
    LAUNCH(p, colmode(p, CM_FWD, b, md, 0, nproj_of(p)));  // tilt (a spectral shift), P1
    b.in = p->M;
    b.t = t;
    b.conj_t = 0;
    b.u1 = nullptr;
    LAUNCH(p, row(p, ROW_MUL_T, b, nproj_of(p)));
    LAUNCH(p, col_q(p, b, 2, 0, nproj_of(p)));              // P2
    b.v = store_v ? p->VSTACK + j * n : nullptr;
    b.f_out = intensity;
    b.mode_w = md.w;
    b.accumulate = j > 0;
    LAUNCH(p, row(p, ROW_MODE_INT, b, nproj_of(p)));
  }
  return PWF_OK;
}

// G (real, f - y or dL/df) in `G`; back-propagate every stored mode and
// accumulate sum_j w_j F_row{conj(s_j) P1^H{conj(t) P2^H{v_j G}}} into ACC
// (as 2-D spectra, then one inverse column pass).
pwf_status modal_backward(pwf_plan* p, PassArgs a, const float2* t, const float* G) {
  const size_t n = (size_t)p->d.batch * p->d.ny * p->d.nx;
  for (size_t j = 0; j < p->modes.size(); j++) {
    const Mode& md = p->modes[j];
    PassArgs b = a;
    b.v = p->VSTACK + j * n;
    b.y = G;
    b.out = p->M;
    LAUNCH(p, row(p, ROW_MODE_VG, b, nproj_of(p)));
    b.in = p->M;
    LAUNCH(p, col_q(p, b, 2, 1, nproj_of(p)));              // P2^H
    b.t = t;
    b.conj_t = 1;
    LAUNCH(p, row(p, ROW_MUL_T, b, nproj_of(p)));
    b.out = p->ACC;
    LAUNCH(p, colmode(p, CM_BACK, b, md, j > 0, nproj_of(p)));  // P1^H, untilt, accumulate (spectra)
  }
  return accumulated_from_spectrum(p, a, nproj_of(p));
}

pwf_status modal_resid(pwf_plan* p, const float* y, const int* active) {
  (void)active;
  const size_t per = (size_t)p->d.ny * p->d.nx;
  dim3 grid((unsigned)((per + 255) / 256 > 64 ? 64 : (per + 255) / 256), (unsigned)nproj_of(p));
  return enqueue(p, "modal_resid", [&] {
           return launch_pass(k_modal_resid, grid, dim3(256), 0, p->stream, pdl_of(p), p->IBUF, y, per, p->acc, 0);
         }) == cudaSuccess
             ? PWF_OK
             : cuda_fail(p, cudaGetLastError(), "k_modal_resid");
}

// The residual passes of the IOTF iteration take the packed form (two real
// rows per complex row, columns kx and nx - kx from one transform pair) where
// the column length has packed shapes, unless PWF_FLAG_UNPACKED_RESID.
bool packed_resid(const pwf_plan* p) {
  return !(p->d.flags & PWF_FLAG_UNPACKED_RESID) && p->kcol->ncolv[COL_RESID_PK] > 0;
}

// A packed-residual shape covers C of the nx/2 positions per tile: it fits a
// plan whose nx/2 it divides. Every other shape fits every plan of its length.
bool shape_fits(const pwf_plan* p, int op, const ColVariant& v) {
  return op != COL_RESID_PK || (p->d.nx / 2) % v.C == 0;
}

// one fused iteration (or the body of pwf_step): X must hold F_row{exp psi}
pwf_status fused_iteration(pwf_plan* p, pwf_state* st, const float* y, const float2* t, float2* psi,
                           bool next_fft, double corr_tol, float2* t_refine = nullptr, double eta_t = 0.0) {
  PassArgs a = base_args(p);
  a.active = st->active;
  a.beta = &st->it->beta;
  pwf_status r;
  if (!p->modes.empty()) {
    // source-mode variant: forward per mode (v_j kept), residual, adjoint per mode.
    // The mode fields were allocated by the caller, outside any stream capture.
    if (!p->VSTACK) return fail(p, PWF_ERR_STATE, "mode field stack not allocated");
    if ((r = modal_forward(p, a, t, p->IBUF, true)) ||
        (r = modal_resid(p, y, st->active)) || (r = modal_backward(p, a, t, p->IBUF)))
      return r;
    a.in = p->ACC;
    a.out = p->X;
    a.psi = psi;
    a.reg = p->REG;
    a.aux = p->S;
    LAUNCH(p, row(p, ROW_GRAD_PACK, a, nproj_of(p)));
    a.in = p->X;
    a.aux_in = p->S;
    LAUNCH(p, col(p, COL_PRECOND_REG, a, nproj_of(p)));
    a.psi_out = psi;
    a.phi = st->phi;
    LAUNCH(p, row(p, next_fft ? ROW_NESTEROV_FFT : ROW_NESTEROV, a, nproj_of(p)));
    LAUNCH(p, enqueue(p, "finalize", [&] {
        return launch_pass(k_finalize, dim3(1), dim3(256), 0, p->stream, pdl_of(p), p->acc, a.B, st->active, st->iters,
                           st->loss, st->corr, st->it, corr_tol);
      }));
    return PWF_OK;
  }
  const bool joint = t_refine != nullptr;
  r = fused_to_detector(p, a, psi, t, joint ? p->S : nullptr, false, nproj_of(p));  // u1 kept for g_t
  if (r) return r;
  a.in = p->X;
  a.out = p->X;
  a.y = y;
  if (p->coherent) {
    LAUNCH(p, row(p, ROW_COH_RESID, a, nproj_of(p)));   // e = y - |v|^2; loss; v (-e)
  } else {
    a.v = p->V;
    a.yhat = p->YH;
    if (packed_resid(p)) {  // |v|^2 and G are real: two rows per complex row, half the columns
      LAUNCH(p, row(p, ROW_INTENSITY_PK, a, nproj_of(p)));  // v stored; F_row{|v|^2}, rows packed in pairs
      LAUNCH(p, col(p, COL_RESID_PK, a, nproj_of(p)));      // as COL_RESID_IOTF2 on bins 0..nx/2
      LAUNCH(p, row(p, ROW_MUL_V_PK, a, nproj_of(p)));      // v F^-1{IOTF F{-e}} from the packed rows
    } else {
      LAUNCH(p, row(p, ROW_INTENSITY, a, nproj_of(p)));   // v stored; F_row{|v|^2}
      LAUNCH(p, col(p, COL_RESID_IOTF2, a, nproj_of(p))); // IOTF (IOTF F{|v|^2} - F{y}); loss (Parseval)
      LAUNCH(p, row(p, ROW_MUL_V, a, nproj_of(p)));       // v F^-1{IOTF F{-e}}
    }
  }
  if ((r = fused_backprop(p, a, t, joint, nproj_of(p), p->GT))) return r;
  a.psi = psi;
  a.reg = p->REG;
  a.aux = p->S;
  LAUNCH(p, row(p, ROW_GRAD_PACK, a, nproj_of(p)));     // Re g; F_row{alpha o psi}; F_row{Im g}
  a.aux_in = p->S;
  LAUNCH(p, col(p, COL_PRECOND_REG, a, nproj_of(p)));   // Gamma^2 H + i P^-1 S
  a.psi_out = psi;
  a.phi = st->phi;
  LAUNCH(p, row(p, next_fft ? ROW_NESTEROV_FFT : ROW_NESTEROV, a, nproj_of(p)));
  LAUNCH(p, enqueue(p, "finalize", [&] {
      return launch_pass(k_finalize, dim3(1), dim3(256), 0, p->stream, pdl_of(p), p->acc, a.B, st->active, st->iters,
                         st->loss, st->corr, st->it, corr_tol);
    }));
  if (joint) {
    // joint refinement: step t along the batch sum of g_t (max|t|^2 of the
    // t this iteration used), then max|t|^2 of the new t for the next one
    const size_t n = (size_t)p->d.ny * p->d.nx;
    LAUNCH(p, enqueue(p, "t_update", [&] {
      k_t_update<<<grid_for(n), 256, 0, p->stream>>>(t_refine, p->GT, a.B, n, (float)eta_t, p->maxt2);
      return cudaGetLastError();
    }));
    pwf_status rr = compute_maxt2(p, t_refine);
    if (rr) return rr;
  }
  return PWF_OK;
}

// The passes of one fused iteration (IOTF or coherent form, the same order
// and arguments as fused_iteration) for the persistent solver, ending with the
// end-of-iteration step.
void persist_schedule(const pwf_plan* p, const pwf_state* st, const float* y, const float2* t, float2* psi,
                      std::vector<PersistPhase>& ph) {
  PassArgs a = base_args(const_cast<pwf_plan*>(p));
  a.active = st->active;
  a.beta = &st->it->beta;
  a.in = p->X;
  a.out = p->X;
  auto row_ph = [&](int op, const PassArgs& b) { ph.push_back({PK_ROW, op, 0, row_args(p, b)}); };
  auto col_ph = [&](int op, const PassArgs& b) { ph.push_back({PK_COL, op, 0, col_args(p, b)}); };
  auto colq_ph = [&](const PassArgs& b, int which, int conj) {
    ph.push_back({PK_COL, COL_Q, 0, colq_args(p, b, which, conj)});
  };
  colq_ph(a, 1, 0);                       // P1
  a.t = t;
  a.conj_t = 0;
  row_ph(ROW_MUL_T, a);                   // t P1{x}
  colq_ph(a, 2, 0);                       // P2
  a.y = y;
  if (p->coherent) {
    row_ph(ROW_COH_RESID, a);             // e = y - |v|^2; loss; v (-e)
  } else {
    a.v = p->V;
    row_ph(ROW_INTENSITY, a);             // v stored; F_row{|v|^2}
    a.yhat = p->YH;
    col_ph(COL_RESID_IOTF2, a);           // IOTF (IOTF F{|v|^2} - F{y}); loss (Parseval)
    row_ph(ROW_MUL_V, a);                 // v F^-1{IOTF F{-e}}
  }
  colq_ph(a, 2, 1);                       // P2^H
  a.conj_t = 1;
  row_ph(ROW_MUL_T, a);                   // conj(t)
  colq_ph(a, 1, 1);                       // P1^H
  a.psi = psi;
  a.reg = p->REG;
  a.aux = p->S;
  row_ph(ROW_GRAD_PACK, a);               // Re g; F_row{alpha o psi}; F_row{Im g}
  a.aux_in = p->S;
  col_ph(COL_PRECOND_REG, a);             // Gamma^2 H + i P^-1 S
  a.psi_out = psi;
  a.phi = st->phi;
  row_ph(ROW_NESTEROV_FFT, a);            // Nesterov; correlation sums; F_row{exp psi}
  ph.back().flush = 1;
  ph.push_back({PK_FINALIZE, 0, 0, a});
}

// All max_iter iterations as one cooperative launch (X holds F_row{exp psi}).
pwf_status persist_solve(pwf_plan* p, pwf_state* st, const float* y, const float2* t, float2* psi, int max_iter,
                         double corr_tol) {
  std::vector<PersistPhase> ph;
  persist_schedule(p, st, y, t, psi, ph);
  if ((int)ph.size() > PERSIST_MAX_PHASES) return fail(p, PWF_ERR_STATE, "too many passes for the persistent solver");
  if (p->cluster > 0 && p->cluster_sched == 1)  // the kernel's transforms run the alternative schedule
    for (PersistPhase& q : ph) {
      const AxisTables& A = q.kind == PK_COL ? p->ay : p->ax;
      q.a.tw_fwd = A.tw_fwd_alt;
      q.a.tw_inv = A.tw_inv_alt;
    }
  PWF_CUDA(p, cudaMemcpyAsync(p->phases, ph.data(), ph.size() * sizeof(PersistPhase), cudaMemcpyHostToDevice,
                              p->stream));
  if (p->cluster == 0) PWF_CUDA(p, cudaMemsetAsync(p->bar, 0, 2 * sizeof(unsigned), p->stream));
  PersistArgs pa{};
  pa.phases = p->phases;
  pa.nphases = (int)ph.size();
  pa.B = p->d.batch;
  pa.max_iter = max_iter;
  pa.corr_tol = corr_tol;
  pa.gpart = p->gpart;
  pa.bar = p->bar;
  pa.cap = p->wait_cap;
  pa.active = st->active;
  pa.iters = st->iters;
  pa.loss = st->loss;
  pa.corr = st->corr;
  pa.it = st->it;
  pa.cit = p->cit;
  if (p->cluster > 0) {
    LAUNCH(p, enqueue(p, "persist_cluster",
                      [&] { return p->kcol->persist_cluster[p->cluster_sched](pa, p->cluster, p->stream); }));
    p->launches++;  // the closing k_persist_cluster_finish
  } else {
    LAUNCH(p, enqueue(p, "persist", [&] { return p->kcol->persist(pa, p->persist_grid, p->stream); }));
  }
  return PWF_OK;
}

// F{y} for every projection (used by the Parseval form of the residual)
pwf_status compute_yhat(pwf_plan* p, const float* y, const int* active) {
  PassArgs a = base_args(p);
  a.active = active;
  a.y = y;
  a.out = p->YH;
  LAUNCH(p, row(p, ROW_REAL_FFT, a, a.B));
  a.in = p->YH;
  LAUNCH(p, col(p, COL_FFT, a, a.B));
  return PWF_OK;
}

// ---- unfused baseline: Algorithm S2 one operation per launch, one projection at a time ----
pwf_status plain_fft2(pwf_plan* p, float2* X, int proj, bool inverse) {
  PassArgs a = base_args(p);
  a.proj0 = proj;
  a.in = X;
  a.out = X;
  if (!inverse) {
    LAUNCH(p, row(p, ROW_FFT, a, 1));
    LAUNCH(p, col(p, COL_FFT, a, 1));
  } else {
    LAUNCH(p, col(p, COL_IFFT, a, 1));
    LAUNCH(p, row(p, ROW_IFFT, a, 1));
  }
  return PWF_OK;
}

pwf_status plain_filter(pwf_plan* p, float2* X, int proj, int which, int L, int conj) {
  pwf_status r;
  if ((r = plain_fft2(p, X, proj, false))) return r;
  const size_t n = (size_t)p->d.ny * p->d.nx;
  float2* Xp = X + (size_t)proj * n;
  k_filter<<<grid_for(n), 256, 0, p->stream>>>(Xp, p->d.ny, p->d.nx, which, L == 1 ? p->ax.q1 : p->ax.q2,
                                                L == 1 ? p->ay.q1 : p->ay.q2, conj, p->ax.iotf, p->ay.iotf,
                                                p->ax.u2, p->ay.u2, p->ax.stf, p->ay.stf,
                                                (p->d.flags & PWF_FLAG_NO_PRECOND) ? 1 : 0);
  PWF_CUDA(p, cudaGetLastError());
  return plain_fft2(p, X, proj, true);
}

pwf_status plain_iteration(pwf_plan* p, pwf_state* st, const float* y, const float2* t, float2* psi, int proj) {
  const size_t n = (size_t)p->d.ny * p->d.nx;
  const size_t o = (size_t)proj * n;
  const int G = grid_for(n);
  cudaStream_t s = p->stream;
  float2 *X = p->X, *V = p->V, *S = p->S, *H = p->YH;
  pwf_status r;
  // forward model, Eq. (1)
  k_exp<<<G, 256, 0, s>>>(psi + o, X + o, n);
  if ((r = plain_filter(p, X, proj, PF_Q, 1, 0))) return r;
  k_mul_t<<<G, 256, 0, s>>>(X + o, t, n, 0);
  if ((r = plain_filter(p, X, proj, PF_Q, 2, 0))) return r;
  k_abs2_keep<<<G, 256, 0, s>>>(X + o, V + o, n);
  if ((r = plain_filter(p, X, proj, PF_IOTF, 0, 0))) return r;
  // e = y - f
  k_resid<<<G, 256, 0, s>>>(X + o, y + o, n, p->acc + (size_t)proj * NACC + ACC_LOSS);
  // Wirtinger derivative (back-propagation)
  if ((r = plain_filter(p, X, proj, PF_IOTF, 0, 0))) return r;
  k_mul_v_real<<<G, 256, 0, s>>>(X + o, V + o, n);
  if ((r = plain_filter(p, X, proj, PF_Q, 2, 1))) return r;
  k_mul_t<<<G, 256, 0, s>>>(X + o, t, n, 1);
  if ((r = plain_filter(p, X, proj, PF_Q, 1, 1))) return r;
  k_grad<<<G, 256, 0, s>>>(X + o, psi + o, n, p->maxt2);
  // Preconditioner
  k_split<<<G, 256, 0, s>>>(X + o, p->REG + o, S + o, n);
  if ((r = plain_filter(p, S, proj, PF_PINV, 0, 0))) return r;
  // regularizer, Eqs. (14)-(15)
  k_copy<<<G, 256, 0, s>>>(psi + o, H + o, n);
  if ((r = plain_filter(p, H, proj, PF_GAMMA2, 0, 0))) return r;
  // Nesterov
  const bool no_reg = (p->d.flags & PWF_FLAG_NO_REG) != 0;
  k_nesterov_plain<<<G, 256, 0, s>>>(p->REG + o, S + o, H + o, psi + o, st->phi + o, n, (float)p->d.eta,
                                     no_reg ? 0.f : (float)p->d.alpha_re, no_reg ? 0.f : (float)p->d.alpha_im,
                                     &st->it->beta, p->acc + (size_t)proj * NACC);
  PWF_CUDA(p, cudaGetLastError());
  return PWF_OK;
}

// Plan-time autotuning of the column passes: every shape variant of every
// column op is run once to warm up and then timed over two launches on the
// plan's own (zeroed) workspace, and the fastest is kept.
pwf_status tune_columns(pwf_plan* p) {
  const size_t n = (size_t)p->d.batch * p->d.ny * p->d.nx;
  PWF_CUDA(p, cudaMemsetAsync(p->X, 0, n * sizeof(float2), p->stream));
  PWF_CUDA(p, cudaMemsetAsync(p->S, 0, n * sizeof(float2), p->stream));
  PWF_CUDA(p, cudaMemsetAsync(p->YH, 0, n * sizeof(float2), p->stream));
  cudaEvent_t e0, e1;
  PWF_CUDA(p, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(p, cudaGetLastError(), "cudaEventCreate");
  }
  PassArgs a = base_args(p);
  a.in = p->X;
  a.out = p->X;
  a.aux_in = p->S;
  a.yhat = p->YH;
  a.tw_fwd = p->ay.tw_fwd;
  a.tw_inv = p->ay.tw_inv;
  a.qx = p->ax.q1;
  a.qy = p->ay.q1;
  a.ix = p->ax.iotf;
  a.iy = p->ay.iotf;
  a.u2x = p->ax.u2;
  a.u2y = p->ay.u2;
  a.ex = p->ax.stf;
  a.ey = p->ay.stf;
  cudaError_t err = cudaSuccess;
  for (int op = 0; op < NUM_COL_OPS && err == cudaSuccess; op++) {
    float best = 1e30f;
    for (int v = 0; v < p->kcol->ncolv[op] && err == cudaSuccess; v++) {
      const PassFn fn = p->kcol->colv[op][v].launch;
      const PassArgs av = sched_tables(p, a, p->kcol->colv[op][v].sched);
      if (!shape_fits(p, op, p->kcol->colv[op][v])) {  // not offered on this plan
        p->coltime[op][v] = 1e30f;
        continue;
      }
      if (p->kcol->colv[op][v].pipe == 5 && fn(av, a.B, p->stream) != cudaSuccess) {
        // a TMA shape whose tensor map the driver would not encode: not offered
        cudaGetLastError();
        p->coltime[op][v] = 1e30f;
        continue;
      }
      if ((err = fn(av, a.B, p->stream)) != cudaSuccess) break;
      cudaEventRecord(e0, p->stream);
      for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) err = fn(av, a.B, p->stream);
      cudaEventRecord(e1, p->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      p->coltime[op][v] = ms / 2.0f;
      if (err == cudaSuccess && ms < best) {
        best = ms;
        p->colsel[op] = v;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(p, err, "column-pass tuning");
  PWF_CUDA(p, cudaMemsetAsync(p->acc, 0, (size_t)p->d.batch * NACC * sizeof(double), p->stream));
  return PWF_OK;
}

// The mode column passes' shapes timed the same way (source-mode plans): CM_FWD
// reads the spectrum X at a shift of (3, 5) bins into M, CM_BACK reads M and
// accumulates into ACC at the same shift.
pwf_status tune_modes(pwf_plan* p) {
  const size_t n = (size_t)p->d.batch * p->d.ny * p->d.nx;
  PWF_CUDA(p, cudaMemsetAsync(p->X, 0, n * sizeof(float2), p->stream));
  PWF_CUDA(p, cudaMemsetAsync(p->M, 0, n * sizeof(float2), p->stream));
  PWF_CUDA(p, cudaMemsetAsync(p->ACC, 0, n * sizeof(float2), p->stream));
  cudaEvent_t e0, e1;
  PWF_CUDA(p, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(p, cudaGetLastError(), "cudaEventCreate");
  }
  PassArgs a = base_args(p);
  a.qx = p->ax.q1;
  a.qy = p->ay.q1;
  a.mode_mx = 3;
  a.mode_my = 5;
  a.mode_w = 1.0f;
  cudaError_t err = cudaSuccess;
  for (int m = 0; m < 2 && err == cudaSuccess; m++) {
    a.in = m == CM_FWD ? p->X : p->M;
    a.out = m == CM_FWD ? p->M : p->ACC;
    a.accumulate = m == CM_BACK;
    float best = 1e30f;
    for (int v = 0; v < p->kcol->ncolmodev[m] && err == cudaSuccess; v++) {
      const ColVariant& sh = p->kcol->colmodev[m][v];
      const PassArgs av = sched_tables(p, a, sh.sched);
      if ((err = sh.launch(av, a.B, p->stream)) != cudaSuccess) break;
      cudaEventRecord(e0, p->stream);
      for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) err = sh.launch(av, a.B, p->stream);
      cudaEventRecord(e1, p->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      p->modetime[m][v] = ms / 2.0f;
      if (err == cudaSuccess && ms < best) {
        best = ms;
        p->modesel[m] = v;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(p, err, "mode column-pass tuning");
  return PWF_OK;
}

// One iteration (enqueued by `body` on the capture stream) as a graph replayed
// once per iteration from the host.
template <class F>
pwf_status capture_step_graph(pwf_plan* p, F&& body) {
  cudaStream_t user = p->stream;
  p->stream = p->capture_stream;
  cudaGraph_t g = nullptr;
  PWF_CUDA(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  const long long before = p->launches;
  pwf_status r = body();
  p->graph_kernels = p->launches - before;
  p->launches = before;
  cudaError_t ce = cudaStreamEndCapture(p->capture_stream, &g);
  p->stream = user;
  if (r) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (ce != cudaSuccess) return cuda_fail(p, ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&p->graph, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return cuda_fail(p, ce, "cudaGraphInstantiate");
  p->graph_loop = false;
  return PWF_OK;
}

// The iteration captured into the body of a conditional WHILE node, closed by
// k_loop_control: one launch runs the loop. PWF_ERR_UNSUPPORTED (with no
// error left pending) when the driver does not take conditional nodes.
template <class F>
pwf_status capture_loop_graph(pwf_plan* p, pwf_state* st, double corr_tol, F&& body) {
  cudaGraph_t g = nullptr;
  PWF_CUDA(p, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams np{};
  cudaGraphNode_t node;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return PWF_ERR_UNSUPPORTED;
  }
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return PWF_ERR_UNSUPPORTED;
  }
  cudaGraph_t loop_body = np.conditional.phGraph_out[0];
  cudaStream_t user = p->stream;
  p->stream = p->capture_stream;
  cudaError_t ce = cudaStreamBeginCaptureToGraph(p->stream, loop_body, nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    p->stream = user;
    cudaGetLastError();
    cudaGraphDestroy(g);
    return PWF_ERR_UNSUPPORTED;
  }
  const long long before = p->launches;
  pwf_status r = body();
  if (r == PWF_OK) {
    ce = launch_pass(k_loop_control, dim3(1), dim3(32), 0, p->stream, pdl_of(p), h, (const DevIter*)st->it, p->loop_ctl,
                     corr_tol);
    if (ce != cudaSuccess) r = cuda_fail(p, ce, "k_loop_control");
    p->launches++;
  }
  p->graph_kernels = p->launches - before;
  p->launches = before;
  cudaGraph_t captured = nullptr;
  ce = cudaStreamEndCapture(p->capture_stream, &captured);
  p->stream = user;
  if (r || ce != cudaSuccess) {
    cudaGraphDestroy(g);
    return r ? r : cuda_fail(p, ce, "cudaStreamEndCapture (loop body)");
  }
  ce = cudaGraphInstantiate(&p->graph, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    p->graph = nullptr;
    return PWF_ERR_UNSUPPORTED;
  }
  p->graph_loop = true;
  return PWF_OK;
}

bool size_ok(int n) { return kernels_for_length(n) != nullptr; }

pwf_status check_plan(pwf_plan* p) {
  if (!p) return PWF_ERR_INVALID_ARG;
  if (p->sticky != PWF_OK) return p->sticky;
  return PWF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* pwf_status_string(pwf_status s) {
  switch (s) {
    case PWF_OK: return "PWF_OK";
    case PWF_ERR_INVALID_ARG: return "PWF_ERR_INVALID_ARG";
    case PWF_ERR_UNSUPPORTED: return "PWF_ERR_UNSUPPORTED";
    case PWF_ERR_NOMEM: return "PWF_ERR_NOMEM";
    case PWF_ERR_CUDA: return "PWF_ERR_CUDA";
    case PWF_ERR_NONFINITE: return "PWF_ERR_NONFINITE";
    case PWF_ERR_STATE: return "PWF_ERR_STATE";
    case PWF_ERR_TIMEOUT: return "PWF_ERR_TIMEOUT";
    case PWF_ERR_BOUNDS: return "PWF_ERR_BOUNDS";
  }
  return "PWF_ERR_UNKNOWN";
}

const char* pwf_plan_last_error(const pwf_plan* plan) { return plan ? plan->err : "null plan"; }

pwf_status pwf_plan_create(const pwf_plan_desc* desc, pwf_plan** out) {
  if (!desc || !out) return PWF_ERR_INVALID_ARG;
  *out = nullptr;
  const pwf_plan_desc& d = *desc;
  if (d.batch < 1 || d.ny < 1 || d.nx < 1 || !(d.pixel_m > 0) || !(d.wavelength_m > 0) || d.L1_m < 0 ||
      d.L2_m < 0 || d.xcoh_m < 0 || d.ycoh_m < 0 || !(d.eta > 0) || d.gamma < 0 ||
      (d.flags & ~(PWF_FLAG_NO_PRECOND | PWF_FLAG_NO_REG | PWF_FLAG_PLAIN | PWF_FLAG_NO_TUNE |
                   PWF_FLAG_PERSISTENT | PWF_FLAG_GRAPH | PWF_FLAG_CLUSTER | PWF_FLAG_NO_PDL |
                   PWF_FLAG_CHECK_FINITE | PWF_FLAG_UNPACKED_RESID)))
    return PWF_ERR_INVALID_ARG;
  {
    const uint32_t solver = d.flags & (PWF_FLAG_PERSISTENT | PWF_FLAG_GRAPH | PWF_FLAG_CLUSTER);
    if (solver & (solver - 1)) return PWF_ERR_INVALID_ARG;  // at most one way to run pwf_solve
    // the scans follow the passes one by one: not inside a single-launch solver
    if ((d.flags & PWF_FLAG_CHECK_FINITE) && (d.flags & (PWF_FLAG_PERSISTENT | PWF_FLAG_CLUSTER)))
      return PWF_ERR_UNSUPPORTED;
  }
  if (!(d.n_modes == 0 || d.n_modes == 1 || d.n_modes == 9 || d.n_modes == 25) || !(d.mode_sigma_px >= 0.0))
    return PWF_ERR_INVALID_ARG;
  if (d.n_modes > 1 && (d.flags & PWF_FLAG_PLAIN)) return PWF_ERR_UNSUPPORTED;  // baseline is the paper's form
  if (!size_ok(d.ny) || !size_ok(d.nx)) return PWF_ERR_UNSUPPORTED;
  // evanescent bins and the separable-propagator bound, in double precision
  {
    const double umax = 0.5 / d.pixel_m, il = 1.0 / d.wavelength_m;
    if (2.0 * umax * umax >= il * il) return PWF_ERR_UNSUPPORTED;
    for (double L : {d.L1_m, d.L2_m}) {
      const double cross = prop_phase(2 * umax * umax, d.wavelength_m, L) - 2 * prop_phase(umax * umax, d.wavelength_m, L);
      if (std::fabs(cross) > 1e-6) return PWF_ERR_UNSUPPORTED;
    }
  }
  pwf_plan* p = new (std::nothrow) pwf_plan();
  if (!p) return PWF_ERR_NOMEM;
  p->d = d;
  p->stream = static_cast<cudaStream_t>(d.stream);
  p->krow = kernels_for_length(d.nx);
  p->kcol = kernels_for_length(d.ny);
  p->coherent = (d.xcoh_m == 0.0 && d.ycoh_m == 0.0);
  if (d.n_modes > 1) p->modes = source_modes(d);
  const size_t n = (size_t)d.batch * d.ny * d.nx;
  pwf_status r;
  if ((r = build_axis(p, p->ax, d.nx, d.pixel_m, d.xcoh_m)) || (r = build_axis(p, p->ay, d.ny, d.pixel_m, d.ycoh_m)) ||
      (r = dalloc(p, &p->X, n)) || (r = dalloc(p, &p->S, n)) || (r = dalloc(p, &p->REG, n)) ||
      (r = dalloc(p, &p->V, n)) || (r = dalloc(p, &p->YH, n)) ||
      (r = dalloc(p, &p->acc, (size_t)d.batch * NACC)) || (r = dalloc(p, &p->maxt2, 1)) ||
      (r = dalloc(p, &p->kstatus, 1)) || (r = dalloc(p, &p->loop_ctl, 2)) ||
      ((d.flags & PWF_FLAG_CHECK_FINITE) && (r = dalloc(p, &p->scan_word, 1))) ||
      (!p->modes.empty() && ((r = dalloc(p, &p->M, n)) || (r = dalloc(p, &p->ACC, n)) ||
                             (r = dalloc(p, &p->IBUF, n))))) {
    pwf_plan_destroy(p);
    return r;
  }
  if (p->scan_word && cudaMemset(p->scan_word, 0xff, sizeof(int)) != cudaSuccess) {  // -1: no pass yet
    pwf_plan_destroy(p);
    return PWF_ERR_CUDA;
  }
  for (int op = 0; op < NUM_ROW_OPS; op++)
    if (p->krow->row_prep[op]() != cudaSuccess) {
      cudaGetLastError();
      pwf_plan_destroy(p);
      return PWF_ERR_CUDA;
    }
  for (int m = 0; m < 2; m++)
    for (int v = 0; v < p->kcol->ncolmodev[m]; v++)
      if (p->kcol->colmodev[m][v].prep() != cudaSuccess) {
        cudaGetLastError();
        pwf_plan_destroy(p);
        return PWF_ERR_CUDA;
      }
  for (int op = 0; op < NUM_COL_OPS; op++)
    for (int v = 0; v < p->kcol->ncolv[op]; v++)
      if (p->kcol->colv[op][v].prep() != cudaSuccess) {
        cudaGetLastError();
        pwf_plan_destroy(p);
        return PWF_ERR_CUDA;
      }
  if (cudaMemset(p->acc, 0, (size_t)d.batch * NACC * sizeof(double)) != cudaSuccess ||
      cudaMemset(p->kstatus, 0, sizeof(int)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    pwf_plan_destroy(p);
    return PWF_ERR_CUDA;
  }
  // persistent solver (PWF_FLAG_PERSISTENT): square IOTF/coherent plans of
  // the built sizes. Not the default: on a GB300 its grid barriers cost more
  // than the graph replay's launch gaps at every size it serves (128^2: 132
  // against 56 us per iteration; 512^2: 180 against 80)
  {
    const bool eligible = p->kcol->persist != nullptr && d.nx == d.ny && p->modes.empty() &&
                          !(d.flags & PWF_FLAG_PLAIN);
    const bool want = (d.flags & PWF_FLAG_PERSISTENT) != 0;
    if ((d.flags & (PWF_FLAG_PERSISTENT | PWF_FLAG_CLUSTER)) && !eligible) {
      pwf_plan_destroy(p);
      return PWF_ERR_UNSUPPORTED;
    }
    // With no solver asked for, the cluster-resident solver takes the plans it
    // measured faster on: lengths with its one-warp-per-transform schedule
    // (128^2: 50 against 58 us per iteration, IOTF), batches that one wave of
    // clusters holds (9 x 128^2 needed two waves: 99 against 58 us).
    const bool no_solver = !(d.flags & (PWF_FLAG_PERSISTENT | PWF_FLAG_GRAPH | PWF_FLAG_CLUSTER));
    const bool try_cluster = eligible && no_solver && !(d.flags & PWF_FLAG_CHECK_FINITE) &&
                             p->kcol->persist_cluster[1] != nullptr && p->ax.tw_fwd_alt && p->ay.tw_fwd_alt;
    if ((d.flags & PWF_FLAG_CLUSTER) || try_cluster) {
      if ((r = dalloc(p, &p->gpart, (size_t)d.batch * PERSIST_MAX_CLUSTER * NACC)) ||
          (r = dalloc(p, &p->cit, (size_t)d.batch)) || (r = dalloc(p, &p->phases, PERSIST_MAX_PHASES))) {
        pwf_plan_destroy(p);
        return r;
      }
      p->cluster_plan = true;
      r = pwf_plan_set_cluster_schedule(p, -1);
      int maxc = 0;
      if (r == PWF_OK && try_cluster &&
          (p->kcol->persist_cluster_prep[p->cluster_sched](d.batch, p->cluster, &maxc) != cudaSuccess ||
           maxc < d.batch)) {
        cudaGetLastError();
        p->cluster = 0;  // more than one wave of clusters: the graph
        p->cluster_plan = false;
      } else if (r != PWF_OK && try_cluster) {
        cudaGetLastError();
        p->cluster = 0;
        p->cluster_plan = false;
        r = PWF_OK;
      }
      if (r) {
        pwf_plan_destroy(p);
        return r;
      }
      p->err[0] = 0;
    }
    if (eligible && want) {
      int per_sm = 0;
      if (p->kcol->persist_prep(d.batch) != cudaSuccess || p->kcol->persist_occupancy(d.batch, &per_sm) != cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        if (d.flags & PWF_FLAG_PERSISTENT) {
          pwf_plan_destroy(p);
          return PWF_ERR_UNSUPPORTED;
        }
      } else {
        p->persist_grid = device_sms();
        if ((r = dalloc(p, &p->gpart, (size_t)p->persist_grid * d.batch * NACC)) || (r = dalloc(p, &p->bar, 2)) ||
            (r = dalloc(p, &p->phases, PERSIST_MAX_PHASES))) {
          pwf_plan_destroy(p);
          return r;
        }
        p->persist = true;
      }
    }
  }
  if (!(d.flags & PWF_FLAG_NO_TUNE) && ((r = tune_columns(p)) != PWF_OK ||
                                        (!p->modes.empty() && (r = tune_modes(p)) != PWF_OK))) {
    pwf_plan_destroy(p);
    return r;
  }
  *out = p;
  return PWF_OK;
}

static void host_pipe_destroy(HostPipe* hp);

pwf_status pwf_plan_destroy(pwf_plan* p) {
  if (!p) return PWF_ERR_INVALID_ARG;
  if (p->pipe) host_pipe_destroy(p->pipe);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->solve_state) pwf_state_destroy(p->solve_state);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  for (void* q : p->allocs) cudaFree(q);
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  delete p;
  return PWF_OK;
}

pwf_status pwf_plan_set_stream(pwf_plan* p, void* stream) {
  if (!p) return PWF_ERR_INVALID_ARG;
  p->stream = static_cast<cudaStream_t>(stream);
  return PWF_OK;
}

size_t pwf_plan_workspace_bytes(const pwf_plan* p) { return p ? p->ws_bytes : 0; }

pwf_status pwf_forward(pwf_plan* p, const void* psi, const void* t, float* f) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!psi || !t || !f) return PWF_ERR_INVALID_ARG;
  if (!a16(psi) || !a16(t) || !a16(f)) return misaligned(p);
  PassArgs a = base_args(p);
  if (!p->modes.empty()) {
    a.psi = (const float2*)psi;
    a.out = p->X;
    LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
    return modal_forward(p, a, (const float2*)t, f, false);
  }
  if ((r = fused_to_detector(p, a, (const float2*)psi, (const float2*)t, nullptr, true, a.B))) return r;
  a.in = p->X;
  a.out = p->X;
  a.f_out = f;
  if (p->coherent) {
    LAUNCH(p, row(p, ROW_INTENSITY_OUT, a, a.B));
  } else {
    a.v = nullptr;
    LAUNCH(p, row(p, ROW_INTENSITY, a, a.B));
    LAUNCH(p, col(p, COL_IOTF, a, a.B));
    LAUNCH(p, row(p, ROW_REAL_OUT, a, a.B));
  }
  return PWF_OK;
}

pwf_status pwf_gradient(pwf_plan* p, const void* psi, const void* t, const float* y, void* g, double* loss) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!psi || !t || !y || !g) return PWF_ERR_INVALID_ARG;
  if (!a16(psi) || !a16(t) || !a16(y) || !a16(g)) return misaligned(p);
  const float2* P = (const float2*)psi;
  if ((r = compute_maxt2(p, (const float2*)t))) return r;
  PWF_CUDA(p, cudaMemsetAsync(p->acc, 0, (size_t)p->d.batch * NACC * sizeof(double), p->stream));
  PassArgs a = base_args(p);
  if (!p->modes.empty()) {
    a.psi = P;
    a.out = p->X;
    LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
    if ((r = ensure_vstack(p)) || (r = modal_forward(p, a, (const float2*)t, p->IBUF, true)) ||
        (r = modal_resid(p, y, nullptr)) || (r = modal_backward(p, a, (const float2*)t, p->IBUF)))
      return r;
    a.in = p->ACC;
    a.g_out = (float2*)g;
    a.div_maxt2 = 1;
    a.gscale = 1.0f;
    LAUNCH(p, row(p, ROW_GRAD_OUT, a, a.B));
    if (loss) {
      k_gather_loss<<<(a.B + 255) / 256, 256, 0, p->stream>>>(p->acc, loss, a.B);
      PWF_CUDA(p, cudaGetLastError());
    }
    return PWF_OK;
  }
  if ((r = fused_to_detector(p, a, P, (const float2*)t, nullptr, true, a.B))) return r;
  a.in = p->X;
  a.out = p->X;
  a.y = y;
  if (p->coherent) {
    LAUNCH(p, row(p, ROW_COH_RESID, a, a.B));
  } else {
    a.v = p->V;
    LAUNCH(p, row(p, ROW_INTENSITY, a, a.B));   // |v|^2, v kept
    LAUNCH(p, col(p, COL_IOTF, a, a.B));        // f = F^-1{IOTF F{|v|^2}}
    LAUNCH(p, row(p, ROW_RESID, a, a.B));       // e = y - f; loss; -e
    LAUNCH(p, col(p, COL_IOTF, a, a.B));        // F^-1{IOTF F{-e}}
    LAUNCH(p, row(p, ROW_MUL_V, a, a.B));       // v g
  }
  if ((r = fused_backprop(p, a, (const float2*)t, false, a.B))) return r;
  a.psi = P;
  a.g_out = (float2*)g;
  a.div_maxt2 = 1;
  a.gscale = 1.0f;
  LAUNCH(p, row(p, ROW_GRAD_OUT, a, a.B));
  if (loss) {
    k_gather_loss<<<(a.B + 255) / 256, 256, 0, p->stream>>>(p->acc, loss, a.B);
    PWF_CUDA(p, cudaGetLastError());
  }
  return PWF_OK;
}

pwf_status pwf_forward_vjp(pwf_plan* p, const void* psi, const void* t, const float* grad_f, void* grad_psi,
                           void* grad_t) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!psi || !t || !grad_f) return PWF_ERR_INVALID_ARG;
  if (!a16(psi) || !a16(t) || !a16(grad_f) || !a16(grad_psi) || !a16(grad_t)) return misaligned(p);
  if (!grad_psi && !grad_t) return PWF_OK;
  const float2* P = (const float2*)psi;
  PassArgs a = base_args(p);
  if (!p->modes.empty()) {
    // per mode: forward to v_j, then straight back (v_j recomputed, never stored)
    const float2* T = (const float2*)t;
    a.psi = P;
    a.out = p->X;
    LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
    if ((r = spectrum_for_modes(p, a, a.B))) return r;
    for (size_t j = 0; j < p->modes.size(); j++) {
      const Mode& md = p->modes[j];
      PassArgs b = a;
      b.in = p->X;
      b.out = p->M;
      LAUNCH(p, colmode(p, CM_FWD, b, md, 0, a.B));
      b.in = p->M;
      b.t = T;
      b.u1 = grad_t ? p->S : nullptr;
      LAUNCH(p, row(p, ROW_MUL_T, b, a.B));
      b.u1 = nullptr;
      LAUNCH(p, col_q(p, b, 2, 0, a.B));
      b.out = p->V;
      LAUNCH(p, row(p, ROW_IFFT, b, a.B));          // v_j
      b.v = p->V;
      b.y = grad_f;
      b.out = p->M;
      LAUNCH(p, row(p, ROW_MODE_VG, b, a.B));       // v_j dL/df
      b.in = p->M;
      LAUNCH(p, col_q(p, b, 2, 1, a.B));            // P2^H
      if (grad_t) {
        b.u1 = p->S;
        b.gt_scratch = p->YH;
        b.mode_w = md.w;
        b.accumulate = j > 0;
        LAUNCH(p, row(p, ROW_GRADT, b, a.B));
        b.u1 = nullptr;
      } else {
        b.conj_t = 1;
        LAUNCH(p, row(p, ROW_MUL_T, b, a.B));
      }
      b.out = p->ACC;
      LAUNCH(p, colmode(p, CM_BACK, b, md, j > 0, a.B));
    }
    if (grad_t) {
      const size_t n = (size_t)p->d.ny * p->d.nx;
      k_batch_sum<<<grid_for(n), 256, 0, p->stream>>>(p->YH, (float2*)grad_t, a.B, n);
      PWF_CUDA(p, cudaGetLastError());
    }
    if (grad_psi) {
      if ((r = accumulated_from_spectrum(p, a, a.B))) return r;
      a.in = p->ACC;
      a.g_out = (float2*)grad_psi;
      a.div_maxt2 = 0;
      a.gscale = 2.0f;
      LAUNCH(p, row(p, ROW_GRAD_OUT, a, a.B));
    }
    return PWF_OK;
  }
  if ((r = fused_to_detector(p, a, P, (const float2*)t, grad_t ? p->S : nullptr, true, a.B))) return r;
  a.in = p->X;
  a.out = p->X;
  if (p->coherent) {
    a.y = grad_f;
    LAUNCH(p, row(p, ROW_COH_VJP, a, a.B));     // v grad_f
  } else {
    a.out = p->V;
    LAUNCH(p, row(p, ROW_IFFT, a, a.B));        // v
    a.out = p->X;
    a.y = grad_f;
    LAUNCH(p, row(p, ROW_REAL_FFT, a, a.B));    // F_row{grad_f}
    LAUNCH(p, col(p, COL_IOTF, a, a.B));        // F^-1{IOTF F{grad_f}}
    a.v = p->V;
    LAUNCH(p, row(p, ROW_MUL_V, a, a.B));       // v G
  }
  if ((r = fused_backprop(p, a, (const float2*)t, grad_t != nullptr, a.B))) return r;
  if (grad_t) {
    const size_t n = (size_t)p->d.ny * p->d.nx;
    k_batch_sum<<<grid_for(n), 256, 0, p->stream>>>(p->YH, (float2*)grad_t, a.B, n);
    PWF_CUDA(p, cudaGetLastError());
  }
  if (grad_psi) {
    a.psi = P;
    a.g_out = (float2*)grad_psi;
    a.div_maxt2 = 0;
    a.gscale = 2.0f;
    LAUNCH(p, row(p, ROW_GRAD_OUT, a, a.B));
  }
  return PWF_OK;
}

pwf_status pwf_state_create(pwf_plan* p, pwf_state** out) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!out) return PWF_ERR_INVALID_ARG;
  pwf_state* s = new (std::nothrow) pwf_state();
  if (!s) return PWF_ERR_NOMEM;
  s->B = p->d.batch;
  s->ny = p->d.ny;
  s->nx = p->d.nx;
  const size_t n = (size_t)s->B * s->ny * s->nx;
  bool ok = cudaMalloc(&s->phi, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&s->active, s->B * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&s->iters, s->B * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&s->loss, s->B * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->corr, s->B * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->it, sizeof(DevIter)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pwf_state_destroy(s);
    return PWF_ERR_NOMEM;
  }
  if ((r = pwf_state_reset(p, s))) {
    pwf_state_destroy(s);
    return r;
  }
  *out = s;
  return PWF_OK;
}

pwf_status pwf_state_destroy(pwf_state* s) {
  if (!s) return PWF_ERR_INVALID_ARG;
  cudaFree(s->phi);
  cudaFree(s->active);
  cudaFree(s->iters);
  cudaFree(s->loss);
  cudaFree(s->corr);
  cudaFree(s->it);
  delete s;
  return PWF_OK;
}

pwf_status pwf_state_reset(pwf_plan* p, pwf_state* s) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!s) return PWF_ERR_INVALID_ARG;
  if (s->B != p->d.batch || s->ny != p->d.ny || s->nx != p->d.nx) return PWF_ERR_STATE;
  PWF_CUDA(p, cudaMemsetAsync(s->phi, 0, (size_t)s->B * s->ny * s->nx * sizeof(float2), p->stream));
  PWF_CUDA(p, cudaMemsetAsync(p->acc, 0, (size_t)s->B * NACC * sizeof(double), p->stream));
  if (p->scan_word) PWF_CUDA(p, cudaMemsetAsync(p->scan_word, 0xff, sizeof(int), p->stream));  // -1: none yet
  k_state_reset<<<1, 256, 0, p->stream>>>(s->it, s->active, s->iters, s->loss, s->corr, s->B);
  p->launches++;
  PWF_CUDA(p, cudaGetLastError());
  return PWF_OK;
}

pwf_status pwf_step(pwf_plan* p, pwf_state* st, const float* y, const void* t, void* psi, double corr_tol) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!st || !y || !t || !psi) return PWF_ERR_INVALID_ARG;
  if (!a16(y) || !a16(t) || !a16(psi)) return misaligned(p);
  if (st->B != p->d.batch || st->ny != p->d.ny || st->nx != p->d.nx) return PWF_ERR_STATE;
  float2* P = (float2*)psi;
  if (!p->modes.empty() && (r = ensure_vstack(p))) return r;
  if ((r = compute_maxt2(p, (const float2*)t))) return r;
  PWF_CUDA(p, cudaMemsetAsync(p->acc, 0, (size_t)p->d.batch * NACC * sizeof(double), p->stream));
  if (p->d.flags & PWF_FLAG_PLAIN) {
    // host-driven: read the convergence flags, then one projection at a time
    std::vector<int> act(p->d.batch);
    PWF_CUDA(p, cudaMemcpyAsync(act.data(), st->active, p->d.batch * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PWF_CUDA(p, cudaStreamSynchronize(p->stream));
    for (int b = 0; b < p->d.batch; b++)
      if (act[b] && (r = plain_iteration(p, st, y, (const float2*)t, P, b))) return r;
    k_finalize<<<1, 256, 0, p->stream>>>(p->acc, p->d.batch, st->active, st->iters, st->loss, st->corr, st->it,
                                         corr_tol);
    PWF_CUDA(p, cudaGetLastError());
    return PWF_OK;
  }
  if (!p->coherent && (r = compute_yhat(p, y, st->active))) return r;
  PassArgs a = base_args(p);
  a.active = st->active;
  a.psi = P;
  a.out = p->X;
  LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
  return fused_iteration(p, st, y, (const float2*)t, P, false, corr_tol);
}

pwf_status pwf_state_read(pwf_plan* p, const pwf_state* s, double* loss_host, double* corr_host,
                          int32_t* iters_host, int32_t* active_host) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!s) return PWF_ERR_INVALID_ARG;
  if (loss_host) PWF_CUDA(p, cudaMemcpyAsync(loss_host, s->loss, s->B * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  if (corr_host) PWF_CUDA(p, cudaMemcpyAsync(corr_host, s->corr, s->B * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  if (iters_host) PWF_CUDA(p, cudaMemcpyAsync(iters_host, s->iters, s->B * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  if (active_host) PWF_CUDA(p, cudaMemcpyAsync(active_host, s->active, s->B * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  PWF_CUDA(p, cudaStreamSynchronize(p->stream));
  DevIter it;
  PWF_CUDA(p, cudaMemcpy(&it, s->it, sizeof(DevIter), cudaMemcpyDeviceToHost));
  int ks = 0;
  PWF_CUDA(p, cudaMemcpy(&ks, p->kstatus, sizeof(int), cudaMemcpyDeviceToHost));
  if (ks != 0) {
    cudaMemset(p->kstatus, 0, sizeof(int));
    if (ks == PWF_ERR_BOUNDS) return fail(p, PWF_ERR_BOUNDS, "an index check of a pass failed");
    return fail(p, PWF_ERR_TIMEOUT, "a bounded wait for a tile copy ran out");
  }
  if (it.status == PWF_ERR_TIMEOUT) return fail(p, PWF_ERR_TIMEOUT, "a grid barrier of the persistent solver ran out");
  if (p->scan_word) {
    int id = -1;
    PWF_CUDA(p, cudaMemcpy(&id, p->scan_word, sizeof(int), cudaMemcpyDeviceToHost));
    if (id >= 0 && id < (int)p->scan_names.size()) {
      char msg[96];
      std::snprintf(msg, sizeof(msg), "first non-finite values written by pass %s", p->scan_names[id]);
      return fail(p, PWF_ERR_NONFINITE, msg);
    }
  }
  if (it.nonfinite) return fail(p, PWF_ERR_NONFINITE, "non-finite loss or iterate");
  return PWF_OK;
}

static pwf_status solve_impl(pwf_plan* p, const float* y, const void* t, void* psi, int32_t max_iter,
                             double corr_tol, int32_t* iters_host, double* loss_host, double eta_t);

pwf_status pwf_solve(pwf_plan* p, const float* y, const void* t, void* psi, int32_t max_iter, double corr_tol,
                     int32_t* iters_host, double* loss_host) {
  return solve_impl(p, y, t, psi, max_iter, corr_tol, iters_host, loss_host, -1.0);
}

pwf_status pwf_solve_joint(pwf_plan* p, const float* y, void* t, void* psi, int32_t max_iter, double eta_t,
                           int32_t* iters_host, double* loss_host) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!(eta_t >= 0.0)) return PWF_ERR_INVALID_ARG;
  if (!p->modes.empty() || (p->d.flags & PWF_FLAG_PLAIN))
    return fail(p, PWF_ERR_UNSUPPORTED, "joint refinement runs the fused single-chain IOTF/coherent path");
  return solve_impl(p, y, t, psi, max_iter, 0.0, iters_host, loss_host, eta_t);
}

static pwf_status solve_impl(pwf_plan* p, const float* y, const void* t, void* psi, int32_t max_iter,
                             double corr_tol, int32_t* iters_host, double* loss_host, double eta_t) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!y || !t || !psi || max_iter < 0) return PWF_ERR_INVALID_ARG;
  if (!a16(y) || !a16(t) || !a16(psi)) return misaligned(p);
  const bool joint = eta_t >= 0.0;
  if (!p->solve_state && (r = pwf_state_create(p, &p->solve_state))) return r;
  if (!p->modes.empty() && (r = ensure_vstack(p))) return r;  // before the graph capture
  if (joint && !p->GT && (r = dalloc(p, &p->GT, (size_t)p->d.batch * p->d.ny * p->d.nx))) return r;
  pwf_state* st = p->solve_state;
  if ((r = pwf_state_reset(p, st))) return r;
  float2* P = (float2*)psi;
  if (p->d.flags & PWF_FLAG_PLAIN) {
    for (int k = 0; k < max_iter; k++)
      if ((r = pwf_step(p, st, y, t, psi, corr_tol))) return r;
  } else if (max_iter > 0) {
    if ((r = compute_maxt2(p, (const float2*)t))) return r;
    if (!p->coherent && (r = compute_yhat(p, y, st->active))) return r;
    PassArgs a = base_args(p);
    a.active = st->active;
    a.psi = P;
    a.out = p->X;
    LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
    if ((p->persist || p->cluster > 0) && !joint) {
      if ((r = persist_solve(p, st, y, (const float2*)t, P, max_iter, corr_tol))) return r;
      if (iters_host || loss_host) return pwf_state_read(p, st, loss_host, nullptr, iters_host, nullptr);
      return PWF_OK;
    }
    // The whole loop as one graph: one fused iteration captured into the body
    // of a conditional WHILE node whose condition the iteration's last kernel
    // sets, so that a solve is a single graph launch and the loop runs on the
    // device (re-captured when the operands change). If the driver refuses
    // conditional nodes, the single-iteration graph is replayed from the host.
    const void* key[4] = {y, t, psi, p->stream};
    if (!p->graph || std::memcmp(key, p->graph_key, sizeof(key)) != 0 || p->graph_tol != corr_tol ||
        p->graph_eta_t != (joint ? eta_t : -1.0)) {
      if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
      }
      auto body = [&]() {
        return joint ? fused_iteration(p, st, y, (const float2*)t, P, true, corr_tol, (float2*)t, eta_t)
                     : fused_iteration(p, st, y, (const float2*)t, P, true, corr_tol);
      };
      if ((r = capture_loop_graph(p, st, corr_tol, body)) == PWF_ERR_UNSUPPORTED) r = capture_step_graph(p, body);
      if (r) return r;
      std::memcpy(p->graph_key, key, sizeof(key));
      p->graph_tol = corr_tol;
      p->graph_eta_t = joint ? eta_t : -1.0;
    }
    if (p->graph_loop) {
      const int ctl[2] = {max_iter, 0};
      PWF_CUDA(p, cudaMemcpyAsync(p->loop_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, p->stream));
      PWF_CUDA(p, cudaGraphLaunch(p->graph, p->stream));
      p->launches += p->graph_kernels * max_iter;  // at most: the loop may stop early
    } else {
      const int check_every = 16;
      for (int k = 0; k < max_iter; k++) {
        PWF_CUDA(p, cudaGraphLaunch(p->graph, p->stream));
        p->launches += p->graph_kernels;
        if (corr_tol > 0.0 && (k + 1) % check_every == 0 && k + 1 < max_iter) {
          DevIter it;
          PWF_CUDA(p, cudaMemcpyAsync(&it, st->it, sizeof(DevIter), cudaMemcpyDeviceToHost, p->stream));
          PWF_CUDA(p, cudaStreamSynchronize(p->stream));
          if (it.n_active == 0) break;
        }
      }
    }
  }
  if (iters_host || loss_host) return pwf_state_read(p, st, loss_host, nullptr, iters_host, nullptr);
  return PWF_OK;
}

// ---------------------------------------------------------------------------
// solve from host buffers
// ---------------------------------------------------------------------------
// The batch streams through the device in chunks of `chunk` projections and
// two device slots, each with a plan of batch `chunk` (its own workspace and
// captured iteration graph): while chunk k is solved on the run stream, the
// inputs of chunk k + 1 arrive on the copy-in stream and the result of chunk
// k - 1 leaves on the copy-out stream. Per-projection results and each
// chunk's status word go to pinned staging on the run stream.
struct HostPipe {
  int chunk = 0;
  pwf_plan* sub[2] = {nullptr, nullptr};
  float* y[2] = {nullptr, nullptr};
  float2* psi[2] = {nullptr, nullptr};
  float2* t = nullptr;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  cudaEvent_t start = nullptr, in_done[2] = {}, run_done[2] = {}, out_done[2] = {};
  int* h_iters = nullptr;   // pinned, [B]
  double* h_loss = nullptr; // pinned, [B]
  DevIter* h_it = nullptr;  // pinned, one per chunk
};

static void host_pipe_destroy(HostPipe* hp) {
  if (!hp) return;
  for (int s = 0; s < 2; s++) {
    if (hp->sub[s]) pwf_plan_destroy(hp->sub[s]);
    if (hp->y[s]) cudaFree(hp->y[s]);
    if (hp->psi[s]) cudaFree(hp->psi[s]);
    for (cudaEvent_t e : {hp->in_done[s], hp->run_done[s], hp->out_done[s]})
      if (e) cudaEventDestroy(e);
  }
  if (hp->t) cudaFree(hp->t);
  if (hp->start) cudaEventDestroy(hp->start);
  for (cudaStream_t st : {hp->s_in, hp->s_run, hp->s_out})
    if (st) cudaStreamDestroy(st);
  if (hp->h_iters) cudaFreeHost(hp->h_iters);
  if (hp->h_loss) cudaFreeHost(hp->h_loss);
  if (hp->h_it) cudaFreeHost(hp->h_it);
  delete hp;
}

// the largest divisor of B that is at most ceil(B / 4): four chunks when B allows
static int default_chunk(int B) {
  const int cap = (B + 3) / 4;
  for (int c = cap; c > 1; c--)
    if (B % c == 0) return c;
  return 1;
}

static pwf_status host_pipe_ensure(pwf_plan* p, int chunk) {
  if (p->pipe && p->pipe->chunk == chunk) return PWF_OK;
  if (p->pipe) {
    host_pipe_destroy(p->pipe);
    p->pipe = nullptr;
  }
  HostPipe* hp = new HostPipe();
  hp->chunk = chunk;
  const size_t npx = (size_t)p->d.ny * p->d.nx, per = (size_t)chunk * npx;
  cudaError_t e = cudaSuccess;
  for (cudaStream_t* st : {&hp->s_in, &hp->s_run, &hp->s_out})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->start, cudaEventDisableTiming);
  for (int s = 0; s < 2 && e == cudaSuccess; s++) {
    for (cudaEvent_t* ev : {&hp->in_done[s], &hp->run_done[s], &hp->out_done[s]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&hp->y[s], per * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&hp->psi[s], per * sizeof(float2));
  }
  if (e == cudaSuccess) e = cudaMalloc(&hp->t, npx * sizeof(float2));
  if (e == cudaSuccess) e = cudaHostAlloc(&hp->h_iters, p->d.batch * sizeof(int), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&hp->h_loss, p->d.batch * sizeof(double), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&hp->h_it, p->d.batch * sizeof(DevIter), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    host_pipe_destroy(hp);
    return e == cudaErrorMemoryAllocation ? fail(p, PWF_ERR_NOMEM, "host pipeline buffers")
                                          : cuda_fail(p, e, "host pipeline setup");
  }
  pwf_plan_desc d = p->d;
  d.batch = chunk;
  d.stream = hp->s_run;
  for (int s = 0; s < 2; s++) {
    pwf_status r = pwf_plan_create(&d, &hp->sub[s]);
    if (r) {
      host_pipe_destroy(hp);
      return fail(p, r, "host pipeline: plan for one chunk");
    }
  }
  p->pipe = hp;
  return PWF_OK;
}

// Enqueues the chunks of one pwf_solve_host call on the pipeline's streams.
static pwf_status host_pipe_enqueue(pwf_plan* p, HostPipe& hp, const float* yh, const void* t_host, float2* ph,
                                    int32_t psi_is_input, int32_t max_iter, double corr_tol) {
  const int chunk = hp.chunk, nch = p->d.batch / chunk;
  const size_t npx = (size_t)p->d.ny * p->d.nx, per = (size_t)chunk * npx;
  pwf_status r;
  // after whatever the caller queued on the plan's stream
  PWF_CUDA(p, cudaEventRecord(hp.start, p->stream));
  PWF_CUDA(p, cudaStreamWaitEvent(hp.s_in, hp.start, 0));
  PWF_CUDA(p, cudaStreamWaitEvent(hp.s_run, hp.start, 0));
  PWF_CUDA(p, cudaMemcpyAsync(hp.t, t_host, npx * sizeof(float2), cudaMemcpyHostToDevice, hp.s_in));
  for (int k = 0; k < nch; k++) {
    const int s = k & 1;
    if (k >= 2) PWF_CUDA(p, cudaStreamWaitEvent(hp.s_in, hp.out_done[s], 0));  // slot s is free again
    PWF_CUDA(p, cudaMemcpyAsync(hp.y[s], yh + k * per, per * sizeof(float), cudaMemcpyHostToDevice, hp.s_in));
    if (psi_is_input)
      PWF_CUDA(p, cudaMemcpyAsync(hp.psi[s], ph + k * per, per * sizeof(float2), cudaMemcpyHostToDevice, hp.s_in));
    else
      PWF_CUDA(p, cudaMemsetAsync(hp.psi[s], 0, per * sizeof(float2), hp.s_in));
    PWF_CUDA(p, cudaEventRecord(hp.in_done[s], hp.s_in));
    PWF_CUDA(p, cudaStreamWaitEvent(hp.s_run, hp.in_done[s], 0));
    pwf_plan* q = hp.sub[s];
    if ((r = solve_impl(q, hp.y[s], hp.t, hp.psi[s], max_iter, corr_tol, nullptr, nullptr, -1.0)))
      return fail(p, r, q->err);
    const pwf_state* st = q->solve_state;
    PWF_CUDA(p, cudaMemcpyAsync(hp.h_iters + k * chunk, st->iters, chunk * sizeof(int), cudaMemcpyDeviceToHost,
                                hp.s_run));
    PWF_CUDA(p, cudaMemcpyAsync(hp.h_loss + k * chunk, st->loss, chunk * sizeof(double), cudaMemcpyDeviceToHost,
                                hp.s_run));
    PWF_CUDA(p, cudaMemcpyAsync(hp.h_it + k, st->it, sizeof(DevIter), cudaMemcpyDeviceToHost, hp.s_run));
    PWF_CUDA(p, cudaEventRecord(hp.run_done[s], hp.s_run));
    PWF_CUDA(p, cudaStreamWaitEvent(hp.s_out, hp.run_done[s], 0));
    PWF_CUDA(p, cudaMemcpyAsync(ph + k * per, hp.psi[s], per * sizeof(float2), cudaMemcpyDeviceToHost, hp.s_out));
    PWF_CUDA(p, cudaEventRecord(hp.out_done[s], hp.s_out));
  }
  return PWF_OK;
}

pwf_status pwf_solve_host(pwf_plan* p, const float* y_host, const void* t_host, void* psi_host, int32_t psi_is_input,
                          int32_t max_iter, double corr_tol, int32_t chunk, int32_t* iters_host, double* loss_host) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!y_host || !t_host || !psi_host || max_iter < 0 || chunk < 0) return PWF_ERR_INVALID_ARG;
  const int B = p->d.batch;
  if (chunk == 0) chunk = default_chunk(B);
  if (chunk > B || B % chunk != 0) return fail(p, PWF_ERR_INVALID_ARG, "chunk must divide the batch");
  if ((r = host_pipe_ensure(p, chunk))) return r;
  HostPipe& hp = *p->pipe;
  r = host_pipe_enqueue(p, hp, y_host, t_host, static_cast<float2*>(psi_host), psi_is_input, max_iter, corr_tol);
  // wait for every stream even after an error: no copy may still be writing
  // the caller's host buffers when the call returns
  const cudaError_t e_out = cudaStreamSynchronize(hp.s_out);
  const cudaError_t e_run = cudaStreamSynchronize(hp.s_run);
  const cudaError_t e_in = cudaStreamSynchronize(hp.s_in);
  if (r) return r;
  for (cudaError_t e : {e_out, e_run, e_in})
    if (e != cudaSuccess) return cuda_fail(p, e, "pwf_solve_host");
  if (iters_host) std::memcpy(iters_host, hp.h_iters, B * sizeof(int));
  if (loss_host) std::memcpy(loss_host, hp.h_loss, B * sizeof(double));
  for (int k = 0; k < B / chunk; k++)
    if (hp.h_it[k].nonfinite) return fail(p, PWF_ERR_NONFINITE, "non-finite loss");
  return PWF_OK;
}

long long pwf_plan_launch_count(const pwf_plan* p) { return p ? p->launches : -1; }

pwf_status pwf_plan_set_wait_limit(pwf_plan* p, int64_t cycles) {
  if (!p || cycles < 0) return PWF_ERR_INVALID_ARG;
  p->wait_cap = (long long)cycles;
  return PWF_OK;
}

int32_t pwf_plan_uses_persistent(const pwf_plan* p) { return p ? (p->cluster > 0 ? 2 : p->persist ? 1 : 0) : -1; }

// threads per transform of length n in schedule set `set` of its kernels
int set_tpf(const LengthKernels* k, int set, int n) {
  int e = 1;
  for (int i = 0; i < k->sched_stages[set]; i++) {
    int a = e, b = k->sched_radix[set][i];
    while (b) {
      const int r = a % b;
      a = b;
      b = r;
    }
    e = e / a * k->sched_radix[set][i];
  }
  return n / e;
}

pwf_status pwf_plan_set_cluster_size(pwf_plan* p, int32_t ctas) {
  if (!p || !p->kcol || !p->kcol->persist_cluster[p->cluster_sched] || !p->cluster_plan || ctas < 0 ||
      ctas > PERSIST_MAX_CLUSTER)
    return PWF_ERR_INVALID_ARG;
  PersistClusterPrepFn prep = p->kcol->persist_cluster_prep[p->cluster_sched];
  if (ctas == 0) {
    // One warp-sized item (32 / (threads per transform) rows or columns) runs
    // as a serial chain on its warp, so the pass takes as long as its longest
    // chain: the default spreads the items over as many SMs as one cluster
    // can hold (measured at 128^2: 105 us per iteration on 2 CTAs, 71 on 8,
    // 71 on 16), at most one CTA per item.
    const int per_item = 32 / set_tpf(p->kcol, p->cluster_sched, p->d.nx);
    const int items = p->d.nx / per_item;
    int cs = PERSIST_MAX_CLUSTER;
    while (cs > 1 && cs > items) cs /= 2;
    for (; cs >= 1; cs /= 2) {
      int maxc = 0;
      if (prep(p->d.batch, cs, &maxc) == cudaSuccess && maxc > 0) break;
      cudaGetLastError();
    }
    if (cs < 1) return fail(p, PWF_ERR_UNSUPPORTED, "no cluster shape of the cluster-resident solver fits");
    p->cluster = cs;
    return PWF_OK;
  }
  int maxc = 0;
  if (prep(p->d.batch, ctas, &maxc) != cudaSuccess || maxc < 1) {
    cudaGetLastError();
    return fail(p, PWF_ERR_UNSUPPORTED, "this cluster shape does not fit on the device");
  }
  p->cluster = ctas;
  return PWF_OK;
}

int32_t pwf_plan_cluster_size(const pwf_plan* p) { return p ? p->cluster : -1; }

pwf_status pwf_plan_set_cluster_schedule(pwf_plan* p, int32_t set) {
  if (!p || !p->kcol || !p->cluster_plan || set < -1 || set > 1) return PWF_ERR_INVALID_ARG;
  const bool alt = p->kcol->persist_cluster[1] != nullptr && p->ax.tw_fwd_alt != nullptr && p->ay.tw_fwd_alt != nullptr;
  if (set == -1) set = alt ? 1 : 0;  // the shorter chains per thread where built
  if (set == 1 && !alt) return fail(p, PWF_ERR_UNSUPPORTED, "no alternative schedule of the cluster solver here");
  if (!p->kcol->persist_cluster[set]) return fail(p, PWF_ERR_UNSUPPORTED, "cluster solver not built for this length");
  const int old = p->cluster_sched;
  p->cluster_sched = set;
  const pwf_status r = pwf_plan_set_cluster_size(p, 0);
  if (r) p->cluster_sched = old;
  return r;
}

int32_t pwf_plan_cluster_schedule(const pwf_plan* p) { return p ? (p->cluster > 0 ? p->cluster_sched : -1) : -1; }

void pwf_debug_fail_alloc(int32_t after) { g_fail_alloc.store(after < 0 ? -1 : after); }

pwf_status pwf_debug_overrun(pwf_plan* p) {
  pwf_status r = check_plan(p);
  if (r) return r;
#ifndef PWF_BOUNDS_CHECK
  return fail(p, PWF_ERR_UNSUPPORTED, "only a bounds-checked build (PWF_BOUNDS_CHECK) runs the overrun check");
#else
  // every row of the extra projection fails its index check before any access
  PassArgs a = base_args(p);
  a.in = p->X;
  a.out = p->X;
  a.pdl = 0;
  const PassArgs ra = row_args(p, a);
  PWF_CUDA(p, p->krow->row[ROW_FFT](ra, p->d.batch + 1, p->stream));
  PWF_CUDA(p, cudaStreamSynchronize(p->stream));
  int ks = 0;
  PWF_CUDA(p, cudaMemcpy(&ks, p->kstatus, sizeof(int), cudaMemcpyDeviceToHost));
  PWF_CUDA(p, cudaMemset(p->kstatus, 0, sizeof(int)));
  if (ks == PWF_ERR_BOUNDS) return fail(p, PWF_ERR_BOUNDS, "rows beyond the plan's batch were caught and skipped");
  return ks ? fail(p, (pwf_status)ks, "unexpected status word") : PWF_OK;
#endif
}

int32_t pwf_plan_column_shapes(const pwf_plan* p, int32_t pass) {
  if (!p || pass < 0 || pass >= NUM_COL_OPS + 2) return -1;
  return pass < NUM_COL_OPS ? p->kcol->ncolv[pass] : p->kcol->ncolmodev[pass - NUM_COL_OPS];
}

pwf_status pwf_plan_set_column_shape(pwf_plan* p, int32_t pass, int32_t shape) {
  if (!p || pass < 0 || pass >= NUM_COL_OPS + 2 || shape < 0 || shape >= pwf_plan_column_shapes(p, pass))
    return PWF_ERR_INVALID_ARG;
  if (pass < NUM_COL_OPS && !shape_fits(p, pass, p->kcol->colv[pass][shape]))
    return fail(p, PWF_ERR_UNSUPPORTED, "column shape does not fit this plan's nx");
  if (pass < NUM_COL_OPS)
    p->colsel[pass] = shape;
  else
    p->modesel[pass - NUM_COL_OPS] = shape;
  if (p->graph) {  // the captured iteration used the previous shapes
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return PWF_OK;
}

size_t pwf_plan_describe(const pwf_plan* p, char* buf, size_t len) {
  if (!p) return 0;
  char tmp[8192];
  size_t o = 0;
  // appends while room is left (a longer description is cut, never overrun)
  auto put = [&](const char* fmt, auto... args) {
    if (o >= sizeof(tmp) - 1) return;
    const int w = std::snprintf(tmp + o, sizeof(tmp) - o, fmt, args...);
    if (w > 0) o = std::min(sizeof(tmp) - 1, o + (size_t)w);
  };
  auto shape = [&](const ColVariant& v) {
    put("C%d%s", v.C, v.pipe == MODE_PAIR ? "x2" : v.pipe == 5 ? "tma2" : v.pipe == 4 ? "s2" : v.pipe == 3 ? "p2"
                      : v.pipe == 2 ? "t" : v.pipe ? "p" : "");
    if (v.sched == 1)  // built with the alternative radix schedule: its radices
      for (int i = 0; i < p->kcol->sched_stages[1]; i++) put("%s%d", i ? "." : "@", p->kcol->sched_radix[1][i]);
  };
  tmp[0] = 0;
  put("ny=%d nx=%d batch=%d solver=%s loop=%s", p->d.ny, p->d.nx, p->d.batch,
      p->cluster > 0 ? "cluster" : p->persist ? "persistent" : "graph",
      p->persist || p->cluster > 0 ? "device" : !p->graph ? "none" : p->graph_loop ? "device" : "host");
  if (p->cluster > 0) {
    put(" cluster_ctas=%d cluster_schedule=", p->cluster);
    for (int i = 0; i < p->kcol->sched_stages[p->cluster_sched]; i++)
      put("%s%d", i ? "." : "", p->kcol->sched_radix[p->cluster_sched][i]);
  }
  for (int op = 0; op < NUM_COL_OPS; op++) {
    put(" %s=", kColNames[op]);
    shape(p->kcol->colv[op][p->colsel[op]]);
    if (p->coltime[op][0] > 0.f) {  // tuned: all candidates with their times
      put("%s", "[");
      for (int v = 0; v < p->kcol->ncolv[op]; v++) {
        shape(p->kcol->colv[op][v]);
        put(":%.3f%s", p->coltime[op][v], v + 1 < p->kcol->ncolv[op] ? "," : "]");
      }
    }
  }
  for (int m = 0; m < 2 && !p->modes.empty(); m++) {
    put(" %s=", m == CM_FWD ? "col_mode_fwd" : "col_mode_back");
    shape(p->kcol->colmodev[m][p->modesel[m]]);
    if (p->modetime[m][0] > 0.f) {
      put("%s", "[");
      for (int v = 0; v < p->kcol->ncolmodev[m]; v++) {
        shape(p->kcol->colmodev[m][v]);
        put(":%.3f%s", p->modetime[m][v], v + 1 < p->kcol->ncolmodev[m] ? "," : "]");
      }
    }
  }
  if (buf && len) std::snprintf(buf, len, "%s", tmp);
  return std::strlen(tmp) + 1;
}

pwf_status pwf_profile_iteration(pwf_plan* p, const float* y, const void* t, void* psi, int32_t iters,
                                 float* pass_ms, const char** pass_names, int32_t* n_passes) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!y || !t || !psi || iters < 1 || !pass_ms || !pass_names || !n_passes) return PWF_ERR_INVALID_ARG;
  if (!a16(y) || !a16(t) || !a16(psi)) return misaligned(p);
  if (p->d.flags & PWF_FLAG_PLAIN) return PWF_ERR_UNSUPPORTED;
  if (!p->solve_state && (r = pwf_state_create(p, &p->solve_state))) return r;
  if (!p->modes.empty() && (r = ensure_vstack(p))) return r;
  pwf_state* st = p->solve_state;
  if ((r = pwf_state_reset(p, st)) || (r = compute_maxt2(p, (const float2*)t))) return r;
  if (!p->coherent && (r = compute_yhat(p, y, st->active))) return r;
  PassArgs a = base_args(p);
  a.active = st->active;
  a.psi = (const float2*)psi;
  a.out = p->X;
  LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
  p->prof_names.clear();
  p->prof_n = 0;
  p->prof = true;
  for (int k = 0; k < iters && r == PWF_OK; k++) r = fused_iteration(p, st, y, (const float2*)t, (float2*)psi, true, 0.0);
  p->prof = false;
  if (r) return r;
  PWF_CUDA(p, cudaStreamSynchronize(p->stream));
  const size_t total = p->prof_names.size();
  const size_t per = total / (size_t)iters;
  if (per == 0 || per > PWF_MAX_PASSES) return fail(p, PWF_ERR_STATE, "unexpected pass count");
  for (size_t i = 0; i < per; i++) {
    double acc_ms = 0.0;
    for (int k = 0; k < iters; k++) {
      float ms = 0.f;
      const size_t j = (size_t)k * per + i;
      PWF_CUDA(p, cudaEventElapsedTime(&ms, p->ev_pool[2 * j], p->ev_pool[2 * j + 1]));
      acc_ms += ms;
    }
    pass_ms[i] = (float)(acc_ms / iters);
    pass_names[i] = p->prof_names[i];
  }
  *n_passes = (int32_t)per;
  return PWF_OK;
}

// ---------------------------------------------------------------------------
// groups: several plans (size classes) iterated together from one graph
// ---------------------------------------------------------------------------
}  // extern "C"

struct pwf_group {
  std::vector<pwf_plan*> plans;
  std::vector<cudaStream_t> branch;  // one per plan, used only while capturing
  cudaStream_t main = nullptr;       // capture origin
  std::vector<cudaEvent_t> ev;       // fork/join events
  cudaGraphExec_t graph = nullptr;
  std::vector<const void*> key;
  double tol = 0.0;
  long long graph_kernels = 0;
  bool loop = false;                 // the graph holds the whole loop (conditional WHILE node)
  DevIter** d_its = nullptr;         // device array of the classes' iteration records
};

namespace {
// The group's device-side loop: ends after ctl[0] bodies (ctl[1] counts them,
// both written by the host before the launch), or earlier once the stopping
// rule has retired every projection of every class.
__global__ void k_group_loop_control(cudaGraphConditionalHandle h, DevIter* const* its, int n, int* ctl,
                                     double corr_tol) {
  pdl_wait();
  if (threadIdx.x == 0) {
    int active = 0;
    for (int i = 0; i < n; i++) active += its[i]->n_active;
    const int done = ++ctl[1];
    const bool more = done < ctl[0] && (corr_tol <= 0.0 || active > 0);
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}
}  // namespace

extern "C" {

pwf_status pwf_group_create(pwf_plan* const* plans, int32_t n, pwf_group** out) {
  if (!plans || n < 1 || !out) return PWF_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; i++) {
    if (!plans[i]) return PWF_ERR_INVALID_ARG;
    if (plans[i]->d.flags & PWF_FLAG_PLAIN) return PWF_ERR_UNSUPPORTED;
    for (int j = 0; j < i; j++)
      if (plans[j] == plans[i]) return PWF_ERR_INVALID_ARG;
  }
  pwf_group* g = new (std::nothrow) pwf_group();
  if (!g) return PWF_ERR_NOMEM;
  g->plans.assign(plans, plans + n);
  bool ok = cudaStreamCreateWithFlags(&g->main, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < n && ok; i++) {
    cudaStream_t s;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) g->branch.push_back(s);
  }
  for (int i = 0; i < 2 * n + 1 && ok; i++) {
    cudaEvent_t e;
    ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) g->ev.push_back(e);
  }
  if (!ok) {
    cudaGetLastError();
    pwf_group_destroy(g);
    return PWF_ERR_CUDA;
  }
  *out = g;
  return PWF_OK;
}

pwf_status pwf_group_destroy(pwf_group* g) {
  if (!g) return PWF_ERR_INVALID_ARG;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  if (g->d_its) cudaFree(g->d_its);
  for (cudaStream_t s : g->branch) cudaStreamDestroy(s);
  if (g->main) cudaStreamDestroy(g->main);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
  return PWF_OK;
}

// classes of at least this many pixels (batch x ny x nx) fill the GPU on their own
constexpr long long kGroupChainPixels = 8LL << 20;

pwf_status pwf_group_solve(pwf_group* g, void* stream, const float* const* y, const void* const* t,
                           void* const* psi, int32_t max_iter, double corr_tol) {
  if (!g || !y || !t || !psi || max_iter < 0) return PWF_ERR_INVALID_ARG;
  const int n = (int)g->plans.size();
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  pwf_status r;
  for (int i = 0; i < n; i++) {
    pwf_plan* p = g->plans[i];
    if ((r = check_plan(p))) return r;
    if (!y[i] || !t[i] || !psi[i]) return PWF_ERR_INVALID_ARG;
    if (!a16(y[i]) || !a16(t[i]) || !a16(psi[i])) return misaligned(p);
  }
  if (max_iter == 0) return PWF_OK;
  // set-up of every class on the caller's stream (Algorithm S1 initialisation)
  for (int i = 0; i < n; i++) {
    pwf_plan* p = g->plans[i];
    p->stream = user;
    if (!p->solve_state && (r = pwf_state_create(p, &p->solve_state))) return r;
    if (!p->modes.empty() && (r = ensure_vstack(p))) return r;
    pwf_state* st = p->solve_state;
    if ((r = pwf_state_reset(p, st)) || (r = compute_maxt2(p, (const float2*)t[i]))) return r;
    if (p->modes.empty() && !p->coherent && (r = compute_yhat(p, y[i], st->active))) return r;
    PassArgs a = base_args(p);
    a.active = st->active;
    a.psi = (const float2*)psi[i];
    a.out = p->X;
    LAUNCH(p, row(p, ROW_EXP_FFT, a, a.B));
  }
  // One graph per iteration. Classes large enough to fill the GPU on their own
  // run one after another on the main chain (largest first): side by side
  // their persistent column passes only contend for the SMs. Smaller classes
  // run on forked branches beside that chain and join at its end.
  std::vector<const void*> key;
  for (int i = 0; i < n; i++) {
    key.push_back(y[i]);
    key.push_back(t[i]);
    key.push_back(psi[i]);
  }
  if (!g->graph || key != g->key || g->tol != corr_tol) {
    if (g->graph) {
      cudaGraphExecDestroy(g->graph);
      g->graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    pwf_plan* p0 = g->plans[0];
    // the loop on the device: the iteration below is captured into the body of a
    // conditional WHILE node (falls back to one launch per iteration)
    std::vector<DevIter*> its;
    for (pwf_plan* p : g->plans) its.push_back(p->solve_state->it);
    if (!g->d_its && cudaMalloc(&g->d_its, n * sizeof(DevIter*)) != cudaSuccess) {
      cudaGetLastError();
      g->d_its = nullptr;
    }
    cudaGraph_t outer = nullptr, loop_body = nullptr;
    cudaGraphConditionalHandle h{};
    if (g->d_its && cudaMemcpy(g->d_its, its.data(), n * sizeof(DevIter*), cudaMemcpyHostToDevice) == cudaSuccess &&
        cudaGraphCreate(&outer, 0) == cudaSuccess &&
        cudaGraphConditionalHandleCreate(&h, outer, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
      cudaGraphNodeParams np{};
      cudaGraphNode_t node;
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      if (cudaGraphAddNode(&node, outer, nullptr, nullptr, 0, &np) == cudaSuccess) loop_body = np.conditional.phGraph_out[0];
    }
    cudaGetLastError();
    if (!loop_body && outer) {
      cudaGraphDestroy(outer);
      outer = nullptr;
    }
    std::vector<int> chain, side;
    for (int i = 0; i < n; i++)
      ((long long)g->plans[i]->d.batch * g->plans[i]->d.ny * g->plans[i]->d.nx >= kGroupChainPixels ? chain : side)
          .push_back(i);
    std::sort(chain.begin(), chain.end(), [&](int a, int b) {
      const pwf_plan_desc &da = g->plans[a]->d, &db = g->plans[b]->d;
      return (long long)da.batch * da.ny * da.nx > (long long)db.batch * db.ny * db.nx;
    });
    if (loop_body)
      PWF_CUDA(p0, cudaStreamBeginCaptureToGraph(g->main, loop_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    else
      PWF_CUDA(p0, cudaStreamBeginCapture(g->main, cudaStreamCaptureModeThreadLocal));
    r = PWF_OK;
    cudaError_t ce = cudaEventRecord(g->ev[0], g->main);
    long long kernels = 0;
    auto run_class = [&](int i, cudaStream_t s) {
      pwf_plan* p = g->plans[i];
      p->stream = s;
      const long long before = p->launches;
      r = fused_iteration(p, p->solve_state, y[i], (const float2*)t[i], (float2*)psi[i], true, corr_tol);
      kernels += p->launches - before;
      p->launches = before;
      p->stream = user;
    };
    for (int i : side) {
      if (r != PWF_OK || ce != cudaSuccess) break;
      ce = cudaStreamWaitEvent(g->branch[i], g->ev[0], 0);
      if (ce != cudaSuccess) break;
      run_class(i, g->branch[i]);
      if (r == PWF_OK) ce = cudaEventRecord(g->ev[1 + i], g->branch[i]);
    }
    for (int i : chain) {
      if (r != PWF_OK || ce != cudaSuccess) break;
      run_class(i, g->main);
    }
    for (int i : side) {
      if (r != PWF_OK || ce != cudaSuccess) break;
      ce = cudaStreamWaitEvent(g->main, g->ev[1 + i], 0);
    }
    if (loop_body && r == PWF_OK && ce == cudaSuccess) {
      ce = launch_pass(k_group_loop_control, dim3(1), dim3(32), 0, g->main, pdl_of(p0), h, (DevIter* const*)g->d_its, n,
                       p0->loop_ctl, corr_tol);
      kernels++;
    }
    cudaError_t ce2 = cudaStreamEndCapture(g->main, &graph);
    for (pwf_plan* p : g->plans) p->stream = user;
    if (r || ce != cudaSuccess || ce2 != cudaSuccess) {
      if (outer) cudaGraphDestroy(outer);
      else if (graph) cudaGraphDestroy(graph);
      if (r) return r;
      return cuda_fail(p0, ce != cudaSuccess ? ce : ce2, "group capture");
    }
    ce = cudaGraphInstantiate(&g->graph, outer ? outer : graph, 0);
    cudaGraphDestroy(outer ? outer : graph);
    if (ce != cudaSuccess) return cuda_fail(p0, ce, "group graph instantiate");
    g->loop = outer != nullptr;
    g->key = key;
    g->tol = corr_tol;
    g->graph_kernels = kernels;
  }
  pwf_plan* p0 = g->plans[0];
  if (g->loop) {
    const int ctl[2] = {max_iter, 0};
    PWF_CUDA(p0, cudaMemcpyAsync(p0->loop_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, user));
    PWF_CUDA(p0, cudaGraphLaunch(g->graph, user));
    p0->launches += g->graph_kernels * max_iter;  // at most: the loop may stop early
    return PWF_OK;
  }
  for (int k = 0; k < max_iter; k++) {
    PWF_CUDA(p0, cudaGraphLaunch(g->graph, user));
    p0->launches += g->graph_kernels;
    if (corr_tol > 0.0 && (k + 1) % 16 == 0 && k + 1 < max_iter) {
      int active = 0;
      for (pwf_plan* p : g->plans) {
        DevIter it;
        PWF_CUDA(p, cudaMemcpyAsync(&it, p->solve_state->it, sizeof(DevIter), cudaMemcpyDeviceToHost, user));
        PWF_CUDA(p, cudaStreamSynchronize(user));
        active += it.n_active;
      }
      if (active == 0) break;
    }
  }
  return PWF_OK;
}

pwf_status pwf_group_read(pwf_group* g, int32_t index, double* loss_host, int32_t* iters_host) {
  if (!g || index < 0 || index >= (int)g->plans.size()) return PWF_ERR_INVALID_ARG;
  pwf_plan* p = g->plans[index];
  if (!p->solve_state) return PWF_ERR_STATE;
  return pwf_state_read(p, p->solve_state, loss_host, nullptr, iters_host, nullptr);
}

pwf_status pwf_calibrate_coherence(pwf_plan* p, const float* I_ref, int32_t max_lag, double* xcoh_m,
                                   double* ycoh_m) {
  pwf_status r = check_plan(p);
  if (r) return r;
  const int ny = p->d.ny, nx = p->d.nx;
  if (!I_ref || !xcoh_m || !ycoh_m || max_lag < 1 || max_lag >= nx / 2 || max_lag >= ny / 2)
    return PWF_ERR_INVALID_ARG;
  if (!a16(I_ref)) return misaligned(p);
  const size_t n = (size_t)ny * nx;
  if (!p->calib && (r = dalloc(p, &p->calib, (size_t)nx + ny + 1))) return r;  // released with the plan
  double* d = p->calib;
  PWF_CUDA(p, cudaMemsetAsync(d, 0, sizeof(double) * (nx + ny + 1), p->stream));
  const int G = grid_for(n);
  k_mean<<<G, 256, 0, p->stream>>>(I_ref, n, d + nx + ny);
  PassArgs a = base_args(p);
  a.proj0 = 0;
  a.in = p->X;
  a.out = p->X;
  for (int axis = 1; axis >= 0; axis--) {  // along x (rows), then along y (columns)
    k_real_to_complex<<<G, 256, 0, p->stream>>>(I_ref, p->X, n);
    const int len = axis == 1 ? nx : ny;
    if (axis == 1) {
      LAUNCH(p, row(p, ROW_FFT, a, 1));
      k_abs2_scale<<<G, 256, 0, p->stream>>>(p->X, n, 1.0f / ((float)len * (float)len));
      LAUNCH(p, row(p, ROW_IFFT, a, 1));
    } else {
      LAUNCH(p, col(p, COL_FFT, a, 1));
      k_abs2_scale<<<G, 256, 0, p->stream>>>(p->X, n, 1.0f / ((float)len * (float)len));
      PassArgs b = a;
      b.scale = 1.0f;
      LAUNCH(p, col(p, COL_IFFT, b, 1));
    }
    k_line_mean<<<len, 256, 0, p->stream>>>(p->X, ny, nx, axis, d + (axis == 1 ? 0 : nx));
    PWF_CUDA(p, cudaGetLastError());
  }
  std::vector<double> h((size_t)nx + ny + 1);
  PWF_CUDA(p, cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  PWF_CUDA(p, cudaStreamSynchronize(p->stream));
  const double m2 = h[nx + ny] * h[nx + ny];
  // least squares of ln(g2 - 1) against D^2 over D = 1..max_lag (reading of Methods)
  auto fit = [&](const double* g, double* out) -> bool {
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int k = 1; k <= max_lag; k++) {
      const double g2 = g[k] / m2 - 1.0;
      if (!(g2 > 0)) return false;
      const double x = (double)k * k, yv = std::log(g2);
      sx += x, sy += yv, sxx += x * x, sxy += x * yv;
    }
    const double m = max_lag, slope = (m * sxy - sx * sy) / (m * sxx - sx * sx);
    if (!(slope < 0)) return false;
    *out = std::sqrt(-M_PI / slope) * p->d.pixel_m;
    return true;
  };
  if (!fit(h.data(), xcoh_m) || !fit(h.data() + nx, ycoh_m))
    return fail(p, PWF_ERR_NONFINITE, "autocorrelation not decreasing over the fitted lags");
  return PWF_OK;
}

pwf_status pwf_diffuser_from_reference(pwf_plan* p, const float* I_ref, double wiener_eps, void* t_out) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!I_ref || !t_out || !(wiener_eps >= 0)) return PWF_ERR_INVALID_ARG;
  if (!a16(I_ref) || !a16(t_out)) return misaligned(p);
  const size_t n = (size_t)p->d.ny * p->d.nx;
  const int G = grid_for(n);
  k_real_to_complex<<<G, 256, 0, p->stream>>>(I_ref, p->X, n);
  PWF_CUDA(p, cudaGetLastError());
  if ((r = plain_fft2(p, p->X, 0, false))) return r;
  k_filter<<<G, 256, 0, p->stream>>>(p->X, p->d.ny, p->d.nx, PF_WIENER, nullptr, nullptr, 0, p->ax.iotf, p->ay.iotf,
                                     nullptr, nullptr, nullptr, nullptr, 0, (float)wiener_eps);
  PWF_CUDA(p, cudaGetLastError());
  if ((r = plain_fft2(p, p->X, 0, true))) return r;
  k_sqrt_clip<<<G, 256, 0, p->stream>>>(p->X, n);
  PWF_CUDA(p, cudaGetLastError());
  if ((r = plain_filter(p, p->X, 0, PF_Q, 2, 1))) return r;  // back over L2
  PWF_CUDA(p, cudaMemcpyAsync(t_out, p->X, n * sizeof(float2), cudaMemcpyDeviceToDevice, p->stream));
  return PWF_OK;
}

size_t pwf_state_bytes(const pwf_state* s) {
  if (!s) return 0;
  return 64 + (size_t)s->B * s->ny * s->nx * sizeof(float2) + s->B * (2 * sizeof(int) + 2 * sizeof(double)) +
         sizeof(DevIter);
}

namespace {
struct CkptHeader {
  char magic[8];
  int32_t B, ny, nx, version;
  char pad[40];
};
}  // namespace

pwf_status pwf_state_save(pwf_plan* p, const pwf_state* s, void* host_buf, size_t bytes) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!s || !host_buf) return PWF_ERR_INVALID_ARG;
  if (bytes < pwf_state_bytes(s)) return PWF_ERR_STATE;
  char* b = static_cast<char*>(host_buf);
  CkptHeader h{};
  std::memcpy(h.magic, "PWFSTAT1", 8);
  h.B = s->B;
  h.ny = s->ny;
  h.nx = s->nx;
  h.version = 2;
  std::memcpy(b, &h, sizeof(h));
  b += 64;
  const size_t nf = (size_t)s->B * s->ny * s->nx * sizeof(float2);
  PWF_CUDA(p, cudaMemcpyAsync(b, s->phi, nf, cudaMemcpyDeviceToHost, p->stream));
  b += nf;
  PWF_CUDA(p, cudaMemcpyAsync(b, s->active, s->B * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  b += s->B * sizeof(int);
  PWF_CUDA(p, cudaMemcpyAsync(b, s->iters, s->B * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  b += s->B * sizeof(int);
  PWF_CUDA(p, cudaMemcpyAsync(b, s->loss, s->B * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  b += s->B * sizeof(double);
  PWF_CUDA(p, cudaMemcpyAsync(b, s->corr, s->B * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  b += s->B * sizeof(double);
  PWF_CUDA(p, cudaMemcpyAsync(b, s->it, sizeof(DevIter), cudaMemcpyDeviceToHost, p->stream));
  PWF_CUDA(p, cudaStreamSynchronize(p->stream));
  return PWF_OK;
}

pwf_status pwf_state_load(pwf_plan* p, pwf_state* s, const void* host_buf, size_t bytes) {
  pwf_status r = check_plan(p);
  if (r) return r;
  if (!s || !host_buf) return PWF_ERR_INVALID_ARG;
  if (bytes < pwf_state_bytes(s)) return PWF_ERR_STATE;
  const char* b = static_cast<const char*>(host_buf);
  CkptHeader h;
  std::memcpy(&h, b, sizeof(h));
  if (std::memcmp(h.magic, "PWFSTAT1", 8) != 0 || h.version != 2 || h.B != s->B || h.ny != s->ny || h.nx != s->nx)
    return PWF_ERR_STATE;
  b += 64;
  const size_t nf = (size_t)s->B * s->ny * s->nx * sizeof(float2);
  PWF_CUDA(p, cudaMemcpyAsync(s->phi, b, nf, cudaMemcpyHostToDevice, p->stream));
  b += nf;
  PWF_CUDA(p, cudaMemcpyAsync(s->active, b, s->B * sizeof(int), cudaMemcpyHostToDevice, p->stream));
  b += s->B * sizeof(int);
  PWF_CUDA(p, cudaMemcpyAsync(s->iters, b, s->B * sizeof(int), cudaMemcpyHostToDevice, p->stream));
  b += s->B * sizeof(int);
  PWF_CUDA(p, cudaMemcpyAsync(s->loss, b, s->B * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  b += s->B * sizeof(double);
  PWF_CUDA(p, cudaMemcpyAsync(s->corr, b, s->B * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  b += s->B * sizeof(double);
  PWF_CUDA(p, cudaMemcpyAsync(s->it, b, sizeof(DevIter), cudaMemcpyHostToDevice, p->stream));
  PWF_CUDA(p, cudaStreamSynchronize(p->stream));
  return PWF_OK;
}

}  // extern "C"
