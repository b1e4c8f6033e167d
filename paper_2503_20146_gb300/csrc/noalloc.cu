// pwf_forward_noalloc: the forward model without any device allocation.
//
// pwf_forward needs a plan, and creating a plan allocates device memory (its
// workspace and filter tables). Some callers cannot do that: a process whose
// device memory is owned by another allocator (a framework's caching pool, a
// fixed budget reserved at start-up for a detector read-out pipeline), or code
// on a latency-critical path where the implicit device-wide synchronisation of
// cudaMalloc / cudaFree would stall other work on the GPU. This entry point
// evaluates the same forward model with the same kernels, but its scratch
// field and its 1-D tables live in file-scope __device__ arrays of fixed size,
// so the library never allocates on its behalf.
//
// Every GPU that loads the library holds these arrays (about 16.2 MiB) until
// the process exits. Every call shares them, and they keep the last call's
// contents: the tables are rewritten at the start of each call, and calls
// that overlap on the GPU (for instance on two streams at once) race on them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/pwf.h"
#include "passes.cuh"

namespace pwf {
const LengthKernels* kernels_for_length(int n);
}

using namespace pwf;

namespace {

constexpr size_t kMaxElems = size_t(1) << 21;  // complex64 scratch elements (16 MiB)
constexpr int kMaxN = 2048;                     // longest transform of the built set
constexpr int kTwMax = 4096;                    // twiddle entries per table
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) float2 g_scratch[kMaxElems];
static __device__ __align__(256) float2 g_tw[4][kTwMax];    // x fwd, x inv, y fwd, y inv
static __device__ __align__(256) float2 g_q[4][kMaxN];      // Q1 x, Q2 x, Q1 y, Q2 y
static __device__ __align__(256) float g_iotf[2][kMaxN];    // IOTF x, y

namespace {

struct DevPtrs {
  bool ready = false;
  float2* scratch = nullptr;
  float2* tw = nullptr;
  float2* q = nullptr;
  float* iotf = nullptr;
};
DevPtrs g_dev[kMaxDevices];
std::mutex g_mu;

struct TableParams {
  int nx, ny;
  double pixel, lambda, L1, L2, xcoh, ycoh;
};

__device__ double fftfreq_d(int k, int n) { return (double)(k < (n + 1) / 2 ? k : k - n) / (double)n; }

__device__ double prop_phase_d(double rho2, double lambda, double L) {
  const double il = 1.0 / lambda;
  const double w = sqrt(il * il - rho2);
  return 2.0 * M_PI * L * (-rho2 / (il + w));
}

// Twiddle entries of one (length, direction): stage k >= 1 of radix R after
// NS points holds exp(D 2 pi i r j / (NS R)) at (r - 1) NS + j.
__device__ void fill_twiddles(float2* tab, int n, int D, int idx) {
  const Sched s = sched_for(n);
  for (int k = 1; k < s.s; k++) {
    const int R = stage_radix(n, D, k), NS = stage_ns(n, D, k), off = stage_twoff(n, D, k);
    const int cnt = (R - 1) * NS;
    if (idx < cnt) {
      const int r = idx / NS + 1, j = idx % NS;
      const long m = ((long)r * j) % ((long)NS * R);
      double sn, cs;
      sincospi(2.0 * (double)m / (double)(NS * R), &sn, &cs);
      tab[off + idx] = make_float2((float)cs, (float)(D * sn));
    }
  }
}

__global__ void k_noalloc_tables(TableParams p, float2* tw, float2* q, float* io) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  fill_twiddles(tw + 0 * kTwMax, p.nx, FWD, idx);
  fill_twiddles(tw + 1 * kTwMax, p.nx, INV, idx);
  fill_twiddles(tw + 2 * kTwMax, p.ny, FWD, idx);
  fill_twiddles(tw + 3 * kTwMax, p.ny, INV, idx);
  for (int axis = 0; axis < 2; axis++) {
    const int n = axis == 0 ? p.nx : p.ny;
    if (idx >= n) continue;
    const double u = fftfreq_d(idx, n) / p.pixel;
    const double coh = axis == 0 ? p.xcoh : p.ycoh;
    double s1, c1, s2, c2;
    sincos(prop_phase_d(u * u, p.lambda, p.L1), &s1, &c1);
    sincos(prop_phase_d(u * u, p.lambda, p.L2), &s2, &c2);
    q[(2 * axis + 0) * kMaxN + idx] = make_float2((float)c1, (float)s1);
    q[(2 * axis + 1) * kMaxN + idx] = make_float2((float)c2, (float)s2);
    io[axis * kMaxN + idx] = (float)exp(-0.5 * M_PI * u * u * coh * coh);
  }
}

// Once per device, with that device current: resolve the device addresses of
// the file-scope arrays (the names are host-side stand-ins in host code) and
// raise the shared-memory limit of the kernels used here.
pwf_status setup_device(DevPtrs** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PWF_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  DevPtrs& d = g_dev[dev];
  if (!d.ready) {
    if (cudaGetSymbolAddress((void**)&d.scratch, g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.tw, g_tw) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.q, g_q) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.iotf, g_iotf) != cudaSuccess) {
      cudaGetLastError();
      return PWF_ERR_CUDA;
    }
    for (int n : {16, 32, 64, 96, 128, 256, 512, 768, 1024, 1536, 2048}) {
      const LengthKernels* k = kernels_for_length(n);
      for (int op : {ROW_EXP_FFT, ROW_MUL_T, ROW_INTENSITY, ROW_INTENSITY_OUT, ROW_REAL_OUT})
        if (k->row_prep[op]() != cudaSuccess) {
          cudaGetLastError();
          return PWF_ERR_CUDA;
        }
      for (int op : {COL_Q, COL_IOTF})
        if (k->colv[op][0].prep() != cudaSuccess) {
          cudaGetLastError();
          return PWF_ERR_CUDA;
        }
    }
    d.ready = true;
  }
  *out = &d;
  return PWF_OK;
}

}  // namespace

extern "C" pwf_status pwf_forward_noalloc(const pwf_plan_desc* desc, const void* psi, const void* t, float* f) {
  if (!desc || !psi || !t || !f) return PWF_ERR_INVALID_ARG;
  // rows are read with 16-byte vector loads and L2 bulk prefetches
  for (const void* q : {psi, t, static_cast<const void*>(f)})
    if (reinterpret_cast<uintptr_t>(q) & 15) return PWF_ERR_INVALID_ARG;
  const pwf_plan_desc& d = *desc;
  if (d.batch < 1 || d.ny < 1 || d.nx < 1 || !(d.pixel_m > 0) || !(d.wavelength_m > 0) || d.L1_m < 0 ||
      d.L2_m < 0 || d.xcoh_m < 0 || d.ycoh_m < 0)
    return PWF_ERR_INVALID_ARG;
  // the n_modes values pwf_plan_create accepts; only the paper's forms (0, 1)
  // are computed here, the source-mode variant needs a plan
  if (!(d.n_modes == 0 || d.n_modes == 1 || d.n_modes == 9 || d.n_modes == 25) || !(d.mode_sigma_px >= 0.0))
    return PWF_ERR_INVALID_ARG;
  if (d.n_modes > 1) return PWF_ERR_UNSUPPORTED;
  const LengthKernels* krow = kernels_for_length(d.nx);
  const LengthKernels* kcol = kernels_for_length(d.ny);
  if (!krow || !kcol) return PWF_ERR_UNSUPPORTED;
  if ((size_t)d.batch * d.ny * d.nx > kMaxElems) return PWF_ERR_UNSUPPORTED;  // scratch limit
  if (twiddle_len(d.nx, FWD) > kTwMax || twiddle_len(d.nx, INV) > kTwMax || twiddle_len(d.ny, FWD) > kTwMax ||
      twiddle_len(d.ny, INV) > kTwMax)
    return PWF_ERR_UNSUPPORTED;
  {  // same geometry checks as pwf_plan_create
    const double umax = 0.5 / d.pixel_m, il = 1.0 / d.wavelength_m;
    if (2.0 * umax * umax >= il * il) return PWF_ERR_UNSUPPORTED;
    for (double L : {d.L1_m, d.L2_m}) {
      auto ph = [&](double r2) { return 2.0 * M_PI * L * (-r2 / (il + std::sqrt(il * il - r2))); };
      if (std::fabs(ph(2 * umax * umax) - 2 * ph(umax * umax)) > 1e-6) return PWF_ERR_UNSUPPORTED;
    }
  }
  DevPtrs* dp = nullptr;
  pwf_status st = setup_device(&dp);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(d.stream);

  TableParams tp{};
  tp.nx = d.nx;
  tp.ny = d.ny;
  tp.pixel = d.pixel_m;
  tp.lambda = d.wavelength_m;
  tp.L1 = d.L1_m;
  tp.L2 = d.L2_m;
  tp.xcoh = d.xcoh_m;
  tp.ycoh = d.ycoh_m;
  k_noalloc_tables<<<(kTwMax + 255) / 256, 256, 0, s>>>(tp, dp->tw, dp->q, dp->iotf);
  if (cudaGetLastError() != cudaSuccess) return PWF_ERR_CUDA;

  PassArgs a{};
  a.B = d.batch;
  a.ny = d.ny;
  a.nx = d.nx;
  a.scale = (float)(1.0 / ((double)d.nx * d.ny));
  a.in = dp->scratch;
  a.out = dp->scratch;
  auto row = [&](int op) {
    PassArgs r = a;
    r.tw_fwd = dp->tw + 0 * kTwMax;
    r.tw_inv = dp->tw + 1 * kTwMax;
    return krow->row[op](r, d.batch, s);
  };
  auto col = [&](int op, int L) {
    PassArgs c = a;
    c.tw_fwd = dp->tw + 2 * kTwMax;
    c.tw_inv = dp->tw + 3 * kTwMax;
    c.qx = dp->q + (L == 1 ? 0 : 1) * kMaxN;
    c.qy = dp->q + (L == 1 ? 2 : 3) * kMaxN;
    c.ix = dp->iotf;
    c.iy = dp->iotf + kMaxN;
    return kcol->colv[op][0].launch(c, d.batch, s);
  };
  const bool coherent = d.xcoh_m == 0.0 && d.ycoh_m == 0.0;
  cudaError_t e;
  a.psi = static_cast<const float2*>(psi);
  a.t = static_cast<const float2*>(t);
  a.f_out = f;
  if ((e = row(ROW_EXP_FFT)) || (e = col(COL_Q, 1)) || (e = row(ROW_MUL_T)) || (e = col(COL_Q, 2))) {
    cudaGetLastError();
    return PWF_ERR_CUDA;
  }
  if (coherent) {
    e = row(ROW_INTENSITY_OUT);
  } else if (!(e = row(ROW_INTENSITY)) && !(e = col(COL_IOTF, 0))) {
    e = row(ROW_REAL_OUT);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PWF_ERR_CUDA;
  }
  return PWF_OK;
}
