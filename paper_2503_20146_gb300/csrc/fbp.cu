// Filtered back projection of the retrieved fields (the tomographic step after
// PWF; Methods, "Reconstruction procedure": standard FBP with the Ram-Lak
// filter, applied to every detector row independently, then the factor
// lambda / p / (2 pi)). Parallel-beam, angles over [0, pi).
//
// Two kernels:
//   * fbp_filter_kernel<L>: one detector row per TPF threads. The nx samples
//     are zero-padded to L = 2 nx (so the circular convolution of length L is
//     the linear one over the row), transformed with the Stockham runner of the
//     PWF passes, multiplied by the length-L DFT of the band-limited ramp
//     (Ram-Lak) kernel, transformed back, and the first nx samples kept. The
//     complex field psi is filtered as is: the kernel is real and even, so the
//     real and the imaginary parts are filtered independently in one pass.
//     The filtered row is stored in the middle of a zeroed row of width 2 nx
//     (detector pixel i at column i + nx/2), so that the back projection of
//     any voxel of the nx x nx grid (|s| <= nx / sqrt(2) + 1) reads inside the
//     row without bounds checks and gets zero outside the detector; each
//     column holds the record (q[o], q[o+1] - q[o]), so one 16-byte load gives
//     both taps of the linear interpolation.
//   * fbp_backproject_kernel: one thread per (x, 8 values of z) of one slice
//     (warps laid out as 8 x 4 voxel patches);
//     per angle, s = x cos(theta) + z sin(theta), linear interpolation
//     q[j] + w (q[j+1] - q[j]) from one record, accumulation in FP32. The angle table sits in shared
//     memory; the filtered rows of one slice are read through L1/L2 (a 32 x 64
//     voxel tile touches at most ~70 samples per angle).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/pwf.h"
#include "host_tables.h"
#include "passes.cuh"

namespace pwf {
namespace {

template <int L>
__global__ void __launch_bounds__(row_threads(L))
    fbp_filter_kernel(const float2* __restrict__ in, float2* __restrict__ out, const float* __restrict__ ramp,
                      const float2* __restrict__ tw_fwd, const float2* __restrict__ tw_inv, long long nrows,
                      int nx) {
  constexpr int EPT = ept_for(L), TPF = tpf_for(L), ROWS = rows_for(L);
  constexpr int RS = first_radix<L, FWD>();
  constexpr int RK = last_radix<L, FWD>();
  extern __shared__ float2 smem[];
  const int rr = threadIdx.x / TPF, t = threadIdx.x - rr * TPF;
  long long row = (long long)blockIdx.x * ROWS + rr;
  // rows past the end repeat the last row (every thread of a warp must reach
  // the warp barriers of the transform) and store nothing
  const bool valid = row < nrows;
  if (!valid) row = nrows - 1;
  const float2* src = in + (size_t)row * nx;
  const RowLayout<TPF, ROWS * TPF> sm{smem + rr * row_smem_len(L), 1 + rr};
  float2 v[EPT];
#pragma unroll
  for (int j = 0; j < EPT; j++) {
    const int i = slot_index<L, RS>(t, j);
    v[j] = i < nx ? src[i] : make_float2(0.f, 0.f);
  }
  fft_run<L, FWD>(v, sm, t, tw_fwd);
#pragma unroll
  for (int j = 0; j < EPT; j++) v[j] = cscale(v[j], __ldg(&ramp[slot_index<L, RK>(t, j)]));
  fft_run<L, INV>(v, sm, t, tw_inv);
  // records (q[o], q[o+1] - q[o]) of the padded row of width L = 2 nx (samples
  // at nx/2 .. 3nx/2 - 1, zeros around): first the samples into shared memory
  // (the transform's buffer is free again; every row of a warp takes part in
  // the barriers), then the records of valid rows
  float2* rowbuf = smem + rr * row_smem_len(L);
  sm.sync();
#pragma unroll
  for (int j = 0; j < EPT; j++) {
    const int i = slot_index<L, RS>(t, j);
    const int o = i + nx / 2;
    rowbuf[o < L ? o : o - L] = i < nx ? v[j] : make_float2(0.f, 0.f);
  }
  sm.sync();
  if (valid) {
    float4* dst = reinterpret_cast<float4*>(out) + (size_t)row * L;
    for (int o = t; o < L; o += TPF) {
      const float2 q0 = rowbuf[o], q1 = rowbuf[o + 1 < L ? o + 1 : o];
      dst[o] = make_float4(q0.x, q0.y, q1.x - q0.x, q1.y - q0.y);
    }
  }
}

template <int L>
cudaError_t launch_filter(const float2* in, float2* out, const float* ramp, const float2* twf, const float2* twi,
                          long long nrows, int nx, cudaStream_t s) {
  constexpr int ROWS = rows_for(L);
  const long long blocks = (nrows + ROWS - 1) / ROWS;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  static const cudaError_t attr = cudaFuncSetAttribute(
      fbp_filter_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem_bytes(L));
  if (attr != cudaSuccess) return attr;
  fbp_filter_kernel<L><<<(unsigned)blocks, row_threads(L), row_smem_bytes(L), s>>>(in, out, ramp, twf, twi, nrows,
                                                                                  nx);
  return cudaGetLastError();
}

using FilterFn = cudaError_t (*)(const float2*, float2*, const float*, const float2*, const float2*, long long, int,
                                 cudaStream_t);

FilterFn filter_for(int L) {
  switch (L) {
    case 32: return launch_filter<32>;
    case 64: return launch_filter<64>;
    case 96: return launch_filter<96>;
    case 128: return launch_filter<128>;
    case 192: return launch_filter<192>;
    case 256: return launch_filter<256>;
    case 384: return launch_filter<384>;
    case 512: return launch_filter<512>;
    case 768: return launch_filter<768>;
    case 1024: return launch_filter<1024>;
    case 1536: return launch_filter<1536>;
    case 2048: return launch_filter<2048>;
    default: return nullptr;
  }
}

constexpr int BP_TX = 32, BP_TY = 8, BP_ZPT = 8;  // tile 32 (x) by 64 (z) voxels

__global__ void __launch_bounds__(BP_TX * BP_TY)
    fbp_backproject_kernel(const float2* __restrict__ q, float2* __restrict__ vol, const float2* __restrict__ cs,
                           int n_angles, int ny, int nx, float scale) {
  extern __shared__ float2 scs[];
  const int tid = threadIdx.y * BP_TX + threadIdx.x;
  for (int i = tid; i < n_angles; i += BP_TX * BP_TY) scs[i] = cs[i];
  __syncthreads();
  // each warp covers a compact 8 (x) by 4 (z) patch per z step, so that its
  // lanes' detector positions span at most 8|cos| + 4|sin| + 1 records (two
  // 128-byte wavefronts) instead of the 32|cos| + 1 of a 32-voxel row
  const int lane = tid & 31, warp = tid >> 5;
  const int x = blockIdx.x * BP_TX + (warp & 3) * 8 + (lane & 7);
  const int zb = blockIdx.y * (BP_TY * BP_ZPT) + (warp >> 2) * 4 + (lane >> 3);
  const int y = blockIdx.z;
  const float half = 0.5f * (float)nx - 0.5f;  // detector index of s = 0
  // voxels past the grid (tile overhang) compute on the last row / column,
  // which keeps their reads inside the padded rows; they store nothing
  const float xc = (float)(x < nx ? x : nx - 1) - half;
  float zc[BP_ZPT];
#pragma unroll
  for (int m = 0; m < BP_ZPT; m++) {
    const int z = zb + m * BP_TY;  // z steps of 8: the block's 8 rows of patches
    zc[m] = (float)(z < nx ? z : nx - 1) - half;
  }
  float2 acc[BP_ZPT];
#pragma unroll
  for (int m = 0; m < BP_ZPT; m++) acc[m] = make_float2(0.f, 0.f);
  // rows of width 2 nx, detector index u at column u + nx/2; every voxel of
  // the grid has |u - half| <= nx / sqrt(2) + 1, so both taps stay in the row
  const int W = 2 * nx;
  const size_t plane = (size_t)ny * W;
  const float4* qy = reinterpret_cast<const float4*>(q) + (size_t)y * W + nx / 2;
#pragma unroll 4
  for (int a = 0; a < n_angles; a++) {
    const float2 c = scs[a];
    const float4* row = qy + (size_t)a * plane;
    const float base = fmaf(xc, c.x, half);
#pragma unroll
    for (int m = 0; m < BP_ZPT; m++) {
      const float u = fmaf(zc[m], c.y, base);
      const float uf = floorf(u);
      const float w = u - uf;
      const float4 qd = __ldg(row + (int)uf);
      acc[m].x += fmaf(w, qd.z, qd.x);
      acc[m].y += fmaf(w, qd.w, qd.y);
    }
  }
  if (x >= nx) return;
#pragma unroll
  for (int m = 0; m < BP_ZPT; m++) {
    const int z = zb + m * BP_TY;
    if (z < nx) vol[((size_t)y * nx + z) * nx + x] = cscale(acc[m], scale);
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct FbpLayout {
  size_t q, ramp, twf, twi, cs, total;
};

FbpLayout fbp_layout(int n_angles, int ny, int nx) {
  FbpLayout l{};
  const int L = 2 * nx;
  std::vector<float2> a, b;
  host_twiddles(L, FWD, a);
  host_twiddles(L, INV, b);
  l.q = 0;
  l.ramp = l.q + align256((size_t)n_angles * ny * 2 * nx * sizeof(float4));
  l.twf = l.ramp + align256((size_t)L * sizeof(float));
  l.twi = l.twf + align256(a.size() * sizeof(float2));
  l.cs = l.twi + align256(b.size() * sizeof(float2));
  l.total = l.cs + align256((size_t)n_angles * sizeof(float2));
  return l;
}

bool fbp_sizes_ok(int n_angles, int ny, int nx) {
  return n_angles >= 1 && n_angles <= PWF_FBP_MAX_ANGLES && ny >= 1 && ny <= 65535 && nx >= 16 &&
         filter_for(2 * nx) != nullptr;
}

}  // namespace
}  // namespace pwf

using namespace pwf;

extern "C" {

size_t pwf_fbp_workspace_bytes(int32_t n_angles, int32_t ny, int32_t nx) {
  if (!fbp_sizes_ok(n_angles, ny, nx)) return 0;
  return fbp_layout(n_angles, ny, nx).total;
}

pwf_status pwf_fbp(const void* psi, int32_t n_angles, int32_t ny, int32_t nx, const double* angles_rad_host,
                   double wavelength_m, double voxel_m, void* vol_out, void* workspace, size_t workspace_bytes,
                   void* stream) {
  if (!psi || !vol_out || !workspace || !angles_rad_host || !fbp_sizes_ok(n_angles, ny, nx) ||
      !(wavelength_m > 0) || !(voxel_m > 0))
    return PWF_ERR_INVALID_ARG;
  const FbpLayout l = fbp_layout(n_angles, ny, nx);
  if (workspace_bytes < l.total || ((uintptr_t)workspace & 255) || ((uintptr_t)psi & 7) || ((uintptr_t)vol_out & 7))
    return PWF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int L = 2 * nx;

  // Ram-Lak kernel h(0) = 1/4, h(k) = -1/(pi^2 k^2) for odd k, placed
  // circularly on length L; its DFT is real and even:
  // H(m) = 1/4 + 2 sum_{odd k < nx} h(k) cos(2 pi k m / L). The inverse
  // transform's 1/L is folded in.
  std::vector<float> ramp(L);
  for (int m = 0; m < L; m++) {
    double h = 0.25;
    for (int k = 1; k < nx; k += 2) h -= 2.0 / (M_PI * M_PI * (double)k * k) * std::cos(2.0 * M_PI * k * m / L);
    ramp[m] = (float)(h / L);
  }
  std::vector<float2> twf, twi, cs(n_angles);
  if (!host_twiddles(L, FWD, twf) || !host_twiddles(L, INV, twi)) return PWF_ERR_UNSUPPORTED;
  for (int a = 0; a < n_angles; a++)
    cs[a] = make_float2((float)std::cos(angles_rad_host[a]), (float)std::sin(angles_rad_host[a]));
  // host vectors are pageable: these copies complete before returning
  if (cudaMemcpyAsync(ws + l.ramp, ramp.data(), L * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(ws + l.twf, twf.data(), twf.size() * sizeof(float2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws + l.twi, twi.data(), twi.size() * sizeof(float2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws + l.cs, cs.data(), cs.size() * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return PWF_ERR_CUDA;
  }
  float2* q = (float2*)(ws + l.q);
  const long long nrows = (long long)n_angles * ny;
  if (filter_for(L)((const float2*)psi, q, (const float*)(ws + l.ramp), (const float2*)(ws + l.twf),
                    (const float2*)(ws + l.twi), nrows, nx, s) != cudaSuccess) {
    cudaGetLastError();
    return PWF_ERR_CUDA;
  }
  // back projection weight pi / N_theta and the factor -lambda / (2 pi p):
  // beta + i delta from psi = -k int beta - i k int delta
  const float scale = (float)(M_PI / n_angles * (-wavelength_m / (2.0 * M_PI * voxel_m)));
  const int tiles = (nx + BP_TX - 1) / BP_TX;
  const dim3 grid(tiles, (nx + BP_TY * BP_ZPT - 1) / (BP_TY * BP_ZPT), ny);
  fbp_backproject_kernel<<<grid, dim3(BP_TX, BP_TY), n_angles * sizeof(float2), s>>>(
      q, (float2*)vol_out, (const float2*)(ws + l.cs), n_angles, ny, nx, scale);
  if (cudaGetLastError() != cudaSuccess) return PWF_ERR_CUDA;
  return PWF_OK;
}

}  // extern "C"
