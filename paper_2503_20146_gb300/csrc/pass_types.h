// Types shared by every translation unit of the library: the arguments of a
// pass, the pass and shape tables of one transform length, and the state of
// the persistent solvers. The kernels themselves live in an inline namespace
// per radix schedule (fft.cuh), so that a length's column passes can be built
// with two schedules side by side; these types are common to both.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace pwf {

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
  const float* ex;         // STF - 1 along x (and y): exp(-pi gamma u^2 xcoh^2) - 1, Eq. (14)
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
  // source-mode variant: tilt bins, weight, accumulate flag
  int mode_mx, mode_my;
  float mode_w;
  int accumulate;
  int* kstatus;            // device word set to PWF_ERR_TIMEOUT (7) when a bounded wait runs out
  int pdl;                 // launch with the programmatic stream-serialization attribute
  int l2pf;                // single-buffered pair shapes: tmap maps `in`; prefetch the next tile into L2
  CUtensorMap tmap;        // TMA map of `in` (filled by the launcher of a TMA-staged or prefetching shape)
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
  ROW_GRADT,           // IFFT -> g2; scratch (+)= 2 w conj(u1) g2; conj(t) g2 -> FFT
  ROW_MODE_INT,        // IFFT -> v_j (stored); I (+)= w |v_j|^2          (mode variant)
  ROW_MODE_VG,         // v_j G (both real-space inputs) -> FFT           (mode variant)
  ROW_INTENSITY_PK,    // IFFT -> v (stored) -> |v|^2 of rows 2y', 2y'+1 packed as one
                       // complex row -> FFT -> packed row y' (even row of the field)
  ROW_MUL_V_PK,        // IFFT of packed row y' -> G of rows 2y' (Re), 2y'+1 (Im); v * G -> FFT
  NUM_ROW_OPS
};

enum ColOp : int {
  COL_Q = 0,           // FFT -> * Q (or conj Q) -> IFFT
  COL_IOTF,            // FFT -> * IOTF -> IFFT
  COL_RESID_IOTF2,     // FFT -> R = IOTF I - Y; loss; * IOTF -> IFFT
  COL_PRECOND_REG,     // FFT(H), FFT(S) -> Gamma^2 H + i P^-1 S -> IFFT
  COL_FFT,             // FFT only
  COL_IFFT,            // IFFT only (scaled)
  COL_RESID_PK,        // COL_RESID_IOTF2 on packed rows: columns kx and nx - kx from one
                       // transform pair (the residual field is real)
  NUM_COL_OPS
};

enum ColModeOp : int { CM_FWD = 0, CM_BACK = 1 };

using PassFn = cudaError_t (*)(const PassArgs&, int nproj, cudaStream_t);
using PrepFn = cudaError_t (*)();

struct PersistArgs;  // persist.cuh
using PersistFn = cudaError_t (*)(const PersistArgs&, int grid, cudaStream_t);
using PersistPrepFn = cudaError_t (*)(int batch);
using PersistOccFn = cudaError_t (*)(int batch, int* per_sm);
// cluster-resident variant: a grid of batch clusters of `cluster` CTAs
using PersistClusterFn = cudaError_t (*)(const PersistArgs&, int cluster, cudaStream_t);
using PersistClusterPrepFn = cudaError_t (*)(int batch, int cluster, int* max_clusters);

struct ColVariant {
  PassFn launch;
  PrepFn prep;
  int C;
  int pipe;
  int sched;  // radix schedule of its transforms (LengthKernels::sched_radix)
};
constexpr int MAX_COL_VARIANTS = 24;
constexpr int MAX_SCHED_STAGES = 6;
constexpr int MAX_MODE_VARIANTS = 12;

// tables of launchers for one length, filled by the per-length translation units
struct LengthKernels {
  int n;
  // radix schedules of this length, in forward order: [0] that of every pass,
  // [1] an alternative some column shapes are also built with (0 stages: none)
  int sched_radix[2][MAX_SCHED_STAGES];
  int sched_stages[2];
  PassFn row[NUM_ROW_OPS];
  PrepFn row_prep[NUM_ROW_OPS];
  ColVariant colv[NUM_COL_OPS][MAX_COL_VARIANTS];
  int ncolv[NUM_COL_OPS];
  // mode column passes (CM_FWD, CM_BACK): shapes, the default first
  ColVariant colmodev[2][MAX_MODE_VARIANTS];
  int ncolmodev[2];
  // persistent solver (square grids of the sizes persist_size accepts; null otherwise)
  PersistFn persist;
  PersistPrepFn persist_prep;
  PersistOccFn persist_occupancy;
  // cluster-resident solver, per radix schedule set (null where not built)
  PersistClusterFn persist_cluster[2];
  PersistClusterPrepFn persist_cluster_prep[2];
};

// defined in the per-length translation units
const LengthKernels* kernels_for_length(int n);

// TMA map of a field of B projections of ny x nx complex values (api.cu)
bool encode_field_tmap(CUtensorMap* m, const void* base, int B, int ny, int nx, int C);

// ---------------------------------------------------------------------------
// persistent solvers (persist.cuh)
// ---------------------------------------------------------------------------
struct DevIter {
  double mu;       // mu of Algorithm S1 after the last completed iteration
  float beta;      // (mu_prev - 1)/mu for the next iteration
  int iter;        // completed iterations
  int n_active;    // projections still iterating
  int nonfinite;   // a non-finite loss was seen
  int status;      // PWF_OK, or PWF_ERR_TIMEOUT once a device-side wait ran out
};

enum PersistKind : int { PK_ROW = 0, PK_COL = 1, PK_FINALIZE = 2 };
constexpr int PERSIST_THREADS = 512;
constexpr int PERSIST_MAX_PHASES = 16;
struct PersistPhase {
  int kind;
  int op;
  int flush;   // after this pass, write the CTA's sums of the iteration out
  PassArgs a;
};

struct PersistArgs {
  const PersistPhase* phases;  // device array of nphases
  int nphases;
  int B;
  int max_iter;
  double corr_tol;
  double* gpart;               // [gridDim.x][B][NACC] per-CTA partial sums
  unsigned* bar;               // grid barrier (2 words, zeroed before the launch)
  long long cap;               // clock64 cycles a barrier may wait
  int* active;
  int* iters;
  double* loss;
  double* corr;
  DevIter* it;
  DevIter* cit;                // [B] per-projection iteration records (cluster-resident variant)
};

}  // namespace pwf
