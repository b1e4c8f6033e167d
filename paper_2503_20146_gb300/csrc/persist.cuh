// End-of-iteration bookkeeping of Algorithm S1 and the persistent solver.
//
// Algorithm S1 ends every iteration with the loss of Eq. (2), the correlation
// of successive fields (the stopping rule of Methods, "Reconstruction
// procedure") and Nesterov's sequence mu. The graph-replayed solver does that
// in k_finalize (api.cu); the persistent solver below does it inside its own
// launch. Both use the helpers of this header.
//
// Persistent solver: for square grids of at most 512^2 the whole solve is one
// cooperative launch of one CTA per SM. Each iteration runs the same passes as
// the graph (the row and column bodies of passes.cuh), separated by grid
// barriers. A pass is split into warp-sized items (32 / TPF rows or columns,
// TPF the threads of one transform), dealt round-robin over the warps of the
// grid with consecutive items on different SMs, so that even a 128^2 field
// spreads over the whole GPU; at these sizes every field stays in L2 and the
// time of a pass is the latency of one item. Reductions go to per-CTA partial
// sums in shared memory, written out once per iteration and summed by CTA 0
// in a fixed order (no global atomics). Every barrier waits at most `cap`
// clock64 cycles; a wait that runs out writes PWF_ERR_TIMEOUT to the status
// word, and every CTA leaves at its next barrier.
#pragma once
#include "../../include/pwf.h"
#include "passes.cuh"

namespace pwf {
inline namespace PWF_KNS {


// Per-projection end of an iteration from its five sums (loss and the three
// correlation sums): loss, correlation, iteration count and the stopping rule.
// Returns 1 while the projection keeps iterating.
__device__ __forceinline__ int finalize_projection(int p, const double* a, int* active, int* iters, double* loss,
                                                   double* corr, double corr_tol, int& nonfinite) {
  if (!active[p]) return 0;
  const double L = a[ACC_LOSS];
  const double c = sqrt(a[ACC_XR] * a[ACC_XR] + a[ACC_XI] * a[ACC_XI]) / sqrt(a[ACC_XNEW] * a[ACC_XOLD]);
  loss[p] = L;
  corr[p] = c;
  iters[p] += 1;
  // the correlation sums run over every element of exp(psi) of both
  // iterates, so a non-finite iterate shows here even where the loss is finite
  if (!isfinite(L) || !isfinite(c)) nonfinite = 1;
  if (corr_tol > 0.0 && c > corr_tol) {
    active[p] = 0;
    return 0;
  }
  return 1;
}

// Nesterov's sequence mu <- (1 + sqrt(1 + 4 mu^2)) / 2 and the momentum
// coefficient (mu_prev - 1)/mu of the next iteration, kept in FP64.
__device__ __forceinline__ void finalize_momentum(DevIter* it, int n_active) {
  const double mu_prev = it->mu;
  const double mu = 0.5 * (1.0 + sqrt(1.0 + 4.0 * mu_prev * mu_prev));
  const double mu_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * mu * mu));
  it->mu = mu;
  it->beta = (float)((mu - 1.0) / mu_next);
  it->iter += 1;
  it->n_active = n_active;
}

// ---------------------------------------------------------------------------
// grid barrier with a bounded wait
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// bar[0] counts arrivals, bar[1] is the generation. Returns false once the
// status word holds an error (this wait ran out, or another CTA's did).
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status, long long cap) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = ld_volatile_i32(status) == PWF_OK;
    if (ok) {
      const unsigned gen = ld_acquire_u32(&bar[1]);
      __threadfence();
      if (atomicAdd(&bar[0], 1u) + 1u == gridDim.x) {
        bar[0] = 0u;
        st_release_u32(&bar[1], gen + 1u);
      } else {
        const long long t0 = clock64();
        while (ld_acquire_u32(&bar[1]) == gen) {
          if (clock64() - t0 > cap) {
            atomicCAS(status, PWF_OK, PWF_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
      ok = ld_volatile_i32(status) == PWF_OK;
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// persistent solver
// ---------------------------------------------------------------------------
__host__ __device__ constexpr bool persist_size(int n) { return n == 64 || n == 128 || n == 256 || n == 512; }


__host__ __device__ constexpr size_t persist_smem_bytes(int n, int batch) {
  return (size_t)(PERSIST_THREADS / 32) * (32 / tpf_for(n)) * row_smem_len(n) * sizeof(float2) +
         (size_t)batch * NACC * sizeof(double);
}

// sum of a thread's float partial over the warp, in FP64
__device__ __forceinline__ double warp_sum(float x) {
  double s = (double)x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// rows of a row pass: item = 32/TPF consecutive rows (one projection)
template <int N, int OP, bool TWS>
__device__ __forceinline__ void persist_rows(const PassArgs& a, int gw, int GW, int lane, float2* wsm, double* s_acc,
                                             int only) {
  constexpr int TPF = tpf_for(N), RPW = 32 / TPF;
  const int sub = lane / TPF, t = lane - sub * TPF;
  const RowLayout<TPF, 32, TWS> sm{wsm + sub * row_smem_len(N), 0};
  // every projection's rows, or (only >= 0) those of projection `only`
  const long long per = (long long)a.ny / RPW;
  const long long i0 = only < 0 ? 0 : only * per, items = only < 0 ? a.B * per : i0 + per;
  for (long long it = i0 + gw; it < items; it += GW) {
    const long long row = it * RPW + sub;
    const int proj = (int)((it * RPW) / a.ny);
    if (skip_proj(a, proj)) continue;  // uniform per warp
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    row_body<N, OP>(a, row, t, sm, part);
    if constexpr (RowT<OP>::nred == 1) {
      const double s = warp_sum(part[0]);
      if (lane == 0) atomicAdd(&s_acc[proj * NACC + ACC_LOSS], s);
    } else if constexpr (RowT<OP>::nred == 5) {
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const double s = warp_sum(part[k]);
        if (lane == 0) atomicAdd(&s_acc[proj * NACC + ACC_XR + k], s);
      }
    }
    __syncwarp();
  }
}

// columns of a column pass: item = 32/TPF adjacent columns of one projection;
// lane = t * CPW + c, so that a warp's loads cover CPW adjacent columns
template <int N, int OP, bool TWS>
__device__ __forceinline__ void persist_cols(const PassArgs& a, int gw, int GW, int lane, float2* wsm, double* s_acc,
                                             int only) {
  constexpr int TPF = tpf_for(N), CPW = 32 / TPF;
  const int c = lane % CPW, t = lane / CPW;
  const RowLayout<TPF, 32, TWS> sm{wsm + c * row_smem_len(N), 0};
  const long long per = (long long)a.nx / CPW;
  const long long i0 = only < 0 ? 0 : only * per, items = only < 0 ? a.B * per : i0 + per;
  for (long long it = i0 + gw; it < items; it += GW) {
    const long long cg = it * CPW;
    const int proj = (int)(cg / a.nx);
    const int col = (int)(cg - (long long)proj * a.nx) + c;
    if (skip_proj(a, proj)) continue;
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    col_body<N, OP>(a, proj, col, t, sm, part);
    if constexpr (OP == COL_RESID_IOTF2) {
      const double s = warp_sum(part[0]);
      if (lane == 0) atomicAdd(&s_acc[proj * NACC + ACC_LOSS], s);
    }
    __syncwarp();
  }
}

template <int N, bool TWS = false>
__device__ __forceinline__ void persist_row_op(int op, const PassArgs& a, int gw, int GW, int lane, float2* wsm,
                                               double* s_acc, int only = -1) {
  switch (op) {
    case ROW_MUL_T: persist_rows<N, ROW_MUL_T, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case ROW_INTENSITY: persist_rows<N, ROW_INTENSITY, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case ROW_MUL_V: persist_rows<N, ROW_MUL_V, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case ROW_COH_RESID: persist_rows<N, ROW_COH_RESID, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case ROW_GRAD_PACK: persist_rows<N, ROW_GRAD_PACK, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case ROW_NESTEROV_FFT: persist_rows<N, ROW_NESTEROV_FFT, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    default: break;
  }
}

template <int N, bool TWS = false>
__device__ __forceinline__ void persist_col_op(int op, const PassArgs& a, int gw, int GW, int lane, float2* wsm,
                                               double* s_acc, int only = -1) {
  switch (op) {
    case COL_Q: persist_cols<N, COL_Q, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case COL_RESID_IOTF2: persist_cols<N, COL_RESID_IOTF2, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    case COL_PRECOND_REG: persist_cols<N, COL_PRECOND_REG, TWS>(a, gw, GW, lane, wsm, s_acc, only); break;
    default: break;
  }
}

template <int N>
__global__ void __launch_bounds__(PERSIST_THREADS, 1) persist_kernel(const PersistArgs pa) {
  constexpr int W = PERSIST_THREADS / 32, RPW = 32 / tpf_for(N);
  extern __shared__ float2 smem[];
  double* s_acc = reinterpret_cast<double*>(smem + W * RPW * row_smem_len(N));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = warp * gridDim.x + blockIdx.x;  // consecutive items on different SMs
  const int GW = gridDim.x * W;
  float2* wsm = smem + warp * RPW * row_smem_len(N);
  int* status = &pa.it->status;
  for (int i = threadIdx.x; i < pa.B * NACC; i += blockDim.x) s_acc[i] = 0.0;

  for (int iter = 0; iter < pa.max_iter; iter++) {
    for (int ph = 0; ph < pa.nphases; ph++) {
      const PersistPhase& P = pa.phases[ph];
      const int kind = P.kind, op = P.op;
      if (kind == PK_ROW) {
        persist_row_op<N>(op, P.a, gw, GW, lane, wsm, s_acc);
      } else if (kind == PK_COL) {
        persist_col_op<N>(op, P.a, gw, GW, lane, wsm, s_acc);
      } else if (kind == PK_FINALIZE && blockIdx.x == 0) {
        __shared__ int s_na, s_nf;
        if (threadIdx.x == 0) s_na = 0, s_nf = 0;
        __syncthreads();
        int na = 0, nf = 0;
        for (int p = threadIdx.x; p < pa.B; p += blockDim.x) {
          double sums[NACC] = {};
          for (int g = 0; g < (int)gridDim.x; g++) {  // fixed order: deterministic
            const double* q = pa.gpart + ((size_t)g * pa.B + p) * NACC;
#pragma unroll
            for (int k = 0; k < 5; k++) sums[k] += q[k];
          }
          na += finalize_projection(p, sums, pa.active, pa.iters, pa.loss, pa.corr, pa.corr_tol, nf);
        }
        atomicAdd(&s_na, na);
        if (nf) atomicOr(&s_nf, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
          if (s_nf) pa.it->nonfinite = 1;
          finalize_momentum(pa.it, s_na);
        }
      }
      if (P.flush) {
        // this CTA's sums of the iteration to its slot (read by CTA 0 after
        // the barrier); zeroed for the next iteration
        __syncthreads();
        double* g = pa.gpart + (size_t)blockIdx.x * pa.B * NACC;
        for (int i = threadIdx.x; i < pa.B * NACC; i += blockDim.x) {
          g[i] = s_acc[i];
          s_acc[i] = 0.0;
        }
      }
      if (!grid_sync(pa.bar, status, pa.cap)) return;
    }
    if (pa.corr_tol > 0.0 && ld_volatile_i32(&pa.it->n_active) == 0) break;
  }
}

// ---------------------------------------------------------------------------
// cluster-resident persistent solver
// ---------------------------------------------------------------------------
// One thread-block cluster per projection runs all of that projection's
// iterations: its CTAs split the rows and columns of every pass, and the
// hardware cluster barrier (release/acquire at cluster scope, which orders the
// pass's global-memory writes before the next pass's reads) separates the
// passes. No CTA waits on another cluster, so clusters start and finish on
// their own, and the wait at a barrier ends once every thread of the cluster,
// all of which run the same sequence of barriers, has arrived. The end of an
// iteration (Algorithm S1's loss, correlation, stopping rule and Nesterov's
// mu) is taken by the cluster's first CTA from the CTAs' partial sums in a
// fixed order, into the projection's own iteration record, whose beta the
// Nesterov pass of the cluster reads.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

constexpr int PERSIST_MAX_CLUSTER = 16;

// dynamic shared memory: the warps' transform buffers, the sums, then a copy
// of the passes' arguments (128-byte aligned)
__host__ __device__ constexpr size_t persist_cluster_phase_offset(int n, int batch) {
  return (persist_smem_bytes(n, batch) + 127) / 128 * 128;
}
// then the forward and inverse twiddle tables of the length (rows and columns
// of a square plan share them)
__host__ __device__ constexpr size_t persist_cluster_tw_offset(int n, int batch) {
  return persist_cluster_phase_offset(n, batch) + PERSIST_MAX_PHASES * sizeof(PersistPhase);
}
__host__ __device__ constexpr size_t persist_cluster_smem_bytes(int n, int batch) {
  return persist_cluster_tw_offset(n, batch) +
         (size_t)(twiddle_len(n, FWD) + twiddle_len(n, INV) + 2) * sizeof(float2);
}

template <int N>
__global__ void __launch_bounds__(PERSIST_THREADS, 1) persist_cluster_kernel(const PersistArgs pa) {
  constexpr int W = PERSIST_THREADS / 32, RPW = 32 / tpf_for(N);
  static_assert(sizeof(PersistPhase) % 16 == 0, "phases are copied in 16-byte words");
  extern __shared__ __align__(128) float2 smem[];
  double* s_acc = reinterpret_cast<double*>(smem + W * RPW * row_smem_len(N));
  PersistPhase* s_ph = reinterpret_cast<PersistPhase*>(reinterpret_cast<char*>(smem) +
                                                       persist_cluster_phase_offset(N, pa.B));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int CS = (int)cluster_count(), cr = (int)cluster_rank();
  const int proj = (int)cluster_index();
  const int gw = warp * CS + cr, GW = CS * W;  // consecutive items on different CTAs
  float2* wsm = smem + warp * RPW * row_smem_len(N);
  DevIter* cit = pa.cit + proj;

  {
    const int4* src = reinterpret_cast<const int4*>(pa.phases);
    int4* dst = reinterpret_cast<int4*>(s_ph);
    const int words = pa.nphases * (int)(sizeof(PersistPhase) / 16);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  for (int i = threadIdx.x; i < pa.B * NACC; i += blockDim.x) s_acc[i] = 0.0;
  __syncthreads();
  // The twiddle tables into shared memory: after a cluster barrier the
  // transforms of the next pass then find them at shared-memory latency. The
  // first phase is a column pass of the plan's column axis; a square plan's
  // row axis has the same tables.
  constexpr int TWF = twiddle_len(N, FWD), TWI = twiddle_len(N, INV);
  float2* s_twf = reinterpret_cast<float2*>(reinterpret_cast<char*>(smem) + persist_cluster_tw_offset(N, pa.B));
  float2* s_twi = s_twf + (TWF > 0 ? TWF : 1);
  for (int i = threadIdx.x; i < TWF; i += blockDim.x) s_twf[i] = s_ph[0].a.tw_fwd[i];
  for (int i = threadIdx.x; i < TWI; i += blockDim.x) s_twi[i] = s_ph[0].a.tw_inv[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int ph = 0; ph < pa.nphases; ph++) {
      // the Nesterov pass reads this projection's beta
      if (s_ph[ph].a.beta == &pa.it->beta) s_ph[ph].a.beta = &cit->beta;
      s_ph[ph].a.tw_fwd = s_twf;
      s_ph[ph].a.tw_inv = s_twi;
    }
    if (cr == 0) {
      *cit = *pa.it;
      cit->n_active = pa.active[proj] ? 1 : 0;
    }
  }
  cluster_barrier();

  for (int iter = 0; iter < pa.max_iter; iter++) {
    for (int ph = 0; ph < pa.nphases; ph++) {
      const PersistPhase& P = s_ph[ph];
      if (P.kind == PK_ROW) {
        persist_row_op<N, true>(P.op, P.a, gw, GW, lane, wsm, s_acc, proj);
      } else if (P.kind == PK_COL) {
        persist_col_op<N, true>(P.op, P.a, gw, GW, lane, wsm, s_acc, proj);
      } else if (P.kind == PK_FINALIZE && cr == 0 && threadIdx.x == 0) {
        double sums[NACC] = {};
        const int b0 = (int)blockIdx.x - cr;
        for (int g = 0; g < CS; g++) {  // fixed order: deterministic
          const double* q = pa.gpart + (size_t)(b0 + g) * NACC;
#pragma unroll
          for (int k = 0; k < 5; k++) sums[k] += q[k];
        }
        int nf = 0;
        const int na = finalize_projection(proj, sums, pa.active, pa.iters, pa.loss, pa.corr, pa.corr_tol, nf);
        if (nf) pa.it->nonfinite = 1;
        finalize_momentum(cit, na);
      }
      if (P.flush) {
        // this CTA's sums of the iteration to its slot (read by the cluster's
        // first CTA after the barrier); zeroed for the next iteration
        __syncthreads();
        double* g = pa.gpart + (size_t)blockIdx.x * NACC;
        if (threadIdx.x < NACC) {
          g[threadIdx.x] = s_acc[proj * NACC + threadIdx.x];
          s_acc[proj * NACC + threadIdx.x] = 0.0;
        }
      }
      cluster_barrier();
    }
    if (pa.corr_tol > 0.0 && ld_volatile_i32(&cit->n_active) == 0) break;
  }
}

// The plan's iteration record after a cluster-resident solve: iteration count,
// mu and beta of the projection that iterated longest, active count summed.
static __global__ void k_persist_cluster_finish(const DevIter* cit, int B, DevIter* it) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int best = 0, na = 0;
    for (int p = 0; p < B; p++) {
      if (cit[p].iter > cit[best].iter) best = p;
      na += cit[p].n_active;
    }
    it->mu = cit[best].mu;
    it->beta = cit[best].beta;
    it->iter = cit[best].iter;
    it->n_active = na;
  }
}

template <int N>
cudaLaunchConfig_t persist_cluster_config(int batch, int cluster, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(batch * cluster));
  cfg.blockDim = dim3(PERSIST_THREADS);
  cfg.dynamicSmemBytes = persist_cluster_smem_bytes(N, batch);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Sets the kernel's attributes for `cluster` CTAs per cluster and reports how
// many such clusters the device holds at once (0: the shape does not fit).
template <int N>
cudaError_t prep_persist_cluster(int batch, int cluster, int* max_clusters) {
  *max_clusters = 0;
  if (cluster < 1 || cluster > PERSIST_MAX_CLUSTER) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(persist_cluster_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)persist_cluster_smem_bytes(N, batch));
  if (e == cudaSuccess && cluster > 8)
    e = cudaFuncSetAttribute(persist_cluster_kernel<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = persist_cluster_config<N>(batch, cluster, nullptr, attr);
  return cudaOccupancyMaxActiveClusters(max_clusters, persist_cluster_kernel<N>, &cfg);
}

template <int N>
cudaError_t launch_persist_cluster(const PersistArgs& pa, int cluster, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = persist_cluster_config<N>(pa.B, cluster, s, attr);
  cudaError_t e = cudaLaunchKernelEx(&cfg, persist_cluster_kernel<N>, pa);
  if (e != cudaSuccess) return e;
  k_persist_cluster_finish<<<1, 32, 0, s>>>(pa.cit, pa.B, pa.it);
  return cudaGetLastError();
}

template <int N>
cudaError_t prep_persist(int batch) {
  return cudaFuncSetAttribute(persist_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)persist_smem_bytes(N, batch));
}

template <int N>
cudaError_t launch_persist(const PersistArgs& pa, int grid, cudaStream_t s) {
  void* args[] = {const_cast<PersistArgs*>(&pa)};
  return cudaLaunchCooperativeKernel((const void*)persist_kernel<N>, dim3(grid), dim3(PERSIST_THREADS), args,
                                     persist_smem_bytes(N, pa.B), s);
}

template <int N>
cudaError_t occupancy_persist(int batch, int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, persist_kernel<N>, PERSIST_THREADS,
                                                       persist_smem_bytes(N, batch));
}

template <int N>
LengthKernels with_persist(LengthKernels k) {
  if constexpr (persist_size(N)) {
    k.persist = launch_persist<N>;
    k.persist_prep = prep_persist<N>;
    k.persist_occupancy = occupancy_persist<N>;
    k.persist_cluster[0] = launch_persist_cluster<N>;
    k.persist_cluster_prep[0] = prep_persist_cluster<N>;
  }
  return k;
}

// The cluster-resident solver built with this translation unit's schedule
// set, registered in that set's slot (lengths whose transform fits one warp).
template <int N>
void add_schedule_cluster(LengthKernels& k) {
  if constexpr (persist_size(N) && tpf_for(N) <= 32) {
    k.persist_cluster[PWF_SCHED_VARIANT] = launch_persist_cluster<N>;
    k.persist_cluster_prep[PWF_SCHED_VARIANT] = prep_persist_cluster<N>;
  }
}

}  // namespace PWF_KNS
}  // namespace pwf
