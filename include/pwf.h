/*
 * pwf.h — C ABI of the GB300 (sm_103a) preconditioned Wirtinger flow library.
 *
 * Method: K. Lee, H. Hugonnet, J.-H. Lim, Y. Park, "Speckle-based X-ray
 * microtomography via preconditioned Wirtinger flow", arXiv 2503.20146.
 * Algorithms S1 (the PWF iteration) and S2 (its forward model, Wirtinger
 * derivative, preconditioner, regularizer and angular-spectrum propagation);
 * forward model Eq. (1); loss Eq. (2); IOTF Eq. (5); preconditioning filter
 * Eq. (11); sample transfer function and regularization window Eqs. (14)-(15).
 * Notation: F, F^-1 the 2-D DFT pair; P(L){x} = F^-1{Q F{x}} propagation over
 * L; P1, P2 over L1, L2; P^H the adjoint (propagation over -L).
 *
 * Conventions shared by every entry point
 *  - Arrays are caller-owned DEVICE memory unless a parameter says "host".
 *    Complex arrays are interleaved complex64 (float re, float im), row-major
 *    [batch][ny][nx]. Real arrays are float32 [batch][ny][nx]. The diffuser t
 *    is one complex64 [ny][nx] field shared by every projection of the batch.
 *    Device arrays passed to plan calls must be 16-byte aligned (rows are read
 *    with 16-byte loads and L2 bulk prefetches); a misaligned one returns
 *    PWF_ERR_INVALID_ARG before any work is queued. Fresh cudaMalloc and
 *    PyTorch allocations are 256-byte aligned. pwf_fbp's own rules are below.
 *  - ny and nx are each one of 16, 32, 64, 96, 128, 256, 512, 768, 1024, 1536,
 *    2048 (other sizes return PWF_ERR_UNSUPPORTED).
 *  - Work is enqueued on the plan's stream (pwf_plan_desc.stream, a
 *    cudaStream_t; NULL means the legacy default stream) and runs
 *    asynchronously, except where a parameter is a host output: then the call
 *    synchronises the stream before returning.
 *  - No entry point throws. Errors are returned as pwf_status; the first CUDA
 *    error seen by a plan is sticky and returned by every later call on it.
 *  - A plan owns its workspace (a few complex fields per projection) and its
 *    1-D filter tables. Plans are not thread-safe; use one per host thread.
 *
 * Deliberate differences from a minimal "plan / forward / gradient / step /
 * solve" interface, and why
 *  - pwf_gradient leaves the per-projection loss in DEVICE memory, so that the
 *    call stays asynchronous and can sit inside a caller's CUDA graph or an
 *    autograd backward; host losses come from pwf_state_read, pwf_solve and
 *    pwf_group_read.
 *  - The diffuser t is an argument of every call, not of plan creation: the
 *    joint refinement (pwf_solve_joint) and autograd change it between calls.
 *  - One plan holds one (ny, nx). Series of mixed sizes are several plans
 *    joined in a pwf_group: each size class then has its own tuned column
 *    shapes, radix schedules and 1-D tables.
 *  - The coherence model is chosen by the descriptor's values, not an enum:
 *    xcoh_m = ycoh_m = 0 coherent, > 0 the paper's IOTF, n_modes = 9 or 25 the
 *    source-mode variant.
 *  - No flag stores or recomputes v: the fused solver always keeps the
 *    detector field of the forward pass for its backward pass, and
 *    pwf_forward_vjp always recomputes it (at most one mode's field at a time).
 *  - No exact-ASM switch: the propagator is applied as the sum of its axis
 *    restrictions, and plan creation rejects (PWF_ERR_UNSUPPORTED) any
 *    geometry where that differs from the exact phase by more than 1e-6 rad.
 *  - Bounds checking is a separate build (libpwf_bc.so, PWF_BOUNDS_CHECK), not
 *    a flag, so the normal library's kernels carry none of its branches.
 *  - dL/dt comes from pwf_forward_vjp (with dL/dpsi), not from pwf_gradient.
 */
#ifndef PWF_H
#define PWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PWF_OK = 0,
  PWF_ERR_INVALID_ARG = 1,  /* null pointer, non-positive size, bad flag value */
  PWF_ERR_UNSUPPORTED = 2,  /* transform length not built, or geometry outside the
                               separable-propagator bound (see pwf_plan_create) */
  PWF_ERR_NOMEM = 3,        /* device allocation failed */
  PWF_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
  PWF_ERR_NONFINITE = 5,    /* a non-finite loss was produced */
  PWF_ERR_STATE = 6,        /* state / plan mismatch or bad checkpoint buffer */
  PWF_ERR_TIMEOUT = 7,      /* a device-side wait of the persistent solver ran
                               out (pwf_plan_set_wait_limit); the GPU context
                               stays usable, psi and the state are not defined */
  PWF_ERR_BOUNDS = 8        /* bounds-checked builds (PWF_BOUNDS_CHECK): a pass
                               met an index outside the plan's arrays and
                               skipped it; results are not defined            */
} pwf_status;

typedef struct pwf_plan pwf_plan;
typedef struct pwf_state pwf_state;

/* plan flags (ablations of Figs. S3-S5 and the unfused baseline) */
#define PWF_FLAG_NO_PRECOND 0x1u /* P^-1 := 1 (Preconditioner off, Fig. S3)        */
#define PWF_FLAG_NO_REG 0x2u     /* alpha := 0 (regularizer off)                   */
#define PWF_FLAG_PLAIN 0x4u      /* unfused per-operation kernels, one projection at
                                    a time: Algorithm S2 executed step by step     */
#define PWF_FLAG_NO_TUNE 0x8u    /* skip the plan-time column-pass autotuning      */
#define PWF_FLAG_PERSISTENT 0x20u /* pwf_solve as ONE cooperative launch for all
                                    iterations (grid barriers between the passes,
                                    every wait bounded); square grids of 64, 128, 256
                                    or 512 only, else PWF_ERR_UNSUPPORTED           */
#define PWF_FLAG_GRAPH 0x40u     /* pwf_solve as one CUDA graph holding the whole
                                    iteration loop (the default, but see CLUSTER)  */
#define PWF_FLAG_CLUSTER 0x80u   /* pwf_solve as ONE launch of one thread-block
                                    cluster per projection for all iterations
                                    (hardware cluster barriers between the passes);
                                    square grids of 64, 128, 256 or 512 only, else
                                    PWF_ERR_UNSUPPORTED. At most one of PERSISTENT,
                                    GRAPH and CLUSTER (else PWF_ERR_INVALID_ARG).
                                    With none of the three, a plan takes this
                                    solver where it measured faster: square
                                    128^2 IOTF/coherent plans whose batch one
                                    wave of clusters holds (not with
                                    PWF_FLAG_CHECK_FINITE)                         */
#define PWF_FLAG_CHECK_FINITE 0x200u /* debug: after every pass a scan of what it
                                    wrote; pwf_state_read (and pwf_solve) then
                                    return PWF_ERR_NONFINITE naming, in
                                    pwf_plan_last_error, the first pass whose
                                    output held a NaN or an infinity. Graph
                                    solver only (PWF_ERR_UNSUPPORTED with
                                    PERSISTENT or CLUSTER)                        */
#define PWF_FLAG_UNPACKED_RESID 0x400u /* the residual passes of the IOTF iteration on
                                    full complex rows and every column (by default
                                    the real intensity and residual fields travel
                                    two rows per complex row, and the column pass
                                    covers bins kx = 0..nx/2 only, the other half
                                    being their conjugates)                       */
#define PWF_FLAG_NO_PDL 0x100u   /* launch the passes without programmatic dependent
                                    launch (by default each pass is scheduled once
                                    the CTAs of the one before it have exited and
                                    waits on the device for that pass's writes)    */

/* Inputs of Algorithm S1 other than y and t. All lengths in metres. */
typedef struct {
  int32_t batch;     /* number of independent projections B >= 1 */
  int32_t ny, nx;    /* detector grid */
  double pixel_m;    /* detector pixel pitch p */
  double wavelength_m;
  double L1_m;       /* sample -> diffuser */
  double L2_m;       /* diffuser -> detector */
  double xcoh_m, ycoh_m; /* coherence lengths of Eqs. (4), (5), (14); both 0 = fully
                            coherent: IOTF = 1 and Gamma^2 = 0 */
  double gamma;      /* oversampling ratio of Eq. (14) (paper: 1) */
  double alpha_re, alpha_im; /* regularization parameter (paper: 0.1 + 0.01i) */
  double eta;        /* step size of Algorithm S1 */
  uint32_t flags;    /* PWF_FLAG_* */
  void* stream;      /* cudaStream_t */
  /* Source-mode variant of the partial-coherence model (not the paper's form;
   * 0 or 1 = the paper's IOTF form). n_modes = 9 or 25: the IPSF convolution of
   * Eq. (1) is replaced by the intensities of K mutually incoherent tilted
   * plane-wave modes summed with weights: f = sum_j w_j |P2{t P1{x s_j}}|^2,
   * s_j = exp(i 2 pi (mx_j x / nx + my_j y / ny)), nodes and weights of the
   * tensor Gauss-Hermite rule (3 or 5 points per axis) of a Gaussian source
   * whose walk-off over L1 + L2 has std mode_sigma_px pixels at the detector;
   * tilts rounded to whole frequency bins. x_coh/y_coh still set the
   * regularization window Gamma^2 (Eqs. (14)-(15)). */
  int32_t n_modes;
  double mode_sigma_px;
} pwf_plan_desc;

/* Creates a plan. Unless PWF_FLAG_NO_TUNE is set, the plan also times every
 * column-pass shape it was built with (columns per tile, pipelined or not) on
 * its own zeroed workspace, on desc->stream, and keeps the fastest per pass
 * (a few launches per shape; the call synchronises that stream).
 * Builds the 1-D frequency tables of Q_k = exp(i 2 pi (w - 1/lambda) L)
 * (angular-spectrum propagation, Algorithm S2, constant piston dropped), IOTF (Eq. (5)),
 * P^-1 = 1/(u^2 + v^2) in cycles per pixel with P^-1(0) = 0 (Eq. (11)) and
 * Gamma^2 = 1 - STF (Eqs. (14)-(15)). The propagator phase is applied as the sum
 * of its two axis restrictions; the plan checks, in double precision, that the
 * neglected cross term is below 1e-6 rad over the grid (it is ~1e-8 rad for
 * hard X-rays on micron pixels) and returns PWF_ERR_UNSUPPORTED otherwise.
 * Returns PWF_ERR_UNSUPPORTED also for evanescent bins (rho^2 >= lambda^-2).
 * *out receives the plan; it must be released with pwf_plan_destroy. */
pwf_status pwf_plan_create(const pwf_plan_desc* desc, pwf_plan** out);
pwf_status pwf_plan_destroy(pwf_plan* plan);
/* Replaces the stream used by later calls on this plan. */
pwf_status pwf_plan_set_stream(pwf_plan* plan, void* stream);
/* Bytes of device workspace the plan holds. */
size_t pwf_plan_workspace_bytes(const pwf_plan* plan);

/* The forward model f(psi) of Eq. (1) (Algorithm S2):
 *   x = exp(psi); v = P2{ t P1{x} }; f = Re F^-1{ IOTF F{|v|^2} }.
 * psi: complex64 [B][ny][nx]; t: complex64 [ny][nx]; f: float32 [B][ny][nx]. */
pwf_status pwf_forward(pwf_plan* plan, const void* psi, const void* t, float* f);

/* The Wirtinger derivative g of Algorithm S2 at psi (the raw, unpreconditioned
 * gradient with the factor 2 dropped, divided by max |t|^2):
 *   g = conj(x) P1^H{ conj(t) P2^H{ v F^-1{IOTF F{f - y}} } } / max|t|^2,
 * and the loss of Eq. (2).
 * g: complex64 [B][ny][nx]; loss: device float64 [B] (may be NULL).
 * The gradient of the loss w.r.t. Re psi and Im psi is 4 max|t|^2 (Re g, Im g). */
pwf_status pwf_gradient(pwf_plan* plan, const void* psi, const void* t, const float* y,
                        void* g, double* loss);

/* Vector-Jacobian product of the forward model f(psi, t) for a real cotangent
 * grad_f = dL/df (float32 [B][ny][nx]), in the convention dL/dRe + i dL/dIm:
 *   grad_psi = 2 conj(x) P1^H{ conj(t) P2^H{ v F^-1{IOTF F{grad_f}} } }
 *   grad_t   = sum over the batch of 2 conj(P1{x}) P2^H{ v F^-1{IOTF F{grad_f}} }
 * (the second is the diffuser gradient of the simultaneous retrieval of
 * Methods / Fig. S12). grad_psi: complex64 [B][ny][nx] (may be NULL);
 * grad_t: complex64 [ny][nx] (may be NULL). Intermediate fields are recomputed
 * from psi and t, not taken from an earlier pwf_forward. */
pwf_status pwf_forward_vjp(pwf_plan* plan, const void* psi, const void* t, const float* grad_f,
                           void* grad_psi, void* grad_t);

/* Solver state of Algorithm S1: phi (the previous Nesterov point), mu, the
 * iteration count, per-projection convergence flags and the last loss and
 * correlation. */
pwf_status pwf_state_create(pwf_plan* plan, pwf_state** out);
pwf_status pwf_state_destroy(pwf_state* state);
/* phi := 0, mu := 1, iteration := 0, every projection active (Algorithm S1 set-up). */
pwf_status pwf_state_reset(pwf_plan* plan, pwf_state* state);

/* One iteration of the while-loop of Algorithm S1 on every still-active
 * projection, updating psi (complex64 [B][ny][nx], in place) and the state.
 * corr_tol > 0 enables the stopping rule of Methods ("Reconstruction
 * procedure"): a projection whose normalized correlation between exp(psi) of
 * this and the previous iteration exceeds corr_tol stops (its psi is left
 * as the converged value). corr_tol <= 0 never stops. */
pwf_status pwf_step(pwf_plan* plan, pwf_state* state, const float* y, const void* t, void* psi,
                    double corr_tol);

/* Reads per-projection results of the last iteration into HOST arrays of
 * length B (any may be NULL): loss of Eq. (2) before the update, correlation,
 * iterations done, and 1/0 active flags. Synchronises the stream. */
pwf_status pwf_state_read(pwf_plan* plan, const pwf_state* state, double* loss_host,
                          double* corr_host, int32_t* iters_host, int32_t* active_host);

/* Algorithm S1 from the caller's psi (Algorithm S1 starts from psi = 0; the
 * caller zeroes psi for that): up to max_iter iterations, with the stopping
 * rule when corr_tol > 0. Fused, batched passes, run one of three ways:
 *  - one CUDA graph (the default): one iteration (its passes and the
 *    end-of-iteration kernel) captured once into the body of a conditional
 *    WHILE node, whose condition a last kernel sets after each iteration, so
 *    the loop runs on the device: one graph launch per call. Where the driver
 *    refuses conditional nodes, the one-iteration graph is launched from a host
 *    loop instead;
 *  - one persistent cooperative launch for all iterations (PWF_FLAG_PERSISTENT;
 *    square IOTF/coherent plans of 64^2..512^2): the passes are split into
 *    warp-sized items over every SM, with grid barriers between passes. Each
 *    barrier waits at most the plan's wait limit; when a wait runs out the
 *    launch ends early, and the call (or the next pwf_state_read) returns
 *    PWF_ERR_TIMEOUT;
 *  - one launch of one thread-block cluster per projection (PWF_FLAG_CLUSTER;
 *    the same plans): each cluster runs its projection's iterations on its
 *    own, with the hardware cluster barrier between passes, and no cluster
 *    waits on another.
 * iters_host / loss_host: HOST arrays of length B (may be NULL); when either is
 * given the call synchronises. psi is updated in place. */
pwf_status pwf_solve(pwf_plan* plan, const float* y, const void* t, void* psi, int32_t max_iter,
                     double corr_tol, int32_t* iters_host, double* loss_host);

/* Algorithm S1 (as pwf_solve) on HOST buffers: y (float32 [B][ny][nx]), t
 * (complex64 [ny][nx]) and psi (complex64 [B][ny][nx]; the initial guess when
 * psi_is_input != 0, else Algorithm S1's psi = 0 and psi_host is output only;
 * the result on return). The batch streams through the device in chunks of
 * `chunk` projections (0: the largest divisor of B not above B/4, rounded up;
 * otherwise chunk must divide B, else PWF_ERR_INVALID_ARG): the host-to-device
 * copy of chunk k + 1 and the device-to-host copy of chunk k - 1 overlap the
 * solve of chunk k. Each projection's iterates are those of pwf_solve on the
 * same inputs up to the column-pass shapes the chunk-sized plans pick.
 * Host buffers should be page-locked (cudaHostAlloc, or torch's pin_memory())
 * for the copies to overlap; pageable memory works but serialises them.
 * iters_host / loss_host: HOST arrays of length B (may be NULL). Returns after
 * the results are on the host; ordered after the work queued on the plan's
 * stream. The first call (and a call with another chunk) allocates two
 * chunk-sized plans and device slots: two chunks of y and psi, one t. */
pwf_status pwf_solve_host(pwf_plan* plan, const float* y_host, const void* t_host, void* psi_host,
                          int32_t psi_is_input, int32_t max_iter, double corr_tol, int32_t chunk,
                          int32_t* iters_host, double* loss_host);

/* Joint refinement of the shared diffuser (Methods, "Diffuser transmission
 * function", and Fig. S12: t is updated across all projections). Runs
 * max_iter iterations of Algorithm S1 over the batch (no stopping rule) and,
 * after each, t <- t - eta_t sum_b g_t,b with g_t = conj(P1{x})
 * P2^H{v F^-1{IOTF F{f - y}}} / max|t|^2 evaluated at the same point as the
 * sample gradient (a plain gradient step; max|t|^2 is recomputed from the new
 * t). t (complex64 [ny][nx], device) is updated in place, as is psi.
 * eta_t = 0 reproduces pwf_solve with corr_tol = 0. Keeps B extra fields of
 * workspace (allocated on the first call). PWF_ERR_UNSUPPORTED for source-mode
 * or plain plans; PWF_ERR_INVALID_ARG if eta_t < 0. It runs on the graph replay
 * (also for PWF_FLAG_PERSISTENT plans). */
pwf_status pwf_solve_joint(pwf_plan* plan, const float* y, void* t, void* psi, int32_t max_iter, double eta_t,
                           int32_t* iters_host, double* loss_host);

/* Groups: batches of mixed sizes. One plan per size class (each with its own
 * sizes, batch, coherence model and tuned column shapes) joined in a group and
 * solved together: pwf_group_solve runs Algorithm S1 on every class, one CUDA
 * graph launch per iteration, the graph forking one branch per class so the
 * classes' passes run concurrently. y, t, psi: arrays of n_plans device
 * pointers, in the order of `plans` (psi updated in place, as pwf_solve).
 * stream: cudaStream_t all work is ordered on (NULL = legacy default stream).
 * A plan may belong to one group at a time and must not be used on its own
 * while the group's solve runs. pwf_group_read reads class `index`'s loss and
 * iteration counts (HOST arrays of that plan's batch; synchronises). */
typedef struct pwf_group pwf_group;
pwf_status pwf_group_create(pwf_plan* const* plans, int32_t n_plans, pwf_group** out);
pwf_status pwf_group_destroy(pwf_group* group);
pwf_status pwf_group_solve(pwf_group* group, void* stream, const float* const* y, const void* const* t,
                           void* const* psi, int32_t max_iter, double corr_tol);
pwf_status pwf_group_read(pwf_group* group, int32_t index, double* loss_host, int32_t* iters_host);

/* Calibration from the reference speckle I_ref (float32 [ny][nx], device; the
 * plan's first projection slot is used as workspace), Methods "Intensity
 * optical transfer function (IOTF)" and "Diffuser transmission function".
 * pwf_calibrate_coherence: normalised intensity autocorrelation along x and
 * along y (circular, averaged over the other axis; Siegert relation), Gaussian
 * model g2 = 1 + A exp(-pi D^2 / coh^2) fitted by least squares on
 * ln(g2 - 1) over lags 1..max_lag; HOST outputs x_coh, y_coh in metres.
 * Synchronises. PWF_ERR_NONFINITE if g2 - 1 is not positive and decreasing
 * over the lags. pwf_diffuser_from_reference: I_coh = Re F^-1{W F{I_ref}},
 * W = IOTF/(IOTF^2 + wiener_eps) with the plan's IOTF, then
 * t = P(-L2){sqrt(max(I_coh, 0))} (phase zero at the detector); t_out is
 * complex64 [ny][nx] device memory. */
pwf_status pwf_calibrate_coherence(pwf_plan* plan, const float* I_ref, int32_t max_lag, double* xcoh_m_host,
                                   double* ycoh_m_host);
pwf_status pwf_diffuser_from_reference(pwf_plan* plan, const float* I_ref, double wiener_eps, void* t_out);

/* Filtered back projection after PWF (Methods, "Reconstruction procedure"):
 * standard parallel-beam FBP with the Ram-Lak filter, one slice per detector
 * row, then the factor -lambda / (2 pi p), which turns the retrieved
 * psi = -k int beta - i k int delta into beta + i delta.
 *   psi      complex64 [n_angles][ny][nx], device, 8-byte aligned; detector
 *            pixel j sits at s = j - nx/2 + 1/2 pixels from the rotation axis
 *   angles_rad_host  n_angles projection angles (host), normally [0, pi)
 *   vol_out  complex64 [ny][nx][nx], device, 8-byte aligned: slice y, row z
 *            (beam direction at angle 0), column x; Re = beta, Im = delta
 *   workspace  device memory of pwf_fbp_workspace_bytes(...) bytes, 256-byte
 *            aligned (filtered rows zero-padded to 2 nx as 16-byte
 *            interpolation records, filter and angle tables; about
 *            32 n_angles ny nx bytes)
 *   stream   cudaStream_t (null: legacy default stream)
 * Ram-Lak: h(0) = 1/4, h(k) = -1/(pi^2 k^2) for odd k, 0 otherwise (unit
 * sampling); linear convolution along the row (zero padding to 2 nx); back
 * projection f = (pi / n_angles) sum_a q_a(x cos theta_a + z sin theta_a) with
 * linear interpolation, zero outside the detector. Sizes: 1 <= n_angles <=
 * PWF_FBP_MAX_ANGLES, ny <= 65535, 2 nx one of 32, 64, 96, 128, 192, 256, 384,
 * 512, 768, 1024, 1536, 2048; otherwise PWF_ERR_INVALID_ARG (workspace_bytes
 * returns 0). A short or misaligned workspace, or misaligned psi / vol_out,
 * also returns PWF_ERR_INVALID_ARG before anything is queued.
 * The tables are copied from the host synchronously on the stream; the two
 * kernels are then enqueued asynchronously. */
#define PWF_FBP_MAX_ANGLES 4096
size_t pwf_fbp_workspace_bytes(int32_t n_angles, int32_t ny, int32_t nx);
pwf_status pwf_fbp(const void* psi, int32_t n_angles, int32_t ny, int32_t nx, const double* angles_rad_host,
                   double wavelength_m, double voxel_m, void* vol_out, void* workspace, size_t workspace_bytes,
                   void* stream);

/* Checkpoint: pwf_state_bytes gives the size of a host buffer that holds the
 * state (phi and the counters); save/load copy it. Loading into a state of a
 * plan with other sizes returns PWF_ERR_STATE. Both synchronise. */
size_t pwf_state_bytes(const pwf_state* state);
pwf_status pwf_state_save(pwf_plan* plan, const pwf_state* state, void* host_buf, size_t bytes);
pwf_status pwf_state_load(pwf_plan* plan, pwf_state* state, const void* host_buf, size_t bytes);

/* Instrumentation.
 * pwf_plan_launch_count: number of kernels this plan has enqueued so far
 * (kernels replayed from the solver's CUDA graph included); -1 for NULL.
 * pwf_profile_iteration: runs Algorithm S1 from the caller's psi for `iters`
 * fused iterations WITHOUT the graph, with a CUDA event pair recorded on the
 * plan's stream around every kernel, and returns for each kernel position of
 * one iteration its mean duration in milliseconds (pass_ms, HOST float array
 * of PWF_MAX_PASSES) and its static name (pass_names, HOST array of
 * PWF_MAX_PASSES pointers); *n_passes receives the count. psi is updated as by
 * pwf_solve. Synchronises. PWF_ERR_UNSUPPORTED for PWF_FLAG_PLAIN plans. */
#define PWF_MAX_PASSES 256
long long pwf_plan_launch_count(const pwf_plan* plan);
/* Writes a one-line description of the plan (sizes and the column-pass shape
 * chosen per pass, e.g. "col_q=C8p" = 8 columns per tile, pipelined) into buf
 * (NUL-terminated, truncated to len); returns the length needed including the
 * NUL. buf may be NULL to query the length. */
size_t pwf_plan_describe(const pwf_plan* plan, char* buf, size_t len);
/* Column-pass shapes (for tests and tuning studies). pass: 0 propagator,
 * 1 IOTF, 2 residual (Parseval), 3 preconditioner + regularizer, 4 forward
 * transform, 5 inverse transform, 6 the packed residual (bins 0..nx/2 of two
 * real rows per complex row), 7 and 8 the source-mode passes (spectral
 * shift + Q1 + inverse transform; transform + conj Q1 + shift back,
 * accumulated). Each pass's shapes cover both radix schedules of the length
 * where it has two. pwf_plan_column_shapes returns how many shapes the plan's
 * column length was built with (-1 on a bad argument);
 * pwf_plan_set_column_shape forces one (0-based), replacing the tuned choice. */
int32_t pwf_plan_column_shapes(const pwf_plan* plan, int32_t pass);
pwf_status pwf_plan_set_column_shape(pwf_plan* plan, int32_t pass, int32_t shape);
pwf_status pwf_profile_iteration(pwf_plan* plan, const float* y, const void* t, void* psi, int32_t iters,
                                 float* pass_ms, const char** pass_names, int32_t* n_passes);
/* Longest wait of one grid barrier of the persistent solver, in SM clock
 * cycles (clock64); default 2^31 (about one second). A limit of 0 makes the
 * first barrier any CTA reaches before the others run out at once, which is
 * how the timeout path is tested. PWF_ERR_INVALID_ARG for a negative limit.
 * pwf_plan_uses_persistent: 1 if pwf_solve takes the persistent launch on
 * this plan, 0 if it replays the graph, -1 for NULL. */
pwf_status pwf_plan_set_wait_limit(pwf_plan* plan, int64_t cycles);
int32_t pwf_plan_uses_persistent(const pwf_plan* plan);
/* CTAs per cluster of a PWF_FLAG_CLUSTER plan: 1..16, or 0 for the default
 * (the largest cluster the device holds, up to 16 and to one CTA per
 * warp-sized item of a pass). PWF_ERR_INVALID_ARG for another
 * plan or a size outside 0..16, PWF_ERR_UNSUPPORTED when the device cannot
 * hold such a cluster. pwf_plan_cluster_size returns the size in use (0 for
 * other plans, -1 for NULL); pwf_plan_uses_persistent returns 2 for these
 * plans. */
pwf_status pwf_plan_set_cluster_size(pwf_plan* plan, int32_t ctas);
int32_t pwf_plan_cluster_size(const pwf_plan* plan);
/* Radix schedule set of a PWF_FLAG_CLUSTER plan's kernel: 0 the default
 * schedule of the length, 1 its alternative (128 = 4.4.4.2, 256 = 4.8.8: one
 * transform per warp, fewer values per thread, so shorter dependent chains in
 * every pass item), -1 the alternative where built, else 0 (the plan's
 * choice). Also resets the cluster size to its default. PWF_ERR_UNSUPPORTED
 * when that set is not built for the length; pwf_plan_cluster_schedule
 * returns the set in use (-1 for other plans). */
pwf_status pwf_plan_set_cluster_schedule(pwf_plan* plan, int32_t set);
int32_t pwf_plan_cluster_schedule(const pwf_plan* plan);

/* Debug aid for the out-of-memory paths: the device allocation `after`
 * allocations from now (0: the next one) fails as if cudaMalloc had, so the
 * call making it returns PWF_ERR_NOMEM after freeing what it had allocated. A
 * negative value turns it off. Process-wide; not thread-safe against
 * concurrent plan creation. */
void pwf_debug_fail_alloc(int32_t after);

/* Debug aid for bounds-checked builds (compiled with PWF_BOUNDS_CHECK: every
 * pass checks the projection index of each CTA against the plan's batch
 * before touching memory, records PWF_ERR_BOUNDS and skips the work). Runs
 * one row transform of the plan's work field over one projection more than
 * the plan holds and synchronises: PWF_ERR_BOUNDS when the checks caught the
 * extra rows. Other builds launch nothing and return PWF_ERR_UNSUPPORTED. */
pwf_status pwf_debug_overrun(pwf_plan* plan);

/* Forward model for callers that cannot allocate device memory. The paper has
 * no counterpart: this is an interface choice, not part of the method.
 * pwf_forward needs a plan, and creating a plan allocates device memory. Some
 * callers cannot allow that: processes whose device memory is owned by another
 * allocator or reserved up front (a framework's caching pool, a fixed budget of
 * an acquisition pipeline), and code that cannot take the device-wide
 * synchronisation cudaMalloc/cudaFree imply. This call computes the same f as
 * pwf_forward (x = exp(psi); v = P2{t P1{x}}; f = Re F^-1{IOTF F{|v|^2}}) with
 * the same kernels, but keeps its scratch field and 1-D tables in fixed
 * file-scope device arrays of the library (about 16.2 MiB on every GPU where
 * the library's code is loaded, held until the process exits). It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   desc: as for pwf_plan_create (eta, gamma, alpha and flags are not used);
 *         the work is enqueued on desc->stream. Only the paper's forms are
 *         served: n_modes 0 or 1 (IOTF, or coherent when x_coh = y_coh = 0).
 *         A source-mode descriptor (n_modes 9 or 25) returns
 *         PWF_ERR_UNSUPPORTED, any other n_modes PWF_ERR_INVALID_ARG, both
 *         before any work.
 *   psi, t, f: as for pwf_forward (caller-owned device memory).
 * Limit: batch * ny * nx <= 2097152 (2^21) complex elements; larger problems
 * return PWF_ERR_UNSUPPORTED before any work. Other errors as pwf_forward.
 * The first call on a device does a one-time set-up on that device (resolves
 * the device addresses of the arrays, raises kernel shared-memory limits);
 * make that first call before any stream capture. Every call rewrites and
 * shares the same arrays, which keep the last call's contents; calls that
 * overlap on the GPU (for example on two streams at once) race on them. */
pwf_status pwf_forward_noalloc(const pwf_plan_desc* desc, const void* psi, const void* t, float* f);

/* Human-readable name of a status code (static storage). */
const char* pwf_status_string(pwf_status s);
/* Last error message recorded on the plan (static per plan; never NULL). */
const char* pwf_plan_last_error(const pwf_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* PWF_H */
