/*
 * pasfm.h -- C ABI of the B300 (sm_103a) differentiable acoustic radiation operator
 * of PA-SFM (tracker-free freehand 3D photoacoustic imaging).
 *
 * The operator (paper, Section 2 "Differentiable Acoustic Radiation", Eq. 1, and
 * Appendix A, Eq. gpu_forward_model with the uniform-spherical-source closed form):
 * every voxel i of a grid P_c is a uniform sphere of radius a0 and amplitude
 * p0_i; element j of frame f sits at x_fj = R_f e_j + t_f (the rigid model of
 * Stage 4).  Seen from x_fj at distance d = |x_fj - r_i| the voxel radiates the
 * N-shaped pulse p0_i (d - c t) / (2 d) for |c t - d| <= a0.  Sample n of a trace
 * is that pulse averaged over the sample interval [t_n - 1/(2 fs), t_n + 1/(2 fs)],
 * t_n = t0 + n / fs, so with h = c / fs, tau_n = c t_n and
 *     W(d, n) = (w_lo^2 - w_hi^2) / (4 d h),
 *     w_lo = clamp(tau_n - h/2 - d, -a0, a0),  w_hi = clamp(tau_n + h/2 - d, -a0, a0):
 * With kernel = PASFM_KERNEL_GAUSS the voxel instead radiates the outgoing
 * Gaussian pulse of Eq. 1 (Appendix A, far-field Gaussian source, kernel K_G):
 * p0_i (d - c t) / (2 d) exp(-(c t - d)^2 / (2 sigma^2)), cut to |c t - d| <= 4 sigma,
 * and its sample-interval average is, with E(w) = exp(-w^2 / (2 sigma^2)) and the
 * same clamped ends (support 4 sigma instead of a0),
 *     W(d, n) = sigma^2 (E(w_hi) - E(w_lo)) / (2 d h).
 * Everything below holds for either kernel.
 *   forward    s[f][j][n] = sum_i p0_i W(d_fji, n)
 *   adjoint    v_i        = sum_{f,j,n} g[f][j][n] W(d_fji, n)            (exact transpose)
 *   pose grad  G_fj = sum_i p0_i sum_n g[f][j][n] dW/dd (x_fj - r_i) / d,
 *              dL/dv_f = sum_j G_fj,  dL/dw_f = sum_j x_fj x G_fj
 *              for the left twist x -> Exp(w) x + v about the world origin.
 *
 * Conventions shared by every call
 *  - Units: mm, microseconds, MHz.  Voxel (ix, iy, iz) has centre
 *    (ox + dx ix, oy + dy iy, oz + dz iz); volumes are [nz][ny][nx], x fastest.
 *  - Signals are [F][E][Nt], samples fastest.  Element templates are double
 *    [E][3] in the array frame; poses are double [F][3][4] = [R | t], row-major.
 *  - Every array argument is caller-owned DEVICE memory on the context's device,
 *    unless stated otherwise.  Outputs are overwritten, never accumulated.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and never synchronise the host, except pasfm_status() and
 *    pasfm_timing_read().
 *  - Return value: PASFM_OK or a negative code; pasfm_last_error() gives a
 *    message for the calling thread.  Argument errors are detected on the host
 *    before any launch.  Geometry errors that depend on device data (an element
 *    within the pulse support of the voxel grid, a device wait that ran out) set the context's
 *    device status word; read it with pasfm_status().  Outputs of a call that
 *    set the status word are unspecified but every access stays in bounds.
 *  - A context owns its workspace and may be used by one host thread and one
 *    stream at a time; use one context per concurrently running stream.
 *  - The library allocates device memory only in pasfm_create(), pasfm_reserve()
 *    and, when the workspace must grow, in the first compute call for a larger
 *    geometry (call pasfm_reserve() first to keep compute calls allocation-free).
 */
#ifndef PASFM_H
#define PASFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PASFM_OK 0
#define PASFM_EINVAL (-1)       /* bad argument: NULL, negative size, non-positive scalar */
#define PASFM_ENOMEM (-2)       /* workspace allocation failed */
#define PASFM_ECUDA (-3)        /* a CUDA runtime call failed */
#define PASFM_ETIMEOUT (-4)     /* a bounded device wait ran out (from pasfm_status) */
#define PASFM_EDEVICE (-5)      /* device status word set: element inside the grid, etc. */
#define PASFM_EUNSUPPORTED (-6) /* geometry outside the compiled kernel range */

/* storage types of the volume and signal arrays */
#define PASFM_F32 0
#define PASFM_BF16 1
#define PASFM_F16 2

/* voxel pulse (pasfm_geom.kernel) */
#define PASFM_KERNEL_SPHERE 0 /* uniform sphere of radius a0 (Appendix A closed form)          */
#define PASFM_KERNEL_GAUSS 1  /* Gaussian of width sigma_mm (Eq. 1, kernel K_G), support 4 sigma */

/* device status word bits (pasfm_status) */
#define PASFM_STATUS_ELEMENT_INSIDE 1u /* an element lies within the pulse support of the voxel grid */
#define PASFM_STATUS_TIMEOUT 2u        /* a bounded shared-memory barrier wait expired */
#define PASFM_STATUS_INDEX_CLAMPED 4u  /* a sample index fell outside its window (clamped) */

/* Acquisition geometry: the problem statement of the paper's Eq. 1 (voxel grid
 * P_c in R^{Nx x Ny x Nz}, sensor positions x_s, time-resolved signals) plus
 * the sampling of the time axis.  Host memory; read during the call only. */
typedef struct pasfm_geom {
  int32_t nx, ny, nz;                  /* voxel grid, x fastest                       */
  int32_t n_elem, n_frames, n_samples; /* E elements, F frames, Nt samples per trace   */
  double dx, dy, dz;                   /* voxel spacing (mm), > 0                      */
  double ox, oy, oz;                   /* centre of voxel (0,0,0) (mm)                 */
  double fs_mhz;                       /* sampling rate (MHz), > 0                     */
  double t0_us;                        /* time of sample 0 (us); t_n = t0 + n / fs     */
  double c_mm_per_us;                  /* speed of sound (mm/us), > 0                  */
  double a0_mm;                        /* voxel sphere radius (mm); <= 0 means min(d)/2 */
  int32_t dtype_vol;                   /* PASFM_F32 | PASFM_BF16 | PASFM_F16 (p0)       */
  int32_t dtype_sig;                   /* PASFM_F32 | PASFM_BF16 | PASFM_F16 (meas, g)  */
  int32_t kernel;                      /* PASFM_KERNEL_SPHERE (0) | PASFM_KERNEL_GAUSS  */
  int32_t reserved;                    /* must be 0                                     */
  double sigma_mm;                     /* Gaussian width (mm), > 0 for PASFM_KERNEL_GAUSS;
                                          a pair then spans floor(8 sigma / h) + 2 <= 32
                                          samples (sigma <= 0.14 mm at h = 0.0375 mm);
                                          the sphere allows floor(2 a0 / h) + 2 <= 16   */
} pasfm_geom;

typedef struct pasfm_ctx pasfm_ctx;

/* Adam state for pasfm_step (paper: Adam for the Eq. 2 objective, Stage 1/5,
 * and gradient steps on the rigid parameters, Stage 4).  Moment arrays are
 * caller-owned device memory, zero before the first step. */
typedef struct pasfm_adam {
  float* m_vol;    /* [Nvox] first moment of the volume                          */
  float* v_vol;    /* [Nvox] second moment of the volume                         */
  double* m_pose;  /* [F][6] first moment of the frame twists (w, v)             */
  double* v_pose;  /* [F][6] second moment of the frame twists                   */
  int64_t step;    /* completed steps; pasfm_step uses step + 1 and increments it */
  double lr_vol, lr_rot, lr_trans; /* learning rates (rad for w, mm for v)       */
  double beta1, beta2, eps;
  uint32_t flags;  /* PASFM_ADAM_* bits                                          */
  uint32_t reserved;
} pasfm_adam;

#define PASFM_ADAM_NONNEG 1u        /* project p0 onto p0 >= 0 after the update      */
#define PASFM_ADAM_FIX_FRAME0 2u    /* frame 0 is the gauge (known pose): not moved  */
#define PASFM_ADAM_FREEZE_POSES 4u  /* no pose update (pure volume reconstruction)  */
#define PASFM_ADAM_FREEZE_VOLUME 8u /* no volume update (pure pose refinement)      */

/* Create a context on CUDA device `device` (allocates its status word).
 * *out receives the context; returns PASFM_ECUDA if the device is unusable. */
int pasfm_create(pasfm_ctx** out, int device);

/* Free the context and its workspace.  NULL is accepted. */
int pasfm_destroy(pasfm_ctx* ctx);

/* Bound, in SM clock cycles, of the kernels' wait for each copy they stage with
 * TMA (default 2e9, about 1 s; a negative value restores it).  A wait that runs
 * out sets PASFM_STATUS_TIMEOUT, the kernel skips its compute, lets its copies in
 * flight land (waiting for them with the default bound) and exits; pasfm_status()
 * then returns PASFM_ETIMEOUT and the outputs are unspecified.  0 makes every such
 * wait report the timeout at once: a deterministic way to exercise that error
 * path.  Calls that stage nothing with TMA (unaligned or 16-bit arrays) have no
 * such wait.  Takes effect for later calls on the context. */
int pasfm_set_wait_limit(pasfm_ctx* ctx, int64_t cycles);

/* Device bytes of workspace the calls need for `geom` (host-only, no CUDA call). */
int pasfm_workspace_size(const pasfm_geom* geom, size_t* bytes);

/* Grow the context's workspace to fit `geom` now, so later calls do not allocate. */
int pasfm_reserve(pasfm_ctx* ctx, const pasfm_geom* geom);

/* Cap the bytes used for per-cube partial results (default 4 GiB); larger
 * problems are processed in frame chunks.  0 restores the default. */
int pasfm_set_partial_budget(pasfm_ctx* ctx, size_t bytes);

/* A1 -- element world positions x_fj = R_f e_j + t_f (Stage 4 rigid model).
 * elem: double [E][3]; pose: double [F][3][4]; xw_out: double [F][E][3].
 * Also checks every x_fj against the grid (status bit ELEMENT_INSIDE). */
int pasfm_element_positions(pasfm_ctx* ctx, const pasfm_geom* geom, const double* elem,
                            const double* pose, double* xw_out, void* stream);

/* A2 -- forward radiation s = A(p0; poses) (Eq. 1 / Eq. gpu_forward_model).
 * p0: [nz][ny][nx] of dtype_vol; sig_out: float [F][E][Nt]. */
int pasfm_forward(pasfm_ctx* ctx, const pasfm_geom* geom, const void* p0, const double* elem,
                  const double* pose, float* sig_out, void* stream);

/* A4 -- adjoint v = A^T g (the gradient with respect to P_c, Section 2).
 * g: [F][E][Nt] of dtype_sig; vol_out: float [nz][ny][nx]. */
int pasfm_adjoint(pasfm_ctx* ctx, const pasfm_geom* geom, const double* elem, const double* pose,
                  const void* g, float* vol_out, void* stream);

/* A5 -- pose gradient (gradient with respect to the sensor coordinates x_s,
 * Section 2, carried to the per-frame rigid parameters of Stage 4).
 * g: [F][E][Nt] of dtype_sig; mask: uint8 [F][E] or NULL (0 drops a trace,
 * the inlier mask of Eq. 4); grad6_out: double [F][6] ordered (w, v);
 * gelem_out: double [F][E][3] element-position gradients, or NULL. */
int pasfm_pose_grad(pasfm_ctx* ctx, const pasfm_geom* geom, const void* p0, const double* elem,
                    const double* pose, const void* g, const uint8_t* mask, double* grad6_out,
                    double* gelem_out, void* stream);

/* A3 -- loss head of the Eq. 2 data term: g = mask (s - S), L = 1/2 sum g^2.
 * sig: float [F][E][Nt]; meas: [F][E][Nt] of dtype_sig; mask: uint8 [F][E] or
 * NULL; g_out: float [F][E][Nt] (may alias sig); loss_out: one device double. */
int pasfm_loss(pasfm_ctx* ctx, const pasfm_geom* geom, const float* sig, const void* meas,
               const uint8_t* mask, float* g_out, double* loss_out, void* stream);

/* A6 -- one gradient step of L = 1/2 |mask (A(p0; poses) - S)|^2 jointly in p0
 * and the frame twists (Algorithm 1, Stage 1 / 4 / 5 updates): forward, loss
 * head, adjoint and pose gradient, then Adam on p0 and on the twists with a
 * left retraction R <- Exp(dw) R, t <- Exp(dw) t + dv.
 * p0 (dtype_vol) and pose are updated in place; elem, meas (dtype_sig) and
 * mask (or NULL) are read; state->step is incremented on the host.
 * loss_out: device double receiving L at the pre-update point, or NULL. */
int pasfm_step(pasfm_ctx* ctx, const pasfm_geom* geom, void* p0, double* pose, const double* elem,
               const void* meas, const uint8_t* mask, pasfm_adam* state, double* loss_out,
               void* stream);

/* A10 -- one gradient step (pasfm_step's semantics and results) for each of n
 * resident scans, issued on one stream as batched launches: the scans whose hot
 * kernels share an instantiation and pulse profile (pulse, slot count, cube and
 * window size, sampling, wait bound; at most 16 per launch) have their forward, its
 * reduction and their fused adjoint / pose gradient each run as ONE persistent launch
 * per frame-chunk round, whose CTAs take (scan, cube, frame, element group) and
 * (scan, cube, part) tiles from a shared list until it is exhausted.  Each scan's
 * tiles are exactly those of its own pasfm_step, so its results are bit-identical
 * alone, in any mix and to pasfm_step.  The small per-scan kernels (element
 * positions, loss sum, part sums, element-gradient sums, Adam) are launched per scan.
 *   ctxs[i]: a distinct context per scan (its workspace), all on one device;
 *   geoms[i], p0[i], pose[i], elem[i], meas[i], mask[i] (mask may be NULL, or mask[i]
 *   NULL), states[i], loss_out[i] (loss_out may be NULL, or loss_out[i] NULL): as for
 *   pasfm_step, per scan.  Host arrays of n entries; each scan's arrays are device
 *   memory as for pasfm_step.
 *   trace_ns: device uint64 [n][2] or NULL; receives per scan the globaltimer
 *   (ns) at its first batched tile's start and its last batched tile's end over the
 *   forward and backward launches (how the scans' work overlapped on the device).
 * n = 0 is a no-op.  Each context's status word receives its own scan's errors. */
int pasfm_step_batch(int n, pasfm_ctx* const* ctxs, const pasfm_geom* geoms, void* const* p0, double* const* pose,
                     const double* const* elem, const void* const* meas, const uint8_t* const* mask,
                     pasfm_adam* states, double* const* loss_out, uint64_t* trace_ns, void* stream);

/* F3 -- smoothed second-order total generalized variation of the volume, the
 * regulariser of Stages 1 and 5 (Eq. 2, lambda L_TGV; lambda folded into the
 * weights):
 *   J(u, w) = sum_i alpha1 sqrt(|D u - w|^2 + eps^2) + alpha0 sqrt(|E(w)|_F^2 + eps^2),
 *   E(w)_ab = (D_a w_b + D_b w_a) / 2,
 * D_a the forward difference along axis a divided by the spacing, zero on the
 * last index; w = (w_x, w_y, w_z) an auxiliary vector field optimised with u.
 * u = p0 [nz][ny][nx] of dtype_vol; w, grad_w: float [3][nz][ny][nx];
 * grad_u: float [nz][ny][nx], dJ/du is added to it when accumulate != 0, else
 * written; grad_w receives dJ/dw; energy_out: one device double, or NULL.
 * alpha1, alpha0 >= 0, eps > 0 (units of u per mm). */
int pasfm_tgv_grad(pasfm_ctx* ctx, const pasfm_geom* geom, const void* p0, const float* w, double alpha1,
                   double alpha0, double eps, float* grad_u, int accumulate, float* grad_w, double* energy_out,
                   void* stream);

/* TGV state for pasfm_step_tgv: the auxiliary field and its Adam moments
 * (caller-owned device memory, [3][nz][ny][nx] floats each, moments zero before
 * the first step), the weights and the learning rate of w. */
typedef struct pasfm_tgv {
  float* w;
  float* m_w;
  float* v_w;
  double alpha1, alpha0, eps;
  double lr_w;
} pasfm_tgv;

/* pasfm_step with the TGV term added to the objective (Stages 1 and 5):
 * L + J(p0, w).  The TGV gradient is added to the volume gradient before the
 * Adam update of p0; w takes its own Adam step (same betas, eps and step count
 * as `state`).  tgv NULL is pasfm_step.  tgv_out: device double receiving J at
 * the pre-update point, or NULL.  Needs p0 updates (no PASFM_ADAM_FREEZE_VOLUME). */
int pasfm_step_tgv(pasfm_ctx* ctx, const pasfm_geom* geom, void* p0, double* pose, const double* elem,
                   const void* meas, const uint8_t* mask, pasfm_adam* state, const pasfm_tgv* tgv,
                   double* loss_out, double* tgv_out, void* stream);

/* A7 support -- twist coordinates for autograd (Stage 4 rigid parameters read
 * as an se(3) left twist xi = (w, v) on top of a base pose).
 * pasfm_apply_twists: pose_out[f] = (Exp(w_f) R_f, Exp(w_f) t_f + v_f).
 * pasfm_twist_grad: chain rule from grad6 (pasfm_pose_grad at the twisted pose)
 * to xi: dL/dv = g_v, dL/dw = J_l(w)^T (g_w - v x g_v), J_l the left Jacobian
 * of SO(3).  pose, pose_out: double [F][3][4]; xi, grad6, grad_xi_out: double
 * [F][6]; all device memory. */
int pasfm_apply_twists(pasfm_ctx* ctx, int n_frames, const double* pose, const double* xi, double* pose_out,
                       void* stream);
int pasfm_twist_grad(pasfm_ctx* ctx, int n_frames, const double* xi, const double* grad6, double* grad_xi_out,
                     void* stream);

/* A8 support -- trilinear resampling of a float volume between two voxel
 * grids (coarse-to-fine level change of the volume estimate).  Only the grid
 * fields of the two geometries are used; destination voxel centres outside the
 * source's outermost centres take the clamped (edge) value.  src: float
 * [sz][sy][sx], dst: float [nz][ny][nx], device memory, must not overlap. */
int pasfm_resample(pasfm_ctx* ctx, const pasfm_geom* src_geom, const float* src, const pasfm_geom* dst_geom,
                   float* dst, void* stream);

/* A8 support -- Gaussian low-pass of every trace along time, optionally
 * decimated: the coarse levels of the coarse-to-fine optimiser fit their wider
 * pulses to band-limited data (the data-side counterpart of the paper's
 * decaying kernel width, Stage 2), on a time grid `decim` times coarser.
 * dst[r][m] = sum_k w_k src[r][m decim + k], |k| <= int(4 sigma + 0.5), w_k ~
 * exp(-k^2 / (2 sigma^2)) normalised to sum 1, zero outside the record (sigma
 * in input samples; sigma <= 0 takes the samples as they are).
 * src: float [n_rows][n_samples], dst: float [n_rows][ceil(n_samples / decim)],
 * device memory; dst may alias src only when decim == 1.  decim >= 1.
 * Synchronises `stream` before returning. */
int pasfm_lowpass(pasfm_ctx* ctx, int64_t n_rows, int n_samples, double sigma, int decim, const float* src,
                  float* dst, void* stream);

/* NC loss of Eq. 3 as a score for candidate poses (the coarse search of Stage
 * 2): for each of n_cand candidate trace sets sim[k] ([n_elem][n_samples] float)
 * against one frame's measured traces meas ([n_elem][n_samples] of dtype_meas),
 * scores_out[k] = mean over elements j with mask[j] != 0 (mask may be NULL) of
 * -Cov(sim_kj, meas_j) / (sigma(sim_kj) sigma(meas_j)); a trace with zero
 * variance scores 0.  Lower is better.  Device memory; scores_out: double [n_cand]. */
int pasfm_nc_scores(pasfm_ctx* ctx, int n_cand, int n_elem, int n_samples, const float* sim, const void* meas,
                    int dtype_meas, const uint8_t* mask, double* scores_out, void* stream);

/* Stages 2 and 4 support -- gradient of the NC loss of Eq. 3 summed over traces:
 * g_out[r][n] = scale * d(sum_r mask[r] NC(sim_r, meas_{r / meas_repeat})) / d sim[r][n],
 * with NC = -<s~, m~> / (|s~| |m~|) on the centred traces s~, m~, and nc_out[r] = NC
 * (0 for masked traces and traces of zero variance, whose gradient is 0).  Each
 * measured trace serves meas_repeat consecutive simulated ones (candidates of one
 * element).  Fed to pasfm_pose_grad as its residual, g gives the element-position
 * and rigid gradients of the NC loss.  sim, g_out: float [n_rows][n_samples]
 * (g_out may alias sim); meas: [n_rows / meas_repeat][n_samples] of dtype_meas;
 * mask: uint8 [n_rows] or NULL; nc_out: double [n_rows] or NULL.  Device memory. */
int pasfm_nc_grad(pasfm_ctx* ctx, int64_t n_rows, int n_samples, const float* sim, const void* meas, int dtype_meas,
                  int meas_repeat, const uint8_t* mask, double scale, float* g_out, double* nc_out, void* stream);

/* A8 support -- x *= alpha over n floats (rescaling a volume estimate when the
 * Gaussian width or the grid spacing changes).  Device memory. */
int pasfm_scale(pasfm_ctx* ctx, int64_t n, double alpha, float* x, void* stream);

/* Measurement aid, no counterpart in the paper -- FMA throughput of `device` in
 * TFLOP/s (an FMA counts 2 flops): independent FMA chains on every SM, scalar FP32
 * (packed = 0), Blackwell's packed two-wide FP32 FMA on float2 (packed = 1), or the
 * packed half-precision FMA on half2 (packed = 2) or bfloat162 (packed = 3); other
 * values return PASFM_EINVAL.  Allocates
 * and frees 4 bytes of device memory, runs on the default stream and synchronises,
 * about 10 ms; not for use while other work runs on the device.  tflops_out: host. */
int pasfm_fp32_probe(int device, int packed, double* tflops_out);

/* Measurement aid, no counterpart in the paper -- shared-memory read-modify-write
 * throughput of `device` in TB/s, for the access pattern of the forward's window
 * (each thread adds into its own column of a [slot][thread] array: one conflict-free
 * 128-byte wavefront per warp load or store).  Same conditions as pasfm_fp32_probe. */
int pasfm_smem_probe(int device, double* tbs_out);

/* Allocation-free pose gradient.  No counterpart in the paper: this is a
 * library service for callers that must not allocate device memory while they
 * run -- code hosted inside an application that owns all device memory through
 * its own pool, or a real-time loop that cannot afford the latency and implicit
 * synchronisation of cudaMalloc/cudaFree.  It computes what pasfm_pose_grad
 * computes (same arguments minus the context, same kernels; the same results
 * within the pose-gradient tolerance, since for the sphere the backward here reads
 * g itself where pasfm_pose_grad stages its first differences) but
 * keeps all of its scratch in one fixed array of PASFM_NOALLOC_SCRATCH_BYTES
 * that the library declares at file scope in device memory; every GPU that
 * loads the library holds that array until the process exits.  It calls no
 * allocation routine.
 *  - Needs F*E*(48 + 24*ncubes) + 256 bytes of scratch (24 fewer per trace when
 *    gelem_out is given), ncubes = number of 16^3 (or 8^3 on coarse grids) voxel
 *    cubes; larger problems return PASFM_EUNSUPPORTED with a message.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one array, which keeps what the last call left in it;
 *    calls whose work overlaps on the GPU (other streams, other host threads)
 *    race on it.  Serialise them.
 *  - There is no context status word.  A device-side failure (an element
 *    within the pulse support of the grid, a staged-copy wait that ran out, a
 *    clamped sample index) is reported by filling grad6_out, and gelem_out when
 *    given, with NaN; the return value is still PASFM_OK.  Accesses stay in
 *    bounds either way. */
#define PASFM_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int pasfm_pose_grad_noalloc(const pasfm_geom* geom, const void* p0, const double* elem, const double* pose,
                            const void* g, const uint8_t* mask, double* grad6_out, double* gelem_out,
                            void* stream);

/* Synchronise `stream` and read (then clear) the context's device status word.
 * *bits receives the PASFM_STATUS_* bits seen (may be NULL).  Returns
 * PASFM_OK, PASFM_ETIMEOUT or PASFM_EDEVICE. */
int pasfm_status(pasfm_ctx* ctx, void* stream, uint32_t* bits);

/* Per-kernel timing with CUDA events recorded around every launch of this
 * context (off by default).  pasfm_timing_read() synchronises the recorded
 * events and returns the summed milliseconds and launch count of kernels whose
 * name is `kernel` ("fwd_cube", "fwd_reduce", "bwd_cube", ... or "*" for all). */
int pasfm_timing_enable(pasfm_ctx* ctx, int enable);
int pasfm_timing_reset(pasfm_ctx* ctx);
int pasfm_timing_read(pasfm_ctx* ctx, const char* kernel, double* ms_total, int64_t* launches);

/* Number of kernels this context launched since creation (all calls). */
int64_t pasfm_launch_count(pasfm_ctx* ctx);

/* Message describing the last error on the calling thread ("" if none). */
const char* pasfm_last_error(void);

/* ABI version of this header (incremented on any signature change). */
int pasfm_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PASFM_H */
