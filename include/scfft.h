/*
 * scfft.h - C ABI of the GB300 (sm_103a) implementation of the method-of-lines
 * right-hand side of the FFT-based 3D bulk-magnetization method of
 * Prigozhin & Sokolovsky ("3D simulation of superconducting magnetic shields
 * and lenses using the fast Fourier transform", §2, Eqs. 1-8), and of its
 * time integrator.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid (§2, "uniform Nx x Ny x Nz grid" on D = {|x|<=Lx, |y|<=Ly, |z|<=Lz}):
 *   nodes are cell centres x_i = -Lx + (i + 1/2) dx, dx = 2 Lx / Nx; every
 *   N_a is even and 16 <= N_a <= 128 with N_a = 2^p 3^q (16, 32, 48, 64, 96, 128).
 * Vector fields: double arrays of 3*N entries, N = Nx*Ny*Nz, laid out
 *   [component x,y,z][z][y][x] (x fastest).  Scalar node fields: N entries
 *   [z][y][x].
 * Units: the dimensionless variables of Eq. 8 (e0 = jc = mu0 = 1 by default).
 * Memory: pointers documented "device" are CUDA device pointers owned by the
 *   caller (the library never frees them); "host" pointers are read during the
 *   call only.  Every device-side call is asynchronous on the context's CUDA
 *   stream unless stated otherwise.
 * Errors: invalid arguments are rejected on the host before any work is
 *   queued (SCFFT_EINVAL, nothing changed).  CUDA failures return SCFFT_ECUDA.
 *   No entry point aborts or throws.
 */
#ifndef SCFFT_H
#define SCFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scfft_ctx scfft_ctx; /* opaque; owns every internal workspace */

typedef enum {
  SCFFT_OK = 0,
  SCFFT_EINVAL = 1,    /* bad argument or unsupported size */
  SCFFT_ENOMEM = 2,    /* device or host allocation failed */
  SCFFT_ECUDA = 3,     /* a CUDA runtime call failed */
  SCFFT_ENOCONV = 4,   /* Eq. 5 iteration stopped at max_iter (result still written) */
  SCFFT_ESTEP = 5,     /* integrator step size fell below its floor */
  SCFFT_ENONFINITE = 6,/* NaN/Inf met in a residual or error norm */
  SCFFT_ETIMEOUT = 7,  /* a bounded device wait gave up (latched; see scfft_inject_fault) */
  SCFFT_ESTATE = 8,    /* call out of order (e.g. rhs before precompute_kernel) */
  SCFFT_ESIZE = 9      /* problem larger than a fixed, preallocated maximum */
} scfft_status;

/* Arithmetic of the FFTs and pointwise steps.  The integrator state and its step control
 * are FP64 in every mode.
 *   SCFFT_PREC_F64   FP64 transforms; FP64 stage sums.
 *   SCFFT_PREC_F32   FP32 transforms and stages, FP64 state with compensated sums.
 *   SCFFT_PREC_DF64  double-float transforms (each value an unevaluated sum of two FP32
 *                    numbers, a 48-bit significand, FP32's exponent range: FP64-equivalent
 *                    accuracy on the FP32 pipes); the node-wise law in FP64; FP64 stage sums.
 *                    Its buffers, entry points and results are those of SCFFT_PREC_F64. */
#define SCFFT_PREC_F64 0
#define SCFFT_PREC_F32 1
#define SCFFT_PREC_DF64 2

typedef struct {
  int nx, ny, nz;      /* nodes per axis */
  double Lx, Ly, Lz;   /* half extents of the box D */
} scfft_grid;

/* Eq. 1: rho(|j|) = (e0/jc) |j/jc|^(n-1) in Omega; rho_out in Omega_out (§2). */
typedef struct {
  double n, e0, jc, rho_out, mu0;
} scfft_material;

typedef struct {
  int precision;       /* SCFFT_PREC_F64, SCFFT_PREC_F32 or SCFFT_PREC_DF64 */
  double delta_it;     /* Eq. 5 stop tolerance (§2 uses 2e-5); 0 = never stop early */
  int max_iter;        /* iteration cap of Eq. 5 (>= 0) */
  double sigma_scale;  /* multiplies sigma = half the cell diagonal (§2); 1 = paper */
  double rtol, atol;   /* integrator tolerances (§2 uses rtol 2e-4) */
} scfft_options;

/* Applied field h_e(t) (§3): piecewise-linear through (t[k], he[3k..3k+2]),
 * constant outside [t[0], t[nknots-1]], plus
 * sin_amp * sin(2 pi (t - sin_t0) / sin_period) * sin_dir for sin_t0 <= t < sin_t1. */
typedef struct {
  int nknots;          /* 1..64 */
  const double* t;     /* host, nknots, strictly increasing */
  const double* he;    /* host, 3*nknots */
  double sin_amp, sin_period, sin_t0, sin_t1;
  double sin_dir[3];
} scfft_field_path;

typedef struct {
  long long launches;      /* CUDA kernels launched by the library */
  long long rhs_calls;     /* right-hand-side evaluations */
  long long iterations;    /* Eq. 5 iterations summed over those calls */
  long long accepted, rejected;
  int last_iters;          /* iterations of the most recent rhs */
  double last_residual;    /* its final Eq. 5 residual */
  double t, dt;            /* integrator time and proposed step */
  long long h2d_bytes;     /* host -> device bytes copied by scfft_step_host */
  long long d2h_bytes;     /* device -> host bytes copied by scfft_step_host */
} scfft_stats;

/* Create a context for one grid.  stream: a cudaStream_t (NULL = legacy
 * default stream).  Allocates every device workspace (sizes grow as
 * (3*N complex) * 8 words in FP64).  Errors: EINVAL for an unsupported grid,
 * nonpositive extents, n < 1, negative rho_out, max_iter < 0; ENOMEM. */
scfft_status scfft_create(const scfft_grid* grid, const scfft_material* mat, const scfft_options* opt,
                          void* stream, scfft_ctx** out);

/* Omega (§2): mask[N] (host, [z][y][x]), nonzero = node in the superconductor.
 * Copied to the device.  EINVAL if Omega is empty or touches the two outermost
 * node layers of any box face (the free-space Phi needs the margin). */
scfft_status scfft_set_geometry(scfft_ctx* ctx, const uint8_t* mask);

/* Per-node critical current density jc(x) (device, N doubles, > 0), or NULL
 * for the uniform material jc.  Copied (converted to the FFT precision). */
scfft_status scfft_set_jc_map(scfft_ctx* ctx, const double* jc_dev);

/* The discrete curl of the right-hand side (j = curl h of Eq. 4, -curl e of Eq. 3 and the
 * curl of dh^i in Eq. 5).  SCFFT_CURL_SPECTRAL (the default) takes the derivatives in Fourier
 * space with the Gaussian smoothing of §2 (the paper's choice).  SCFFT_CURL_FD is a local
 * alternative the paper does not use: second-order central differences on the periodic grid,
 * (f(i+1) - f(i-1)) / (2 d_a), no smoothing; the unpadded grid's FFT passes then drop out of
 * every rhs.  scfft_curl keeps the spectral curl either way.  The reverse mode covers the
 * spectral curl only (SCFFT_ESTATE otherwise).  EINVAL for another kind; ENOMEM if the
 * stencil's buffer (3N values) cannot be allocated.  Synchronises the stream. */
#define SCFFT_CURL_SPECTRAL 0
#define SCFFT_CURL_FD 1
scfft_status scfft_set_curl(scfft_ctx* ctx, int kind);

/* Launch schedule of the FP32 passes that carry the transforms of Eqs. 3-7: how the spectral
 * columns are tiled over CTAs and whether the padded y passes load through TMA.  A schedule
 * never changes the arithmetic of a column: every schedule gives the same results bit for
 * bit (x_update_split: see there), only their speed differs by grid size.
 *   z_kernel_tile    padded z pass with the Biot-Savart kernel product (Eq. 7): 4 or 8 columns
 *   z_curl_tile      z pass of the smoothed curl (Eq. 4): 8 or 16 columns
 *   y_unpadded_tile  y passes on the unpadded grid: 8 or 16 columns
 *   y_padded_tma     padded y passes: 1 = TMA-fed persistent kernel, 0 = plain loads
 *   z_kernel_tmem    padded z pass of a 256-point z transform (nz = 128): 1 = each thread keeps the
 *                    spectra of two components between the forward transforms, the product and
 *                    the inverse transforms in tensor memory, 0 = in shared memory; 2 = tensor
 *                    memory as in 1 with two shared-memory transpose buffers instead of three and
 *                    at most 80 registers per thread (six CTAs per SM instead of four), the
 *                    default where it exists; 0 on other grids
 *   box_fused        Eq. 5 iteration with the spectral curl: 1 = the curl's inverse y pass, the
 *                    mask/pad x pass and the padded forward y pass, which see only Omega's
 *                    bounding box, run as one launch with one CTA per (component, plane of the
 *                    box) and their intermediates in shared memory; 0 = three launches.  Applies
 *                    where nx = ny and the box's rows fit shared memory (the three passes run
 *                    otherwise)
 *   x_update_split   Eq. 5 update pass: 1 = the three components' transforms side by side in
 *                    three warp groups of a CTA (their input rows in flight at once), 0 = one
 *                    component after another.  The iterate and dh/dt are the same bits; the
 *                    residual's per-thread partial sums cover other nodes, so its last bits (and,
 *                    on an exact tie with the stop threshold, the iteration count) may differ
 *   us               scfft_autotune only: mean time (microseconds) of the candidates in the order
 *                    z_kernel 8, 4; z_curl 8, 16; y_unpadded 8, 16 (forward + inverse);
 *                    y_padded TMA, plain (forward + inverse); z_kernel_tmem 2, 1, 0; box_fused 0,
 *                    1 (the three passes, the fused pass); x_update_split 0, 1; 0 where not
 *                    timed. */
typedef struct {
  int z_kernel_tile;
  int z_curl_tile;
  int y_unpadded_tile;
  int y_padded_tma;
  int z_kernel_tmem;
  int box_fused;
  int x_update_split;
  double us[15];
} scfft_schedule;

/* Autotuner of the schedule: times each candidate of each knob on the context's own workspace
 * (ten launches each after three, CUDA events on its stream; the scratch spectra are
 * overwritten, no state is touched), keeps the fastest (an alternative to the first candidate
 * only when it is more than 3% faster), and caches the choice per device and grid for the
 * process, so that later contexts of that grid (a batch) reuse it without timing; retune != 0
 * times again.  Rebuilds the context's captured graphs on their next launch.  FP64 and
 * double-float contexts have no schedule: SCFFT_OK, nothing timed.  out (may be NULL)
 * receives the schedule in use.  Errors: SCFFT_EINVAL (NULL ctx), SCFFT_ECUDA. */
scfft_status scfft_autotune(scfft_ctx* ctx, int retune, scfft_schedule* out);
/* The schedule in use (out->us zero). */
scfft_status scfft_get_schedule(scfft_ctx* ctx, scfft_schedule* out);
/* Impose a schedule (FP32 contexts; SCFFT_EINVAL for a value outside the lists above, for
 * y_padded_tma = 1 without TMA descriptors, for z_kernel_tmem = 1 when nz != 128, or for
 * another precision). */
scfft_status scfft_set_schedule(scfft_ctx* ctx, const scfft_schedule* sched);

/* The e(j, h) law in Omega.  §2 (after Eq. 1) notes that another current-voltage relation,
 * e(j) or e(j, h) with h the local magnetic field, can replace the power law; two are
 * provided, alone or together:
 *   Kim's field-dependent critical current  jc(h) = jc / (1 + |h| / kim_h0)  (kim_h0 > 0;
 *     0 = jc independent of h), with |h| the state h at the node;
 *   an anisotropic power law  e = (e0/jc)(|j|_A / jc)^(n-1) A^2 j,  A = diag(aniso),
 *     |j|_A = |A j|, the gradient of the convex potential (e0 jc/(n+1)) (|j|_A / jc)^(n+1),
 *     so the critical current density along axis a is jc / aniso[a].
 * kim_h0 = 0 with aniso = (1, 1, 1) is Eq. 1 (the default).  EINVAL for kim_h0 < 0 or a
 * non-positive or non-finite aniso.  The reverse mode (scfft_rhs_vjp, scfft_adjoint_*)
 * covers Eq. 1 only and returns SCFFT_ESTATE while another law is set. */
typedef struct {
  double kim_h0;
  double aniso[3];
} scfft_ej_law;
scfft_status scfft_set_ej_law(scfft_ctx* ctx, const scfft_ej_law* law);

/* Applied-field path h_e(t); copied.  EINVAL on bad knots. */
scfft_status scfft_set_field_path(scfft_ctx* ctx, const scfft_field_path* path);

/* Sample grad G_sigma (G_sigma = G of Eq. 2 smoothed by a Gaussian of std sigma)
 * on the offsets of the zero-padded 2Nx x 2Ny x 2Nz grid, with the offset -N_a
 * planes zeroed so the kernel is odd (transform 0 at k = 0, the rule under
 * Eq. 7), and keep its purely imaginary transform on one octant.  Queued on
 * the stream; must precede rhs. */
scfft_status scfft_precompute_kernel(scfft_ctx* ctx);

/* One right-hand side dh/dt at time t (§2, Eqs. 1, 3, 4, 5):
 *   j = curl_S h; e = rho(|j|) j in Omega, rho_out j outside;
 *   dh_in = -curl_S e / mu0 on Omega; dh^0 = dh_in on Omega, warm on Omega_out;
 *   dh^{i+1} = dh^i on Omega, dh_e/dt + Phi[chi_Omega curl_S dh^i] on Omega_out,
 *   until mean_{Omega_out} |dh^{i+1} - dh^i| < delta_it max(|dh_e/dt|, 1) or max_iter.
 * left != 0 evaluates dh_e/dt as the left derivative at a kink of the path.
 * h, warm, hdot: device, 3*N doubles; warm is read (its Omega_out part is the
 * initial approximation of Eq. 5) and then overwritten with hdot.  hdot must
 * not alias h.  iters_out: host int* or NULL; if non-NULL the call waits for
 * the stream and stores the iteration count (and returns ENOCONV if the cap
 * stopped it); if NULL the call returns after queueing the work (the early
 * stop of Eq. 5 is decided on the device). */
scfft_status scfft_rhs(scfft_ctx* ctx, double t, int left, const double* h, double* warm, double* hdot,
                       int* iters_out);

/* Smoothed spectral curl alone (§2, derivatives of Eqs. 3-4): out = curl_S f.
 * f, out: device, 3*N doubles (may not alias).  Asynchronous. */
scfft_status scfft_curl(scfft_ctx* ctx, const double* f, double* out);

/* Biot-Savart operator alone (Eqs. 6-7 by zero padding): out = Phi_d[j] on the
 * grid, j taken as given (no mask).  j, out: device, 3*N doubles.  Asynchronous. */
scfft_status scfft_phi(scfft_ctx* ctx, const double* j, double* out);

/* Integrate dh/dt = rhs from t0 to t1 by the Bogacki-Shampine 3(2) FSAL pair
 * (the method of Matlab ode23 used in §2) with error norm
 * max_i |err_i| / max(rtol |y_i|, rtol |y_new,i|, atol), accept if <= 1,
 * dt <- dt min(5, max(0.2, 0.9 err^(-1/3))).  Steps end exactly on the
 * path's kinks, on each snapshot time and on t1.  dt0 > 0 is the first trial
 * step.  h: device, 3*N doubles, in: h(t0), out: h(t1).  tsnap: host, nsnap
 * increasing times in (t0, t1]; snaps: device, nsnap*3*N doubles (may be NULL
 * when nsnap = 0).  warm: device 3*N doubles, in/out warm start of Eq. 5
 * (NULL: dh_e/dt(t0) everywhere).  dt_fixed: host array of nfixed steps for
 * fixed-step mode (no error control), or NULL.  Synchronous: returns when
 * done.  stats: host or NULL. */
scfft_status scfft_integrate(scfft_ctx* ctx, double t0, double t1, double dt0, int nsnap, const double* tsnap,
                             double* h, double* snaps, double* warm, const double* dt_fixed, int nfixed,
                             scfft_stats* stats);

/* One accepted BS23 step (the pair and error control of scfft_integrate) from
 * *t with trial step *dt; rejected trials are retried with smaller steps.  The
 * step never passes tstop or a kink of the path and ends exactly on them when
 * clipped.  On return *t is the new time and *dt the proposed next step.
 * h, warm: device, 3*N doubles, in/out (state and Eq. 5 warm start).  The
 * first stage is reused from the previous accepted step when it was taken on
 * the same h and warm buffers and ended at *t (FSAL).  rejected: host int* or
 * NULL (rejected trials).  Synchronous (reads the error norm). */
scfft_status scfft_step(scfft_ctx* ctx, double* t, double* dt, double tstop, double* h, double* warm,
                        int* rejected);

/* Up to nsteps accepted BS23 steps (the pair, error control and kink handling of scfft_step,
 * the method of lines of §2) without the host between steps.  On the FP32 path the whole
 * sequence is one CUDA graph launch: a WHILE node over trials whose body computes on the
 * device the trial step, dh_e/dt and the Eq. 5 stop threshold at its stage times, the stage
 * states, the three stage right-hand sides (each with its Eq. 5 loop as a nested WHILE node),
 * the error norm and the step controller, and applies an accepted step.  The graph is built
 * on the first call for the buffers h, warm and rebuilt when they or a setting change.  The
 * call returns after nsteps accepted steps, or when t reaches tstop or the next kink of the
 * path (the step that reaches it ends there, as in scfft_step), whichever comes first.  On
 * the FP64 path, and while profiling, the host drives the same steps.  Results equal
 * scfft_step's up to the rounding of the device's cos and pow in the path rate and the step
 * controller.  h, warm: device, 3*N doubles, in/out; steps_done: host int* or NULL (accepted
 * steps taken).  Statuses as scfft_step.  Synchronous. */
scfft_status scfft_advance(scfft_ctx* ctx, double* t, double* dt, double tstop, int nsteps, double* h, double* warm,
                           int* steps_done);

/* scfft_step (one BS23 step of the method of lines of §2) with the state kept in host memory:
 * h_host, warm_host (host, 3*N doubles each,
 * in/out; page-locked memory makes the copies fast) are copied into h, warm (device, 3*N
 * doubles, caller-owned: the buffers scfft_step would take), the step runs on those, and the
 * new h and warm are copied back before the call returns.  h is copied in on every call; warm
 * only when the step reads it, i.e. always on the FP64 path and on the FP32 path unless the
 * step continues the context's own trajectory on these device buffers (FSAL, as in
 * scfft_step), whose warm start the context then holds itself.  The bytes copied are added to
 * scfft_stats.h2d_bytes / d2h_bytes.  warm_host may be NULL: the warm start then lives only
 * in the device buffer warm (a caller that continues its trajectory on this context, or that
 * has put a warm start into warm itself) and is copied in neither direction.  Statuses as
 * scfft_step; on an error nothing is copied back.  Synchronous. */
scfft_status scfft_step_host(scfft_ctx* ctx, double* t, double* dt, double tstop, double* h_host,
                             double* warm_host, double* h, double* warm, int* rejected);

/* Checkpoint and resume of a trajectory stepped with scfft_step (the method of lines of §2,
 * "ode23"; the paper itself does not describe checkpoints).  A checkpoint holds the time t and
 * proposed step dt, the state h and the Eq. 5 warm start (FP64), and the integrator state the
 * next step would reuse: the first-stage derivative (FSAL; FP64, or FP32 on the FP32 path) and,
 * on the FP32 path, the compensation terms of the accepted-state sums.  Resuming from it
 * continues the trajectory with the same results, bit for bit, as the uninterrupted run.
 *
 * scfft_checkpoint_save: h, warm: device, 3*N doubles, the buffers the trajectory was stepped
 * on (the FSAL stage is saved when the context's last accepted step was taken on them and ended
 * at t; otherwise the resumed step recomputes it, as the uninterrupted run would).  buf: host,
 * caller-owned; with buf = NULL only *size is set to the bytes needed; otherwise *size gives
 * buf's capacity (SCFFT_EINVAL if too small) and returns the bytes written.  Synchronises the
 * context's stream.
 *
 * scfft_checkpoint_load: buf/size as written by save for a context of the same grid and
 * precision (SCFFT_EINVAL otherwise).  Writes *t, *dt, and h, warm (device, 3*N doubles,
 * caller-owned); the next scfft_step(ctx, t, dt, .., h, warm, ..) continues the saved
 * trajectory.  Synchronous. */
scfft_status scfft_checkpoint_save(scfft_ctx* ctx, double t, double dt, const double* h, const double* warm,
                                   void* buf, size_t* size);
scfft_status scfft_checkpoint_load(scfft_ctx* ctx, const void* buf, size_t size, double* t, double* dt, double* h,
                                   double* warm);

/* Per-pass profiling: when enabled, every kernel the library launches is
 * bracketed by CUDA events on the context's stream and its elapsed time is
 * added to the counter of its pass kind.  Enabling resets the counters.
 * profile_read waits for the stream and fills counts[SCFFT_NKINDS] and
 * ms[SCFFT_NKINDS] (host arrays). */
enum {
  SCFFT_K_X_FWD = 0,       /* x pass: state rows -> R2C                          */
  SCFFT_K_X_POWERLAW = 1,  /* x pass: C2R, Eq. 1 / rho_out, R2C                   */
  SCFFT_K_X_ASSEMBLE = 2,  /* x pass: C2R, dh^0 assembly, R2C                     */
  SCFFT_K_X_MASKPAD = 3,   /* x pass: C2R, mask, zero pad, padded R2C             */
  SCFFT_K_X_UPDATE = 4,    /* x pass: padded C2R, Eq. 5 update + residual, R2C    */
  SCFFT_K_Y_FWD_U = 5,     /* y pass, unpadded, forward                           */
  SCFFT_K_Y_INV_U = 6,     /* y pass, unpadded, inverse                           */
  SCFFT_K_Z_CURL = 7,      /* z pass: forward, curl multiply, inverse             */
  SCFFT_K_Y_FWD_P = 8,     /* y pass, padded, forward (pruned input)              */
  SCFFT_K_Y_INV_P = 9,     /* y pass, padded, inverse (pruned output)             */
  SCFFT_K_Z_KERNEL = 10,   /* z pass, padded: forward, K^ x F (Eq. 7), inverse    */
  SCFFT_K_FINALIZE = 11,   /* dh/dt and warm start written out                    */
  SCFFT_K_RK = 12,         /* integrator stage sums and error norm                */
  SCFFT_K_OTHER = 13,      /* passes of scfft_curl / scfft_phi                    */
  SCFFT_K_BOX = 14,        /* fused on Omega's box: y inverse, mask/pad x, padded y forward */
  SCFFT_NKINDS = 15
};
scfft_status scfft_profile(scfft_ctx* ctx, int enable);
scfft_status scfft_profile_read(scfft_ctx* ctx, long long* counts, double* ms);
const char* scfft_kind_name(int kind);

/* Batched instances: advance nb independent contexts (one problem each: its own grid,
 * geometry, material, applied-field path) by one accepted BS23 step each, as scfft_step does.
 * When every context computes in FP32 (and none is profiling), one CUDA graph launch advances
 * them all: the graph holds each instance's trial loop (the device-resident step of
 * scfft_advance) as a WHILE node of its own, side by side, so the instances run concurrently
 * on the GPU with no host involvement between their kernels; the graph is kept and reused
 * while the batch (contexts, buffers, settings) stays the same.  Otherwise the contexts'
 * steps are driven from up to 64 host threads (give every context a distinct stream at
 * scfft_create so that the GPU overlaps them).  t, dt, tstop: host arrays of nb; h, warm: host
 * arrays of nb device pointers (3N_i doubles each).  status: host array of nb or NULL
 * (per-instance result).  Returns the first non-OK status (all instances are attempted).
 * Synchronous. */
scfft_status scfft_batch_step(scfft_ctx** ctxs, int nb, double* t, double* dt, const double* tstop, double** h,
                              double** warm, scfft_status* status);

/* Reverse-mode derivative (vector-Jacobian product) of the rhs map
 * F(h, warm, jc, dh_e/dt) = dh/dt of scfft_rhs taken with exactly max_iter
 * Eq. 5 iterations (no early stop; with a converged forward iteration this is
 * the derivative of the converged map up to the residual).  The map is the
 * chain of §2 (j = curl h, Eq. 1, Eq. 3, Eq. 5); its transpose runs the same
 * operators backwards: the iteration's transpose is chi + curl chi Phi (1-chi)
 * (the curl and Phi are symmetric), the power law's Jacobian is
 * rho (I + (n-1) jhat jhat^T) in Omega and rho_out outside.
 * h: device 3N (the point of linearisation), lam: device 3N (cotangent of
 * dh/dt).  Outputs: mu_h device 3N; mu_g device 3N or NULL (cotangent of the
 * warm start); mu_jc device N or NULL (cotangent of the per-node jc, 0 outside
 * Omega); mu_a host double[3] or NULL (cotangent of dh_e/dt, summed over
 * nodes).  The transposed passes run in FP64 or FP32 as the context's
 * precision.  Synchronous. */
scfft_status scfft_rhs_vjp(scfft_ctx* ctx, const double* h, const double* lam, double* mu_h, double* mu_g,
                           double* mu_jc, double* mu_a);

/* Discrete adjoint of the fixed-step BS23 map y_0 -> y_S over the whole run at once (built
 * on scfft_adjoint_record / scfft_adjoint_step below, with step times t0 + dts[0] + ... and
 * the first warm start dh_e/dt(t0)): steps dts[0..nsteps-1] (host), first stage
 * k1 = rhs(y_0), FSAL, each stage's warm start = the previous rhs result, every rhs taking
 * exactly max_iter Eq. 5 iterations (delta_it is ignored during the call), dh_e/dt taken at
 * the stage times (right derivative; a step whose end time equals a kink of the path ends
 * on it as in scfft_adjoint_record).  For J = <lam_T, y_S> it returns mu_y0 = dJ/dy_0
 * (device 3N), mu_jc = dJ/djc (device N or NULL), mu_a = dJ/d(dh_e/dt) summed over every
 * rhs call and the first warm start (host double[3] or NULL) and y_S (device 3N or NULL).
 * States are checkpointed every checkpoint_every steps in the forward sweep and each
 * segment is recomputed during the reverse sweep (memory: about
 * (16 + 2 nsteps/checkpoint_every + 2 checkpoint_every) * 3N doubles, allocated and freed
 * by the call; it also drops any recording of scfft_adjoint_record).  y0, lam_T: device 3N.
 * Synchronous. */
scfft_status scfft_adjoint_integrate(scfft_ctx* ctx, double t0, const double* dts, int nsteps, const double* y0,
                                     const double* lam_T, double* y_end, double* mu_y0, double* mu_jc,
                                     double* mu_a, int checkpoint_every);

/* Reverse mode step by step over a recorded trajectory of the method of lines (§2, "ode23";
 * the paper has no reverse mode): the map is the fixed-step BS23 map of scfft_integrate's
 * fixed-step mode over the given step times, with every rhs taking exactly max_iter Eq. 5
 * iterations (delta_it is ignored during these calls) and the warm-start chain of the
 * forward run (each rhs starts Eq. 5 from the previous rhs result).  A step that ends on a
 * kink of the applied-field path takes its last stage with the left derivative of h_e there
 * and the next step restarts its first stage with the right one, as scfft_step does, so the
 * recorded map reproduces an adaptive run from its accepted step times.
 *
 * scfft_adjoint_record: runs the forward map from y0 (device 3N) at t = ts[0] through the step
 * times ts[0..nsteps] (host, increasing; the accepted step end times of a scfft_step run end
 * exactly on the path's kinks, and a step whose end time equals a kink is treated as ending
 * on it).  warm0: device 3N first warm start, or NULL for dh_e/dt(ts[0]) at every node.  The
 * states (y_n, first stage k1_n) are checkpointed every checkpoint_every steps; y_end (device
 * 3N or NULL) receives y at ts[nsteps].  The context keeps the recording (about
 * (16 + 2 nsteps/checkpoint_every + 2 checkpoint_every) * 3N doubles of device memory,
 * allocated here) until the next record or scfft_destroy.  Synchronous.
 *
 * scfft_adjoint_step: the reverse of step n = step_index; call it for n = nsteps-1, nsteps-2,
 * ..., 0 in this order (SCFFT_ESTATE otherwise).  lambda_h (device 3N, in/out): on entry the
 * cotangent of y_{n+1} (the caller may add dJ/dy_{n+1} of an objective between calls), on
 * return that of y_n; after step 0 it is the full dJ/dy_0.  The recomputation of a checkpoint
 * segment happens in the call that enters it.  grad_jc: device N doubles or NULL, += dJ/djc
 * (per node) over this step's rhs calls.  grad_path: host, 3*nknots + 1 doubles or NULL,
 * += dJ/d(path parameters): entries 3k..3k+2 the knot amplitudes he[3k..3k+2] of
 * scfft_field_path (they enter through the rates dh_e/dt of the linear pieces), entry 3*nknots
 * the sine amplitude sin_amp; step 0 also adds the cotangent of the default first warm start
 * dh_e/dt(ts[0]) (not that of an explicit warm0).  Synchronous. */
scfft_status scfft_adjoint_record(scfft_ctx* ctx, const double* ts, int nsteps, const double* y0, const double* warm0,
                                  int checkpoint_every, double* y_end);
scfft_status scfft_adjoint_step(scfft_ctx* ctx, int step_index, double* lambda_h, double* grad_jc, double* grad_path);

/* Allocation-free spectral curl: out = curl_S f, the same result as
 * scfft_curl (FP64) on the same grid and sigma_scale, for callers that cannot
 * allocate device memory when they need it (inside a region where cudaMalloc
 * is forbidden or unsafe, under a fixed memory budget, or under a host
 * framework that owns every allocation).  This entry point has no counterpart
 * in the paper; it only repackages the curl.
 * It needs no context: grid (host) gives the sizes and half extents;
 * stream is a cudaStream_t (NULL = legacy default stream) of the current
 * device (SCFFT_EINVAL if it belongs to another device); f, out: device,
 * 3*N doubles, not aliased; sigma_scale finite and >= 0.  Its scratch is one
 * static 8 MiB device array per GPU (grids up to 64^3 nodes fit); larger grids
 * return SCFFT_ESIZE and nothing is queued.  It calls no allocator.  Every call
 * made outside a stream capture looks up that array's device address on the
 * current device (so a device reset between calls is harmless); a call made
 * while the stream is capturing reuses the address found by an earlier call on
 * that device, and returns SCFFT_ESTATE if there was none: make the first call
 * on a device before any stream capture.  Calls share the array: calls that
 * overlap on the GPU (other streams or host threads on the same device) race
 * and must be serialized.  SCFFT_ECUDA leaves its cause in
 * scfft_last_cuda_error().  Asynchronous on stream. */
scfft_status scfft_curl_noalloc(const scfft_grid* grid, double sigma_scale, const double* f, double* out,
                                void* stream);

/* Wait for the stream; returns the first latched device-side status. */
scfft_status scfft_sync(scfft_ctx* ctx);

/* Fault injection for tests of the device-side timeout path; the paper has no counterpart.
 * kind = SCFFT_FAULT_TMA_WAIT arms a one-shot fault for an FP32 context: the next TMA-fed
 * padded y pass launched directly by the library (scfft_phi, or an rhs while profiling; not
 * the Eq. 5 loop graph, whose launches were captured before) makes the first stage buffer of
 * every CTA expect 16 bytes more than its copy brings, so that bounded wait gives up after
 * about a second.  The pass then latches SCFFT_ETIMEOUT in the context (scfft_sync and later
 * calls return it) and its output is not valid; no trap is raised, and the GPU and the other
 * contexts stay usable.  kind = 0 disarms.  Returns SCFFT_EINVAL for an unknown kind or an
 * FP64 context. */
#define SCFFT_FAULT_TMA_WAIT 1
scfft_status scfft_inject_fault(scfft_ctx* ctx, int kind);

/* Counters since create (host copy). */
scfft_status scfft_get_stats(scfft_ctx* ctx, scfft_stats* out);

const char* scfft_status_string(scfft_status s);

/* Text of the CUDA error behind the most recent SCFFT_ECUDA returned by any
 * entry point in this process ("" if none); for diagnostics. */
const char* scfft_last_cuda_error(void);

/* Free every workspace.  NULL is a no-op. */
void scfft_destroy(scfft_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SCFFT_H */
