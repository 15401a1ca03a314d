/*
 * fwi.h -- C ABI of the B300 time-domain FWI hot path.
 *
 * The library computes, for a 3D sound-speed model c0 on a regular grid, the
 * paper's time-reversal based misfit gradient (Alg. 1, App. B): a forward
 * k-space pseudospectral simulation of the lossless split-density acoustic
 * system (first-order system of Sec. 2.1 with the k-space derivative of
 * Eqs. 18-19 and PML multipliers), a time-reversed re-simulation of the forward
 * field driven by its trace on a boundary layer of Gamma (Eq. 11, Sec. 3.1),
 * and an adjoint simulation driven by the time-integrated residual; the product
 * 2/(dt c0^3) (p+ - 2 p0 + p-) p_adj is accumulated in FP64 over time on Gamma
 * (discrete form of Eq. 10).  Sources are encoded super-shots
 * s_hat = sum_i w_i s_i (Sec. 3.2).
 *
 * Conventions shared by every call
 *   - Grid arrays are linear in i + nx*(j + ny*k) (x fastest), FP32 unless noted.
 *   - "device" pointers are CUDA global-memory pointers owned by the caller;
 *     "host" pointers are ordinary CPU memory read during the call only.
 *   - Calls that take a stream are asynchronous on that stream (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).  Their outputs are valid
 *     once the stream has reached them.  A plan must not be used from two
 *     host threads or on two streams at once; distinct plans are independent.
 *   - Errors are returned as fwi_status; nothing is thrown across the ABI.
 *     Argument and index validation is done on the host at plan creation and
 *     at each call.  The sound speed is range-checked on the device
 *     (0 < c0 <= c_ref, the stability condition of App. B); a violation makes
 *     the call's kernels skip their work and is reported by fwi_plan_status().
 *   - No device memory is allocated after fwi_plan_bind_workspace(): every
 *     buffer lives in the caller-provided workspace.
 */
#ifndef FWI_H
#define FWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fwi_status {
  FWI_OK = 0,
  FWI_EINVAL = 1,       /* bad argument, size or index list                        */
  FWI_ENOMEM = 2,       /* workspace too small / host allocation failed            */
  FWI_EUNSTABLE = 3,    /* c0 outside (0, c_ref]: scheme unstable (App. B)         */
  FWI_ETIMEOUT = 4,     /* reserved: no kernel here waits on a device flag         */
  FWI_ECUDA = 5,        /* a CUDA runtime call failed                              */
  FWI_ECANCELLED = 6,   /* work was cancelled before it ran                        */
  FWI_ENOTSUP = 7       /* grid shape not supported by the library                 */
} fwi_status;

typedef enum fwi_pairing {
  /* Alg. 1 as printed: adjoint steps n = 1..Nt-1 inject the cumulative residual
   * Q^n and are paired with the TR second difference centred at t_(Nt-n).      */
  FWI_PAIRING_LITERAL = 0,
  /* exact discrete adjoint of the PML-free scheme: adjoint steps j = 0..Nt
   * inject Q^j and are paired with p_(Nt-j) - 2 p_(Nt-j-1) + p_(Nt-j-2).      */
  FWI_PAIRING_EXACT = 1
} fwi_pairing;

/* Problem description (host memory, copied by fwi_plan_create). */
typedef struct fwi_problem {
  int32_t nx, ny, nz;       /* FFT grid including the PML; each a product of 2, 3, 5  */
  int32_t pml[3];           /* PML thickness per axis in cells, inside the grid       */
  double dx;                /* grid spacing [m]                                       */
  double dt;                /* time step [s]; stability needs c0 <= c_ref             */
  double c_ref;             /* reference speed of the kappa correction (Eq. 18)       */
  double rho0;              /* constant ambient density [kg/m^3]                      */
  double pml_alpha;         /* PML strength: sigma = alpha c_ref/dx (d/P)^4           */
  double c_rec;             /* >0: gradient returned as dD/dc (raw accumulator times
                               dx*c_rec/2, exact when every receiver sits in c_rec);
                               0: the raw Alg. 1 accumulator                          */
  int32_t nt;               /* time samples = forward iterations (Nt + 1)             */
  int32_t n_src;            /* emitters                                               */
  int32_t n_rec;            /* receivers (measurement channels, operator M)           */
  int32_t n_layer;          /* voxels of the TR boundary layer (subset of Gamma)      */
  int32_t n_gamma;          /* voxels of the reconstruction region Gamma              */
  const int32_t *src_idx;   /* host [n_src] linear voxel index of each emitter        */
  const int32_t *rec_idx;   /* host [n_rec] linear voxel index of each receiver       */
  const int32_t *layer_idx; /* host [n_layer] strictly increasing, each in gamma_idx  */
  const int32_t *gamma_idx; /* host [n_gamma] strictly increasing                     */
  const float *wavelet;     /* host [nt] emitted pressure signal s(t_n)               */
  int32_t pairing;          /* fwi_pairing                                            */
  int32_t max_shots;        /* largest K (super-shots per call) this plan serves      */
  int32_t sims_per_launch;  /* 0: all simulations of a phase share each launch
                               (K shots, adjoint and TR together); 1: the plain form,
                               one simulation per launch sequence                    */
  int32_t per_shot_models;  /* 0: one sound-speed model per call, the gradient is the
                               mean over the K super-shots; 1: super-shot k is an
                               instance of its own -- model c + k N in, gradient
                               grad + k N out (c and grad are [K][N]) -- so instances
                               that share grid and transducers share every launch    */
} fwi_problem;

typedef struct fwi_plan fwi_plan;

/*
 * Validate `prob`, build the host-side tables (wavenumbers, kappa inputs,
 * staggering shifts, PML profiles, FFT radix schedules, per-plane sparse lists)
 * and report the device workspace size needed.  No device memory is touched.
 *   workspace_bytes: out, bytes the caller must provide to fwi_plan_bind_workspace.
 *   out: out, the new plan (free with fwi_plan_destroy).
 * Errors: FWI_EINVAL (bad sizes/indices, duplicate or unsorted gamma/layer, layer
 * voxel outside gamma, nt < 3), FWI_ENOTSUP (a dimension with a prime factor
 * other than 2, 3, 5, or a plane too large for shared memory), FWI_ENOMEM.
 */
fwi_status fwi_plan_create(const fwi_problem *prob, size_t *workspace_bytes, fwi_plan **out);

/*
 * Give the plan its device workspace (>= the reported size, 256-byte aligned)
 * and upload the constant tables (synchronous).  The memory stays owned by the
 * caller and must outlive every call made with the plan.
 * Errors: FWI_EINVAL (NULL or misaligned), FWI_ENOMEM (too small), FWI_ECUDA.
 */
fwi_status fwi_plan_bind_workspace(fwi_plan *plan, void *dev_ptr, size_t bytes);

/*
 * Time-reversal re-simulation on a box enclosing Gamma (Sec. 3.1: the TR simulation
 * domain only needs to enclose Gamma).  After this call, fwi_gradient runs its TR
 * simulations on the box [origin, origin + size) of the grid, a grid of its own with the
 * same dx, dt and c_ref, its own PML of pml[a] cells inside the box (same profile rule and
 * pml_alpha as the plan), and c0 cropped from the model given to each call; the adjoint
 * simulations stay on the whole grid.  The boundary history and the Gamma values are
 * shared, so the gradient keeps its layout.  Forward calls are unchanged.
 *   origin, size, pml: host [3] (x, y, z) in cells; size is the box's FFT grid (each a
 *                product of 2, 3, 5); every Gamma voxel must lie inside the box and
 *                outside its PML.
 *   workspace_bytes: out, the plan's new workspace size (the box plan's workspace and
 *                the cropped c0 added, the whole-grid TR simulations removed).
 * Must be called before fwi_plan_bind_workspace; calling it again replaces the box.
 * The box keeps the default schedule of its own grid: fwi_plan_set_schedule changes the
 * whole-grid simulations only (the box's launches follow the plan's stream groups).
 * Errors: FWI_EINVAL (bound plan, box outside the grid, Gamma outside the box interior),
 * FWI_ENOTSUP (box size not supported), FWI_ENOMEM.
 */
fwi_status fwi_plan_set_tr_box(fwi_plan *plan, const int32_t origin[3], const int32_t size[3],
                               const int32_t pml[3], size_t *workspace_bytes);

/*
 * Forward simulations of K encoded super-shots (Alg. 1, forward loop).
 *   c:       device [nx*ny*nz] sound speed c0 [m/s] ([K][nx*ny*nz] with per_shot_models)
 *   weights: device [K][n_src] encoding weights w (Sec. 3.2), e.g. Rademacher +-1
 *   traces:  device out [K][nt][n_rec], f^n = M p after iteration n
 * Errors: FWI_EINVAL (K outside 1..max_shots, NULL pointer), FWI_ECUDA.
 */
fwi_status fwi_forward(fwi_plan *plan, const float *c, const float *weights, int32_t K,
                       float *traces, void *stream);

/*
 * Misfit and sound-speed gradient, averaged over K encoded super-shots
 * (Alg. 1 whole; mean of independent estimates, Sec. 4.5).
 *   c:        device [N] sound speed ([K][N], one model per super-shot, with per_shot_models)
 *   weights:  device [K][n_src]
 *   observed: device observed data; observed_encoded = 1: [K][nt][n_rec], already
 *             encoded as f_hat = sum_i w_i f_i; observed_encoded = 0: raw per-source
 *             data [n_src][nt][n_rec], encoded on the device with `weights`.
 *   misfit:   device out [K] FP64, D_k = 0.5 ||q_k||^2
 *   grad:     device out [N] FP64, (1/K) sum_k of the gradient on Gamma, 0 elsewhere;
 *             with per_shot_models [K][N], the gradient of each super-shot alone
 *   traces:   device out [K][nt][n_rec] simulated traces, or NULL
 * Errors: FWI_EINVAL, FWI_ECUDA.
 */
fwi_status fwi_gradient(fwi_plan *plan, const float *c, const float *weights, int32_t K,
                        const float *observed, int32_t observed_encoded, double *misfit,
                        double *grad, float *traces, void *stream);

/*
 * Delayed source encoding (Sec. 3.2, Eq. 13): emitter i of super-shot k fires the
 * plan's wavelet delayed by delay[k][i] time steps, s_hat(t_n) = sum_i w_ki
 * s(t_n - delay_ki dt), and the observed data are encoded with the same delays,
 * f_hat[n] = sum_i w_ki f_i[n - delay_ki].  The random delays d_i tau of Eq. 13 are
 * given as whole time steps (0 <= delay < nt); the plan's nt must cover the data
 * length plus the largest delay (T + tau), and its wavelet is the undelayed pulse
 * (zero-padded to nt).  Delays outside [0, nt) simply emit nothing in the window.
 *   delay:       device [K][n_src] int32
 *   observed:    observed_encoded = 1: [K][nt][n_rec] already delay-encoded;
 *                observed_encoded = 0: raw per-source data [n_src][observed_nt][n_rec],
 *                1 <= observed_nt <= nt, zero beyond its samples
 * Other arguments, outputs and errors as for fwi_forward / fwi_gradient.  All delays
 * zero give exactly the results of fwi_forward / fwi_gradient.
 */
fwi_status fwi_forward_delayed(fwi_plan *plan, const float *c, const float *weights,
                               const int32_t *delay, int32_t K, float *traces, void *stream);
fwi_status fwi_gradient_delayed(fwi_plan *plan, const float *c, const float *weights,
                                const int32_t *delay, int32_t K, const float *observed,
                                int32_t observed_encoded, int32_t observed_nt, double *misfit,
                                double *grad, float *traces, void *stream);

/*
 * Stochastic L-BFGS (Alg. 2) on the device: an L-BFGS history of at most m pairs
 * (s, y) of n-vectors, stored in FP32 in a caller-owned workspace, with every dot
 * product accumulated in FP64.  Alg. 2 evaluates the gradient estimator twice per
 * iteration with the same stochastic approximation and stores the pair
 * (nu z, G_z - G_u); the two-loop recursion gives the step z = -H G.
 *   fwi_lbfgs_create:  sizes the workspace (2 m n floats + small scratch).
 *   fwi_lbfgs_bind_workspace: caller-owned device memory, 256-byte aligned; empties
 *                      the history.
 *   fwi_lbfgs_push:    adds the pair (s, y) (device FP64 [n] each) unless s'y <= 0
 *                      (the pair is then skipped, *stored = 0), dropping the oldest
 *                      pair beyond m.  Synchronous on `stream` (it reads s'y and y'y).
 *   fwi_lbfgs_apply:   out = H g (device FP64 [n]; out may equal g), H_0 = h0 I, or
 *                      (s'y / y'y) I of the newest pair if h0 <= 0 (I if empty).
 *                      Asynchronous.
 *   fwi_lbfgs_size:    number of stored pairs.
 * Errors: FWI_EINVAL (NULL, n <= 0, m outside 1..1024, unbound or misaligned
 * workspace), FWI_ECUDA.
 */
typedef struct fwi_lbfgs fwi_lbfgs;
fwi_status fwi_lbfgs_create(int64_t n, int32_t m, size_t *workspace_bytes, fwi_lbfgs **out);
fwi_status fwi_lbfgs_bind_workspace(fwi_lbfgs *lbfgs, void *dev_ptr, size_t bytes);
fwi_status fwi_lbfgs_push(fwi_lbfgs *lbfgs, const double *s, const double *y, void *stream,
                          int32_t *stored);
fwi_status fwi_lbfgs_apply(fwi_lbfgs *lbfgs, const double *g, double h0, double *out, void *stream);
int32_t fwi_lbfgs_size(const fwi_lbfgs *lbfgs);
fwi_status fwi_lbfgs_destroy(fwi_lbfgs *lbfgs);

/*
 * Elementwise steps of Alg. 2 and of the parameterisations of Sec. 3.3, on device
 * vectors of length n (asynchronous on `stream`):
 *   fwi_vec_step_project: u <- min(max(u + nu z, u_min), u_max)   (projection step)
 *   fwi_vec_accumulate:   acc <- acc + w u                         (iterate averaging)
 *   fwi_param_to_speed:   c <- c(u) for u = c (kind 0), u = 1/c (1, slowness),
 *                         u = 1/c^2 (2, squared slowness)
 *   fwi_grad_to_param:    g_u <- g_c dc/du: 1, -c^2, -c^3 / 2 for kinds 0, 1, 2
 * Errors: FWI_EINVAL (NULL, n <= 0, bad kind, u_min > u_max), FWI_ECUDA.
 */
fwi_status fwi_vec_step_project(int64_t n, double *u, const double *z, double nu, double u_min,
                                double u_max, void *stream);
fwi_status fwi_vec_accumulate(int64_t n, double *acc, const double *u, double w, void *stream);
fwi_status fwi_param_to_speed(int64_t n, int32_t kind, const double *u, float *c, void *stream);
fwi_status fwi_grad_to_param(int64_t n, int32_t kind, const float *c, const double *gc, double *gu,
                             void *stream);

/*
 * Grid transfers of the coarse-to-fine scheme (Sec. 3.3, App. C): separable periodic
 * Fourier resampling of a real array [n2][n1][n0] (axis 0 fastest) to [m2][m1][m0].
 * Along each axis a the output sample i is the windowed trigonometric interpolant of
 * the input at t = i n_a / m_a over the band |k| <= K = floor((min(n_a, m_a) - 1) / 2):
 *   out_i = (1/n_a) sum_j in_j (w(0) + 2 sum_{k=1..K} w(k) cos(2 pi k (t - j) / n_a)),
 * window[a]: 0 = none (plain Fourier interpolation), 1 = Blackman (model up-sampling),
 * 2 = Kaiser with parameter kaiser_beta (time-series low-pass); both windows are 1 at
 * k = 0 and vanish just beyond the band.  Axes with n_a = m_a and window 0 are left as
 * they are.  The output is multiplied by `scale` (eta^(d-1) for data down-sampled in time,
 * App. C; 1 otherwise; it needs at least one resampled axis).  FP32 arrays, FP64
 * accumulation.
 *   fwi_resampler_create: host; reports the workspace size (matrices + two intermediates).
 *   fwi_resampler_bind_workspace: caller-owned device memory, 256-byte aligned; uploads
 *                         the matrices (synchronous).
 *   fwi_resample:         in (device [n2][n1][n0]) -> out (device [m2][m1][m0]); in and
 *                         out must not overlap.  Asynchronous on `stream`.
 * Errors: FWI_EINVAL (NULL, sizes outside 1..8192, bad window, beta < 0, unbound),
 * FWI_ENOMEM, FWI_ECUDA.
 */
typedef struct fwi_resampler fwi_resampler;
fwi_status fwi_resampler_create(const int32_t n_in[3], const int32_t n_out[3], const int32_t window[3],
                                double kaiser_beta, double scale, size_t *workspace_bytes,
                                fwi_resampler **out);
fwi_status fwi_resampler_bind_workspace(fwi_resampler *resampler, void *dev_ptr, size_t bytes);
fwi_status fwi_resample(fwi_resampler *resampler, const float *in, float *out, void *stream);
fwi_status fwi_resampler_destroy(fwi_resampler *resampler);

/*
 * Wait for the plan's last call and report its device-side status:
 * FWI_EUNSTABLE if its sound speed was outside (0, c_ref] (the call's outputs are
 * then undefined), FWI_ECUDA on an asynchronous CUDA error, else FWI_OK.
 */
fwi_status fwi_plan_status(fwi_plan *plan);

/* Voxel-steps one call performs: (forward + adjoint iterations) * voxels * K, plus TR
 * iterations * (box or grid) voxels * K for a gradient. */
int64_t fwi_plan_voxel_steps(const fwi_plan *plan, int32_t K, int32_t gradient);

/* Number of kernel launches one fwi_forward (gradient = 0) or fwi_gradient (1) call
 * with encoded observed data issues under the plan's current schedule (for launch
 * accounting; raw observed data add one encoding launch). */
int64_t fwi_plan_launches(const fwi_plan *plan, int32_t K, int32_t gradient);

/*
 * FFT schedule of a plan (what the autotuner searches).
 *   specialized: 1 = compile-time transforms where the library has them (square planes
 *                of 32, 64, 96, 128, 160; z lengths 32..128), 0 = runtime schedules,
 *                2 = two-step register-transform kernels where the library has them:
 *                whole square planes of 32, 64, 96, 128, 135, 160; split square planes of
 *                243, 256, 480; z lengths 32, 48, 64, 80, 96, 128, 135, 256 (the other
 *                passes as for 1; FWI_ENOTSUP when none applies)
 *   radix_order: runtime radix schedule: 0 = radix 8, 4, 2 then 3, 5; 1 = radix 4, 2
 *                then 3, 5 (no radix 8); 2 = small radices first (2, 3, 4, 5, 8 order
 *                reversed: the largest pass last)
 *   z_tile:      spectrum columns per z-pass CTA, 16 or 32
 *   split_plane: 0 = one CTA transforms a whole z-plane in shared memory; 1 = the XY
 *                work of a plane is split into column (y) and row-pair (x) passes
 *                through global memory (always used when a plane does not fit)
 *   stream_groups: 1 = all simulations of a call advance in one launch sequence; 2 or
 *                4 = the super-shots are split into that many groups (at most K; for
 *                gradients each shot's adjoint and TR simulations stay together) that
 *                advance on separate streams, so that kernels of one group fill SMs the
 *                others leave idle.  Results are bit-identical.
 * fwi_plan_create picks the first of {2, 0, 32, 0, 4}, {2, 0, 32, 1, 4}, {1, 0, 32, 0, 4},
 * {1, 0, 32, 1, 4} that applies (split planes only where a plane does not fit).  Setting a schedule keeps the workspace size;
 * it may be changed after binding (between calls).  Results differ only by FP32
 * rounding order.  Errors: FWI_EINVAL (bad values), FWI_ENOTSUP (the shared memory
 * the schedule needs exceeds the device limit).
 */
typedef struct fwi_schedule {
  int32_t specialized;
  int32_t radix_order;
  int32_t z_tile;
  int32_t split_plane;
  int32_t stream_groups;
} fwi_schedule;
fwi_status fwi_plan_set_schedule(fwi_plan *plan, const fwi_schedule *schedule);
fwi_status fwi_plan_get_schedule(const fwi_plan *plan, fwi_schedule *schedule);

/* Kernels that can be timed by the profiling hook. */
typedef enum fwi_kernel {
  FWI_K_ZPASS_MOMENTUM = 0, FWI_K_PLANE_MOMENTUM = 1, FWI_K_ZPASS_MASS = 2, FWI_K_PLANE_MASS = 3
} fwi_kernel;

/*
 * Profiling hook: with enable = 1, every later launch of a kernel whose bit is
 * set in `kernel_mask` (bit k = fwi_kernel k) is bracketed by CUDA events on
 * its stream; at most `capacity` launches are kept, later ones are not timed.
 * enable = 0 stops recording and keeps the totals.  Launches issued into a stream
 * that is being captured (a batch graph, a serving graph) are not timed: an event
 * recorded during capture is only a graph dependency.  Host-side event objects
 * only; no device memory is allocated.  Errors: FWI_EINVAL, FWI_ECUDA.
 */
fwi_status fwi_plan_profile(fwi_plan *plan, int32_t kernel_mask, int32_t enable, int32_t capacity);

/*
 * Synchronise and read the profile, per fwi_kernel k (arrays of 4): total device
 * time ms[k] of the timed launches, their number launches[k], and the number of
 * simulations they processed sims[k] (a launch over s simulations counts s).
 * Resets the totals.
 */
fwi_status fwi_plan_profile_read(fwi_plan *plan, double *ms, int64_t *launches, int64_t *sims);

/*
 * Allocation-free adjoint source (no counterpart in the paper; added for callers
 * that cannot allocate device memory).  Same arithmetic as the adjoint-source
 * stage inside fwi_gradient: q^n = f^(Nt-n) - f_obs^(Nt-n), D_k = 0.5 ||q_k||^2
 * (FP64), Q^n = sum_{m<=n} q^m (FP64 running sum, stored FP32).
 *
 * Who needs it: callers that manage every byte of device memory themselves --
 * a fixed pool carved out once at start-up, or a host process that must keep its
 * device footprint constant while it runs -- and can neither call cudaMalloc nor
 * hand the library a workspace for this step.  The block partial sums of D live
 * in a file-scope __device__ array of FWI_NOALLOC_MAX_PARTIALS doubles (64 KiB)
 * that every GPU which loads the library holds until the process exits.
 *   traces, observed: device [K][nt][n_rec] simulated and observed (encoded) traces
 *   qcum:   device out [K][nt][n_rec] FP32 cumulative residual Q
 *   misfit: device out [K] FP64
 * Limits: K * ceil(n_rec / 256) <= FWI_NOALLOC_MAX_PARTIALS and 1 <= K <= 32,
 * else FWI_EINVAL (nothing is launched).  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents: every partial is written before it is read,
 * so no clearing is needed, but calls that overlap on the GPU (on different
 * streams) race on it.  Allocates nothing: no cudaMalloc, no cudaFree.
 */
#define FWI_NOALLOC_MAX_PARTIALS 8192
fwi_status fwi_adjoint_source_noalloc(const float *traces, const float *observed, int32_t K,
                                      int32_t nt, int32_t n_rec, float *qcum, double *misfit,
                                      void *stream);

/*
 * Batched form: gradients of n independent problems (plans, possibly of different
 * grid sizes, each with its own workspace) submitted as one CUDA graph launch.
 * The first fwi_batch_gradient call with a given set of arguments captures every
 * plan's launch sequence into one graph, one stream branch per plan, so the
 * instances overlap on the GPU; later calls with identical arguments replay it
 * (any change of pointer or K, and any fwi_plan_bind_workspace or
 * fwi_plan_set_schedule on a member plan since the capture, re-captures).  The
 * output pointers are part of the key: callers that want replays pass the same
 * misfit and grad buffers on every call.  Plans must not be used elsewhere
 * while a batch that contains them runs.  Results are identical to n separate
 * fwi_gradient calls.  Each plan appears once (a plan listed twice, or one
 * without a bound workspace, is FWI_EINVAL).  Errors: FWI_EINVAL, FWI_ECUDA.
 */
typedef struct fwi_batch fwi_batch;
fwi_status fwi_batch_create(int32_t n, fwi_plan *const *plans, fwi_batch **out);
/* Arrays of n entries, element i as in fwi_gradient for plans[i]; traces may be NULL. */
fwi_status fwi_batch_gradient(fwi_batch *batch, const float *const *c, const float *const *weights,
                              const int32_t *K, const float *const *observed,
                              const int32_t *observed_encoded, double *const *misfit,
                              double *const *grad, void *stream);
/* Kernel launches the captured graph holds (0 before the first capture). */
int64_t fwi_batch_nodes(const fwi_batch *batch);
/*
 * Concurrency of the batch graph: plan i runs on chain chain[i] (host [n], values 0..n-1);
 * the chains run side by side, each chain's plans one after another in batch order.
 * chain = NULL (the default) gives every plan a chain of its own; all zeros runs the
 * plans in sequence.  Plans that each fill the GPU (several super-shots or stream groups)
 * keep their data in L2 between their own launches when they do not run side by side;
 * small ones fill the SMs that a large one leaves idle when they do.  Results are identical
 * for every assignment.  The next fwi_batch_gradient re-captures.
 * Errors: FWI_EINVAL (NULL batch, a chain outside 0..n-1).
 */
fwi_status fwi_batch_set_chains(fwi_batch *batch, const int32_t *chain);
fwi_status fwi_batch_destroy(fwi_batch *batch);

/* Release the plan's host memory (not the workspace, which the caller owns). */
fwi_status fwi_plan_destroy(fwi_plan *plan);

/* Static description of a status code. */
const char *fwi_status_string(fwi_status status);

/* Name and description of the last CUDA runtime error that made a call of this
 * thread return FWI_ECUDA ("" if none).  Valid until the thread's next call. */
const char *fwi_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FWI_H */
