/*
 * kpdhg.h - C ABI of the GB300 (sm_103a) library for k-space-preconditioned PDHG
 * reconstruction of multi-coil non-Cartesian MRI (Ong, Uecker & Lustig,
 * "Accelerating Non-Cartesian MRI Reconstruction Convergence using k-space
 * Preconditioning", arXiv 1902.09657).
 *
 * Problem statement (Sec. 2, Eq. model_i / model / obj):
 *   y_c[i] = N^{-1/2} sum_n s_c[n] x[n] exp(-i 2 pi sum_d f_{i,d} n_d / N_d) + w_c[i],
 *   x_hat = argmin_x 1/2 ||A x - y||^2 + g(x),  g = lambda ||x||^2/2  or  lambda ||W x||_1.
 * A is applied as a Kaiser-Bessel NUFFT (Sec. 6: oversampling 1.25, width 4, following
 * Beatty et al.).
 *
 * Conventions used by every entry point:
 *   - Images are complex64 (interleaved re, im float32), row-major, slowest axis first
 *     ((y, x) in 2D, (z, y, x) in 3D); pixel index j_d holds the centred position
 *     n_d = j_d - N_d/2.
 *   - Trajectories are float32 [M][ndim] in cycles per field of view, column d matching
 *     image axis d; every coordinate must lie in [-N_d/2, N_d/2].
 *   - k-space arrays (y, dual variable, preconditioner) are coil-major [C][M].
 *   - Coil maps are [C][N] complex; storage type given by a kp_cdtype.
 *   - All pointers named *_dev are device pointers owned by the caller, 16-byte aligned,
 *     contiguous, and must stay valid until the stream work that uses them completes.
 *     The library never frees caller memory; a plan owns only its own workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Work is
 *     ordered on that stream.  Calls documented as "synchronous" wait for it to finish.
 *   - No C++ exception crosses the boundary.  Every call returns a kp_status; on failure
 *     kp_last_error() returns a thread-local message.
 *   - A plan is not thread-safe: do not use one plan from two host threads or two
 *     streams at the same time.
 */
#ifndef KPDHG_H
#define KPDHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kp_plan_s* kp_plan;

typedef enum {
    KP_OK = 0,
    KP_EINVAL = 1,       /* invalid argument (sizes, null pointer, coordinate range, p <= 0) */
    KP_ENOMEM = 2,       /* device or host allocation failed */
    KP_ECUDA = 3,        /* a CUDA runtime call failed */
    KP_ECUFFT = 4,       /* a cuFFT call failed */
    KP_EDIVERGED = 5,    /* objective exceeded 1e3 x its first value */
    KP_ENONFINITE = 6,   /* NaN/Inf met (objective, power-method norm, or a non-positive
                            preconditioner denominator in kp_make_preconditioner) */
    KP_ETIMEOUT = 7,     /* a bounded device-side wait gave up */
    KP_EINTERNAL = 8
} kp_status;

/* Complex storage types.  Arithmetic is always float32 with float64 reductions. */
typedef enum {
    KP_C64 = 0,          /* complex float32 */
    KP_C32_BF16 = 1,     /* complex bfloat16 (re, im) */
    KP_C32_FP16 = 2      /* complex float16 (re, im) */
} kp_cdtype;

typedef enum {
    KP_REG_L2 = 0,           /* g(x) = lambda ||x||^2 / 2                       (Sec. 2) */
    KP_REG_L1_WAVELET = 1,   /* g(x) = lambda ||W x||_1, W periodised orthonormal
                                8-tap Daubechies, `wavelet_levels` levels       (Sec. 2, 6) */
    KP_REG_TV = 2            /* g(x) = lambda ||G x||_1, G periodic forward differences
                                along every axis, |.| of each complex difference (Sec. 4.2) */
} kp_reg;

typedef struct {
    int ndim;              /* 2 or 3 */
    int64_t img[3];        /* N_d, slowest axis first; entries beyond ndim ignored */
    int ncoils;            /* C >= 1 */
    int64_t nsamples;      /* M >= 1 */
    float oversamp;        /* grid oversampling alpha (1.25 in the paper); G_d = ceil(alpha N_d), even */
    int kernel_width;      /* Kaiser-Bessel width W in grid units; 4 (the paper's) is supported */
    int wavelet_levels;    /* levels of W for KP_REG_L1_WAVELET; each N_d divisible by 2^levels */
} kp_params;

#define KP_NPHASES 12      /* phases of one PDHG iteration reported by profiling */

typedef struct {
    int iters;             /* iterations run */
    double lmax;           /* lambda_max(P A A^H) used for tau_0 */
    double pmin;           /* min_i p_i used by the step-size schedule */
    double sigma_last;     /* sigma, tau after the last iteration */
    double tau_last;
    double final_obj;      /* objective at the returned x if a trace was requested, else NaN */
    double phase_ms[KP_NPHASES];  /* with profiling on: summed GPU time per phase (ms):
                                     0 coil/apodise/pad, 1 FFT, 2 interpolation + dual update,
                                     3 spreading, 4 split-tile reduction, 5 inverse FFT,
                                     6 adjoint + primal step, 7 DWT, 8 soft threshold,
                                     9 inverse DWT, 10 extrapolation, 11 iteration counter */
} kp_stats;

/* Human-readable name of a status; never NULL. */
const char* kp_status_string(kp_status s);

/* Thread-local message describing the last failure on this host thread ("" if none). */
const char* kp_last_error(void);

/* Create a plan: validates `params`, allocates all device workspace (grids, sort buffers,
 * cuFFT plans) and uploads the apodisation and wavelet tables.  Synchronous.
 * Errors: KP_EINVAL (ndim not 2/3, non-positive sizes, width != 4, oversamp < 1,
 * levels incompatible with the image), KP_ENOMEM, KP_ECUFFT. */
kp_status kp_plan_create(kp_plan* out, const kp_params* params, void* stream);

/* Release a plan and all its workspace.  Synchronises the device first.  NULL is a no-op. */
kp_status kp_plan_destroy(kp_plan plan);

/* Set the trajectory (Sec. 2: sampling points f_i): converts to grid coordinates
 * t = f G/N (formed in float64; kept as the first tap and a float32 offset), sorts samples
 * by grid tile (counting sort) and builds the
 * per-tile lists used by the spreading kernel.  traj_dev: float32 [M][ndim].
 * Synchronous (it checks the coordinate range).  Errors: KP_EINVAL if any coordinate is
 * outside [-N_d/2, N_d/2] or not finite. */
kp_status kp_plan_set_trajectory(kp_plan plan, const float* traj_dev, void* stream);

/* Set the coil sensitivity maps s_c (Sec. 2), [C][N] of type maps_t; copied into the
 * plan (converted to the plan's storage: float32 for KP_C64, half types kept half).
 * Asynchronous. */
kp_status kp_plan_set_maps(kp_plan plan, const void* maps_dev, kp_cdtype maps_t, void* stream);

/* y = A x (Sec. 2, Eq. model_i), NUFFT approximation: coil multiply, apodisation,
 * oversampled FFT, Kaiser-Bessel interpolation.  x_dev: complex64 [N];
 * y_dev: [C][M] of type y_t.  Asynchronous. */
kp_status kp_sense_forward(kp_plan plan, const void* x_dev, void* y_dev, kp_cdtype y_t, void* stream);

/* x = A^H y, the exact adjoint of kp_sense_forward (spreading, inverse FFT, apodisation,
 * conjugate coil combine).  y_dev: [C][M] of type y_t; x_dev: complex64 [N].  Asynchronous. */
kp_status kp_sense_adjoint(kp_plan plan, const void* y_dev, kp_cdtype y_t, void* x_dev, void* stream);

/* l2-optimised diagonal k-space preconditioner (Sec. 5 and App. A), computed by the fast
 * route of Sec. 5.1 (Fig. 2): autocorrelations of s_c s_d^* by FFT on a 2N grid,
 * point-spread function h by a type-1 NUFFT of ones, one type-2 NUFFT per coil.
 * multichannel = 1: Eq. mc_precond, p_c[i]^{-1} = 1/(||s_c||^2 N) sum_j sum_d
 *   |sum_n s_c s_d^* e^{-i 2 pi (f_i - f_j) n/N}|^2;
 * multichannel = 0: Eq. sc_precond with the 1/N^2 prefactor of the general form
 *   (C = 1, s = 1), the same value written for every coil.
 * FFTs and gridding in float32; the denominator sums (R_c = sum_d |Q_cd|^2 and the taps of the
 * last type-2 interpolation) accumulate in float64.
 * p_dev: float32 [C][M], sample order of the trajectory.  Synchronous.
 * Errors: KP_ENONFINITE if a denominator came out non-positive (NUFFT error). */
kp_status kp_make_preconditioner(kp_plan plan, int multichannel, float* p_dev, void* stream);

/* lambda_max(P A A^H) by `iters` power iterations on A^H P A (Sec. 6: 30 iterations),
 * started from v0_dev (complex64 [N]) or from the all-ones image if v0_dev is NULL.
 * p_dev: float32 [C][M] or NULL for P = I.  *lmax receives ||A^H P A v|| for the last
 * normalised v.  Synchronous. */
kp_status kp_max_eig(kp_plan plan, const float* p_dev, const void* v0_dev, int iters,
                     double* lmax, void* stream);

/* Preconditioned PDHG (Sec. 4.1):
 *   u <- (I + sigma_k P)^{-1} (u + sigma_k P (A xbar - y))
 *   x <- prox_{tau_k g}(x - tau_k A^H u),  xbar <- x + theta_k (x - x_old)
 *   sigma_0 = 1, tau_0 = 1/lmax, theta_k = 1/(1 + 2 sigma_k min p),
 *   sigma_{k+1} = theta_k sigma_k, tau_{k+1} = tau_k / theta_k;  x_0 = xbar_0 = 0, u_0 = 0.
 * y_dev: [C][M] of type y_t.  p_dev: float32 [C][M]; NULL computes the multi-channel
 * preconditioner first.  lmax <= 0 runs 30 power iterations from the all-ones image.
 * x_dev: complex64 [N] output.  obj_trace: host double[iters] receiving F(x_k) after each
 * iteration, or NULL (tracing adds a forward NUFFT per iteration).  stats: host or NULL.
 * KP_REG_TV follows Sec. 4.2 instead: a second dual variable v [ndim][N],
 *   v <- projection of v + sigma G xbar onto {|v_i| <= lambda},
 *   x <- x - tau (A^H u + G^H v),  xbar <- 2 x - x_old,
 * with sigma = 1, theta = 1 and tau = 1/(lmax + 4 ndim) at every iteration, v_0 = 0.
 * The iteration is replayed from a CUDA graph captured once per plan and regulariser.
 * Synchronous.  Errors: KP_EINVAL (iters < 0, lambda < 0, wavelet levels 0 for l1,
 * non-positive p or lmax found on the device), KP_ENONFINITE (the returned x holds a NaN or
 * Inf, checked on the device after every solve, or a non-finite objective in the trace),
 * KP_EDIVERGED (traced objective above 1e3 x its first value), KP_ETIMEOUT (a bounded device
 * wait gave up: see kp_plan_set_wait_limit). */
kp_status kp_pdhg_solve(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev,
                        kp_reg reg, float lambda, int iters, double lmax, void* x_dev,
                        double* obj_trace, kp_stats* stats, void* stream);

/* kp_pdhg_solve with the measurements in page-locked host memory (y_host: [C][M] of type y_t,
 * allocated with cudaHostAlloc or pinned).  The library copies y into its own device buffer on
 * a copy stream of the plan while the preconditioner and the power method run, and waits for
 * the copy only before the measurements are first read (the sorted load ahead of the first
 * dual step), so the host-to-device transfer overlaps the set-up.  The copy starts after the
 * work already queued on `stream`.  Same result as kp_pdhg_solve on a device copy of y.
 * Synchronous.  Errors: those of kp_pdhg_solve; KP_EINVAL if y_host is not page-locked. */
kp_status kp_pdhg_solve_host(kp_plan plan, const void* y_host, kp_cdtype y_t, const float* p_dev, kp_reg reg,
                             float lambda, int iters, double lmax, void* x_dev, double* obj_trace, kp_stats* stats,
                             void* stream);

/* State of a PDHG run (Sec. 4.1) between iterations, for checkpoints and warm starts: the
 * iterates x_k, xbar_k and the dual variable u_k, and the number k of iterations already taken
 * (the step sizes sigma_k, tau_k, theta_k follow from k, lambda_max and min p).  All pointers
 * are device buffers owned by the caller: x and xbar complex64 [N]; u complex64 [C][M] in the
 * trajectory's sample order; v complex64 [ndim][N], the dual variable of Sec. 4.2, used with
 * KP_REG_TV only (NULL otherwise). */
typedef struct {
    void* x;
    void* xbar;
    void* u;
    void* v;
    int k;
} kp_pdhg_state;

/* kp_pdhg_solve with a state in and out.  start: NULL runs from x_0 = xbar_0 = 0, u_0 = 0
 * (v_0 = 0), k = 0 like kp_pdhg_solve; otherwise the run continues from that state, so
 * `a` iterations followed by `b` iterations resumed from the returned state equal a + b
 * iterations in one call (same y, p, lambda and lambda_max; pass the lambda_max the first call
 * used, found in kp_stats.lmax).  end: receives the state after the last iteration; end->x is
 * required (the reconstruction), the other pointers may be NULL (not written); end->k is set.
 * start and end may point at the same buffers.  Synchronous.  Errors as kp_pdhg_solve, and
 * KP_EINVAL for start->k < 0, a NULL start->x, start->xbar or start->u, or a NULL start->v with
 * KP_REG_TV. */
kp_status kp_pdhg_solve_ex(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, kp_reg reg,
                           float lambda, int iters, double lmax, const kp_pdhg_state* start, kp_pdhg_state* end,
                           double* obj_trace, kp_stats* stats, void* stream);

/* l2-regularised reconstruction through the dual (appendix on the connection to Trzasko
 * et al.): (A A^H + lambda I) w = lambda y by `iters` conjugate-gradient iterations with the
 * diagonal p as preconditioner, from w = 0, then x = A^H w / lambda, the minimiser of
 * 1/2 ||A x - y||^2 + lambda/2 ||x||^2 (w = -u for the dual u of kp_pdhg_solve with KP_REG_L2).
 * y_dev: complex64 [C][M].  p_dev: float32 [C][M] (every entry positive), or NULL for none.
 * x_dev: complex64 [N] output.  res_trace: host double[iters + 1] receiving
 * ||lambda y - (A A^H + lambda I) w|| before the first and after each iteration, or NULL.
 * Uses the plan's PDHG work buffers.  Synchronous.  Errors: KP_EINVAL (lambda <= 0,
 * iters < 0, no trajectory or maps, a p entry not positive), KP_ENONFINITE (a residual not
 * finite). */
kp_status kp_dual_l2_solve(kp_plan plan, const void* y_dev, const float* p_dev, float lambda, int iters,
                           void* x_dev, double* res_trace, void* stream);

/* Comparison systems of Sec. 6 (the experiments compare PDHG with the proposed k-space
 * preconditioners against CG, CG with a circulant preconditioner and FISTA).
 *
 * l2-optimised circulant preconditioner (App. B): P = argmin over circulant P of
 * ||A^H A - P||_F^2, P[m, n] = c[(m - n) mod N] per axis, c[k] = 1/N sum over s in {0,1}^ndim
 * of r[k - s N] h[k - s N] with r[d] = N^{-1/2} sum_c sum_{m - n = d} s_c^*[m] s_c[n] (FFTs on the
 * 2N grid, float64 sums) and h the point-spread function of Sec. 5.1.  The 1/N is the average
 * over a circulant diagonal that the appendix's closed form leaves out (a uniform scale).  Kept in
 * the plan as the eigenvalues of P (the DFT of c); eig_dev: float32 [N] copy of them, or NULL.
 * Recomputed after a new trajectory or new maps.  Synchronous. */
kp_status kp_make_circulant_preconditioner(kp_plan plan, float* eig_dev, void* stream);

/* Conjugate gradients on (A^H A + lambda I) x = A^H y (the l2 problem of Eq. obj), from x = 0,
 * plain (circulant = 0) or preconditioned by P + lambda I with P the circulant above
 * (circulant = 1; computed first if the plan holds none for its trajectory and maps).
 * y_dev complex64 [C][M] (trajectory order); x_dev complex64 [N] out; obj_trace host double[iters]
 * receiving F(x_k) = 1/2 ||A x_k - y||^2 + lambda/2 ||x_k||^2 after each iteration (A x_k kept by
 * recurrence), or NULL.  Uses the plan's PDHG work buffers.  Synchronous.
 * Errors: KP_EINVAL, KP_ENONFINITE (objective not finite), KP_ETIMEOUT. */
kp_status kp_cg_l2_solve(kp_plan plan, const void* y_dev, float lambda, int iters, int circulant, void* x_dev,
                         double* obj_trace, void* stream);

/* FISTA (Beck & Teboulle) on 1/2 ||A x - y||^2 + g(x), g = lambda ||x||^2/2 (KP_REG_L2) or
 * lambda ||W x||_1 (KP_REG_L1_WAVELET), from x_0 = z_0 = 0, t_0 = 1, step 1/L with L = lmax, or,
 * for lmax <= 0, 1.01 x the 30-iteration power-method estimate of lambda_max(A^H A).
 * y_dev complex64 [C][M]; x_dev complex64 [N] out; obj_trace host double[iters] or NULL (an extra
 * forward NUFFT per iteration).  Uses the plan's PDHG work buffers.  Synchronous. */
kp_status kp_fista_solve(kp_plan plan, const void* y_dev, kp_reg reg, float lambda, int iters, double lmax,
                         void* x_dev, double* obj_trace, void* stream);

/* Trajectory gradient through y = A x (differentiable reconstruction; Sec. 6 operator with the
 * Kaiser-Bessel derivative phi'): gtraj[i][d] = Re sum_c conj(gy_c[i]) d y_c[i] / d f_{i,d},
 * taps held fixed (y jumps where a coordinate crosses a grid line, at the window edge).
 * x_dev complex64 [N]; gy_dev complex64 [C][M] (user order); gtraj_dev float32 [M][ndim]
 * (overwritten).  Asynchronous. */
kp_status kp_sense_forward_traj_grad(kp_plan plan, const void* x_dev, const void* gy_dev, float* gtraj_dev,
                                     void* stream);

/* Trajectory gradient through x = A^H u: gtraj[i][d] = Re sum_n conj(gx[n]) d x[n] / d f_{i,d}
 * = Re sum_c conj(u_c[i]) d (A gx)_c[i] / d f_{i,d}.  u_dev [C][M], gx_dev [N], gtraj_dev
 * [M][ndim] (overwritten).  Asynchronous. */
kp_status kp_sense_adjoint_traj_grad(kp_plan plan, const void* u_dev, const void* gx_dev, float* gtraj_dev,
                                     void* stream);

/* Unrolled l2 PDHG for differentiation: `iters` iterations of Sec. 4.1 with
 * g = lambda ||x||^2 / 2 (same schedule, start and preconditioner rules as kp_pdhg_solve,
 * complex64 y), keeping xbar_k, u_{k+1} and x_{k+1} of every iteration in the plan (per-
 * iteration checkpoints, (2N + CM) complex values each).  x_dev receives x_K.  Synchronous. */
kp_status kp_unrolled_forward(kp_plan plan, const void* y_dev, const float* p_dev, float lambda, int iters,
                              double lmax, void* x_dev, void* stream);

/* Reverse sweep of the last kp_unrolled_forward: given gx = dL/dRe x_K + i dL/dIm x_K
 * (complex64 [N]), returns dL/dy (complex64 [C][M], user order, or NULL), dL/dlambda (host,
 * or NULL) and dL/df (float32 [M][ndim], or NULL), with p, lambda_max and the step sizes held
 * constant.  Synchronous. */
kp_status kp_unrolled_backward(kp_plan plan, const void* gx_dev, void* gy_dev, double* glambda, float* gtraj_dev,
                               void* stream);

/* Periodised multilevel Daubechies-4 wavelet transform W (forward = 1) or W^H
 * (forward = 0) of a complex64 [N] image, Mallat layout, plan's wavelet_levels.
 * in_dev and out_dev may alias.  Asynchronous. */
kp_status kp_wavelet(kp_plan plan, const void* in_dev, void* out_dev, int forward, void* stream);

/* Profiling switch: when enable != 0, kp_pdhg_solve launches each iteration's kernels
 * directly (no CUDA graph), records a CUDA event at every phase boundary on the caller's
 * stream, and returns the per-phase GPU time in kp_stats.phase_ms. */
kp_status kp_plan_set_profiling(kp_plan plan, int enable);

/* Limit, in SM clock cycles, of every bounded wait inside this plan's kernels (the bulk-copy
 * staging of the interpolation, the grid barriers of the persistent primal kernel); the default
 * 2e9 is about a second.  A wait that reaches it gives up: the kernel records the timeout,
 * still lets its own copies in flight land (waiting up to the default limit for them), and
 * finishes; results of that launch are then invalid and the next synchronous call on the plan
 * (kp_pdhg_solve, kp_plan_sync, ...) returns KP_ETIMEOUT.  cycles >= 0.  Captured iteration
 * graphs are dropped (they hold the limit). */
kp_status kp_plan_set_wait_limit(kp_plan plan, long long cycles);

/* Waits for the stream and reports device-side conditions recorded by the plan's asynchronous
 * calls since the last check (kp_sense_forward, kp_sense_adjoint, kp_wavelet): KP_ETIMEOUT if a
 * bounded wait gave up.  The recorded condition is cleared.  Synchronous. */
kp_status kp_plan_sync(kp_plan plan, void* stream);

/* Number of this library's own kernel launches issued through this plan so far (kernels
 * inside replayed CUDA graphs included; cuFFT's kernels not included). */
kp_status kp_plan_launch_count(kp_plan plan, int64_t* count);

/* Out-of-range accesses recorded by the bounds-checked build of this library
 * (libkpdhg_checked.so, compiled with -DKP_CHECKED as a stand-in for a memory checker: the
 * hot kernels test each computed global-memory index against its buffer's extent, skip an
 * access out of range and record it).  Synchronises the device, then returns and clears the
 * records: *checked = 1 for the checked build, 0 for the release build (whose records are
 * always empty); *count = accesses skipped since the last call; *first_site and *first_index
 * = the first one's check site (numbered in the library's internal header) and index, 0 when
 * none.  Any pointer may be NULL.  Errors: KP_ECUDA if the device reports an error. */
kp_status kp_bounds_report(int* checked, uint32_t* count, uint32_t* first_site, int64_t* first_index);

/* x = A^H y like kp_sense_adjoint, but with no plan and no device allocation: for callers
 * that reserve all device memory up front and may not let a library allocate afterwards
 * (for example a real-time reconstruction service with a fixed memory pool).  The paper has
 * no counterpart; this is a deployment variant of the adjoint.
 * params: sizes as for kp_plan_create (wavelet_levels ignored); traj_dev float32 [M][ndim];
 * maps_dev complex64 [C][N]; y_dev complex64 [C][M]; x_dev complex64 [N] (output).
 * Work space is one fixed 4 MiB device array built into the library (2^19 complex64 values,
 * held on every GPU that loads the library until exit); problems needing more than
 * C x (G + G / g_last x n_last) values are rejected with KP_EINVAL (G = prod g_d, g_d the
 * oversampled grid).  Its device address is looked up on every call, on the current device;
 * the first call on a device also loads the library's device code there, so make that first
 * call before any stream capture.  The grid is
 * cleared at the start of every call; calls that overlap on the GPU share the array and race,
 * so issue them one at a time.  The inverse DFT is evaluated directly (no cuFFT plan), so the
 * result matches kp_sense_adjoint to float32 rounding (float64 grid coordinates, like the plan).  Samples with a coordinate outside
 * [-N_d/2, N_d/2] or not finite are skipped (this path cannot report them without a
 * synchronisation; kp_plan_set_trajectory validates a trajectory).  Asynchronous. */
kp_status kp_sense_adjoint_noalloc(const kp_params* params, const float* traj_dev, const void* maps_dev,
                                   const void* y_dev, void* x_dev, void* stream);

/* Batched reconstruction of independent cases (the paper solves one problem at a time; a
 * batch is many Sec. 4.1 solves sharing the GPU).  A batch refers to `ncases` existing plans
 * (each with its own sizes, trajectory and maps; the plans stay owned by the caller, must
 * outlive the batch, and must not be used by another call while a batch solve runs).
 * Errors: KP_EINVAL (null pointer, ncases < 1), KP_ECUDA. */
typedef struct kp_batch_s* kp_batch;
kp_status kp_batch_create(kp_batch* out, kp_plan* plans, int ncases);

/* How a batch's PDHG iteration is laid out in its CUDA graph.
 * KP_BATCH_PER_CASE (default): every case's own iteration kernels on its own forked stream, so
 *   one case's FFTs overlap another case's interpolation or spreading.
 * KP_BATCH_PHASES: one kernel launch per phase over all cases (interpolation + dual step,
 *   split-tile clearing, spreading, primal step, each wavelet level, pre-step, counters; each
 *   block finds its case in a table of block offsets), with the cases' cuFFT transforms on
 *   forked streams between the phases.  Applies when every case is 2D, l2 or l1-wavelet, and
 *   the cases share one k-space and one maps storage type; otherwise the solve uses the
 *   per-case layout.  All cases spread with the single-pass interleaved-pair kernel.
 * On 64 uneven 2D cases (96..320 pixels, 4..32 coils) the per-case layout measured 7.1 ms per
 * iteration of all cases on a GB300 and the phase layout 8.7 ms. */
typedef enum { KP_BATCH_PER_CASE = 0, KP_BATCH_PHASES = 1 } kp_batch_form;
/* Selects the layout of later solves (the graph is captured again).  Errors: KP_EINVAL. */
kp_status kp_batch_set_form(kp_batch batch, kp_batch_form form);

/* Runs `iters` PDHG iterations (Sec. 4.1; Sec. 4.2 for KP_REG_TV cases) on every case of the
 * batch.  Arrays of length ncases:
 * y_devs[i] ([C_i][M_i] of type y_types[i]), p_devs[i] (float32 [C_i][M_i], or NULL entries /
 * a NULL array for the multi-channel preconditioner), regs[i], lambdas[i], x_devs[i]
 * (complex64 [N_i] output).  Start, step sizes and power method follow kp_pdhg_solve per case.
 * Set-up runs case by case, each case on its own stream; the 29 power iterations after the
 * first replay one graph of all cases.  The iteration of all cases is one CUDA graph in the
 * batch's form (captured on the first call and again when the form, regs, lambdas, y types or
 * a plan's buffers change), replayed `iters` times on `stream`.  Each case's result equals
 * that case's kp_pdhg_solve up to float32 rounding order.
 * Synchronous.  Errors: KP_EINVAL (iters < 0, an unknown regulariser, l1 case without wavelet
 * levels, non-positive p or lambda_max of some case), KP_ECUDA, KP_ECUFFT. */
kp_status kp_batch_solve(kp_batch batch, const void* const* y_devs, const kp_cdtype* y_types,
                         const float* const* p_devs, const kp_reg* regs, const float* lambdas, int iters,
                         void* const* x_devs, void* stream);

/* Frees the batch's streams, events and graph (not the plans).  Waits for the device. */
kp_status kp_batch_destroy(kp_batch batch);

/* Number of grid tiles and the longest tile's sample count after kp_plan_set_trajectory
 * (diagnostics for load balance). */
kp_status kp_plan_tile_stats(kp_plan plan, int64_t* ntiles, int64_t* max_tile_samples);

/* The spreading configuration the autotuner chose at the plan's first trajectory: kernel
 * variant (0: warp-private tile copies, 4 coils x 4 warps per CTA; 1: one shared accumulator
 * with shared-memory atomics, up to 16 coils per CTA; 2: one warp per 4 coils, all coils per
 * CTA; 3, 4, 5: warp-private copies with 2 coils x 8 warps, 1 coil x 8 warps, 2 coils x 4 warps;
 * 6, 7: warp-private copies of interleaved coil pairs, 4 coils x 4 or 8 warps; 8, 9 (3D): each
 * warp owns one z-plane of a single accumulator, 8 or 4 coils; 10, 11 (3D): two phases, padded
 * tiles of each tile's own samples then a gather over tiles, 8 or 4 coils; 12 (2D): the same two
 * phases with warp-private padded tiles of 4 coils),
 * samples per work item, number of work items and of split tiles (tiles cut into several items,
 * accumulated with global atomics).  Any pointer may be NULL.  KP_EINVAL before a trajectory
 * is set.  The environment variables KPDHG_SPREAD_VARIANT and KPDHG_SPREAD_CHUNK, read at that
 * moment, fix either choice instead of timing it. */
kp_status kp_plan_spread_config(kp_plan plan, int* variant, int* chunk, int64_t* n_items, int64_t* n_split);

#ifdef __cplusplus
}
#endif
#endif /* KPDHG_H */
