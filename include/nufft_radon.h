/*
 * nufft_radon.h -- C ABI of the GB300 NUFFT parallel-beam Radon library.
 *
 * The operators follow arXiv 2304.12934 (tomoCAM):
 *   A   = discrete Radon transform R (Sec. 2.1 Eq. radon_transform, Eq. line_eqn),
 *         evaluated through the Fourier-slice theorem (Eq. fourier_radon) with a
 *         NUFFT: row DFT, gridding on a 2x oversampled Cartesian grid, 2D FFT and
 *         deapodisation (Sec. 2.2 Eqs. nufft, nufft2, nufft3, run backwards, as Sec. 2.2 notes for the Radon transform).
 *   A^T = its exact adjoint R* (Sec. 3 Eq. transpose).
 *   MBIR objective  Phi(f) = 1/2 ||A f - b||_W^2 + lambda H(f)  (Sec. 3 Eq. objfn,
 *         gradient Eq. gradient), H the qGGMRF prior (Sec. 3 Eqs. reg2, reg3).
 *   Solver: accelerated gradient with restart (Sec. 3, last paragraph).
 *
 * Discrete conventions (shared by every entry point):
 *   image   x[b][iy][ix], float32, row-major, pixel centre (ix - N/2, iy - N/2)
 *   sinogram y[b][a][i], float32, detector coordinate t_i = i - D/2
 *   angle   theta_a (default a*pi/A); projection coordinate x cos(theta) + y sin(theta)
 *   A is the band-limited operator y(a,i) = sum_n f_n K_D(t_i - s_n(a)) with the
 *   Dirichlet kernel K_D of the length-D detector DFT (Nyquist bin weighted 1/2).
 *
 * Memory: every array argument is a DEVICE pointer unless stated otherwise; the
 * caller owns it.  The plan owns its own scratch (allocated in tc_plan_create).
 * Calls are asynchronous on the given stream (a cudaStream_t passed as void*,
 * NULL = legacy default stream) unless stated otherwise; an error detected on
 * the host is returned immediately, an asynchronous device error surfaces at a
 * later call or synchronisation.  No C++ exception crosses this interface.
 * A plan is not thread safe: calls on one plan must be serialised by the caller
 * (one stream at a time).
 */
#ifndef NUFFT_RADON_H
#define NUFFT_RADON_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
#define TC_OK                0
#define TC_ERR_INVALID_ARG  -1   /* bad size, NULL pointer, unsupported parameter */
#define TC_ERR_OOM          -2   /* device or host allocation failed */
#define TC_ERR_CUDA         -3   /* a CUDA runtime call failed */
#define TC_ERR_TIMEOUT      -4   /* a bounded device wait expired */
#define TC_ERR_UNSUPPORTED  -5   /* valid request this build does not implement */

/* Human-readable text for a status code (static storage, never NULL). */
const char *tc_status_string(int status);

/* Text of the last CUDA error seen by this library on this thread (or ""). */
const char *tc_last_error_detail(void);

/* ------------------------------------------------------------ geometry ---- */
/* Scan geometry of one family of slices (Sec. 2.1; Sec. 2.2 for sigma and w).
 *   n             image side N; power of two, 16 <= N <= 4096
 *   n_angles      A >= 1
 *   n_det         D; even, 4 <= D <= 16384.  tc_plan_create returns
 *                 TC_ERR_UNSUPPORTED when the detector DFT of one CTA would
 *                 exceed 200 KB of shared memory: lengths with a prime
 *                 factor > 32 use Bluestein with L = 2^k >= 2D - 1 (up to
 *                 L = 8192, i.e. D <= 4096), other lengths (and longer ones)
 *                 a mixed-radix DFT needing about 24 D bytes (D <~ 8500)
 *   angles        HOST pointer to A angles in radians, or NULL for a*pi/A;
 *                 copied during tc_plan_create
 *   oversample    sigma, the grid oversampling factor; must be 2
 *   kernel_width  w, spreading-kernel width in grid points (Sec. 2.2: w about
 *                 log10(1/eps)); 2 <= w <= 8; 7 gives ~1e-6 relative error
 *   center_offset delta, rotation-axis offset in detector bins: the axis
 *                 projects to detector coordinate D/2 + delta, so pixel x_n
 *                 lands at t = s_n(theta) + delta.  Applied as the Fourier
 *                 shift exp(-2 pi i m delta / D) of every projection's
 *                 spectrum (Sec. 4.1, axis correction by the shift property);
 *                 the adjoint applies the conjugate phase.  Finite and
 *                 |delta| <= D/2, else TC_ERR_INVALID_ARG.  0 (a
 *                 zero-initialised struct) means the axis at the centre.
 */
typedef struct {
    int n;
    int n_angles;
    int n_det;
    const double *angles;
    int oversample;
    int kernel_width;
    double center_offset;
} tc_geom;

typedef struct tc_plan tc_plan;

/* Build a plan: FP64 deapodisation factors, polar-point gridding tables sorted
 * into per-row bins, twiddle tables, and scratch for max_batch slices per
 * launch (larger batches are processed in chunks of max_batch).  Synchronous.
 * Allocates device memory with cudaMalloc on the current device.
 * Returns TC_OK and *out, or an error (and *out = NULL). */
int tc_plan_create(const tc_geom *geom, int max_batch, tc_plan **out);

/* Release a plan and its device memory (synchronises the device first).
 * NULL is accepted. */
int tc_plan_destroy(tc_plan *plan);

/* Device bytes held by the plan (tables + scratch). */
long long tc_plan_device_bytes(const tc_plan *plan);

/* Launch-shape autotuner (an engineering addition; the paper has none).
 * Times radon_fwd + radon_adj on the caller's buffers for every candidate of
 *   chunk      slices per launch: max_batch, max_batch/2, ..., 1 (smaller
 *              chunks keep the grid rows of the column pass in L2 for the
 *              row pass), and
 *   col_pairs  image column pairs per CTA of the column passes (1, 2, 4),
 * keeps the fastest in the plan and reports it (chunk_out, cp_out: HOST, may
 * be NULL).  x [batch][N][N] and y [batch][A][D] are DEVICE scratch buffers
 * (overwritten).  Synchronous.  The operators' outputs do not depend on the
 * choice (bit-identical images and sinograms; only the summation order of the
 * FP64 objective across chunks changes).  reps: timed repetitions per
 * candidate (>= 1). */
int tc_plan_autotune(tc_plan *plan, const float *x, float *y, int batch, int reps,
                     int *chunk_out, int *cp_out, void *stream);

/* Set the launch shape directly: chunk in [1, max_batch]; col_pairs 1, 2, 4
 * (0 keeps the current value).  Returns TC_ERR_INVALID_ARG if unsupported. */
int tc_plan_set_launch(tc_plan *plan, int chunk, int col_pairs);

/* Entries per chunk of the spreading pass (A^T): 256, 512 or 1024 (the
 * default).  Each grid row's key-sorted entries are staged in shared memory
 * one chunk at a time, with one gather record per touched cell and chunk;
 * larger chunks need fewer records and barriers, smaller ones less shared
 * memory.  Rebuilds the record tables (host, then upload; synchronises the
 * device).  A cell's contributions are summed chunk by chunk, so a different
 * chunk regroups that FP32 sum: A^T changes at the rounding level only (each
 * chunk size on its own is bit-reproducible).  TC_ERR_INVALID_ARG for other
 * sizes. */
int tc_plan_set_spread_chunk(tc_plan *plan, int entries);
/* The plan's current spreading chunk (or TC_ERR_INVALID_ARG for NULL). */
int tc_plan_get_spread_chunk(const tc_plan *plan);
/* Autotuner of the spreading chunk: times radon_adj of y [batch][A][D] into
 * x [batch][N][N] (DEVICE scratch, overwritten) reps times for each chunk
 * size and keeps the fastest (reported in *chunk_out, HOST, may be NULL).
 * Synchronous. */
int tc_plan_autotune_spread(tc_plan *plan, const float *y, float *x, int batch, int reps,
                            int *chunk_out, void *stream);

/* --------------------------------------------------------------- operators */
/* y = A x  (Sec. 2.2 NUFFT steps in reverse order).
 *   x  [batch][N][N] float32 in;  y [batch][A][D] float32 out (overwritten).
 *   batch >= 0 (0 is a no-op).  x and y must not overlap. */
int radon_fwd(tc_plan *plan, const float *x, float *y, int batch, void *stream);

/* x = A^T y  (Sec. 3 Eq. transpose; exact adjoint of radon_fwd's operator).
 *   y  [batch][A][D] float32 in;  x [batch][N][N] float32 out (overwritten). */
int radon_adj(tc_plan *plan, const float *y, float *x, int batch, void *stream);

/* x_out = A^T A x, the Hessian of the unweighted data term (Sec. 3 Eqs.
 * gradient and transpose), without gridding.  For even D (with the Nyquist
 * pair weighted 1/2, as in radon_fwd) the detector-bin sum of two shifted
 * Dirichlet kernels is exact in closed form, which makes A^T A Toeplitz plus
 * Hankel in the pixel coordinates:
 *   (A^T A x)(p') = sum_p x(p) [T(p' - p) + H(p' + p)],
 *   T(d) = sum_a K(s_d(a)) - cos(pi s_d(a)) / 2D,
 *   H(e) = sum_a cos(pi (s_e(a) + 2 delta)) / 2D,
 * with s_d(a) = d_x cos(theta_a) + d_y sin(theta_a) and K the Dirichlet
 * kernel.  Both are convolutions on the 2N-periodic grid: one 2D FFT of the
 * image (half plane), a pointwise product with the precomputed spectra of T
 * and H, and the inverse 2D FFT at the N x N pixels.  The result equals
 * radon_adj(radon_fwd(x)) up to FP32 rounding and the NUFFT's own kernel
 * error, and costs no interpolation, spreading or detector transforms.
 *   x, x_out  [batch][N][N] float32 DEVICE (may be the same buffer).
 * The first call on a plan builds the spectra (FP64, synchronous on the
 * stream; device memory about 12 (N+1) 2N bytes, plus a 16 (2N)^2-byte
 * temporary), as tc_plan_prepare_normal does; later calls are asynchronous. */
int radon_normal(tc_plan *plan, const float *x, float *x_out, int batch, void *stream);

/* Builds the spectra of radon_normal's kernels if not yet built (idempotent,
 * synchronous).  Call it before capturing radon_normal into a CUDA graph. */
int tc_plan_prepare_normal(tc_plan *plan, void *stream);

/* ---------------------------------------------------------------- prior --- */
/* qGGMRF prior (Sec. 3 Eqs. reg2, reg3; defaults of Sec. 5):
 *   H(f) = sum_m sum_{n in N(m)} w_mn rho(f_m - f_n),
 *   rho(d) = (|d|/sigma)^2 / (c + (|d|/sigma)^(2-p)),
 *   w_mn proportional to 1/||m-n|| and summing to one over the neighbourhood.
 *   dims = 2: 8 in-plane neighbours; dims = 3: 26 neighbours across slices
 *   (slices of one call are consecutive along z).  Neighbours outside the
 *   volume are left out without renormalising the weights.
 *   lambda >= 0 scales H in the objective (0 disables the prior). */
typedef struct {
    double p;       /* 1.2 */
    double sigma;   /* 1/0.7 */
    double c;       /* 1e-4 */
    double lambda;  /* 1.0 */
    int dims;       /* 2 or 3 */
} tc_prior;

/* ----------------------------------------------------------------- MBIR --- */
/* Gradient of Phi at x (Sec. 3 Eq. gradient plus the prior gradient):
 *   grad = A^T W (A x - b) + lambda grad H(x)
 *   b      [batch][A][D] measured sinogram (Beer-Lambert, Sec. 5)
 *   w      [batch][A][D] statistical weights, or NULL for W = I
 *   prior  HOST pointer, or NULL for no prior
 *   grad   [batch][N][N] out
 *   obj    DEVICE pointer to 2 doubles or NULL: obj[0] = 1/2 sum W (Ax-b)^2,
 *          obj[1] = lambda H(x); FP64 reductions in a fixed order. */
int mbir_grad(tc_plan *plan, const float *x, const float *b, const float *w,
              const tc_prior *prior, float *grad, double *obj, int batch,
              void *stream);

/* Largest eigenvalue of A^T W A by power iteration (step-size estimate).
 *   v      [batch][N][N] start vector in (must be nonzero), last iterate out
 *   work   [batch][N][N] scratch
 *   w      weights or NULL
 *   lam_out HOST pointer: last Rayleigh quotient <v, A^T W A v>, ||v|| = 1.
 * Synchronises the stream before returning. */
int mbir_power_norm(tc_plan *plan, const float *w, float *v, float *work,
                    int batch, int n_iter, double *lam_out, void *stream);

/* Accelerated gradient with restart (reading of Sec. 3's "monotonic
 * accelerated gradient method with restart"), v = z_k - step * grad Phi(z_k):
 *   restart = 1 (gradient test):  x_{k+1} = v;
 *       if <grad Phi(z_k), x_{k+1} - x_k> > 0 then t_k := 1
 *   restart = 2 (monotone, function-value test): x_{k+1} = v if Phi(v) <=
 *       Phi(x_k), else x_{k+1} = x_k and t_k := 1, so Phi(x_k) never
 *       increases; costs one more forward projection and prior value per
 *       iteration, and Phi(x) once per call
 *   restart = 0: x_{k+1} = v (plain FISTA momentum)
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
 *   z_{k+1} = x_{k+1} + ((t_k - 1) / t_{k+1}) (x_{k+1} - x_k)
 * All scalars (objective, inner products, t, momentum, the accept test) are
 * FP64 on the device; no host round trip inside the loop. */
typedef struct {
    int n_iter;      /* iterations to run in this call (>= 0) */
    double step;     /* > 0: the constant step 1/L, with L >= ||A^T W A|| + lambda * 8/(sigma^2 c).
                        <= 0: the library derives it (reading of Sec. 3: a constant step 1/L):
                        L = 1.05 lambda_max + lambda * 8 / (sigma^2 c), lambda_max the largest
                        eigenvalue of A^T W A by power_iter power iterations over the whole batch
                        from a seeded start (FP64 norms on the device), the prior term the bound
                        4 max rho'' = 8 / (sigma^2 c) on the Hessian of H with unit-sum weights.
                        The derivation runs when state->k == 0, using state->z and state->g as
                        its work vectors before the iteration starts, and the step is returned
                        in state->step; a resumed call (state->k > 0) with step <= 0 reuses
                        state->step (TC_ERR_INVALID_ARG when that is not > 0). */
    int restart;     /* 0, 1 or 2 as above; anything else is TC_ERR_INVALID_ARG */
    int normal;      /* 1: unweighted data term (w must be NULL) through radon_normal's
                        embedding: grad = A^T A z - A^T b, with A^T b (in state->atb)
                        and ||b||^2 formed once per call.  Restart 0 or 1 only; the
                        reported data term 1/2 <z, A^T A z> - <z, A^T b> + 1/2 ||b||^2
                        loses relative precision as the residual vanishes.  The first
                        normal-mode call builds the embedding's tables (allocating and
                        synchronising): call tc_plan_prepare_normal before capturing a
                        normal-mode solve into a CUDA graph (inside a capture the
                        unprepared call returns TC_ERR_UNSUPPORTED).  0: the gridded
                        operators. */
    int power_iter;  /* power iterations of a derived step (0: 30) */
} tc_solve_opts;

/* Solver state; resuming with the same state continues the iteration exactly.
 *   z, g   caller-owned DEVICE buffers [batch][N][N] (momentum point; g is
 *          scratch: the gradient or the next momentum point, depending on the
 *          step).  A solve with a prior may exchange the two pointers (see
 *          mbir_solve): z always names the momentum point on return
 *   t      momentum scalar t_k (host copy, updated on return)
 *   k      iterations completed; k == 0 starts fresh (z := x, t := 1)
 *   n_restarts  restarts taken so far (monotone variant: rejected steps)
 *   obj    objective terms (data, lambda H) at the last gradient point z;
 *          with restart = 2, at the returned x
 *   atb    with opts->normal: caller-owned DEVICE buffer [batch][N][N] that
 *          receives A^T b (else ignored, may be NULL) */
typedef struct {
    float *z;
    float *g;
    double t;
    int k;
    int n_restarts;
    double obj[2];
    float *atb;
    double step;     /* the step the iteration used (set on return; input for a resumed
                        call whose opts->step <= 0) */
    double dots[2];  /* set on return (restart 0 or 1; 0 for restart 2): the inner products
                        of the last iteration's restart test, <grad Phi(z_k), z_k - x_k> and
                        <grad Phi(z_k), grad Phi(z_k)>, reduced on the device from the FP32
                        vectors with error-free products and compensated sums (as exact as
                        an FP64 reduction of the same vectors) */
} tc_solve_state;

/* Run opts->n_iter iterations on device buffers.
 *   b, w   [batch][A][D] (w may be NULL);  x [batch][N][N] in/out.
 * With a prior (lambda != 0) and restart 0 or 1, each iteration forms z_{k+1}
 * inside the prior pass: x_{k+1} is written over x_k and the momentum point
 * of an iteration without restart over the gradient buffer, so the buffers
 * behind state->z and state->g exchange roles every iteration (after a
 * restart a check-and-copy kernel sets z_{k+1} = x_{k+1}).  On return x holds
 * x_k, and the call may have EXCHANGED the pointers state->z and state->g:
 * state->z then names the buffer that holds z_k (read the pointers back
 * after every call; on an error return the state is undefined).
 * Synchronises the stream before returning (to fill the host fields of state). */
int mbir_solve(tc_plan *plan, const float *b, const float *w, float *x, int batch,
               const tc_prior *prior, const tc_solve_opts *opts,
               tc_solve_state *state, void *stream);

/* Same solve, end to end from HOST memory: b_host, w_host (or NULL) and
 * x_host are HOST pointers (page-locked memory gives asynchronous copies);
 * dev_b, dev_w, dev_x are caller-owned DEVICE buffers of the same sizes that
 * receive the copies.  Inputs are copied host-to-device in slabs of max_batch
 * slices on a copy stream, and the result comes back on another (both
 * created and destroyed by the call); the first iteration's chunk c starts as
 * soon as slab c is resident (for a resumed solve with a prior, as soon as its
 * b and w are: only the prior reads x, and it waits for its slab), so the
 * copies overlap the first iteration's Radon work, and in the last iteration
 * (gradient restart or plain momentum with a prior) each slab's result leaves
 * as soon as its prior is done.  The result x is copied
 * back to x_host and is also left in dev_x.  Synchronises before returning. */
int mbir_solve_host(tc_plan *plan, const float *b_host, const float *w_host,
                    float *x_host, float *dev_b, float *dev_w, float *dev_x,
                    int batch, const tc_prior *prior, const tc_solve_opts *opts,
                    tc_solve_state *state, void *stream);

/* ------------------------------------------------------- plan groups ------ */
/* Uneven batches (an engineering addition for batches of slices whose image
 * side, angle count or detector width differ; the paper reconstructs one
 * geometry at a time).  A group holds one plan per geometry, sized for all of
 * that geometry's slices (counts[i] slices of geoms[i]), and a work list per
 * pipeline stage over every (geometry, slice, tile) item.  Each stage runs as
 * one launch per geometry class (the geometries of one image side and, for
 * the detector passes, one detector-transform kind), one CTA per item, with up
 * to four geometries in the launch's parameter block and the costliest items
 * first.  The class launches of a stage, and the per-geometry prior launches,
 * are independent and run side by side on up to 7 streams the group owns,
 * forked from and joined back into the caller's stream with events.  Stage
 * boundaries are kernel boundaries (no CTA waits for another).
 * Results are those of the per-geometry plans to within 1e-6 relative (the
 * group kernels are separate compilations of the same pass bodies, so a
 * multiply-add may be fused differently), and deterministic.
 * Arrays of a group are the geometries' slices concatenated in the order
 * given: images geoms[0] x counts[0] slices of N0 x N0, then geoms[1]'s, ...;
 * sinograms likewise with A_i x D_i.  Calls are asynchronous, capturable into
 * a CUDA graph once the group exists, and not thread safe per group.
 * tc_plan_group_create allocates (synchronous); 1 <= n_geoms <= 256 and
 * 1 <= counts[i] <= 65535, each geometry as for tc_plan_create. */
typedef struct tc_plan_group tc_plan_group;
int tc_plan_group_create(const tc_geom *geoms, const int *counts, int n_geoms, tc_plan_group **out);
int tc_plan_group_destroy(tc_plan_group *group);
long long tc_plan_group_device_bytes(const tc_plan_group *group);
/* y = A x and x = A^T y for every slice of the group (concatenated layouts). */
int radon_fwd_group(tc_plan_group *group, const float *x, float *y, void *stream);
int radon_adj_group(tc_plan_group *group, const float *y, float *x, void *stream);
/* grad = A^T W (A x - b) + lambda grad H(x) for every slice, the prior over
 * each geometry's slices as one volume (dims = 3) or slice by slice (dims =
 * 2); w may be NULL (W = I), prior may be NULL.  obj: DEVICE pointer to
 * 2 n_geoms doubles or NULL: obj[2 i] = 1/2 sum W (A x - b)^2 and
 * obj[2 i + 1] = lambda H(x) of geometry i. */
int mbir_grad_group(tc_plan_group *group, const float *x, const float *b, const float *w,
                    const tc_prior *prior, float *grad, double *obj, void *stream);

/* --------------------------------------------------------- checkpoints --- */
/* Solver checkpoint on storage (no counterpart in the paper, whose solver
 * state lives in host memory between partitions, Sec. 4; it lets a long solve
 * stop and resume in another process).  One file: a one-line JSON header
 * (ASCII, ending in a newline) naming the format, the geometry (n, n_angles,
 * n_det), batch, the scalar state (k, t, n_restarts, step, obj, each double
 * printed with 17 significant digits, which round-trips exactly), followed by
 * the raw float32 arrays x then z, [batch][N][N] each, in the host's byte
 * order (little-endian on the supported machines).
 *   tc_checkpoint_save: x (DEVICE) and state->z are copied to the host in
 *     bounded chunks and written to `path` (created or truncated).
 *   tc_checkpoint_load: reads `path` back into x and state->z (DEVICE) and the
 *     scalar fields of state; the header must match the plan's geometry and
 *     batch, else TC_ERR_INVALID_ARG (checked before any device copy).
 * A solve resumed from a loaded checkpoint continues exactly as the
 * uninterrupted solve would (state->g and state->atb are scratch at the start
 * of every call).  Both synchronise `stream`.  Host I/O failures return
 * TC_ERR_INVALID_ARG (unreadable or malformed file) or TC_ERR_CUDA. */
int tc_checkpoint_save(const char *path, const tc_plan *plan, const float *x, int batch,
                       const tc_solve_state *state, void *stream);
int tc_checkpoint_load(const char *path, const tc_plan *plan, float *x, int batch,
                       tc_solve_state *state, void *stream);

/* --------------------------------------------------------- testing hooks -- */
/* Failure injection on the host (for tests of the error paths; no GPU fault
 * is involved).  After `after` more host-to-device or device-to-host copies
 * issued by mbir_solve_host, the next one is not issued and reports a CUDA
 * failure instead, as if cudaMemcpyAsync had returned an error; the call then
 * waits for the copies already in flight and returns TC_ERR_CUDA.  A negative
 * value switches injection off (the default).  Process wide. */
int tc_test_fail_copy_after(int after);

/* ------------------------------------------------------------ profiling --- */
/* Per-kernel device timing with CUDA events (no counterpart in the paper; it
 * supports the roofline measurements).  While enabled, every kernel launch of
 * this library is bracketed by two events on its stream.  Enabling (or
 * re-enabling) discards earlier records. */
int tc_profile_enable(int on);

/* Synchronises the recorded events and fills counts[i] (launches) and ms[i]
 * (summed device milliseconds) for kernel ids i < max_kernels (HOST arrays).
 * Returns the number of kernel ids the library defines, or an error. */
int tc_profile_collect(int max_kernels, long long *counts, double *ms);

/* Name of kernel id (static storage; "" for an unknown id). */
const char *tc_profile_kernel_name(int id);

/* Kernel launches issued by this library since it was loaded (host counter). */
long long tc_launch_count(void);

/* Throughput of the special-function unit on the current device (no
 * counterpart in the paper; it is the roof of the prior kernel, whose pair
 * evaluations take one lg2, one ex2 and one rcp per cell): op 0 lg2.approx,
 * 1 ex2.approx, 2 rcp.approx.  Runs independent chains of the operation on
 * 8 CTAs of 256 threads per SM and returns lane operations per second in
 * *lane_ops_per_s (HOST).  Synchronous on `stream`; allocates nothing on the
 * device.  TC_ERR_INVALID_ARG for another op or a NULL output. */
int tc_sfu_throughput(int op, double *lane_ops_per_s, void *stream);

/* ------------------------------------------------------ device status --- */
/* Kernels that wait on a device barrier (the TMA-staged forward column pass)
 * bound each wait to one second; on expiry they record TC_ERR_TIMEOUT in the
 * plan's device status and return early, leaving their outputs incomplete.
 * mbir_solve, mbir_solve_host and mbir_power_norm (which synchronise)
 * report that status when they return; after radon_fwd, radon_adj or
 * mbir_grad (asynchronous), tc_plan_status synchronises the device, returns
 * the status (TC_OK or TC_ERR_TIMEOUT) and clears it. */
int tc_plan_status(tc_plan *plan);

/* Self-test of the bounded wait: one kernel waits on a barrier that never
 * completes, with a 2 ms limit.  Returns TC_ERR_TIMEOUT when the wait
 * expired and the kernel returned as designed (the context stays usable);
 * synchronises the given stream. */
int tc_selftest_wait_timeout(void *stream);

/* ------------------------------------------------------ no allocation --- */
/* Prior gradient and value without any device allocation.  There is no
 * counterpart of this entry point in the paper; it exists for callers that
 * cannot call cudaMalloc -- for example code running under a framework whose
 * caching allocator owns the device memory budget, or a latency-critical loop
 * that must not risk the implicit device synchronisation of an allocation --
 * and who therefore cannot create a plan.
 *
 * Computes the qGGMRF prior of the tc_prior block (same definition and kernel
 * as the prior inside mbir_grad):
 *   grad += lambda * grad H(x)       (accumulated into the caller's grad)
 *   *h_out = lambda * H(x)           (h_out: DEVICE pointer to one double, or NULL)
 *   x, grad  DEVICE float32 [batch][n][n], 16-byte aligned, caller-owned;
 *            they must not overlap (the kernel writes grad at one slice while
 *            other blocks still read x at the slices above and below), else
 *            TC_ERR_INVALID_ARG
 *   1 <= n <= 4096, 1 <= batch <= 65535; anything else returns TC_ERR_INVALID_ARG.
 * Scratch: the per-block FP64 partial sums live in a fixed array of 65536
 * doubles (512 KiB) declared at file scope in the library's device code; every
 * GPU that loads the library holds it until the process exits.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current) and caches it, so make the first call on each device
 * before any stream capture.  All calls share the array and each call
 * overwrites the part it uses (nothing has to start at zero), so calls that
 * overlap on the GPU (concurrent streams) race and must be serialised.
 * Asynchronous on `stream`; calls no cudaMalloc, cudaFree or allocating
 * library routine, and records no profiler events (tc_profile_enable does not
 * apply to it: its launches are counted by tc_launch_count only). */
int tc_prior_grad_noalloc(const float *x, float *grad, int n, int batch,
                          const tc_prior *prior, double *h_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NUFFT_RADON_H */
