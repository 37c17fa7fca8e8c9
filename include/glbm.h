/*
 * glbm.h - C ABI of the GB300 generalized lattice Boltzmann model (GLBM)
 * library: gas flow through a voxelised two-phase shale matrix in which every
 * lattice node carries its own porosity eps(x) and apparent permeability
 * K(x), after Wang, Chen, Kang & Rahman, arXiv:1601.00704, Sec. 2.3.
 *
 * One time step (Eq. 29) is: pull-stream the distributions, form rho and the
 * first moment (Eqs. 32-33), the temporal velocity v (Eq. 35), the node
 * velocity u from the explicit quadratic solve (Eq. 34 with c0, c1 of
 * Eqs. 36-37), the total body force F (Eq. 27; Eq. 28 when F_eps = 0), the
 * porosity-weighted equilibrium (Eq. 30) and the forcing term (Eq. 31), then
 * BGK-collide.  The loop repeats until the mean velocity converges; the
 * sample's apparent permeability then follows from Darcy's law.
 *
 * Conventions (all entry points):
 *  - Lattice units: dx = dt = c = 1, D2Q9, c_s^2 = 1/3, nu = (tau - 1/2)/3.
 *  - Arrays are row-major [ny][nx] (x fastest), FP64, unless stated.
 *  - Pointer arguments are BORROWED for the duration of the call: the caller
 *    keeps ownership; nothing is retained.  `device_ptrs != 0` means the
 *    arrays live in device memory of the handle's GPU, else host memory.
 *  - The handle OWNS all device memory it allocates (distribution buffers,
 *    packed coefficients, reduction scratch) and frees it in glbm_destroy.
 *  - No C++ exception crosses this boundary.  Every entry point returns a
 *    glbm_status; on failure glbm_last_error() describes it and the handle's
 *    state is unchanged unless stated.
 *  - A handle is not thread-safe; use one handle per host thread / stream.
 *    Work is enqueued on the stream given to glbm_create.
 *  - The solver and batch entry points (set_medium, init_equilibrium, step,
 *    mean_velocity, permeability, save, load, batch_set_medium, batch_step)
 *    each open an NVTX range of their own name for a profiler's timeline;
 *    without a tool attached the ranges record nothing.
 */
#ifndef GLBM_H
#define GLBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glbm *glbm_t;

typedef enum {
    GLBM_OK = 0,
    GLBM_EINVAL = -1, /* bad argument (size, range, NaN, missing force) */
    GLBM_ENOMEM = -2, /* device or pinned allocation failed */
    GLBM_ECUDA = -3,  /* a CUDA runtime call or kernel launch failed */
    GLBM_ENAN = -4,   /* a non-finite mean velocity was detected */
    GLBM_ESTATE = -5  /* call not valid in the current state */
} glbm_status;

/* Storage precision of the distributions.  Collision arithmetic runs in
 * FP32 for the 32/16-bit formats and FP64 for GLBM_F64; the convergence
 * reduction always accumulates in FP64.  All formats store deviations
 * g_i = f_i - w_i * rho0 (rho0 = 1) rather than f_i.  The 16-bit formats
 * round stochastically by default (a counter-based hash of node, step and
 * population decides each rounding direction, so runs are reproducible):
 * nearest rounding freezes the slow pressure mode once its per-step change
 * falls below half an ulp.  FP16 stores g*S with a power-of-two scale S that
 * the library chooses from G (or the warm-start state) and then keeps the
 * largest stored magnitude between 2^8 and 2^13, checked at the end of
 * every chunk (so FP16 runs read a status back every chunk); BF16 has
 * FP32's exponent range and stores g unscaled. */
typedef enum {
    GLBM_F32 = 0,
    GLBM_F64 = 1,
    GLBM_F16DEV = 2,  /* FP16 deviations times a power-of-two scale */
    GLBM_BF16DEV = 3  /* BF16 deviations times a power-of-two scale */
} glbm_storage;

/* Boundary flags (the paper states none; see glbm_create). */
#define GLBM_WALLS_Y 0u    /* halfway bounce-back walls at y=-1/2, ny-1/2 */
#define GLBM_PERIODIC_Y 1u /* periodic in y */
/* 16-bit storage rounds to nearest instead of stochastically (for studies of
 * the stagnation that nearest rounding causes; not recommended). */
#define GLBM_NEAREST16 2u

/*
 * Create a solver for an nx-by-ny lattice (x is always periodic).
 *   tau      BGK relaxation time (Eq. 29), must be > 1/2.
 *   storage  distribution storage format (above).
 *   flags    GLBM_WALLS_Y (default) or GLBM_PERIODIC_Y, optionally or-ed
 *            with GLBM_NEAREST16.
 *   stream   cudaStream_t to enqueue on; NULL = the legacy default stream.
 *   out      receives the handle.
 * Allocates both distribution buffers, the coefficient planes and the
 * reduction scratch on the current CUDA device.  nx, ny >= 2 and
 * nx*ny < 2^31.  Errors: EINVAL, ENOMEM, ECUDA.
 */
glbm_status glbm_create(int nx, int ny, double tau, glbm_storage storage,
                        unsigned flags, void *stream, glbm_t *out);

/*
 * Load the medium: per-node porosity eps in (0, 1] and apparent permeability
 * K > 0 (+inf = clear fluid), each [ny][nx] FP64.  F_eps selects the
 * Forchheimer geometric function of Eq. 27, which the paper leaves unset:
 * 0 = none (the paper's Eq. 28), > 0 = that constant, < 0 = Ergun's
 * 1.75/sqrt(150 eps^3) per node.  Packs the per-node coefficients
 * (eps*nu/K, eps and, with F_eps != 0, eps*F_eps/sqrt(K); Eqs. 36-37) on the
 * device, resets the distributions to f_eq(rho = 1, u = 0), the step count to
 * zero and the convergence history.  Invalid values: EINVAL, state unchanged.
 */
glbm_status glbm_set_medium(glbm_t h, const double *eps, const double *K,
                            double F_eps, int device_ptrs);

/* External body force G (per unit mass, lattice units) of Eq. 27.  Keeps the
 * distributions; clears the convergence history. */
glbm_status glbm_set_force(glbm_t h, double gx, double gy);

/*
 * Warm start: set the distributions to the porosity equilibrium of Eq. 30,
 * f_i = f_eq_i(rho, u; eps), per node.  rho may be NULL (rho = 1); ux and uy
 * must both be given or both NULL (u = 0).  Resets the step count and the
 * convergence history.  Requires a medium (ESTATE otherwise).
 */
glbm_status glbm_init_equilibrium(glbm_t h, const double *rho,
                                  const double *ux, const double *uy,
                                  int device_ptrs);

/*
 * Advance at most n steps.  The steps run in chunks of check_every; the mean
 * velocity U (FP64 over all nodes, the Eq. 34 velocities of that step) is
 * formed at the end of every chunk when tol > 0, and at the end of the call
 * in any case.  With tol > 0 the call stops once
 * |Ux - Ux_prev| <= tol * |Ux| (Ux_prev = the previous such value, kept
 * between calls) and reads a 32-byte status back after each chunk; with
 * tol <= 0 it runs exactly n steps and returns without waiting for the GPU.
 *   steps_done, converged  (out, may be NULL)
 * Errors: ESTATE (no medium), EINVAL (n < 0, check_every < 1), ENAN (the
 * state is kept for inspection), ECUDA.
 */
glbm_status glbm_step(glbm_t h, long long n, double tol, int check_every,
                      long long *steps_done, int *converged);

/*
 * Convergence test of glbm_step: converged once `patience` CONSECUTIVE
 * checks each pass |Ux - Ux_prev| <= tol * |Ux| (default 1: the first pass).
 * With 16-bit storage the stochastic rounding leaves a noise floor on Ux:
 * near that floor two checks can agree by chance while the slow mode is
 * still drifting, and a patience of a few checks guards against such early
 * stops.  The count of passes so far is kept between glbm_step calls and
 * cleared with the history (set_medium, set_force, init_equilibrium).
 * EINVAL unless 1 <= patience <= 1e6.
 */
glbm_status glbm_set_convergence(glbm_t h, int patience);

/* Mean velocity (Ux, Uy) of the last completed step; waits for the stream.
 * ESTATE before the first step, ENAN if it is not finite. */
glbm_status glbm_mean_velocity(glbm_t h, double out[2]);

/* Darcy apparent permeability of the sample, K_app = nu * Ux / Gx in lattice
 * units (multiply by dx^2 for physical units).  EINVAL if Gx = 0. */
glbm_status glbm_permeability(glbm_t h, double *kxx);

/* The Eq. 34 velocity field of the last completed step, [ny][nx] FP64 each
 * (recomputed from the pre-step state with the step's own arithmetic). */
glbm_status glbm_get_velocity(glbm_t h, double *ux, double *uy,
                              int device_ptrs);

/* The current post-collision distributions as absolute f_i in FP64,
 * laid out [9][ny][nx] with the D2Q9 order e0=(0,0), e1..e4=(1,0),(0,1),
 * (-1,0),(0,-1), e5..e8=(1,1),(-1,1),(-1,-1),(1,-1). */
glbm_status glbm_get_distributions(glbm_t h, double *f, int device_ptrs);

/* Steps since the last reset, and the number of kernels this handle has
 * launched in total (either pointer may be NULL). */
glbm_status glbm_counters(glbm_t h, long long *steps, long long *launches);

/*
 * One FP32 time step plus the mean-velocity reduction, without allocating.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory themselves, such as applications whose host
 * framework owns the whole device-memory budget and hands out every buffer,
 * or pipelines that must not risk the implicit device synchronisation that
 * cudaMalloc/cudaFree can cause in the middle of their loop.  It runs the
 * same fused step kernel as glbm_step on buffers the caller owns; the
 * kernel's reduction scratch (one FP64 pair per block, plus a 40-byte status)
 * is a fixed 1 MiB array compiled into the library, held on every GPU that
 * loads it until the process exits.  No cudaMalloc, cudaFree or allocating
 * library routine is called.
 *
 *   g_src   device, FP32 deviations g_i = f_i - w_i of the current
 *           post-collision state, laid out [9][plane] (plane i holds node
 *           y*nx + x), D2Q9 order as in glbm_get_distributions.  Read only.
 *   g_dst   device, same layout, receives the state after the step; must not
 *           overlap g_src or the coefficient arrays.  Start from zeros for
 *           f_eq(rho = 1, u = 0).
 *   alpha   device [ny][nx] FP32: eps*nu/K per node, nu = (tau - 1/2)/3
 *           (0 for K = +inf).
 *   eps     device [ny][nx] FP32 porosity.
 *   beta    device [ny][nx] FP32 eps*F_eps/sqrt(K), or NULL for the paper's
 *           Forchheimer-free model.
 *   plane   elements per population plane: >= nx*ny and a multiple of 4;
 *           every array must be 16-byte aligned.
 *   flags   GLBM_WALLS_Y or GLBM_PERIODIC_Y.
 *   mean_u  device, 2 doubles: receives (Ux, Uy) of this step.
 *   stream  cudaStream_t (NULL = legacy default stream); all work is
 *           enqueued on it and the call returns without waiting.
 *
 * Limit: the lattice may need at most 65536 reduction blocks, where one
 * block covers 512 nodes of a row when nx is a multiple of 4 (else 128):
 * e.g. 4096 x 8192 fits.  Larger lattices, misaligned arrays, a g_dst or
 * mean_u that overlaps any array the step reads (g_src, alpha, eps, beta;
 * mean_u may not overlap g_dst either) and other bad arguments return
 * GLBM_EINVAL with a message in glbm_last_error(NULL).
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: a cudaDeviceReset (or anything else that destroys and recreates
 * the device's primary context) may move the array and leave the kept
 * address stale, so do not call this entry point on a device after resetting
 * it.  Every call shares the one scratch array, which keeps the last call's
 * contents (the status is cleared at the start of each call): calls that
 * overlap on the GPU, e.g. on two streams at once, race.
 */
glbm_status glbm_step_reduce_noalloc(const float *g_src, float *g_dst,
                                     const float *alpha, const float *eps,
                                     const float *beta, int nx, int ny,
                                     long long plane, double tau, double gx,
                                     double gy, unsigned flags,
                                     double *mean_u, void *stream);

/*
 * Checkpoint and resume (no counterpart in the paper: long runs of the time
 * loop are restartable).  glbm_save writes the handle's current
 * distributions, packed medium coefficients, body force, step counts, FP16
 * scale, stochastic-rounding seed and convergence history to the file
 * `path` (overwritten), with a checksum; it waits for the stream.
 * glbm_load reads such a file into a handle created with the same nx, ny,
 * tau, storage and flags (no glbm_set_medium needed) and replaces its whole
 * state; continuing from there gives the same bits as the run that was
 * saved would have.  The file is host-endian and not meant to move between
 * machines of different byte order.
 * Errors: EINVAL (cannot open/read/write, not a checkpoint, another
 * geometry or format, checksum mismatch; the handle is then unchanged),
 * ESTATE (save before any medium), ECUDA.
 */
glbm_status glbm_save(glbm_t h, const char *path);
glbm_status glbm_load(glbm_t h, const char *path);

/* Release all device memory of the handle.  NULL-safe. */
void glbm_destroy(glbm_t h);

/*
 * Test hook for the error paths (no counterpart in the paper): the kernel
 * launch of glbm_step or glbm_batch_step that comes `after` launches from
 * now (0 = the next one) is refused on the host with GLBM_ECUDA, as a
 * rejected cudaLaunchKernelEx would be, without calling CUDA, so nothing
 * faults.  A refusal while a chunk is being captured into a CUDA graph ends
 * and discards the capture and leaves the handle's state, step count and
 * launch count as they were before that chunk.  after < 0 switches the hook
 * off (the default).  Process-wide; not for production use.
 */
void glbm_debug_fail_launch(long long after);

/*
 * Memory-safety check without a sanitizer (no counterpart in the paper):
 * every device buffer a handle allocates (distributions, coefficients,
 * reduction scratch, status words, input staging) carries 4 KB guard zones
 * before and after it, filled with the byte 0xA5 when allocated.  Sets
 * *damaged to the number of guard bytes that no longer hold it: 0 unless a
 * kernel or copy wrote outside its buffer.  poke != 0 first overwrites one
 * guard byte (and restores it after counting), so that *damaged = 1 shows
 * the count works.  Waits for the handle's stream.
 */
glbm_status glbm_debug_guards(glbm_t h, int poke, long long *damaged);

/* ===========================================================================
 * Batched media: many lattices of uneven size advanced together.
 *
 * All media share tau, the storage format (GLBM_F32 or GLBM_BF16DEV), the
 * boundary flags and the body force; each has its own eps and K.  Every time
 * step is ONE kernel launch over the row tiles of all media that have not
 * converged; chunks of check_every steps are captured into CUDA graphs and
 * replayed.  Per medium the arithmetic is exactly that of glbm_step on a
 * lone lattice (same kernel body), so each medium's distributions match a
 * single-lattice run bit for bit.  The model is the paper's Forchheimer-free
 * one (Eq. 28).  Batches enqueue on their own stream when `stream` is NULL
 * (graph capture needs a non-legacy stream).  The handle owns its memory.
 * ======================================================================== */
typedef struct glbm_batch *glbm_batch_t;

/* count media with sizes nx[m] x ny[m] (nx[m] a multiple of 4, ny[m] >= 2).
 * Errors: EINVAL (sizes, storage other than F32/BF16DEV), ENOMEM, ECUDA;
 * the message is in glbm_batch_last_error(NULL). */
glbm_status glbm_batch_create(int count, const int *nx, const int *ny,
                              double tau, glbm_storage storage, unsigned flags,
                              void *stream, glbm_batch_t *out);

/* eps and K of medium `index`, [ny][nx] FP64 as in glbm_set_medium; packs
 * its coefficients and puts it at rest. */
glbm_status glbm_batch_set_medium(glbm_batch_t b, int index, const double *eps,
                                  const double *K, int device_ptrs);

/* Convergence test of glbm_batch_step per medium, as glbm_set_convergence:
 * a medium converges once `patience` consecutive checks pass (default 1). */
glbm_status glbm_batch_set_convergence(glbm_batch_t b, int patience);

/* Body force G for every medium; clears the convergence histories. */
glbm_status glbm_batch_set_force(glbm_batch_t b, double gx, double gy);

/* Every medium back to rest (f = f_eq(1, 0)), step counts and convergence
 * histories cleared, all media active again. */
glbm_status glbm_batch_reset(glbm_batch_t b);

/* Block schedule: threads per block (64, 128 or 256) and tile order (0 =
 * media in index order, 1 = largest media first, 2 = largest and smallest
 * media alternating). */
glbm_status glbm_batch_set_schedule(glbm_batch_t b, int threads, int order);

/* Persistent variant (on != 0): each chunk of glbm_batch_step is ONE
 * cooperative launch in which the blocks loop over the tile table for every
 * time step and meet at a grid-wide barrier between steps (every wait is
 * bounded, about a second, after which the call returns ECUDA instead of
 * hanging); off (default): one launch per time step, chunks replayed from
 * captured CUDA graphs.  Both give the same bits.  The autotuner tries both.
 * glbm_batch_get_persistent reports the current choice. */
glbm_status glbm_batch_set_persistent(glbm_batch_t b, int on);
glbm_status glbm_batch_get_persistent(glbm_batch_t b, int *on);

/* glbm_debug_guards for the batch's device buffers. */
glbm_status glbm_batch_debug_guards(glbm_batch_t b, int poke, long long *damaged);

/* Time every schedule (threads x order x persistent or not) for
 * 2 x trial_steps steps on this batch, keep the fastest (threads/order
 * returned, either may be NULL; see glbm_batch_get_persistent) and reset
 * the batch (the trials advance it).  Requires every medium set. */
glbm_status glbm_batch_autotune(glbm_batch_t b, int trial_steps, int *threads,
                                int *order);

/* Advance at most n steps in chunks of check_every.  With tol > 0 each
 * medium's mean u_x is tested at every chunk end as in glbm_step, and a
 * medium whose relative change is <= tol leaves the batch (its state is
 * kept); the call returns early when none is left.  steps_done and
 * active_left (media still running) may be NULL.  ENAN names the medium. */
glbm_status glbm_batch_step(glbm_batch_t b, long long n, double tol,
                            int check_every, long long *steps_done,
                            int *active_left);

/* Per medium: Darcy permeability nu*Ux/Gx (kxx[count]), mean velocity
 * (mean_u[2*count], Ux Uy pairs), steps run (steps[count]) and whether it
 * converged (converged[count]); any pointer may be NULL. */
glbm_status glbm_batch_results(glbm_batch_t b, double *kxx, double *mean_u,
                               long long *steps, int *converged);

/* Absolute distributions of medium `index`, [9][ny][nx] FP64 (as
 * glbm_get_distributions). */
glbm_status glbm_batch_get_distributions(glbm_batch_t b, int index, double *f,
                                         int device_ptrs);

/* Density (Eq. 32) and Eq. 34 velocity of medium `index` at its last step,
 * [ny][nx] FP64 each (rho may be NULL).  ESTATE before the first step. */
glbm_status glbm_batch_get_fields(glbm_batch_t b, int index, double *rho,
                                  double *ux, double *uy, int device_ptrs);

/* Current schedule, kernels launched so far and total node count. */
glbm_status glbm_batch_info(glbm_batch_t b, int *threads, int *order,
                            long long *launches, long long *nodes);

void glbm_batch_destroy(glbm_batch_t b);
const char *glbm_batch_last_error(glbm_batch_t b);

/* ===========================================================================
 * Per-node apparent permeability from the DGM + GMS model (Sec. 2.1): Eq. 18
 * for inorganic nodes (organic[i] = 0) and Eq. 19 for organic nodes, with
 * K0 and K_c from Eq. 4 (pore diameter d = 2 r[i]), D_K from Eq. 3 and the
 * ideal-gas density rho_g = P M / (R T).  SI inputs: r (m, per node), eps
 * (per node, in (0, 1)), P (Pa), T (K), M (kg/mol), eta (Pa s), tort
 * (tortuosity), qsat (mol/m^3), b (1/Pa), Ds (m^2/s), dx (lattice spacing,
 * m).  K[i] receives K_app / dx^2 (lattice units, ready for set_medium).
 * n values each; device_ptrs as elsewhere; work is enqueued on `stream`
 * (NULL = legacy default) and the call returns when K is written.  EINVAL
 * (message in glbm_last_error(NULL)) for a non-positive radius or bad
 * scalars.
 * ======================================================================== */
glbm_status glbm_kapp_field(const double *r, const unsigned char *organic,
                            const double *eps, long long n, double P, double T,
                            double M, double eta, double tort, double qsat,
                            double b, double Ds, double dx, double *K,
                            int device_ptrs, void *stream);

/* Eq. 38: saturation concentration q_sat,k (mol per m^3 of kerogen) from a
 * Langmuir volume q_sat,b (m^3 of methane per kg of bulk shale):
 * q_sat,b rho_b / ((1 - eps) TOC) * rho_CH4 / M_CH4.  Host arithmetic only;
 * returns NaN for a non-positive (1 - eps) TOC or M_CH4. */
double glbm_qsat_from_langmuir_volume(double qsat_b, double rho_b, double eps,
                                      double toc, double rho_ch4,
                                      double M_ch4);

/* Message of the last failure on this handle (h = NULL: the last failure of
 * glbm_create or glbm_step_reduce_noalloc on this host thread).  Never NULL. */
const char *glbm_last_error(glbm_t h);

/* ===========================================================================
 * EM fit of a one-dimensional Gaussian mixture (Sec. 2.2, Eqs. 20-24), the
 * paper's way of splitting a measured pore-size distribution into OM and IOM
 * components.  Each iteration computes the E-step responsibilities (Eqs.
 * 20-21; Eq. 21 read with the minus sign its exponent lacks as printed) and
 * the M-step fractions, means and variances (Eqs. 22-24; Eq. 24 with the
 * means just updated), in FP64 with deterministic reductions.
 *   x              m samples (host or device per device_ptrs)
 *   k              components, 1..8
 *   phi, mu, var   host arrays of k: initial guess in, estimate out
 *   max_iter, tol  stop after max_iter iterations or when the mean
 *                  log-likelihood changes by less than tol (tol <= 0: never)
 *   iters, loglik  iterations done and the mean log-likelihood of the last
 *                  E-step (either may be NULL)
 * EINVAL (message in glbm_last_error(NULL)) for bad sizes or non-positive
 * initial fractions/variances; ENAN when the estimate is no longer finite
 * (a component collapsed onto one sample: zero variance), with the
 * arrays still written.
 * ======================================================================== */
glbm_status glbm_em_gmm1d(const double *x, long long m, int k, double *phi,
                          double *mu, double *var, int max_iter, double tol,
                          int *iters, double *loglik, int device_ptrs,
                          void *stream);

/* ===========================================================================
 * Network kernels of the learned warm start.  The paper has no surrogate:
 * these exist so that a small U-Net, trained by this library on the solver's
 * own converged fields, can predict the steady density deviation and
 * velocity of a new medium, from which glbm_init_equilibrium starts the
 * solver.  FP32, NCHW device tensors; each tensor is passed as (pointer,
 * per-sample stride in floats), so a layer may read or write a channel slice
 * of a larger tensor.  Convolutions use zero padding ksize/2 (ksize 1 or 3)
 * and weights laid out [cout][cin][ksize][ksize].  All calls enqueue on
 * `stream` and return EINVAL for bad sizes or NULL pointers, ECUDA for a
 * failed launch.
 * ======================================================================== */

/* y = conv(x) + bias (bias may be NULL), then max(., 0) when relu != 0. */
glbm_status glbm_nn_conv_fwd(const float *x, long long xbs, int cin, float *y,
                             long long ybs, int cout, int n, int h, int w,
                             int ksize, const float *wt, const float *bias,
                             int relu, void *stream);

/* dx = dL/dx of y = conv(x) given dy; wt_scratch holds cout*cin*ksize^2
 * floats (the flipped, transposed weights). */
glbm_status glbm_nn_conv_bwd_data(const float *dy, long long dybs, int cout,
                                  float *dx, long long dxbs, int cin, int n,
                                  int h, int w, int ksize, const float *wt,
                                  float *wt_scratch, void *stream);

/* dw += dL/dw and db += dL/db (db may be NULL); the caller zeroes them. */
glbm_status glbm_nn_conv_bwd_weight(const float *x, long long xbs, int cin,
                                    const float *dy, long long dybs, int cout,
                                    int n, int h, int w, int ksize, float *dw,
                                    float *db, void *stream);

/* dy[i] = 0 where y[i] <= 0 (ReLU backward, in place). */
glbm_status glbm_nn_relu_bwd(const float *y, long long ybs, float *dy,
                             long long dybs, int c, int n, int h, int w,
                             void *stream);

/* dst[:, 0:c] = src[:, 0:c] (accumulate != 0: +=). */
glbm_status glbm_nn_copy_channels(const float *src, long long sbs, float *dst,
                                  long long dbs, int c, int n, int h, int w,
                                  int accumulate, void *stream);

/* 2x2 average pool of an h x w input; backward != 0: x is dy (h/2 x w/2),
 * y receives dx (h x w), += when accumulate != 0. */
glbm_status glbm_nn_pool2(const float *x, long long xbs, float *y,
                          long long ybs, int c, int n, int h, int w,
                          int backward, int accumulate, void *stream);

/* Nearest 2x upsample of an h x w input; backward != 0: x is dy (2h x 2w),
 * y receives dx (h x w). */
glbm_status glbm_nn_upsample2(const float *x, long long xbs, float *y,
                              long long ybs, int c, int n, int h, int w,
                              int backward, void *stream);

/* loss += sum_c channel_weight[c] * mean over (n, pixels) of
 * (pred - target)^2 (loss: one device double); grad = dloss/dpred (may be
 * NULL).  Contiguous NCHW tensors. */
glbm_status glbm_nn_mse(const float *pred, const float *target,
                        const float *channel_weight, int c, int n, int h,
                        int w, float *grad, double *loss, void *stream);

/* Adam update of count parameters (step t >= 1, bias-corrected). */
glbm_status glbm_nn_adam(float *p, const float *g, float *m, float *v,
                         long long count, float lr, float beta1, float beta2,
                         float eps, int t, void *stream);

/* ===========================================================================
 * Tensor-core inference of the same network (tcgen05, sm_103a).  Activations
 * are NHWC BF16 device tensors whose pixel stride equals their channel count
 * unless stated; weights are BF16 [ksize^2][cout][cin]; accumulation is FP32
 * in tensor memory.  Like the FP32 kernels above this has no counterpart in
 * the paper.  All calls enqueue on `stream`; EINVAL for bad sizes, NULL or
 * misaligned pointers, ECUDA for a failed launch.
 * ======================================================================== */

/* y = conv(concat(x0, x1)) + bias, then max(., 0) when relu != 0; zero
 * padding ksize/2 (ksize 1 or 3).  x0 holds c0 channels, x1 (may be NULL
 * when c1 = 0) c1 channels of the same n x h x w images; c0 >= 32 and c1 are
 * multiples of 32, or c1 = 0 and c0 a multiple of 16 (a first layer of few
 * input channels padded to 16 rather than 32; the kernels read its last
 * 32-channel chunk with zeros in place of the missing channels).  wt: BF16
 * [ksize^2][cout][c0 + c1]; bias: cout FP32;
 * cout a multiple of 16 in [16, 256].  Output: f32_nchw = 0 -> BF16 NHWC at
 * y with pixel stride ys >= cout (a multiple of 8; y may point at a channel
 * slice of a wider tensor); f32_nchw != 0 -> the first cout_store channels
 * as FP32 NCHW.  *err (device int, zeroed by the caller) receives a nonzero
 * code if a pipeline wait in the kernel timed out (never in a correct run);
 * the kernel then returns without hanging.  All pointers 16-byte aligned. */
glbm_status glbm_nn_tc_conv(const void *x0, int c0, const void *x1, int c1,
                            int n, int h, int w, int ksize, const void *wt,
                            const float *bias, int cout, void *y,
                            long long ys, int relu, int f32_nchw,
                            int cout_store, int *err, void *stream);

/*
 * The band kernel of a 3x3 convolution with 32 or 64 output channels (as in
 * glbm_nn_tc_conv, bias and ReLU applied) with outputs fused into its
 * epilogue, so that the layers that follow need no pass of their own:
 *   y       BF16 NHWC output (pixel stride ys), or NULL when only the fused
 *           outputs are wanted;
 *   pool_y  if not NULL, the 2x2 average of the BF16 output, BF16 NHWC
 *           (n, h/2, w/2, cout), computed as glbm_nn_pool2_nhwc does (h, w
 *           even);
 *   head_y  if not NULL (32 output channels only), a 1x1 convolution (the
 *           network's head) of the BF16 output: head_w BF16 [head_out][32],
 *           head_b FP32 [head_out], head_out in 1..4, written FP32 NCHW
 *           (n, head_out, h, w).
 * EINVAL when the layer does not fit the band kernel (rows of >= 128 pixels,
 * input channels as in glbm_nn_tc_conv, weights within shared memory; with
 * 32 output channels the stacked or streaming form).
 */
glbm_status glbm_nn_tc_conv_fused(const void *x0, int c0, const void *x1,
                                  int c1, int n, int h, int w, const void *wt,
                                  const float *bias, int cout, void *y,
                                  long long ys, int relu, void *pool_y,
                                  const void *head_w, const float *head_b,
                                  int head_out, float *head_y, int *err,
                                  void *stream);

/* As glbm_nn_tc_conv (3x3, BF16 output, bias and ReLU when relu != 0) for a
 * layer with 32 or 64 output channels, but written 2x nearest-upsampled:
 * y is BF16 NHWC (n, 2h, 2w) with pixel stride ys >= cout (a multiple of
 * 8), and each output pixel (r, x) of the convolution fills (2r + a, 2x + b)
 * for a, b in {0, 1} -- what glbm_nn_upsample2_nhwc would make of the plain
 * output, without the plain output or the extra pass.  Runs on the
 * streaming kernel only (its epilogue stages each finished row pair in
 * shared memory and writes it with four TMA stores per row); EINVAL when
 * the layer does not fit it (rows of >= 128 pixels, segments of >= 16 rows
 * per SM, weights within shared memory). */
glbm_status glbm_nn_tc_conv_up2(const void *x0, int c0, const void *x1,
                                int c1, int n, int h, int w, const void *wt,
                                const float *bias, int cout, void *y,
                                long long ys, int relu, int *err,
                                void *stream);

/* Test hook for the kernels' timeout path: the next tensor-core launch
 * (glbm_nn_tc_conv, glbm_nn_tc_conv_fused or glbm_nn_tc_conv_wgrad) arms the
 * TMA barrier of its stage number `stage` (counted from 1 in the first CTA's
 * ring) but issues none of its copies, so the MMA warp's bounded wait for
 * that stage runs out after about 2 s.  The kernel then writes its error
 * code to *err, waits (bounded) for its copies and MMAs in flight, frees its
 * tensor memory and returns; the CUDA context stays usable.  One launch
 * takes the setting and clears it; 0 clears it.  Process-wide. */
void glbm_nn_tc_debug_starve(int stage);

/* Choice of tensor-core convolution kernel for glbm_nn_tc_conv and
 * glbm_nn_tc_conv_fused (process-wide):
 * 0 (default) = per layer: 3x3 layers with BF16 output, rows of >= 128
 * pixels and 32 or 64 output channels where one CTA per (image, 128-pixel
 * strip) leaves segments of >= 16 rows per SM run the streaming kernel (each
 * CTA walks down its strip, each input row multiplied once into a ring of
 * row accumulators in tensor memory; the three vertical taps stacked into
 * one MMA of 96 or 192 columns where the weights fit shared memory with
 * their zero tiles; 64-channel layers whose weights exceed it take them
 * along with each stage); other such layers whose weights fit shared memory
 * run the band kernel (weights resident, each band's halo loaded once per
 * 32-channel chunk; stacked taps for 32 output channels); the rest run the
 * tile kernel (one 128-pixel tile per CTA, one TMA tile per tap; a 3-stage
 * TMA ring, or an 8-stage one when the grid has at most one CTA per SM);
 * 1 = tile kernel always (and glbm_nn_tc_conv_wgrad in its per-tap form);
 * 2 = as 0 but the tile kernel always with the
 * 3-stage ring; 3 = band kernel where it applies but never stacked or
 * streaming; 4 = band kernel, stacked, never streaming; 5 = as 0 with
 * streaming however short its segments.  All compute the same convolution;
 * other values reset to 0. */
void glbm_nn_tc_set_variant(int variant);

/* FP32 [cout][cin][ksize][ksize] -> BF16 [ksize^2][cout_pad][cin_pad] (the
 * padding is zero). */
glbm_status glbm_nn_tc_pack_weights(const float *w, int cout, int cin,
                                    int ksize, int cout_pad, int cin_pad,
                                    void *wt, void *stream);

/* Training on the tensor cores: weight gradient of a k x k convolution
 * (zero padding k/2), dw[o][c][tap] += sum over images and pixels p of
 * dy[p][o] * x[p + shift(tap)][c], from BF16 NHWC activations: x with cx
 * channels (pixel stride cx, a multiple of 32; the first cin are real), dy
 * with cy channels (a multiple of 32, <= 256; the first cout are real).  dw
 * is FP32 [cout][cin][k][k] on the device and is accumulated into (FP32
 * reductions from many CTAs: the last bits depend on their order; 16-byte
 * vector reductions where cin is a multiple of 4 and dw is 16-byte
 * aligned).  FP32 accumulation of BF16 products in tensor memory.  3x3
 * layers run in band form: each CTA loads bands of 8 (or 4, 2, 1) dy rows
 * and the input rows they meet once, and one MMA covers all nine taps of a
 * 32-channel input chunk and output chunk; with glbm_nn_tc_set_variant(1),
 * and for 1x1 layers, one MMA atom per (tap, 32-channel chunk).  *err as in
 * glbm_nn_tc_conv.  16-byte aligned x and dy.  EINVAL for bad sizes. */
glbm_status glbm_nn_tc_conv_wgrad(const void *x, int cx, int cin,
                                  const void *dy, int cy, int cout, int n,
                                  int h, int w, int k, float *dw, int *err,
                                  void *stream);

/* Weights of the input-gradient convolution (dx = conv(dy, these)) from FP32
 * forward weights w [cout][cin][k][k], for the input channels c_begin ..
 * c_begin + c_pad - 1 (the gradient convolution's outputs; at most 256 per
 * call): BF16 [k^2][c_pad][cout_pad] with wt[tap][cc][o] =
 * w[o][c_begin + cc][k^2 - 1 - tap] (flipped in space, channels swapped),
 * zero where c_begin + cc >= cin or o >= cout. */
glbm_status glbm_nn_tc_pack_weights_flip(const float *w, int cout, int cin,
                                         int k, int c_begin, int c_pad,
                                         int cout_pad, void *wt, void *stream);

/* Bias gradient db[c] += sum over images and pixels of dy, FP32 NCHW dy with
 * per-sample stride dybs. */
glbm_status glbm_nn_bias_grad(const float *dy, long long dybs, int c, int n,
                              int h, int w, float *db, void *stream);

/* FP32 NCHW (n, c, h, w) -> BF16 NHWC with c_pad >= c channels (zero);
 * c_pad a multiple of 8, y 16-byte aligned. */
glbm_status glbm_nn_nchw_to_nhwc(const float *x, int n, int c, int h, int w,
                                 void *y, int c_pad, void *stream);

/* 3x3 patches of FP32 NCHW (n, c, h, w) as BF16 NHWC channels: channel
 * ci * 9 + 3 (dy + 1) + (dx + 1) of output pixel (y, x) is x[ci][y + dy]
 * [x + dx] (zero outside the image), channels 9c .. c_pad - 1 are zero.
 * A 3x3 convolution with zero padding of x then equals the 1x1 convolution
 * (glbm_nn_tc_conv with ksize 1) of this tensor with the FP32 weights
 * [cout][c][3][3] read as [cout][9c][1][1].  c_pad >= 9c, a multiple of 8;
 * y 16-byte aligned. */
glbm_status glbm_nn_im2col3_nhwc(const float *x, int n, int c, int h, int w,
                                 void *y, int c_pad, void *stream);

/* 2x2 average pool, BF16 NHWC (n, h, w, c) -> (n, h/2, w/2, c); c, h, w even. */
glbm_status glbm_nn_pool2_nhwc(const void *x, int n, int c, int h, int w,
                               void *y, void *stream);

/* Nearest 2x upsample, BF16 NHWC (n, h, w, c) -> (n, 2h, 2w, c); c a
 * multiple of 8. */
glbm_status glbm_nn_upsample2_nhwc(const void *x, int n, int c, int h, int w,
                                   void *y, void *stream);

/* Warm-start input of one medium of npix nodes (FP64 eps and K on the
 * device) -> x, 3 x npix FP32 (one NCHW sample): (eps - 0.05)/0.05,
 * (log10 K + 2)/2 and log10|G| + 6, in FP32 arithmetic on the rounded
 * inputs. */
glbm_status glbm_nn_warm_features(const double *eps, const double *K,
                                  long long npix, double G, float *x,
                                  void *stream);

/* Network output y (3 x npix FP32) -> FP64 warm-start fields on the device:
 * rho = 1 + y0 (G rho_scale), ux = (y1 K) (G / nu), uy = (y2 K) (G / nu)
 * (the scalar factors formed first), ready for glbm_init_equilibrium with
 * device_ptrs = 1. */
glbm_status glbm_nn_warm_decode(const float *y, const double *K,
                                long long npix, double G, double nu,
                                double rho_scale, double *rho, double *ux,
                                double *uy, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GLBM_H */
