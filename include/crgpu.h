/*
 * crgpu.h -- C ABI of the GB300 P-APG convex-regression solver.
 *
 * Method: Aybat & Wang, "A Parallel Method for Large Scale Convex Regression
 * Problems" (arXiv:1407.7220).  The library solves problem (regularize)
 * (Sec. II-C)
 *
 *     min_{y in R^N, xi in R^{N x n}}  1/2 ||y - ybar||^2 + gamma/2 ||xi||^2
 *     s.t.  y_{l1} - y_{l2} - xi_{l2}^T (x_{l1} - x_{l2}) >= 0   for all l1 != l2,
 *
 * by P-APG (Fig. 2) on its dual (lambda_dual) with every one of the N(N-1)
 * pairwise constraints dualized (the partition of Sec. II-A taken to
 * singletons, K = N).  Step 1 of P-APG then has a closed form (the "fold"),
 * Step 2 is the projected update of the N x N multiplier array, and Steps 3-4
 * are the momentum of Fig. 2.  The y >= 0 rows of C (Eq. (eq:C)) are kept and
 * made inactive by the shift of the observations described after
 * Eq. (omega_primal).  The same multiplier-array machinery also runs ALCC with
 * its MAPG inner solver (Sec. II-D) on (regularize) directly (cr_alcc_*).
 *
 * Conventions for every entry point:
 *  - Host pointers are plain C arrays; "device" pointers are CUDA device
 *    addresses on the handle's device.  Matrices are row-major.
 *  - X is N x n (row l = x_l), ybar has N entries.
 *  - The library copies every input; outputs go to caller-owned buffers.
 *  - No C++ exception crosses this boundary.  Every call returns a cr_status;
 *    on failure cr_last_error(h) returns a message (per handle).
 *  - A handle is used by one host thread at a time.  Work is enqueued on the
 *    handle's stream (cr_options.stream, or a stream the library creates).
 *  - There is no CPU fallback: without a usable sm_103a device every call
 *    that needs one returns CR_ECUDA.
 */
#ifndef CRGPU_H
#define CRGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cr_ctx *cr_handle;

typedef enum {
    CR_OK = 0,
    CR_NOT_CONVERGED = 1, /* cr_solve reached max_iter (not an error) */
    CR_EINVAL = -1,       /* invalid argument (sizes, gamma <= 0, non-finite input, N < n + 1) */
    CR_ENOMEM = -2,       /* device or host allocation failed */
    CR_ECUDA = -3,        /* CUDA runtime error (message in cr_last_error) */
    CR_ETIMEOUT = -4,     /* a bounded device-side wait gave up; the handle must be reset */
    CR_ENUMERIC = -5,     /* a non-finite value appeared in the iteration */
    CR_ESTATE = -6        /* call not valid in the handle's current state */
} cr_status;

/* Storage type of the multiplier array theta.  F32, BF16, F16: the per-pair math is FP32.
 * F64: the multipliers and the whole per-pair step (residual, projection, adjoint sums) are
 * FP64, for problems that must be solved below the KKT floor of FP32 multipliers (measured
 * near 5e-5 at N = 500, n = 2 with stochastic rounding); n <= 10, CUDA-core pass, single
 * instances, no record_every.  GB300's FP64 rate makes it the mode for small problems (both arrays in L2). */
enum { CR_THETA_F32 = 0, CR_THETA_BF16 = 1, CR_THETA_F16 = 2, CR_THETA_F64 = 3 };

/* Iteration driver. */
enum {
    CR_DRIVER_AUTO = 0,       /* persistent if the cooperative launch fits, else phase kernels */
    CR_DRIVER_PERSISTENT = 1, /* one cooperative launch runs many iterations (bounded grid barriers) */
    CR_DRIVER_PHASES = 2      /* one kernel launch per phase per iteration */
};

/* Pair-pass engine (cr_options.pair_engine).  The pair pass needs, per stage of 16 rows x 256
 * columns, the residual dot products xi_l2 . x_l1 and the adjoint sums sum_l1 theta x_l1,
 * sum_l1 theta: two rank-n products. */
enum {
    CR_PAIR_AUTO = 0,         /* tensor cores for a 16-bit theta with n >= 8 or an FP32 theta with n >= 16,
                                 unless record_every > 0 or the persistent driver; CUDA cores otherwise */
    CR_PAIR_CUDA_CORES = 1,   /* packed FP32 FMA on the CUDA cores (bitwise reproducible by cr_backward) */
    CR_PAIR_TENSOR_CORES = 2  /* tcgen05 TF32 MMA, three TF32 products per FP32 product (~FP32 accuracy);
                                 not with record_every > 0 and not in a batch */
};

typedef struct {
    double gamma;   /* Tikhonov parameter of (regularize), > 0.  The paper gives no value; default 1e-2 */
    double L;       /* step constant L_g of Eq. (eq:lischitz); <= 0: the closed-form bound
                       (1 + 2N + max_l lambda_max(sum_m (x_m-x_l)(x_m-x_l)^T)) / gamma */
    double shift;   /* observation shift s (after Eq. (omega_primal)); < 0: max(0,-min ybar) + range(ybar) */
    int32_t theta_dtype;      /* CR_THETA_F32 / _BF16 / _F16 / _F64 */
    int32_t stochastic_round; /* 1: unbiased stochastic rounding of every theta store (counter-based hash) */
    int32_t kkt_every;        /* cr_solve evaluates the KKT residual every this many iterations (>= 1) */
    int32_t momentum;         /* 1: P-APG (Fig. 2); 0: dual gradient ascent (the paper's comparator, Sec. III) */
    int32_t restart;          /* NOT IN THE PAPER. 1: reset the momentum (t <- 1) when the dual value decreases;
                                 default 0 (plain P-APG, which converged faster in our measurements) */
    int32_t driver;           /* CR_DRIVER_* */
    int32_t grid;             /* CTAs used by the pair pass; 0 = tuned per device and size */
    int32_t fp16_exponent;    /* CR_THETA_F16 only: theta is stored as theta * 2^fp16_exponent */
    uint64_t seed;            /* seed of the stochastic-rounding hash */
    void *stream;             /* cudaStream_t; NULL = a stream owned by the handle */
    int32_t barrier_timeout_ms; /* bound of every device-side grid-barrier wait; 0 = 4000 ms.  A wait
                                   that runs out sets an error word, every CTA returns, and the call
                                   reports CR_ETIMEOUT (the context stays usable; cr_reset recovers) */
    int32_t test_barrier_extra; /* test hook, 0 in use: barriers wait for this many extra arrivals
                                   that never come, so the bounded wait runs out on purpose */
    int32_t profile;          /* 1: record CUDA events around every kernel launch (see cr_profile) */
    int32_t record_every;     /* > 0: cr_iterate keeps a checkpoint every this many iterations so that
                                 cr_backward can differentiate the unrolled iterations (FP32 theta, n <= 10) */
    int32_t pair_engine;      /* CR_PAIR_*: where the pair pass computes its two dense products */
    int32_t batch_stage_rows; /* batches only: rows per pipeline stage of the pair pass (the tile shape), 16
                                 or 8; 0 (default): the batch autotuner picks one */
    int32_t reserved[2];
    double restart_tol;       /* restart only when the dual value fell by more than restart_tol * |previous|
                                 (guards the test against rounding noise); default 1e-7 */
    double B_theta;           /* radius of the ball in Q_2 = {lambda >= 0, ||lambda||_2 <= B_theta} of Eq.
                                 (lambda_dual), lambda = (theta, mu) all dual variables; <= 0 (default) or
                                 infinite: no ball.  Finite: Step 2 projects on Q_2 exactly, the clamp at 0
                                 followed by the radial factor min(1, B_theta / ||clamped lambda||_2), which
                                 costs a norm pass and, when the ball binds, a scaling pass over the array.
                                 FP32 or FP64 multipliers, CUDA-core pass, phase driver, no record_every */
    double promote_at;        /* BF16 or FP16 multipliers: > 0 makes cr_solve a precision schedule, solving
                                 in the 16-bit format until the FP64-confirmed KKT residual reaches
                                 promote_at, then widening to FP32 in place (cr_promote) and solving on to
                                 its tol.  0 (default): no widening.  Measured on recipe (2) at N = 20,000:
                                 0.1 for FP16 and 0.2 for BF16, just before each format stalls */
} cr_options;

/* Fills *opt with the defaults documented above. */
void cr_options_default(cr_options *opt);

/* Creates a solver for one instance.  X: host, N x n row-major FP64; ybar: host, N FP64.
 * opt may be NULL (defaults).  Requires n >= 1, N >= n + 1 (uniqueness of y*, stated after
 * problem (original)) and finite inputs, else CR_EINVAL.  The state is Iteration 0 of Fig. 2
 * (theta^(1)_0 = theta^(2)_1 = 0, t_1 = 1).  Device memory: two N x ceil128(N) theta arrays of
 * the chosen dtype plus O(N n) vectors and O(N^2/32) partial sums. */
cr_status cr_create(const double *X, const double *ybar, int64_t N, int32_t n, const cr_options *opt,
                    cr_handle *out);

/* Same as cr_create with device-resident FP32 inputs (e.g. torch tensors), copied on the
 * handle's stream. */
cr_status cr_create_device(const float *dX, const float *dybar, int64_t N, int32_t n,
                           const cr_options *opt, cr_handle *out);

/* Returns the handle to Iteration 0 of Fig. 2 (theta = 0, t = 1). */
cr_status cr_reset(cr_handle h);

/* Widens the stored multipliers of a BF16 or FP16 handle to FP32 in place of the iteration:
 * both stored iterates (theta^(1)_l, theta^(1)_{l-1}) are converted exactly, the momentum state,
 * the FP64 aggregates and the iteration count are kept, and later iterations run with FP32
 * multipliers (a precision schedule: cheap 16-bit iterations while the updates are large, FP32
 * once the 16-bit rounding floor is reached).  The tensor-core pass stays when the options allow
 * it at FP32 (n >= 16 or pair_engine = CR_PAIR_TENSOR_CORES); otherwise the CUDA-core pass.
 * Allocates the two FP32 arrays and frees the 16-bit ones.  CR_EINVAL for any other
 * conversion.  Blocks. */
cr_status cr_promote(cr_handle h, int32_t theta_dtype);

/* Enqueues k iterations of P-APG (Fig. 2, steps 1-4) on the handle's stream and returns
 * without waiting.  Each iteration streams the multiplier array once (read theta^(1)_l,
 * theta^(1)_{l-1}; write theta^(1)_{l+1}). */
cr_status cr_iterate(cr_handle h, int64_t k);

/* Runs iterations until the KKT residual (see cr_kkt_residual) at the current dual iterate
 * is <= tol -- checked every kkt_every iterations with an FP32 screen and confirmed in FP64 --
 * or until max_iter more iterations.  Blocks.  *iters_done (nullable) receives the iterations
 * run by this call.  Returns CR_OK on convergence, CR_NOT_CONVERGED at max_iter. */
cr_status cr_solve(cr_handle h, double tol, int64_t max_iter, int64_t *iters_done);

/* FP64 objective values at the current dual iterate theta^(1)_l and its minimizer
 * eta = (y, xi) (Step 1 map):  primal = 1/2||y - ybar||^2 + gamma/2||xi||^2,
 * dual = g_gamma(theta) (Eq. (eq:g_gamma)), gap = primal - dual = theta^T C eta
 * (the paper's duality gap, Sec. III).  Any pointer may be NULL.  Blocks. */
cr_status cr_objective(cr_handle h, double *primal, double *dual, double *gap);

/* FP64 KKT residual at the current dual iterate (Sec. III metrics plus the reading used by
 * this library): with sigma = max(1, max ybar - min ybar) and g_p = (C eta)_p,
 *   pri  = max(max_p (-g_p)_+, max_l (-y_l)_+) / sigma
 *   comp = max(max_p theta_p |g_p|, max_l mu_l |y_l|) / sigma^2
 *   kkt  = max(pri, comp)           (stationarity holds exactly by the closed form)
 *   infeas_norm = ||(A_1 y + A_2 xi)_-||_2 / sqrt(N^2 - N)    (Sec. III)
 *   gap_norm    = theta^T C eta / (N^2 - N)                    (Sec. III)
 * Every per-pair term is evaluated in FP64.  Any pointer may be NULL.  Blocks. */
cr_status cr_kkt_residual(cr_handle h, double *kkt, double *infeas_norm, double *gap_norm);

/* Reverse mode through the iterations run so far (all by cr_iterate from Iteration 0 with
 * record_every > 0): given dL_dyhat (device, N floats) = dLoss/dyhat of the current fitted
 * values, writes dLoss/dybar (device, N floats) and dLoss/dX (device, N x n floats).  The
 * iterations are plain P-APG (restart = 0) with gamma, L and the shift s held fixed; the
 * projection max(0, .) differentiates to its active indicator (0 at a tie).  Every
 * record_every iterations form a segment: the segment is recomputed from its checkpoint
 * (bit for bit) and then reversed.  The handle's state is restored afterwards.  Workspace:
 * record_every + 3 multiplier arrays plus O(N n) vectors.  Blocks. */
cr_status cr_backward(cr_handle h, const float *dL_dyhat, float *dL_dybar, float *dL_dX);

/* Fitted values yhat (N, shift removed) and subgradients xi (N x n, row-major) at the current
 * dual iterate, in FP64, to host buffers (either may be NULL).  Blocks. */
cr_status cr_get_solution(cr_handle h, double *yhat, double *xi);

/* The same values into caller-owned DEVICE buffers (yhat: N doubles, xi: N x n doubles,
 * row-major; either may be NULL), written by a kernel on the handle's stream; returns after
 * that stream has finished the copy, so the buffers may be used from any stream.  For callers
 * that keep the fit on the device (the autograd binding) and would otherwise copy through the
 * host.  The buffers must not overlap the handle's own state. */
cr_status cr_get_solution_device(cr_handle h, double *yhat, double *xi);

/* Iterations run since creation/reset, momentum restarts so far, the step constant L used,
 * and the shift s.  Any pointer may be NULL. */
cr_status cr_get_info(cr_handle h, int64_t *iters, int64_t *restarts, double *L, double *shift);

/* The pair-pass engine the handle resolved at creation: CR_PAIR_CUDA_CORES or
 * CR_PAIR_TENSOR_CORES (CR_PAIR_AUTO is decided by n and record_every). */
cr_status cr_get_engine(cr_handle h, int32_t *engine);

/* The problem constants the solvers derive on the host, without a device: the step constant
 * bound L = (1 + sigma_max^2(A_1) + sigma_max^2(A_2)) / gamma of cr_options.L (Eq. (eq:lischitz)
 * with sigma_max^2(C) <= 1 + ||A_1||^2 + ||A_2||^2), the default shift s (after Eq.
 * (omega_primal)), sigma_max^2(A_1) = 2N and sigma_max^2(A_2) = max_l lambda_max(sum_m (x_m - x_l)
 * (x_m - x_l)^T) (Fig. `fig:alcc` step 1).  X, ybar: host arrays as for cr_create.  Any output
 * pointer may be NULL.  CR_EINVAL (message in cr_last_error(NULL)) on bad sizes, non-finite
 * inputs or gamma <= 0. */
cr_status cr_problem_constants(const double *X, const double *ybar, int64_t N, int32_t n, double gamma, double *L,
                               double *shift, double *sigma2_A1, double *sigma2_A2);

/* Kernel timing collected since the last call when cr_options.profile = 1 (CUDA events on the
 * handle's stream around each launch).  kind: 0 = pair pass (Step 2 + fused adjoint, the
 * multiplier-array stream), 1 = folds (Step 1 and reductions), 2 = KKT passes, 3 = persistent
 * launches (all phases of many iterations).  *ms = summed device time, *launches = count.
 * Blocks; resets the counters. */
cr_status cr_profile(cr_handle h, int32_t kind, double *ms, int64_t *launches);

/* Device addresses of the handle's current iterate, without copying: theta^(1)_l (N rows of
 * ld elements, row-major, in the handle's theta_dtype), X (N x n FP64), y (N FP64, the fitted
 * values plus the shift s), xi (N x n FP64), mu (N FP64, multipliers of the y >= 0 rows) and
 * the data scale sigma used by the KKT residual.  The buffers stay owned by the handle; the
 * addresses are valid until the next call that iterates, resets or destroys it.  Any output
 * pointer may be NULL. */
cr_status cr_get_device_state(cr_handle h, const void **dtheta, int64_t *ld, const double **dX, const double **dy,
                              const double **dxi, const double **dmu, double *sigma);

/* KKT residual without any allocation, for callers that cannot allocate device memory when
 * they check convergence: processes that reserve their whole device-memory budget up front
 * and forbid later allocation, and loops that must avoid cudaMalloc/cudaFree because those
 * calls can synchronize the device.  The paper has no counterpart; this is a service of this
 * library.
 *
 * Computes the same five FP64 values as cr_kkt_residual (kkt, pri, comp, infeas_norm,
 * gap_norm, in that order) for a caller-described dual point: theta (device, FP32, N rows of
 * ld >= N elements, row-major; the diagonal is ignored), X (device, N x n FP64), y (device, N
 * FP64, the minimizer's y including the shift), xi (device, N x n FP64), mu (device, N FP64,
 * or NULL for zero) and sigma > 0; the five results are written to dout (device, 5 doubles).
 * Work is enqueued on `stream` (cudaStream_t, NULL = legacy default stream) and the call
 * returns without waiting.
 *
 * Scratch: a fixed array of 65,536 x 4 doubles (2 MiB) inside the library, held by every
 * device that loads the library until the process exits.  N > 65,536 is rejected with
 * CR_EINVAL (message in cr_last_error(NULL)).  The first call on a device is its set-up: with
 * that device current it looks up the array's device address (cudaGetSymbolAddress).  Under
 * CUDA's lazy module loading (the default) that first call is also when the driver loads the
 * library's module, reserves the 2 MiB and loads the two kernels, so a caller with a fixed
 * memory budget makes one warm-up call at start-up; later calls on that device change no
 * device-memory figure.  Make the first call before any stream capture.  The address is kept
 * per device together with the current context; a device reset (cudaDeviceReset) destroys
 * that context, and the next call, made in the new context, repeats the set-up.  All calls
 * share the array, so calls that overlap on the GPU (for example on two streams at once) race
 * and must be ordered by the caller.  The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine. */
cr_status cr_kkt_residual_noalloc(int64_t N, int32_t n, const float *dtheta, int64_t ld, const double *dX,
                                  const double *dy, const double *dxi, const double *dmu, double sigma, void *stream,
                                  double *dout);

/* Releases every resource of the handle (NULL is a no-op). */
void cr_destroy(cr_handle h);

/* ---- ALCC with the MAPG inner solver on the full problem (Sec. II-D) ---------------------
 * ALCC (Fig. `fig:alcc`) solves (regularize) directly, without the y >= 0 rows and without a
 * shift.  Outer iteration k:
 *   1. L^y_k = 1/mu_k + sigma_max^2(A_1), L^xi_k = gamma/mu_k + sigma_max^2(A_2), with
 *      sigma_max^2(A_1) = 2N and sigma_max^2(A_2) = max_l lambda_max(sum_m (x_m-x_l)(x_m-x_l)^T);
 *   2. ell^max_k = 4 sqrt((L^y_k Bbar_y^2 + L^xi_k Bbar_xi^2) / tau_k);
 *   3. (y_k, xi_k) = MAPG on the subproblem P_k of Eq. (eq:subproblem) from (y_{k-1}, xi_{k-1}):
 *      block steps 1/L^y_k and 1/L^xi_k projected on the balls Q_y = {||y - ybar|| <= Bbar_y} and
 *      Q_xi = {||xi|| <= Bbar_xi}, momentum, stopped when both step lengths are <= alpha^y_k and
 *      alpha^xi_k or at ell^max_k.  The pair pass reads FP32 copies of y and xi, so the thresholds
 *      are taken no smaller than 2^-23 ||y|| and 2^-23 ||xi|| (a shorter step cannot change those
 *      copies); fixed_inner turns the test off;
 *   4. theta_{k+1} = (mu_k/mu_{k+1}) (A_1 y_k + A_2 xi_k - theta_k)_-;
 *   5-6. mu_{k+1} = c mu_k; tau and the alphas are divided by (c k^(1+kappa))^2.
 * Readings where the paper is silent: theta_1 = 0; (y_0, xi_0) = (ybar, 0); the radii come from
 * the feasible point (mean(ybar) 1, 0): Bbar = ||ybar - mean(ybar)||, Bbar_y = Bbar,
 * Bbar_xi = Bbar / sqrt(gamma); mu_1, tau_1 and the alphas are set relative to these scales.
 *
 * Device memory: ONE N x ceil128(N) FP32 multiplier array (read once per MAPG iteration, read and
 * written once per outer iteration) plus O(N n) vectors and O(N^2/32) partial sums.  Each MAPG
 * iteration is a cooperative launch's pair pass plus two row folds in FP64; a launch runs up to
 * launch_iters MAPG iterations.  The handle answers cr_get_solution ((y_k, xi_k)),
 * cr_get_info (iters = outer iterations), cr_get_device_state, cr_reset and cr_destroy; the
 * P-APG calls (cr_iterate, cr_solve, cr_kkt_residual, cr_objective, cr_backward) return
 * CR_ESTATE on it. */
typedef struct {
    double mu1_scale;      /* mu_1 = mu1_scale / sigma_max^2(A_1); default 1e3 */
    double tau1_rel;       /* tau_1 = tau1_rel * Bbar^2 / mu_1; default 1e-2 */
    double alpha1_rel;     /* alpha^y_1 = alpha1_rel * Bbar_y, alpha^xi_1 = alpha1_rel * Bbar_xi; default 1e-2 */
    double c;              /* > 1; default 2 */
    double kappa;          /* > 0; default 0.1 */
    int64_t lmax_cap;      /* > 0: at most this many MAPG iterations per outer iteration; 0: ell^max_k only */
    int64_t fixed_inner;   /* > 0: every MAPG call runs exactly this many iterations (stopping test off) */
    int64_t launch_iters;  /* MAPG iterations per cooperative launch; 0 = chosen from N */
    double mu_max_scale;   /* NOT IN THE PAPER.  > 0: mu_k stops growing at mu_max_scale / sigma_max^2(A_1)
                              (the multiplier update alone then drives feasibility); 0 = the paper's
                              unbounded mu_{k+1} = c mu_k */
    double reserved[3];
} cr_alcc_options;

/* Fills *o with the defaults documented above. */
void cr_alcc_options_default(cr_alcc_options *o);

/* Creates an ALCC solver.  X, ybar as for cr_create; opt (nullable) supplies gamma, grid, stream,
 * barrier_timeout_ms and profile, and must ask for FP32 theta and not for the tensor-core pass;
 * aopt may be NULL (defaults).  CR_EINVAL on bad sizes, non-finite inputs or options (c <= 1,
 * kappa <= 0, mu1_scale/tau1_rel/alpha1_rel <= 0); CR_ECUDA when the cooperative launch does not
 * fit.  The state is Iteration 0 of Fig. `fig:alcc`. */
cr_status cr_alcc_create(const double *X, const double *ybar, int64_t N, int32_t n, const cr_options *opt,
                         const cr_alcc_options *aopt, cr_handle *out);

/* Runs k outer iterations (steps 1-6 each).  inner (nullable, k entries) receives the MAPG
 * iterations of each.  Blocks. */
cr_status cr_alcc_iterate(cr_handle h, int64_t k, int64_t *inner);

/* Runs outer iterations until the KKT residual of cr_alcc_metrics is <= tol or max_outer more
 * outer iterations; *outer_done (nullable) = outer iterations run by this call.  CR_OK on
 * convergence, CR_NOT_CONVERGED otherwise.  Blocks. */
cr_status cr_alcc_solve(cr_handle h, double tol, int64_t max_outer, int64_t *outer_done);

/* FP64 KKT residual of (regularize) after the last outer iteration k, at (y_k, xi_k) with the
 * multiplier estimate lambda = mu_{k+1} theta_{k+1}; with sigma = max(1, max ybar - min ybar):
 *   stat = max(max_l |y_l - ybar_l - (A_1^T lambda)_l|, max_lk |gamma xi_lk - (A_2^T lambda)_lk|) / sigma
 *   pri  = max_p (-(A_1 y + A_2 xi)_p)_+ / sigma
 *   comp = max_p lambda_p |(A_1 y + A_2 xi)_p| / sigma^2,      kkt = max(stat, pri, comp).
 * CR_ESTATE before the first outer iteration.  Any pointer may be NULL. */
cr_status cr_alcc_metrics(cr_handle h, double *kkt, double *stat, double *pri, double *comp);

/* Outer iterations run, MAPG iterations run in total, the current mu_k and the ell^max_k of the
 * next outer iteration.  Any pointer may be NULL. */
cr_status cr_alcc_info(cr_handle h, int64_t *outer, int64_t *inner_total, double *mu, int64_t *lmax_next);

/* ---- batched solves: many independent fits in one persistent launch ---------------------
 * B independent instances (sizes N[i] x n[i], host FP64 arrays X[i], ybar[i]) advance together:
 * one cooperative launch runs every phase of every instance, separated by bounded grid
 * barriers.  Work items (a slice of an instance's stripes and rows) are spread over the
 * physical CTAs by pair count; the item size is chosen at creation by an autotuner that
 * times a few iterations per candidate (cr_options.grid > 0 fixes the granularity factor
 * instead).  The launch is captured once in a CUDA graph and replayed chunk after chunk.
 * Each instance keeps its own L, shift, momentum scalars and KKT test; an instance whose
 * KKT residual reaches tol leaves the work, and its state stays at that iterate.  All
 * instances share the options (gamma, theta_dtype ...), padded to the largest n. */
typedef struct cr_batch_ctx *cr_batch_handle;

cr_status cr_batch_create(int32_t B, const int64_t *N, const int32_t *n, const double *const *X,
                          const double *const *ybar, const cr_options *opt, cr_batch_handle *out);
/* Iterates until every instance reached KKT <= tol (checked every kkt_every iterations) or
 * max_iter iterations; *converged (nullable) = instances that converged.  Blocks. */
cr_status cr_batch_solve(cr_batch_handle b, double tol, int64_t max_iter, int64_t *converged);
/* k iterations of every instance still running (no convergence test).  Blocks. */
cr_status cr_batch_iterate(cr_batch_handle b, int64_t k);
/* Every instance back to Iteration 0 of Fig. 2. */
cr_status cr_batch_reset(cr_batch_handle b);
/* Handle of instance i (owned by the batch): use cr_get_solution, cr_get_info, cr_objective or
 * cr_kkt_residual on it; do not iterate or destroy it directly. */
cr_status cr_batch_instance(cr_batch_handle b, int32_t i, cr_handle *h);
/* Granularity factor picked by the autotuner, physical CTAs, iterations run. */
cr_status cr_batch_info(cr_batch_handle b, int32_t *factor, int32_t *grid, int64_t *iters);
/* How the batch launches ran: *graph_live = 1 when the launch is held as an instantiated CUDA
 * graph (0 when capture of the cooperative launch was refused and the batch launches directly);
 * graph_launches / direct_launches count the launches of each kind so far; *tuned = candidates
 * the autotuner timed, tune_ms (nullable, room for 8) the milliseconds per iteration of the first
 * 8 of them (cr_batch_tuning lists every candidate).  Any pointer may be NULL. */
cr_status cr_batch_stats(cr_batch_handle b, int32_t *graph_live, int64_t *graph_launches, int64_t *direct_launches,
                         int32_t *tuned, double *tune_ms);
/* The batch autotuner's choice and measurements.  The candidates are the tile shapes (rows per
 * pipeline stage of the pair pass: 16, then 8) times the work granularities (factors 1, 2, 4,
 * 8, 16), each timed over a few iterations from the initial point; *stage_rows and *factor are
 * the pair in use (the fastest, or the one the options fixed).  *count = candidates timed (0 when
 * the options fixed both); the first min(count, cap) are written to cand_rows, cand_factor and
 * cand_ms (milliseconds per iteration).  Any pointer may be NULL. */
cr_status cr_batch_tuning(cr_batch_handle b, int32_t cap, int32_t *count, int32_t *stage_rows, int32_t *factor,
                          int32_t *cand_rows, int32_t *cand_factor, double *cand_ms);
void cr_batch_destroy(cr_batch_handle b);
const char *cr_batch_last_error(cr_batch_handle b);

/* ---- P-APG with K blocks (Sec. II-A, Fig. 2) -------------------------------------------------
 * The points are partitioned into blocks (block_of[l] = block of point l, any ids in [0, N)).
 * The pairwise constraints between blocks and the y >= 0 rows of C (Eq. (eq:C)) are dualized and
 * P-APG (plain momentum) runs on their dual; Step 1 separates into one problem per block,
 *     min 1/2 ||y_i - a_i||^2 + gamma/2 ||xi_i - b_i||^2  s.t. the pairwise constraints inside block i,
 * with a = ybar + s + A_1^T theta^(2) + mu^(2) and b = A_2^T theta^(2) / gamma (dualized rows only).
 * The library solves all block problems together by an inner P-APG on their duals (FP64, the
 * pairs inside the blocks), warm-started from the previous call's inner multipliers with the
 * momentum restarted (as from Iteration 0), for inner_iters (even, >= 2) iterations per outer
 * iteration: an inexact Step 1, as the paper's ALCC or interior-point block solves.  K = N (every
 * point its own block) is the P-APG of cr_create; K = 1 makes Step 1 the whole problem.
 * Multipliers and arithmetic are FP64 (n <= 10); device memory: 4 N x ceil128(N) FP64 arrays
 * (outer and inner iterates).  The handles hold the points sorted by block (stable); the inner
 * pass visits, in each 256-column stripe, only the rows of the blocks its columns belong to, and
 * cr_blocks_solution returns the points in the caller's order.  The handle answers cr_get_info
 * and cr_destroy; cr_reset and the P-APG calls of cr_create return CR_ESTATE on it. */
cr_status cr_blocks_create(const double *X, const double *ybar, int64_t N, int32_t n, const int32_t *block_of,
                           const cr_options *opt, int32_t inner_iters, cr_handle *out);
/* k outer iterations, then Step 1 once more at the dual iterate theta^(1)_l (the primal point of
 * Theorem 1, read by cr_blocks_solution).  Blocks. */
cr_status cr_blocks_iterate(cr_handle h, int64_t k);
/* The primal point (yhat with the shift removed, xi), host buffers (either may be NULL).  Blocks. */
cr_status cr_blocks_solution(cr_handle h, double *yhat, double *xi);

/* Static description of a status code. */
const char *cr_status_str(cr_status s);

/* Last error message recorded on the handle ("" if none).  Valid until the next call. */
const char *cr_last_error(cr_handle h);

#ifdef __cplusplus
}
#endif

#endif /* CRGPU_H */
