/*
 * mnl.h - C ABI of the GB300 multinomial-logit Newton-Raphson library.
 *
 * Model (Sec. 2.1, eq. "unormalized utility"): observation i chooses one of K
 * alternatives (k = 0 is the base, Sec. 2.1 "normalizing") with utility
 *     U_ik = X_i . beta_k + Y_ik . gamma_k + Z_ik . alpha
 * X: individual-specific data with per-alternative coefficients beta_k
 * (beta_0 = 0; an intercept is an X column of ones, Sec. 3.1); Y: alternative-
 * specific data with per-alternative coefficients gamma_k; Z: alternative-
 * specific data with one generic coefficient alpha.  P_ik is the softmax of
 * U_i. over k (eqs. "probability", "base probability"), l the log-likelihood
 * (eq. "log-lik function"), and one Newton-Raphson step (eq. "NR update",
 * Sec. 3.1) is  theta <- theta + t (-H)^{-1} g  with t = 1, 1/2, ... chosen by
 * step halving until l does not decrease.
 *
 * Coefficient vector theta (eq. "theta vec"), float64:
 *     [ beta_1 .. beta_{K-1} (p each) | gamma_{1 or 0} .. gamma_{K-1} (d each) | alpha (f) ]
 * gamma_base = 0 (default): gamma_0 is fixed at 0 and the k = 0 rows of Y are
 *   ignored; n_theta = (K-1)(p+d) + f.
 * gamma_base = 1: gamma_0 is estimated as in the paper (Sec. 2.3 "1 x K";
 *   eq. "theta vec"); n_theta = (K-1)p + Kd + f, needs d >= 1.  Supported by
 *   the single-problem handle (mnl_create and every call on it); the batched,
 *   serving and allocation-free calls return MNL_ERR_UNSUPPORTED for it.
 *   The library solves it as the equivalent gamma_base = 0 problem with d more
 *   generic columns (z'_ikj = y_i0j for k = 0, else 0: only differences
 *   against alternative 0 enter, and z'_ik - z'_i0 = -y_i0 for k >= 1 is the
 *   paper's -Y_i0 gamma_0 term); theta, the gradient, the Hessian and the
 *   standard errors are returned in the order above.
 *
 * Data layout (all row-major, float32, read-only, owned by the caller):
 *     X      [N][p]       individual-specific columns
 *     Y      [N][K][d]    alternative-specific, per-alternative coefficients (NULL if d = 0)
 *     Z      [N][K][f]    alternative-specific, generic coefficient; raw values, the
 *                         library uses only differences against alternative 0 (NULL if f = 0)
 *     choice [N]          int32 in [0, K), the observed alternative
 *
 * Devices and streams: every entry point works on the CUDA device that was
 * current at mnl_create and enqueues its work on the stream given there (NULL:
 * the legacy default stream).  Pointers documented as "device" must be device
 * (or managed) memory of that device.
 *
 * Errors: every int-returning function returns MNL_OK (0) or one of the
 * MNL_ERR_* codes below; no C++ exception crosses this boundary.  After
 * MNL_ERR_CUDA the handle should be destroyed.  mnl_status_string gives text.
 */
#ifndef MNL_H
#define MNL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MNL_API __attribute__((visibility("default")))
#else
#define MNL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MNL_OK = 0,
  MNL_ERR_INVALID_ARG = 1, /* bad size, NULL required pointer, choice out of range          */
  MNL_ERR_OOM = 2,         /* a device allocation failed                                     */
  MNL_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed                              */
  MNL_ERR_NOT_PD = 4,      /* Cholesky of -H found a non-positive pivot: singular design     */
  MNL_ERR_NONFINITE = 5,   /* NaN/Inf in the data, the log-likelihood or the gradient        */
  MNL_ERR_LINESEARCH = 6,  /* no step size 2^-j, j <= max_halvings, kept l from decreasing    */
  MNL_MAXITER = 7,         /* mnl_fit: maxiter reached without meeting a tolerance (non-fatal) */
  MNL_ERR_TIMEOUT = 8,     /* a bounded device-side wait gave up; the result is invalid      */
  MNL_ERR_UNSUPPORTED = 9, /* valid request that the library does not implement             */
  MNL_PENDING = 10         /* mnl_server_poll: the request has not finished yet (non-fatal)  */
};

/* Arithmetic of the Hessian contraction.  In every mode the Cholesky solve,
 * the reductions across blocks and the convergence tests are float64.
 *   MNL_FP64: every step in float64 (CUDA-core DFMA).
 *   MNL_TF32: utilities, softmax, log-likelihood and gradient in float32 with
 *             compensated sums; A^T A on tcgen05 tensor cores with TF32 inputs
 *             and float32 accumulation; other Hessian blocks float32.
 *   MNL_BF16: as MNL_TF32 with BF16 tensor-core inputs, rounded stochastically
 *             (unbiased, reproducible); problems with fewer than 1024
 *             observations, too few for the rounding errors to average out,
 *             use TF32 inputs instead. */
typedef enum { MNL_FP64 = 0, MNL_TF32 = 1, MNL_BF16 = 2 } mnl_precision;

typedef struct mnl_dims {
  int64_t N;          /* observations, >= 1                       */
  int32_t K;          /* alternatives, >= 2                        */
  int32_t p, d, f;    /* columns of X, Y, Z (each >= 0, p+d+f >= 1) */
  int32_t gamma_base; /* 0 or 1, see above                         */
} mnl_dims;

typedef struct mnl_data {
  const float *X;
  const float *Y;
  const float *Z;
  const int32_t *choice;
} mnl_data;

typedef struct mnl_handle mnl_handle;

/* One Newton-Raphson iteration (mnl_newton_step). */
typedef struct mnl_step_info {
  double loglik_old; /* l(theta) before the step                    */
  double loglik_new; /* l(theta + t*delta) after the accepted step   */
  double grad_inf;   /* max_j |g_j| at theta before the step         */
  double step_inf;   /* max_j |t*delta_j|                            */
  double theta_inf;  /* max_j |theta_j| after the step               */
  double step_scale; /* t = 2^-halvings                              */
  double ls_noise;   /* tolerance tau the line search allowed        */
  int32_t halvings;  /* j of the accepted step                       */
  int32_t ls_evals;  /* log-likelihood evaluations in the line search */
  /* Device time per phase (CUDA events on the handle's stream):
   * pass = utilities/softmax/l/g; hess = every Hessian kernel; chol = factor + solve; ls = line search. */
  float t_pass_ms, t_hess_ms, t_chol_ms, t_ls_ms;
  /* Inside the Hessian and solve phases: operand build, A^T A contraction (all class blocks),
   * diagonal class blocks, Z blocks, assembly, factorisation (the whole mixed solve for
   * MNL_SOLVE_MIXED), triangular solves, float64 fallback of a mixed solve (0 when not taken). */
  float t_build_ms, t_syrk_ms, t_band_ms, t_zblk_ms, t_asm_ms, t_factor_ms, t_solve_ms, t_fallback_ms;
  int32_t launches;    /* kernels this library launched for the step        */
  int32_t solve_mode;  /* MNL_SOLVE_FP64 or MNL_SOLVE_MIXED, as used          */
  int32_t refine_steps;/* refinement steps of a mixed solve                 */
  int32_t fallback;    /* 1 when a mixed solve fell back to float64          */
  int32_t factor_kind; /* factorisation of the (first) solve: MNL_FACTOR_*   */
  int32_t wait_errors; /* after MNL_ERR_TIMEOUT: MNL_WAIT_* bits of the kernels whose waits gave up */
  int32_t cg_iters;    /* truncated Newton (MNL_CREATE_TRUNCATED): conjugate-gradient iterations */
} mnl_step_info;

/* mnl_step_info.wait_errors: which kernels' bounded device waits gave up
 * (the tensor-core contraction of the Hessian, the pass's tile copies, the
 * cooperative factorisation's grid barrier, the tensor-core trailing updates
 * of the panel factorisation). */
enum { MNL_WAIT_SYRK = 15, MNL_WAIT_PASS = 16, MNL_WAIT_COOP = 32, MNL_WAIT_PANEL = 64 };

/* mnl_step_info.factor_kind: the cooperative blocked Cholesky on the CUDA
 * cores (float32 in a mixed solve, float64 otherwise), or the panel
 * factorisation whose trailing updates run on the tensor cores (mixed solves
 * with n_theta >= 4096; environment variable MNL_TC_CHOL_MIN_N, read by
 * mnl_create, moves that threshold).  The panel factorisation runs the next
 * panel's diagonal and panel steps on a second stream that the handle owns,
 * ordered by events after the work already on the handle's stream and before
 * anything enqueued there later, so the stream semantics above still hold. */
enum { MNL_FACTOR_NONE = 0, MNL_FACTOR_COOP = 1, MNL_FACTOR_TENSOR = 2 };

typedef struct mnl_fit_opts {
  int32_t maxiter;      /* Newton iterations at most (paper default 50)              */
  int32_t max_halvings; /* line-search halvings at most                              */
  double gtol;          /* stop when max|g| < gtol before a step                     */
  double ftol;          /* stop when |l_new - l_old| < ftol after a step (0: off)      */
  double steptol;       /* stop when max|step| <= steptol * max(1, max|theta|) (0: off;
                           < 0: 1e-10 for MNL_FP64, 1e-7 for MNL_TF32 / MNL_BF16, whose
                           float32 gradient has a noise floor near 1e-8 relative)   */
} mnl_fit_opts;

/* Defaults: maxiter 50, max_halvings 30, gtol 1e-8, ftol 0, steptol -1 (per precision). */
MNL_API void mnl_fit_opts_default(mnl_fit_opts *opts);

/* MNL_STOP_NOISE (TF32 / BF16 only): the relative step stopped shrinking (it
 * fell by less than half in one iteration) while already below 1e-5, i.e. the
 * iterates reached the noise floor of the float32 gradient. */
enum { MNL_STOP_GTOL = 1, MNL_STOP_FTOL = 2, MNL_STOP_STEPTOL = 3, MNL_STOP_MAXITER = 4, MNL_STOP_NOISE = 5 };

typedef struct mnl_fit_info {
  int32_t iters;       /* Newton iterations taken                          */
  int32_t ls_evals;    /* log-likelihood evaluations in line searches      */
  int32_t stop_reason; /* MNL_STOP_* (0 when the fit ended in an error)     */
  int32_t status;      /* same value mnl_fit returned                      */
  double loglik;       /* l at the returned theta                          */
  double grad_inf;     /* max|g| at the last gradient evaluation           */
  double dloglik;      /* l change of the last step                        */
  double step_rel;     /* max|step| / max(1, max|theta|) of the last step    */
  double t_total_ms;   /* wall time of mnl_fit                             */
  double t_pass_ms, t_hess_ms, t_chol_ms, t_ls_ms; /* summed device time per phase */
} mnl_fit_info;

/* Number of coefficients, (K-1)p + (K-1 or K)d + f; -1 for invalid dims. */
MNL_API int64_t mnl_num_params(const mnl_dims *dims);

/* Static text for a status code (never NULL). */
MNL_API const char *mnl_status_string(int status);

/* Device bytes mnl_create would allocate for these dims and precision (0 on error). */
MNL_API size_t mnl_workspace_bytes(const mnl_dims *dims, int precision);

/* mnl_create_ex flags.  MNL_CREATE_TRUNCATED: a Hessian-free handle for
 * problems whose n_theta^2 Hessian does not fit (the paper's closing
 * discussion of inexact Newton for larger problems): every Newton step solves
 * (-H) delta = g approximately by conjugate gradients whose products -H v come
 * from a pass over the data (mnl_hessian_vec), stopped at a relative residual
 * eta = min(0.1, ||g||^(1/2)) (tending to 0 with g, so convergence stays fast
 * near the optimum), then the step halving of mnl_newton_step.  The handle
 * holds the data pass's buffers and a few n_theta vectors, no Hessian,
 * operand or factor workspaces; mnl_hessian, mnl_std_errors, mnl_shard_* and
 * mnl_set_solve (other than AUTO) return MNL_ERR_UNSUPPORTED on it. */
enum { MNL_CREATE_TRUNCATED = 1 };

/* Create a handle for one problem.
 *   dims      sizes (copied).
 *   data      DEVICE pointers to the caller's arrays, which must stay valid
 *             and unchanged until mnl_destroy; or NULL, in which case the
 *             handle allocates its own device copies, to be filled by
 *             mnl_upload before any computation.
 *   precision an mnl_precision value.
 *   stream    cudaStream_t (as void*) all work is enqueued on; NULL = default.
 *   out       receives the handle (NULL on error).
 * Allocates every workspace up front (mnl_workspace_bytes) and, when data is
 * given, validates it on the device: a choice outside [0, K) returns
 * MNL_ERR_INVALID_ARG, a NaN/Inf in X, Y or Z returns MNL_ERR_NONFINITE.
 * Synchronises the stream. */
MNL_API int mnl_create(const mnl_dims *dims, const mnl_data *data, int precision, void *stream, mnl_handle **out);
/* mnl_create with flags (0 or MNL_CREATE_TRUNCATED). */
MNL_API int mnl_create_ex(const mnl_dims *dims, const mnl_data *data, int precision, int flags, void *stream,
                          mnl_handle **out);

/* Hessian-vector product at theta (paper sign: H v, H negative definite),
 * without forming H: with u_ik = j_ik . v (j_ik the derivative of alternative
 * k's utility with respect to theta) and P the probabilities at theta,
 * -H v = sum_i sum_k P_ik (u_ik - sum_m P_im u_im) j_ik (App. A's Hessian
 * applied to v), one pass over the data.  theta, v, Hv: DEVICE [n_theta]
 * float64.  Synchronises.  Any handle. */
MNL_API int mnl_hessian_vec(mnl_handle *h, const double *theta, const double *v, double *Hv);
/* Conjugate-gradient iterations per truncated Newton step at most (default 500). */
MNL_API int mnl_set_cg_max(mnl_handle *h, int32_t iters);

/* Copy HOST arrays into the handle's own device buffers (handles created with
 * data = NULL only; otherwise MNL_ERR_INVALID_ARG), then validate them as
 * mnl_create does.  The copy is split into 32 MiB pieces over four internal
 * copy streams (several copy engines); it starts after the work already on
 * the handle's stream and completes before anything enqueued there later.
 * Pinned host memory makes the copy asynchronous and fast; pageable memory
 * works too.  Synchronises the stream. */
MNL_API int mnl_upload(mnl_handle *h, const mnl_data *host_data);

/* Log-likelihood and gradient at theta (eq. "log-lik function", eq. "loglik gradient").
 *   theta   DEVICE [n_theta] float64.
 *   loglik  HOST double, or NULL.  When given, the call synchronises the stream.
 *   grad    DEVICE [n_theta] float64, or NULL; written in stream order. */
MNL_API int mnl_loglik_grad(mnl_handle *h, const double *theta, double *loglik, double *grad);

/* Hessian of l at theta (eq. "hessian block"), paper sign (negative definite).
 *   theta DEVICE [n_theta] float64.
 *   H     DEVICE [n_theta][n_theta] float64, column-major, both triangles
 *         written (the matrix is symmetric); enqueued in stream order. */
MNL_API int mnl_hessian(mnl_handle *h, const double *theta, double *H);

/* One Newton-Raphson iteration with step halving (eq. "NR update", Sec. 3.1):
 * computes l, g, H at theta, solves (-H) delta = g by Cholesky, evaluates
 * l(theta + 2^-j delta) for j = 0, 1, ... and accepts the first step whose
 * log-likelihood is not lower than l(theta) by more than the rounding noise
 * of the sum (info->ls_noise).  theta is DEVICE [n_theta] float64, updated in
 * place only when the call returns MNL_OK.  info (HOST) may be NULL.
 * Synchronises the stream.  Errors: MNL_ERR_NOT_PD, MNL_ERR_NONFINITE,
 * MNL_ERR_LINESEARCH, MNL_ERR_TIMEOUT, MNL_ERR_CUDA. */
MNL_API int mnl_newton_step(mnl_handle *h, double *theta, mnl_step_info *info);

/* Newton-Raphson to convergence (Sec. 3.1; stopping rules of Sec. 2.3:
 * maxiter, ftol, gtol; plus the relative step test steptol).
 *   opts  HOST, or NULL for mnl_fit_opts_default.
 *   theta DEVICE [n_theta] float64: start in, estimate out.
 *   info  HOST, may be NULL.
 * Returns MNL_OK when a tolerance was met, MNL_MAXITER when maxiter ran out
 * (theta holds the last iterate), or an error of mnl_newton_step. */
MNL_API int mnl_fit(mnl_handle *h, const mnl_fit_opts *opts, double *theta, mnl_fit_info *info);

/* Asymptotic standard errors at theta (normally the estimate): se_j =
 * sqrt((F^{-1})_jj), F = -H the observed information (the coefficient table
 * of the package's summary method, Sec. 2.3).  F is formed as by
 * mnl_hessian (in the handle's precision), factored in float64 together with
 * the inverse of its factor, F^{-1} = L^{-T} L^{-1}, and se_j is the norm of
 * column j of L^{-1}.  The first call allocates an n_theta^2 float64 buffer,
 * kept until mnl_destroy.
 *   theta  DEVICE [n_theta] float64;  se  DEVICE [n_theta] float64.
 * Synchronises the stream.  MNL_ERR_NOT_PD when F is not positive definite. */
MNL_API int mnl_std_errors(mnl_handle *h, const double *theta, double *se);

/* Choice probabilities at theta (the package's predict method, Sec. 2.3;
 * eqs. "probability", "base probability"), for the handle's data - a handle
 * on new data predicts for those.
 *   P       DEVICE [N][K] float64, row-major.
 *   loglik  HOST, or NULL: l(theta) of the handle's choices (synchronises).
 * Computed by the same pass as mnl_loglik_grad (float32 in the TF32 / BF16
 * modes, float64 in MNL_FP64). */
MNL_API int mnl_predict(mnl_handle *h, const double *theta, double *P, double *loglik);

/* Collinearity check of the data (the `linDepTol` argument of the package's
 * mnlogit call, Sec. 2.3; App. B's necessary conditions for a non-singular
 * Hessian): X and every Y_k need linearly independent columns, and so do the
 * generic variables' normalized columns (the N (K-1) rows Z_ik - Z_i0, k >= 1,
 * stacked).  Within each block the columns are taken in order and column j is
 * flagged when the part of it orthogonal to the unflagged earlier columns has
 * a norm of at most tol * ||column j|| - a rank-revealing factorisation that
 * drops the later columns of a collinear set one by one.  Computed on the
 * device in float64: the blocks' Gram matrices from one pass over the data
 * (float32 products are exact in float64), then per block an in-order Cholesky
 * factorisation that flags column j when its pivot is at most tol^2 times the
 * column's squared norm.  Observation weights play no part.
 *   tol       > 0 (the package's default linDepTol is 1e-6).
 *   flags     HOST int32 [p + K d + f]: X column j at j; column j of Y_k at
 *             p + k d + j (Y_0's entries are 0 unless gamma_base = 1); Z column
 *             j at p + K d + j.  1: dependent, 0: kept.
 *   ndropped  HOST, or NULL: the number of flags set.
 * Synchronises.  Allocates (and frees before returning) scratch for the Gram
 * matrices (the sum of the blocks' cols^2 doubles) and their partial tiles.
 * MNL_ERR_INVALID_ARG for tol <= 0 or NULL flags. */
MNL_API int mnl_check_collinear(mnl_handle *h, double tol, int32_t *flags, int32_t *ndropped);

/* Remove flagged columns from the model, as the package does with collinear
 * columns before it fits.  Their coefficients - beta_k[j] for every k when X
 * column j is flagged, gamma_k[j] for column j of Y_k, alpha[j] for Z column j
 * - are held at their current values (zero in a fit from theta = 0, which is
 * the fit of the model without those columns) by mnl_newton_step, mnl_fit,
 * mnl_shard_solve and mnl_std_errors (whose entries for them are NaN): their
 * gradient entries count as zero and their rows and columns of -H are those
 * of the identity in the Newton system.  mnl_loglik_grad, mnl_hessian,
 * mnl_hessian_vec and mnl_predict still describe the full model.
 *   flags  HOST int32 [p + K d + f] in the layout of mnl_check_collinear (Y_0
 *          entries are ignored when gamma_base = 0), or NULL to restore the
 *          full model.
 * MNL_ERR_INVALID_ARG for a flag other than 0 or 1.  Synchronises. */
MNL_API int mnl_drop_columns(mnl_handle *h, const int32_t *flags);

/* How mnl_newton_step / mnl_fit solve (-H) delta = g.
 *   MNL_SOLVE_FP64:  blocked float64 Cholesky and float64 triangular solves.
 *   MNL_SOLVE_MIXED: float32 Cholesky of -H and float64 iterative refinement
 *                    (residuals g - (-H) delta in float64) until the correction
 *                    is below 1e-12 of delta or stagnates below 1e-8 of it;
 *                    if the float32 factorisation or the refinement fails, the
 *                    step falls back to MNL_SOLVE_FP64.  On GB300 float64 runs
 *                    at about 1/67 of the float32 rate, which makes this the
 *                    faster route to a float64-accurate step.
 *   MNL_SOLVE_AUTO (default): FP64 for MNL_FP64 handles, MIXED otherwise. */
enum { MNL_SOLVE_AUTO = 0, MNL_SOLVE_FP64 = 1, MNL_SOLVE_MIXED = 2 };
MNL_API int mnl_set_solve(mnl_handle *h, int mode);

/* ------------------------------------------------------------------------
 * Observation sharding (several GPUs, one process each).  l, g and -H are
 * sums over the observations (eqs. "log-lik function", "loglik gradient",
 * "hessian block"), so with the observations split over the GPUs one Newton
 * step is: every rank forms its partial sums (mnl_shard_grad_hess), the sums
 * are added across ranks (one all-reduce of mnl_shard_sums_size doubles),
 * every rank solves the same system (mnl_shard_solve: identical inputs give
 * identical steps), and each line-search trial adds the ranks' partial
 * log-likelihoods (mnl_shard_loglik; an all-reduce of two doubles).  The
 * exchange itself is the caller's (e.g. NCCL); gamma_base = 1 handles return
 * MNL_ERR_UNSUPPORTED.
 * ------------------------------------------------------------------------ */

/* 2 + n + n (n + 1) / 2 for n = n_theta (-1 for invalid dims). */
MNL_API int64_t mnl_shard_sums_size(const mnl_dims *dims);
/* This handle's partial sums at theta (DEVICE [n_theta] float64) into sums
 * (DEVICE float64 [mnl_shard_sums_size]): [0] l, [1] sum_i |l_i| (the line
 * search's rounding allowance), [2 .. 2 + n) g, then the lower triangle of
 * -H packed column by column (entry (r, c), r >= c, at 2 + n + c n - c (c - 1)
 * / 2 + r - c).  Synchronises. */
MNL_API int mnl_shard_grad_hess(mnl_handle *h, const double *theta, double *sums);
/* delta (DEVICE [n_theta]) solving (-H) delta = g from summed sums (DEVICE),
 * with the handle's solve mode (as mnl_newton_step).  info (HOST, may be
 * NULL) receives solve_mode, factor_kind, refine_steps, fallback and
 * t_factor_ms.  Synchronises.  MNL_ERR_NOT_PD for a singular -H. */
MNL_API int mnl_shard_solve(mnl_handle *h, const double *sums, double *delta, mnl_step_info *info);
/* This handle's partial [l, sum_i |l_i|] at theta + t delta (delta NULL:
 * at theta) into l2 (DEVICE [2] float64).  Synchronises. */
MNL_API int mnl_shard_loglik(mnl_handle *h, const double *theta, const double *delta, double t, double *l2);
/* Unit roundoff of the arithmetic of this handle's log-likelihood (2^-53 in
 * MNL_FP64, 2^-24 otherwise): a line search over summed l accepts a step when
 * l_new >= l_old - 8 u sum_i |l_i|, as mnl_newton_step does. */
MNL_API double mnl_loglik_roundoff(const mnl_handle *h);

/* Observation weights (the `weights` argument of the package's mnlogit call,
 * Sec. 2.3), read as case weights: observation i counts w_i times in l, g and
 * H (l = sum_i w_i l_i; integer weights equal repeated rows).
 *   w  DEVICE [N] float32, 16-byte aligned, finite and >= 0, owned by the
 *      caller and unchanged until the handle is destroyed or the weights are
 *      replaced; NULL removes them (all ones).
 * Validates on the device (synchronises): MNL_ERR_NONFINITE for NaN/Inf,
 * MNL_ERR_INVALID_ARG for a negative weight or a misaligned pointer. */
MNL_API int mnl_set_weights(mnl_handle *h, const float *w);

/* Bound, in nanoseconds, of every bounded device-side wait of this handle's
 * kernels (pipeline stages, tile copies, grid barriers); 0 restores their
 * defaults (2 s, 4 s for a grid barrier).  A wait that runs out makes every
 * block of its kernel stop (after waiting, with the default bound, for the
 * copies and tensor-core operations it has issued) and the call returns
 * MNL_ERR_TIMEOUT; the handle stays usable.  A bound shorter than the work
 * between two waits makes every call time out: it exists to test that path. */
MNL_API int mnl_set_wait_bound(mnl_handle *h, uint64_t ns);

/* Free the handle and every device buffer it owns (NULL is a no-op). */
MNL_API int mnl_destroy(mnl_handle *h);

/* ------------------------------------------------------------------------
 * Batched fits: many independent problems of uneven N, K, p, d, f advanced
 * together (Sec. 3.1 Newton-Raphson with step halving, per problem).  Every
 * Newton phase is one grouped kernel launch over all problems still
 * iterating; one iteration is captured once as a CUDA graph and replayed.
 * ------------------------------------------------------------------------ */
typedef struct mnl_batch mnl_batch;

typedef struct mnl_batch_problem_info {
  int32_t status;      /* MNL_OK (a tolerance was met), MNL_MAXITER, or an MNL_ERR_* */
  int32_t stop_reason; /* MNL_STOP_* (0 after an error)                          */
  int32_t iters;       /* Newton iterations taken                                 */
  int32_t ls_evals;    /* log-likelihood evaluations in line searches             */
  double loglik;       /* l at the returned theta                                 */
  double grad_inf;     /* max|g| at the last gradient evaluation                  */
} mnl_batch_problem_info;

typedef struct mnl_batch_info {
  mnl_batch_problem_info *problems; /* HOST [count] or NULL, filled by mnl_batch_fit */
  int32_t iterations;  /* Newton iterations of the slowest problem      */
  int32_t converged;   /* problems that met a tolerance                 */
  int32_t failed;      /* problems that ended with an error             */
  int32_t pass_rows;   /* observations per tile of the grouped pass (autotuned) */
  double t_total_ms;   /* wall time of mnl_batch_fit                    */
  double t_graph_ms;   /* device time of the replayed iteration graphs  */
} mnl_batch_info;

/* Create a batch of `count` problems.
 *   dims[i], data[i]  as for mnl_create, DEVICE pointers that must stay valid
 *                     and unchanged until mnl_batch_destroy (not validated).
 *   precision         as for mnl_create; the Newton solves run per problem in
 *                     one CTA (float32 factor + float64 refinement for TF32 /
 *                     BF16, float64 for MNL_FP64).
 *   stream            cudaStream_t (as void*): mnl_batch_fit orders its work
 *                     after, and before, the caller's work on this stream (it
 *                     runs on an internal stream so it can capture a graph).
 * Allocates every workspace (one arena) and autotunes the pass tile height
 * (timed once; cached per batch shape in the process and, if the environment
 * variable MNL_TUNE_CACHE names a file, in that file).  Limits: n_theta <= 1400
 * per problem, K <= 256; else MNL_ERR_UNSUPPORTED. */
MNL_API int mnl_batch_create(int count, const mnl_dims *dims, const mnl_data *data, int precision, void *stream,
                             mnl_batch **out);

/* Total number of coefficients; offsets (HOST [count], may be NULL) receives
 * where problem i's coefficients start in the packed theta vector. */
MNL_API int64_t mnl_batch_num_params(const mnl_batch *b, int64_t *offsets);

/* Fit every problem from the start values in theta (DEVICE, packed, float64,
 * mnl_batch_num_params entries; estimates are written back in place).
 * opts: as for mnl_fit (NULL: defaults).  info (HOST, may be NULL).
 * Returns MNL_OK when every problem met a tolerance, else the status of the
 * first problem that ended with an error, else MNL_MAXITER; per-problem
 * results are in info->problems.  Synchronises. */
MNL_API int mnl_batch_fit(mnl_batch *b, const mnl_fit_opts *opts, double *theta, mnl_batch_info *info);

MNL_API int mnl_batch_destroy(mnl_batch *b);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of fit requests.  Requests are admitted while
 * their device state fits in a fixed memory budget; every mnl_server_step
 * ("tick") runs one Newton iteration for all admitted requests together (the
 * same grouped launches as mnl_batch_fit), retires the ones that finished and
 * frees their memory for the next admissions.  Each request's data,
 * coefficients, P, gradient and Hessian stay on the device from admission to
 * retirement.  Submit and poll may be called from other threads.
 * ------------------------------------------------------------------------ */
typedef struct mnl_server mnl_server;

typedef struct mnl_server_opts {
  size_t mem_budget;   /* device bytes for admitted requests (one pool, allocated at create) */
  int32_t precision;   /* an mnl_precision value                                        */
  int32_t max_active;  /* admitted requests at most                                     */
  int32_t max_skips;   /* times a queued request may be passed over by later, smaller
                          ones before admission waits for it (FIFO fairness)            */
  int32_t pad;
  mnl_fit_opts fit;    /* stopping rules of every request                               */
} mnl_server_opts;

typedef struct mnl_request_result {
  int32_t status;      /* MNL_OK, MNL_MAXITER or an MNL_ERR_*          */
  int32_t stop_reason; /* MNL_STOP_*                                   */
  int32_t iters;       /* Newton iterations (= ticks while admitted)   */
  int32_t ls_evals;
  double loglik, grad_inf;
  double latency_ms;   /* submit -> retirement (host clock)            */
  double queue_ms;     /* submit -> admission                          */
} mnl_request_result;

/* Defaults: 80 GiB budget, MNL_BF16, 4096 active, 8 skips, mnl_fit_opts_default. */
MNL_API void mnl_server_opts_default(mnl_server_opts *opts);
MNL_API int mnl_server_create(const mnl_server_opts *opts, void *stream, mnl_server **out);
/* Queue a request.  host: HOST arrays (copied before the call returns);
 * theta0: HOST [n_theta] start values or NULL (zeros).  MNL_ERR_OOM when the
 * request could never fit the budget; MNL_ERR_INVALID_ARG for a choice out of
 * range; MNL_ERR_UNSUPPORTED for gamma_base = 1, K > 256 or more than 16384
 * raw gradient sums ((K-1)(p+d) + K f).  Requests with n_theta up to 1400 are
 * solved by one CTA each inside the grouped launches; larger ones by the
 * multi-CTA mixed (or, in MNL_FP64, float64) factorisation, one at a time. */
MNL_API int mnl_server_submit(mnl_server *s, const mnl_dims *dims, const mnl_data *host, const double *theta0,
                              uint64_t *ticket);
/* One tick: admit, iterate, retire.  Returns the numbers still admitted and queued. */
MNL_API int mnl_server_step(mnl_server *s, int32_t *n_active, int32_t *n_queued);
/* MNL_OK and the result (theta: HOST [n_theta] or NULL) once the request has
 * finished - the ticket is then released; MNL_PENDING before that. */
MNL_API int mnl_server_poll(mnl_server *s, uint64_t ticket, double *theta, mnl_request_result *result);
/* Tickets of requests that finished since the previous call (up to cap of
 * them, oldest first; those beyond cap are kept for the next call), so that a
 * caller polls only requests that are done.  *count receives how many were
 * written to tickets (HOST [cap]). */
MNL_API int mnl_server_finished(mnl_server *s, uint64_t *tickets, int32_t cap, int32_t *count);
/* Device bytes held by admitted requests. */
MNL_API size_t mnl_server_memory_in_use(const mnl_server *s);
MNL_API int mnl_server_destroy(mnl_server *s);

/* Log-likelihood and gradient, as mnl_loglik_grad, without allocating any
 * device memory.  The paper has no counterpart: this is for callers that
 * cannot call cudaMalloc when they need l and g - code whose device memory
 * is owned by an arena or pool, plug-ins of hosts that forbid allocation
 * after start-up, latency-critical loops where an allocation could block or
 * fail.  It creates no handle; every input and output belongs to the caller.
 *   dims, data  as for mnl_create (DEVICE pointers).  The data are not
 *               validated: choices must lie in [0, K) and values be finite.
 *   precision   MNL_FP64: the pass runs in float64; MNL_TF32 / MNL_BF16:
 *               float32 with compensated sums (the Hessian precision does not
 *               matter here).
 *   theta       DEVICE [n_theta] float64.
 *   loglik      DEVICE, one float64.
 *   grad        DEVICE [n_theta] float64.
 *   P           DEVICE [N][K] choice probabilities (float64 for MNL_FP64,
 *               float32 otherwise).
 *   zbar        DEVICE [N][f] expected Z per observation, sum_k P_ik Z_ik
 *               (same type as P); NULL when f = 0.
 *   stream      cudaStream_t (as void*); the call only enqueues work.
 * Limits: (K-1)(p+d) + K f <= 16384 raw gradient sums and K <= 256, and the
 * pass's tile of one observation's X, Y, Z rows must fit its shared memory
 * (p + K (d + f) up to about 50000 floats); beyond them the call returns
 * MNL_ERR_UNSUPPORTED (the size limits before any CUDA call).
 * Scratch: a fixed 4 MiB array inside the library holds the per-block partial
 * sums between the two kernels of the pass ((K-1)(p+d) + f + 2 doubles per
 * block; large problems run on fewer blocks so that they fit); every GPU that
 * loads the library keeps it until the process exits.  The first call on each
 * device (and after a device reset, in the new context) looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.
 * All calls share the one array: calls that can overlap on the GPU (other
 * streams, other threads) race and corrupt each other's results, so order
 * them, e.g. on one stream.  Nothing in the array needs to start at zero;
 * every call overwrites what it later reads. */
MNL_API int mnl_loglik_grad_noalloc(const mnl_dims *dims, const mnl_data *data, int precision, const double *theta,
                                    double *loglik, double *grad, void *P, void *zbar, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MNL_H */
