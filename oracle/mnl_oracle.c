/*
 * Plain FP64 CPU oracle for the multinomial-logit Newton-Raphson fit.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or constant
 * with the CUDA implementation.
 *
 * The oracle is the plain definition of what the method computes, written in
 * the paper's notation (Sec. 2.1 and Sec. 3):
 *
 *   normalized utility (eq. "normalized utility"), base alternative k = 0:
 *     V_i0 = 0,
 *     V_ik = X_i.beta_k + Y_ik.gamma_k - Y_i0.gamma_0 + (Z_ik - Z_i0).alpha,   k = 1..K-1
 *     (the Y_i0.gamma_0 term exists only when gamma_0 is estimated, gamma_base = 1;
 *      with gamma_base = 0 the Y_i0 block is ignored and gamma_0 = 0)
 *   probabilities (eqs. "probability", "base probability"):
 *     P_i0 = 1 / (1 + sum_{k>=1} exp V_ik),   P_ik = P_i0 exp V_ik
 *   log-likelihood (eq. "log-lik function"):
 *     l = sum_i [ -log(1 + sum_{k>=1} exp V_ik) + sum_{k>=1} V_ik I(y_i = k) ]
 *
 * Let j_ik = dV_ik/dtheta (the "design row" of alternative k; j_i0 = 0).
 * Because V is affine in theta, differentiating l gives (App. A)
 *     dl/dtheta   = sum_i ( j_{i,y_i} - sum_k P_ik j_ik )
 *     -d2l/dtheta2 = sum_i [ sum_k P_ik j_ik j_ik^T - jbar_i jbar_i^T ],  jbar_i = sum_k P_ik j_ik,
 * which, block by block, is eq. "hessian block" with W_nm = diag(P_n (delta_nm - P_m)).
 * The negative Hessian is formed by explicit rank-1 updates per observation.
 *
 * Coefficient order (eq. "theta vec"): beta_1..beta_{K-1} (p each),
 * gamma_0..gamma_{K-1} (d each; gamma_0 only when gamma_base = 1), alpha (f).
 *
 * Observation weights (the `weights` argument of the package's mnlogit call,
 * Sec. 2.3; the paper does not define them further) are read as case weights:
 * observation i counts w_i times, so l, dl/dtheta and d2l/dtheta2 are the sums
 * above with each term multiplied by w_i (NULL weights: all ones).
 *
 * Readings of points the paper leaves open: exp/log use a max shift (equal in
 * exact arithmetic to eq. "base probability"); the line search accepts the
 * first halved step whose log-likelihood is not lower (Sec. 3.1), "not lower"
 * meaning not lower by more than the rounding noise of the FP64 sum
 * (ls_rel_tol*|l|, a few units of roundoff), with a cap on the number of
 * halvings; the Newton system is solved by a textbook Cholesky factorisation
 * of -H.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t N;
  int32_t K, p, d, f, gamma_base;
  const float *X;        /* [N][p]    */
  const float *Y;        /* [N][K][d] */
  const float *Z;        /* [N][K][f] */
  const int32_t *choice; /* [N], 0..K-1, 0 = base */
  const float *w;        /* [N] observation weights (>= 0), or NULL for all ones */
} oracle_problem;

typedef struct {
  int32_t maxiter;      /* Newton iterations at most                       */
  int32_t max_halvings; /* line-search halvings at most                    */
  double gtol;          /* stop when max_j |g_j| < gtol                    */
  double ftol;          /* stop when |l_new - l_old| < ftol (0 disables)    */
  double steptol;       /* stop when max|step| <= steptol*max(1,max|theta|) */
  int32_t nthreads;     /* threads for the Hessian (<= 0: all)             */
  double ls_rel_tol;    /* line search accepts l_new >= l_old - ls_rel_tol*|l_old| */
} oracle_fit_opts;

typedef struct {
  int32_t iters;      /* Newton iterations taken                  */
  int32_t ls_evals;   /* log-likelihood evaluations in line searches */
  int32_t stop;       /* 1 gtol, 2 ftol, 3 steptol, 4 maxiter, <0 error */
  int32_t pad;
  double loglik;      /* l at the returned theta                   */
  double grad_inf;    /* max |g| at the last gradient evaluation   */
} oracle_fit_stats;

int64_t oracle_num_params(int K, int p, int d, int f, int gamma_base) {
  return (int64_t)(K - 1) * p + (int64_t)(gamma_base ? K : K - 1) * d + f;
}

static int64_t n_params(const oracle_problem *P) {
  return oracle_num_params(P->K, P->p, P->d, P->f, P->gamma_base);
}
static int64_t beta_off(const oracle_problem *P, int k) { return (int64_t)(k - 1) * P->p; }
static int64_t gamma_off(const oracle_problem *P, int k) {
  int64_t b = (int64_t)(P->K - 1) * P->p;
  return P->gamma_base ? b + (int64_t)k * P->d : b + (int64_t)(k - 1) * P->d;
}
static int64_t alpha_off(const oracle_problem *P) { return n_params(P) - P->f; }

/* Sparse design row j_ik: its nonzero positions and values. */
typedef struct {
  int64_t *idx;
  double *val;
  int n;
} srow;

static void design_row(const oracle_problem *P, int64_t i, int k, srow *r) {
  r->n = 0;
  if (k == 0) return; /* V_i0 = 0 */
  const int p = P->p, d = P->d, f = P->f, K = P->K;
  const float *x = P->X + i * p;
  for (int j = 0; j < p; ++j) { r->idx[r->n] = beta_off(P, k) + j; r->val[r->n++] = (double)x[j]; }
  const float *y = P->Y + (i * K + k) * d;
  for (int j = 0; j < d; ++j) { r->idx[r->n] = gamma_off(P, k) + j; r->val[r->n++] = (double)y[j]; }
  if (P->gamma_base) {
    const float *y0 = P->Y + (i * K) * d;
    for (int j = 0; j < d; ++j) { r->idx[r->n] = gamma_off(P, 0) + j; r->val[r->n++] = -(double)y0[j]; }
  }
  const float *z = P->Z + (i * K + k) * f;
  const float *z0 = P->Z + (i * K) * f;
  for (int j = 0; j < f; ++j) { r->idx[r->n] = alpha_off(P) + j; r->val[r->n++] = (double)z[j] - (double)z0[j]; }
}

static int row_capacity(const oracle_problem *P) { return P->p + 2 * P->d + P->f + 1; }

/* Weight of observation i (1 when no weights are given). */
static double weight(const oracle_problem *P, int64_t i) { return P->w ? (double)P->w[i] : 1.0; }

typedef struct {
  srow *rows; /* K rows */
  double *V;  /* K */
  double *pr; /* K */
  int64_t *idx_store;
  double *val_store;
} obs_work;

static int work_init(const oracle_problem *P, obs_work *w) {
  const int K = P->K, cap = row_capacity(P);
  w->rows = (srow *)malloc(sizeof(srow) * K);
  w->V = (double *)malloc(sizeof(double) * K);
  w->pr = (double *)malloc(sizeof(double) * K);
  w->idx_store = (int64_t *)malloc(sizeof(int64_t) * (size_t)K * cap);
  w->val_store = (double *)malloc(sizeof(double) * (size_t)K * cap);
  if (!w->rows || !w->V || !w->pr || !w->idx_store || !w->val_store) return -1;
  for (int k = 0; k < K; ++k) {
    w->rows[k].idx = w->idx_store + (size_t)k * cap;
    w->rows[k].val = w->val_store + (size_t)k * cap;
  }
  return 0;
}
static void work_free(obs_work *w) {
  free(w->rows); free(w->V); free(w->pr); free(w->idx_store); free(w->val_store);
}

/* Design rows, utilities V_ik, probabilities P_ik and the log-likelihood term
 * of observation i.  Returns l_i. */
static double observation(const oracle_problem *P, const double *theta, int64_t i, obs_work *w) {
  const int K = P->K;
  double vmax = 0.0; /* V_i0 = 0 */
  for (int k = 0; k < K; ++k) {
    design_row(P, i, k, &w->rows[k]);
    double v = 0.0;
    for (int e = 0; e < w->rows[k].n; ++e) v += w->rows[k].val[e] * theta[w->rows[k].idx[e]];
    w->V[k] = v;
    if (v > vmax) vmax = v;
  }
  /* log(1 + sum_{k>=1} exp V_ik) with a max shift. */
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += exp(w->V[k] - vmax);
  const double lse = vmax + log(s);
  for (int k = 0; k < K; ++k) w->pr[k] = exp(w->V[k] - lse);
  return w->V[P->choice[i]] - lse;
}

int oracle_check(const oracle_problem *P) {
  if (P->N < 0 || P->K < 2 || P->p < 0 || P->d < 0 || P->f < 0) return -1;
  for (int64_t i = 0; i < P->N; ++i)
    if (P->choice[i] < 0 || P->choice[i] >= P->K) return -2;
  if (P->w)
    for (int64_t i = 0; i < P->N; ++i)
      if (!(P->w[i] >= 0.0f) || !isfinite(P->w[i])) return -4;
  return 0;
}

/* Probabilities P[i][k] and l. */
int oracle_probs(const oracle_problem *P, const double *theta, double *prob, double *loglik) {
  obs_work w;
  if (oracle_check(P)) return -1;
  if (work_init(P, &w)) return -3;
  double l = 0.0;
  for (int64_t i = 0; i < P->N; ++i) {
    l += weight(P, i) * observation(P, theta, i, &w);
    for (int k = 0; k < P->K; ++k) prob[i * P->K + k] = w.pr[k];
  }
  work_free(&w);
  if (loglik) *loglik = l;
  return 0;
}

/* l and dl/dtheta = sum_i (j_{i,y_i} - sum_k P_ik j_ik). */
int oracle_loglik_grad(const oracle_problem *P, const double *theta, double *loglik, double *grad) {
  obs_work w;
  if (oracle_check(P)) return -1;
  if (work_init(P, &w)) return -3;
  const int64_t n = n_params(P);
  if (grad) memset(grad, 0, sizeof(double) * n);
  double l = 0.0;
  for (int64_t i = 0; i < P->N; ++i) {
    const double wi = weight(P, i);
    l += wi * observation(P, theta, i, &w);
    if (!grad) continue;
    const srow *ry = &w.rows[P->choice[i]];
    for (int e = 0; e < ry->n; ++e) grad[ry->idx[e]] += wi * ry->val[e];
    for (int k = 0; k < P->K; ++k)
      for (int e = 0; e < w.rows[k].n; ++e) grad[w.rows[k].idx[e]] -= wi * w.pr[k] * w.rows[k].val[e];
  }
  work_free(&w);
  if (loglik) *loglik = l;
  return 0;
}

/* Negative Hessian F = -d2l/dtheta2 (n x n, row-major, full symmetric):
 *   F = sum_i [ sum_k P_ik j_ik j_ik^T - jbar_i jbar_i^T ].
 * The lower triangle is accumulated by rank-1 updates observation by
 * observation; threads own disjoint bands of rows of F, so the result does
 * not depend on the thread count. */
int oracle_neg_hessian(const oracle_problem *P, const double *theta, double *F, int nthreads) {
  if (oracle_check(P)) return -1;
  const int64_t n = n_params(P), N = P->N;
  const int K = P->K;
  memset(F, 0, sizeof(double) * (size_t)n * n);
  double *prob = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * K);
  if (!prob) return -3;
  if (oracle_probs(P, theta, prob, NULL)) { free(prob); return -1; }
  const int64_t RB = 64;
  const int64_t nblk = (n + RB - 1) / RB;
  int err = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t blk = 0; blk < nblk; ++blk) {
    const int64_t a0 = blk * RB, a1 = (a0 + RB < n) ? a0 + RB : n;
    obs_work w;
    double *jbar = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (work_init(P, &w) || !jbar) { err = 1; continue; }
    for (int64_t i = 0; i < N; ++i) {
      const double *pr = prob + i * K;
      const double wi = weight(P, i);
      for (int k = 0; k < K; ++k) design_row(P, i, k, &w.rows[k]);
      /* jbar_i = sum_k P_ik j_ik (only entries below a1 are needed) */
      for (int64_t a = 0; a < a1; ++a) jbar[a] = 0.0;
      for (int k = 0; k < K; ++k)
        for (int e = 0; e < w.rows[k].n; ++e)
          if (w.rows[k].idx[e] < a1) jbar[w.rows[k].idx[e]] += pr[k] * w.rows[k].val[e];
      /* + sum_k P_ik j_ik j_ik^T */
      for (int k = 0; k < K; ++k) {
        const srow *r = &w.rows[k];
        for (int e = 0; e < r->n; ++e) {
          const int64_t a = r->idx[e];
          if (a < a0 || a >= a1) continue;
          const double wa = wi * pr[k] * r->val[e];
          for (int e2 = 0; e2 < r->n; ++e2)
            if (r->idx[e2] <= a) F[a * n + r->idx[e2]] += wa * r->val[e2];
        }
      }
      /* - jbar_i jbar_i^T */
      for (int64_t a = a0; a < a1; ++a) {
        const double ja = wi * jbar[a];
        if (ja == 0.0) continue;
        double *Fa = F + a * n;
        for (int64_t b = 0; b <= a; ++b) Fa[b] -= ja * jbar[b];
      }
    }
    work_free(&w);
    free(jbar);
  }
  free(prob);
  if (err) return -3;
  for (int64_t a = 0; a < n; ++a)
    for (int64_t b = 0; b < a; ++b) F[b * n + a] = F[a * n + b];
  return 0;
}

/* Value of j_ik at coefficient position a (0 when a is not in alternative k's row). */
static double design_entry(const oracle_problem *P, int64_t i, int k, int64_t a) {
  if (k == 0) return 0.0;
  const int p = P->p, d = P->d, f = P->f, K = P->K;
  const int64_t ab = beta_off(P, 1), ag = gamma_off(P, P->gamma_base ? 0 : 1), aa = alpha_off(P);
  if (a >= aa) {
    const int j = (int)(a - aa);
    return (double)P->Z[(i * K + k) * f + j] - (double)P->Z[(i * K) * f + j];
  }
  if (a >= ag) {
    const int64_t r = a - ag;
    const int cls = (int)(r / d) + (P->gamma_base ? 0 : 1), j = (int)(r % d);
    if (cls == 0) return -(double)P->Y[(i * K) * d + j];
    return cls == k ? (double)P->Y[(i * K + k) * d + j] : 0.0;
  }
  const int cls = (int)((a - ab) / p) + 1, j = (int)((a - ab) % p);
  return cls == k ? (double)P->X[i * p + j] : 0.0;
}

/* Selected entries F[rows[e]][cols[e]] of the negative Hessian, each summed
 * over all observations from the definition above. */
int oracle_neg_hessian_entries(const oracle_problem *P, const double *theta, int64_t E, const int64_t *rows,
                               const int64_t *cols, double *out, int nthreads) {
  if (oracle_check(P)) return -1;
  const int64_t N = P->N;
  const int K = P->K;
  double *prob = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * K);
  if (!prob) return -3;
  if (oracle_probs(P, theta, prob, NULL)) { free(prob); return -1; }
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t e = 0; e < E; ++e) {
    const int64_t a = rows[e], b = cols[e];
    double acc = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      const double *pr = prob + i * K;
      double s = 0.0, ja = 0.0, jb = 0.0;
      for (int k = 1; k < K; ++k) {
        const double va = design_entry(P, i, k, a), vb = design_entry(P, i, k, b);
        s += pr[k] * va * vb;
        ja += pr[k] * va;
        jb += pr[k] * vb;
      }
      acc += weight(P, i) * (s - ja * jb);
    }
    out[e] = acc;
  }
  free(prob);
  return 0;
}

/* Textbook column Cholesky A = L L^T (row-major n x n, lower triangle used).
 * Returns 0, or -1 when a pivot is not positive (A not positive definite). */
int oracle_cholesky(int64_t n, double *A) {
  for (int64_t j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0) || !isfinite(s)) return -1;
    const double ljj = sqrt(s);
    A[j * n + j] = ljj;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n - j > 256)
#endif
    for (int64_t i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / ljj;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
  return 0;
}

/* Solve L L^T x = b in place (forward then back substitution). */
int oracle_cholesky_solve(int64_t n, const double *L, double *b) {
  for (int64_t i = 0; i < n; ++i) {
    double t = b[i];
    for (int64_t k = 0; k < i; ++k) t -= L[i * n + k] * b[k];
    b[i] = t / L[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (int64_t k = i + 1; k < n; ++k) t -= L[k * n + i] * b[k];
    b[i] = t / L[i * n + i];
  }
  return 0;
}

static double max_abs(const double *v, int64_t n) {
  double m = 0.0;
  for (int64_t j = 0; j < n; ++j) if (fabs(v[j]) > m) m = fabs(v[j]);
  return m;
}

/* Newton-Raphson (eq. "NR update"): theta_new = theta + t * dtheta with
 * dtheta = (-H)^{-1} g, and t = 1, 1/2, 1/4, ... until l(theta_new) >= l(theta). */
int oracle_fit(const oracle_problem *P, const oracle_fit_opts *o, double *theta, oracle_fit_stats *st) {
  if (oracle_check(P)) return -1;
  const int64_t n = n_params(P);
  double *g = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *F = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (n > 0 ? n : 1));
  double *step = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *trial = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  if (!g || !F || !step || !trial) { free(g); free(F); free(step); free(trial); return -3; }
  memset(st, 0, sizeof(*st));
  int rc = 0;
  double l = 0.0;
  st->stop = 4;
  for (int it = 0; it < o->maxiter; ++it) {
    oracle_loglik_grad(P, theta, &l, g);
    st->loglik = l;
    st->grad_inf = max_abs(g, n);
    if (st->grad_inf < o->gtol) { st->stop = 1; break; }
    if (oracle_neg_hessian(P, theta, F, o->nthreads)) { rc = -3; break; }
    if (oracle_cholesky(n, F)) { rc = -2; st->stop = -2; break; }
    memcpy(step, g, sizeof(double) * n);
    oracle_cholesky_solve(n, F, step);
    double t = 1.0, lt = 0.0;
    int accepted = 0;
    for (int h = 0; h <= o->max_halvings; ++h) {
      for (int64_t j = 0; j < n; ++j) trial[j] = theta[j] + t * step[j];
      oracle_loglik_grad(P, trial, &lt, NULL);
      st->ls_evals++;
      if (lt >= l - o->ls_rel_tol * fabs(l)) { accepted = 1; break; }
      t *= 0.5;
    }
    st->iters = it + 1;
    if (!accepted) { rc = -4; st->stop = -4; break; }
    memcpy(theta, trial, sizeof(double) * n);
    const double dl = lt - l;
    l = lt;
    st->loglik = l;
    if (o->ftol > 0 && fabs(dl) < o->ftol) { st->stop = 2; break; }
    if (t * max_abs(step, n) <= o->steptol * fmax(1.0, max_abs(theta, n))) { st->stop = 3; break; }
  }
  free(g); free(F); free(step); free(trial);
  return rc;
}
