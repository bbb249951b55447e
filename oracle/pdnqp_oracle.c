/*
 * PDNQP oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential FP64 CPU implementation of the PDNQP method
 * ("PDNQP: A GPU-based Factorization-free Method for Large-scale Nonconvex
 * Quadratic Programming", Chen & Lu): the practical proximal augmented-
 * Lagrangian outer iteration (Algorithm 3) driving the practical diagonal
 * rAPDHG inner solver (Algorithm 4) on the residual-form subproblem
 * (Eq. prox-alm-subproblem / inner-qp).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the
 * CUDA path; the inner QP is formed here EXPLICITLY (H_k, B, B^T as sparse
 * matrices, Sec. 2.2), scaled literally (Eq. inner-penalty-scaling + inner
 * Ruiz, Sec. 3.3.2), and every product H w_md, B w, B^T y is recomputed from
 * its definition instead of being cached.  Loops run in natural order; the
 * file is meant to be compiled with -ffp-contract=off.
 *
 * Readings of points where the paper is silent (the CUDA path uses the same
 * readings):
 *   - Two-sided rows l_c <= Ax <= u_c: rows with l_c == u_c are equality rows,
 *     every other row is an "inequality" row whose slack lives in [l_c, u_c].
 *     With u_c = +inf this is exactly Eq. projected-multipliers.
 *   - N_p = N_d = accepted steps in the current restart epoch (Eq. pdqp-trial).
 *   - Averages: wbar <- (1 - alpha_t) wbar + alpha_t w_{t+1} (Algorithm 4).
 *   - Rejection: both step vectors are multiplied by a common factor kappa,
 *     kappa <- kappa * shrink; kappa resets to 1 whenever the steps are rebuilt.
 *   - Restart: PDLP-style KKT criteria (sufficient / necessary / artificial
 *     decay) on KKT_w(w,y) = sqrt(w*||Bw-h||^2 + ||w - P(w - g)||^2 / w) in the
 *     scaled inner space, evaluated at the periodic stopping check.
 *   - Inner Ruiz equilibrates the KKT matrix [[H, B^T], [B, 0]] (8 sweeps,
 *     l_inf norms) after the penalty scaling; inner termination is measured on
 *     the outer-scaled, inner-unscaled QP of Eq. inner-qp.
 *   - Outer Ruiz equilibrates [[Q, A^T], [A, 0]] (the constraint matrix alone
 *     lets a column with one tiny entry take a huge scale, which wrecks D Q D).
 *   - Objective scalar c_s = 1/max(1, ||D Q D||_inf, ||D c||_inf) with the
 *     induced (max row-sum) norm for the matrix.
 *   - Initial penalties follow QPALM's formula; the growth factor is capped and
 *     penalties stop growing once the primal part of the termination test holds.
 *   - The center-update tolerances never drop below the final tolerances.
 *   - Outer termination is evaluated on the unscaled problem.
 *   - Infeasibility tests (Sec. "Infeasibility detection") use the changes of
 *     lambda and x over one outer iteration on the scaled problem, normalised
 *     in l_inf, with one tolerance (1e-5): approximate Farkas certificate /
 *     recession direction with objective decrease (see infeasibility()).
 *   - Anderson acceleration (Type-II, m_A = 5 stored iterates of (lambda, z))
 *     runs while the primal termination test holds on two consecutive outer
 *     iterations; its memory is cleared otherwise, a step that raised the
 *     relative KKT residual pauses it for m_A iterations, and no step moves
 *     G(u_k) by more than 10 ||f_k|| (see aa_step()).
 *
 * Parity pins are in the test-suite: brute-force active-set enumeration,
 * closed forms, invariants (see tests/test_oracle_*.py).  The initial-penalty
 * and penalty-growth rules (QPALM-style; constants not printed in the paper)
 * are "parity unpinned" against the paper.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#include <time.h>

#define OR_BIG 1e20

/* ------------------------------------------------------------------------ */
/* Public (ctypes) structures.  Layouts are mirrored in oracle/oracle.py.    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n, m;
  const int *q_rp, *q_ci;
  const double *q_v;
  const double *c;
  const int *a_rp, *a_ci;
  const double *a_v;
  const double *lc, *uc, *lx, *ux;
  const double *x0;   /* may be NULL: x0 = 0 */
  const double *lam0; /* may be NULL: lambda0 = 0 (original row order) */
} or_problem;

typedef struct {
  double eps_abs, eps_rel;
  double time_limit;
  long long k_out, k_in;
  double sigma_init, theta_sigma, delta_gamma;
  double rho_in_min, rho_in_max, rho_z;
  int ruiz_outer, ruiz_inner;
  int lanczos_steps;
  int k_chk;
  double beta_suff, beta_nec, beta_art;
  int rej_limit;
  double kappa_shrink;
  double delta_sigma, sigma_max, tol_floor;
  double gamma_override; /* > 0: use this gamma instead of the Lanczos choice */
  int no_scaling;        /* 1: skip outer Ruiz and the objective scalar */
  int verbose;           /* 1: one line per outer iteration on stderr */
  double eps_inf;        /* infeasibility tolerance on l_inf-normalised directions; 0: 1e-5 */
  int anderson;          /* 1: Anderson acceleration of (lambda, z) (Sec. "Anderson acceleration") */
  int anderson_mem;      /* stored outer iterates m_A */
} or_params;

typedef struct {
  int status;
  long long outer_iters, inner_iters, trials, restarts;
  double r_p, r_d, s_p, s_d, rel_kkt;
  double gamma, lambda_min, obj;
  double seconds;
} or_result;

enum { OR_SOLVED = 0, OR_PRIMAL_INFEASIBLE = 1, OR_DUAL_INFEASIBLE = 2, OR_ITER_LIMIT = 3,
       OR_TIME_LIMIT = 4, OR_NUMERICAL_ERROR = 5 };
enum { IN_CONVERGED = 0, IN_ITER_LIMIT = 1, IN_NUMERICAL_ERROR = 2 };

#define SNAP_SCALARS 8

void or_default_params(or_params *p) {
  /* Table tab:parameters, plus the readings listed in the header. */
  p->eps_abs = 1e-4; p->eps_rel = 1e-4;
  p->time_limit = 1e30;
  p->k_out = 2147483647LL; p->k_in = 40000;
  p->sigma_init = 20.0; p->theta_sigma = 0.25; p->delta_gamma = 1e-2;
  p->rho_in_min = 0.3; p->rho_in_max = 0.95; p->rho_z = 0.95;
  p->ruiz_outer = 8; p->ruiz_inner = 8;
  p->lanczos_steps = 64;
  p->k_chk = 64;
  p->beta_suff = 0.2; p->beta_nec = 0.8; p->beta_art = 0.36;
  p->rej_limit = 60; p->kappa_shrink = 0.5;
  p->delta_sigma = 2.0; p->sigma_max = 1e6; p->tol_floor = 0.1;
  p->gamma_override = 0.0;
  p->no_scaling = 0;
  p->verbose = 0;
  p->eps_inf = 0.0;
  p->anderson = 1;
  p->anderson_mem = 5;
}

/* ------------------------------------------------------------------------ */
/* Small helpers                                                            */
/* ------------------------------------------------------------------------ */
typedef struct { int nr, nc, nnz; int *rp, *ci; double *v; } ocsr;

static void *xcalloc(size_t n, size_t s) { void *p = calloc(n ? n : 1, s); return p; }
static double *dvec(size_t n) { return (double *)xcalloc(n, sizeof(double)); }

static void ocsr_init(ocsr *M, int nr, int nc, int nnz) {
  M->nr = nr; M->nc = nc; M->nnz = nnz;
  M->rp = (int *)xcalloc((size_t)nr + 1, sizeof(int));
  M->ci = (int *)xcalloc((size_t)nnz, sizeof(int));
  M->v = dvec((size_t)nnz);
}
static void ocsr_free(ocsr *M) { free(M->rp); free(M->ci); free(M->v); memset(M, 0, sizeof(*M)); }
static void ocsr_copy(ocsr *dst, const ocsr *src) {
  ocsr_init(dst, src->nr, src->nc, src->nnz);
  memcpy(dst->rp, src->rp, sizeof(int) * ((size_t)src->nr + 1));
  memcpy(dst->ci, src->ci, sizeof(int) * (size_t)src->nnz);
  memcpy(dst->v, src->v, sizeof(double) * (size_t)src->nnz);
}
/* y = M x */
static void ocsr_mv(const ocsr *M, const double *x, double *y) {
  for (int i = 0; i < M->nr; ++i) {
    double s = 0.0;
    for (int k = M->rp[i]; k < M->rp[i + 1]; ++k) s += M->v[k] * x[M->ci[k]];
    y[i] = s;
  }
}
static void ocsr_transpose(const ocsr *M, ocsr *T) {
  ocsr_init(T, M->nc, M->nr, M->nnz);
  for (int k = 0; k < M->nnz; ++k) T->rp[M->ci[k] + 1]++;
  for (int i = 0; i < M->nc; ++i) T->rp[i + 1] += T->rp[i];
  int *pos = (int *)xcalloc((size_t)M->nc, sizeof(int));
  for (int i = 0; i < M->nc; ++i) pos[i] = T->rp[i];
  for (int i = 0; i < M->nr; ++i)
    for (int k = M->rp[i]; k < M->rp[i + 1]; ++k) {
      int d = pos[M->ci[k]]++;
      T->ci[d] = i; T->v[d] = M->v[k];
    }
  free(pos);
}
static double proj(double v, double lo, double hi) {
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return v;
}
/* Componentwise Euclidean projection onto a box (Sec. 1.2), exported for tests. */
void or_project(int n, const double *v, const double *lo, const double *hi, double *out) {
  for (int i = 0; i < n; ++i) out[i] = proj(v[i], lo[i], hi[i]);
}
static double norm_inf(const double *v, int n) {
  double r = 0.0;
  for (int i = 0; i < n; ++i) if (fabs(v[i]) > r) r = fabs(v[i]);
  return r;
}
static double dot(const double *a, const double *b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
static double clean_bound(double v) {
  if (v >= OR_BIG) return HUGE_VAL;
  if (v <= -OR_BIG) return -HUGE_VAL;
  return v;
}
static double dmax(double a, double b) { return a > b ? a : b; }
/* Maxima of termination-test terms.  A residual term that is not finite (NaN
 * or infinite data) counts as +inf, so a point with such entries never passes
 * (a plain comparison-based maximum would drop a NaN).  A scale term that is
 * not finite is left out: an infinite scale would excuse any residual. */
static double rmax(double a, double b) { return isfinite(b) ? (a > b ? a : b) : INFINITY; }
static double smax(double a, double b) { return (isfinite(b) && b > a) ? b : a; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* The i-th output (i = 0, 1, ...) of the splitmix64 generator seeded with
 * `seed` (Steele, Lea, Flood 2014; Vigna's reference constants), mapped to a
 * double in [-0.5, 0.5).  Used for the Lanczos start vector. */
static double splitmix_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: outer scaling (Eq. scaled-problem) and the objective scalar.   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n, m, mE, mI;
  ocsr Q;              /* scaled Q: c_s * Dx Q Dx */
  ocsr A;              /* scaled A = Dc A Dx, rows ordered E then I */
  ocsr At;             /* its transpose */
  double *c, *lx, *ux; /* scaled */
  double *lc, *uc;     /* scaled row bounds (lc == uc on E rows) */
  double *Dc, *Dx;     /* row / column Ruiz factors (permuted row order) */
  double cs;
  int *perm;           /* perm[k] = original index of internal row k */
  double qnorm;        /* ||Q||_inf of the scaled Q (max row abs-sum) */
} sqp_t;

/* Ruiz equilibration (Ruiz 2001) of the symmetric matrix [[Q, A^T], [A, 0]]:
 * each sweep divides every row and column by the square root of its l_inf
 * norm, so the column of variable i sees both Q's column i and A's column i
 * and row j of A sees A's row j.  Zero rows/columns keep factor 1.  The
 * values of Q are only read (the caller applies Dx Q Dx afterwards); A's
 * values are scaled in place.  Q may be NULL (constraint matrix only). */
void or_ruiz_outer(int m, int n, const int *rp, const int *ci, double *v, const int *qrp, const int *qci,
                   const double *qv, int sweeps, double *Dc, double *Dx) {
  double *rn = dvec((size_t)m), *cn = dvec((size_t)n);
  for (int i = 0; i < m; ++i) Dc[i] = 1.0;
  for (int j = 0; j < n; ++j) Dx[j] = 1.0;
  for (int s = 0; s < sweeps; ++s) {
    for (int i = 0; i < m; ++i) rn[i] = 0.0;
    for (int j = 0; j < n; ++j) cn[j] = 0.0;
    for (int i = 0; i < m; ++i)
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        double a = fabs(v[k]);
        if (a > rn[i]) rn[i] = a;
        if (a > cn[ci[k]]) cn[ci[k]] = a;
      }
    if (qrp)
      for (int i = 0; i < n; ++i)
        for (int k = qrp[i]; k < qrp[i + 1]; ++k) {
          double a = fabs(Dx[i] * qv[k] * Dx[qci[k]]);
          if (a > cn[qci[k]]) cn[qci[k]] = a;
        }
    for (int i = 0; i < m; ++i) rn[i] = rn[i] > 0.0 ? 1.0 / sqrt(rn[i]) : 1.0;
    for (int j = 0; j < n; ++j) cn[j] = cn[j] > 0.0 ? 1.0 / sqrt(cn[j]) : 1.0;
    for (int i = 0; i < m; ++i)
      for (int k = rp[i]; k < rp[i + 1]; ++k) v[k] = v[k] * rn[i] * cn[ci[k]];
    for (int i = 0; i < m; ++i) Dc[i] *= rn[i];
    for (int j = 0; j < n; ++j) Dx[j] *= cn[j];
  }
  free(rn); free(cn);
}

static double csr_norm_inf_rowsum(const ocsr *M) {
  double r = 0.0;
  for (int i = 0; i < M->nr; ++i) {
    double s = 0.0;
    for (int k = M->rp[i]; k < M->rp[i + 1]; ++k) s += fabs(M->v[k]);
    if (s > r) r = s;
  }
  return r;
}

static void sqp_build(const or_problem *P, const or_params *prm, sqp_t *S) {
  int n = P->n, m = P->m;
  memset(S, 0, sizeof(*S));
  S->n = n; S->m = m;
  /* Row classification (reading of Eq. qp for two-sided rows) and E-then-I order. */
  S->perm = (int *)xcalloc((size_t)m, sizeof(int));
  int k = 0;
  for (int i = 0; i < m; ++i) {
    double l = clean_bound(P->lc[i]), u = clean_bound(P->uc[i]);
    if (l == u) S->perm[k++] = i;
  }
  S->mE = k;
  for (int i = 0; i < m; ++i) {
    double l = clean_bound(P->lc[i]), u = clean_bound(P->uc[i]);
    if (!(l == u)) S->perm[k++] = i;
  }
  S->mI = m - S->mE;
  /* Permuted copy of A. */
  int nnzA = m ? P->a_rp[m] : 0;
  ocsr_init(&S->A, m, n, nnzA);
  int pos = 0;
  for (int r = 0; r < m; ++r) {
    int i = S->perm[r];
    for (int kk = P->a_rp[i]; kk < P->a_rp[i + 1]; ++kk) {
      S->A.ci[pos] = P->a_ci[kk];
      S->A.v[pos] = P->a_v[kk];
      ++pos;
    }
    S->A.rp[r + 1] = pos;
  }
  S->Dc = dvec((size_t)m); S->Dx = dvec((size_t)n);
  or_ruiz_outer(m, n, S->A.rp, S->A.ci, S->A.v, P->q_rp, P->q_ci, P->q_v,
                prm->no_scaling ? 0 : prm->ruiz_outer, S->Dc, S->Dx);
  ocsr_transpose(&S->A, &S->At);
  /* Q_hat = Dx Q Dx, c_hat = Dx c */
  int nnzQ = P->q_rp[n];
  ocsr_init(&S->Q, n, n, nnzQ);
  memcpy(S->Q.rp, P->q_rp, sizeof(int) * ((size_t)n + 1));
  memcpy(S->Q.ci, P->q_ci, sizeof(int) * (size_t)nnzQ);
  for (int i = 0; i < n; ++i)
    for (int kk = P->q_rp[i]; kk < P->q_rp[i + 1]; ++kk)
      S->Q.v[kk] = S->Dx[i] * P->q_v[kk] * S->Dx[P->q_ci[kk]];
  S->c = dvec((size_t)n);
  for (int i = 0; i < n; ++i) S->c[i] = S->Dx[i] * P->c[i];
  /* Objective scalar (reading of "an additional scalar balances the objective"). */
  double qn = csr_norm_inf_rowsum(&S->Q), cn = norm_inf(S->c, n);
  S->cs = prm->no_scaling ? 1.0 : 1.0 / dmax(1.0, dmax(qn, cn));
  for (int kk = 0; kk < nnzQ; ++kk) S->Q.v[kk] *= S->cs;
  for (int i = 0; i < n; ++i) S->c[i] *= S->cs;
  S->qnorm = csr_norm_inf_rowsum(&S->Q);
  /* Bounds in scaled coordinates: x = Dx xbar, rows scaled by Dc. */
  S->lx = dvec((size_t)n); S->ux = dvec((size_t)n);
  for (int i = 0; i < n; ++i) {
    S->lx[i] = clean_bound(P->lx[i]) / S->Dx[i];
    S->ux[i] = clean_bound(P->ux[i]) / S->Dx[i];
  }
  S->lc = dvec((size_t)m); S->uc = dvec((size_t)m);
  for (int r = 0; r < m; ++r) {
    int i = S->perm[r];
    S->lc[r] = clean_bound(P->lc[i]) * S->Dc[r];
    S->uc[r] = clean_bound(P->uc[i]) * S->Dc[r];
    if (r < S->mE) S->uc[r] = S->lc[r];
  }
}

static void sqp_free(sqp_t *S) {
  ocsr_free(&S->Q); ocsr_free(&S->A); ocsr_free(&S->At);
  free(S->c); free(S->lx); free(S->ux); free(S->lc); free(S->uc);
  free(S->Dc); free(S->Dx); free(S->perm);
  memset(S, 0, sizeof(*S));
}

/* ------------------------------------------------------------------------ */
/* Eq. R-choice: Lanczos estimate of lambda_min(Q).                         */
/* ------------------------------------------------------------------------ */
/* Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm). */
static int sturm_count(const double *a, const double *b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}
/* Smallest eigenvalue of the tridiagonal matrix by bisection. */
double or_tridiag_min_eig(const double *a, const double *b, int k) {
  double lo = HUGE_VAL, hi = -HUGE_VAL;
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    lo = dmin(lo, a[i] - r);
    hi = dmax(hi, a[i] + r);
  }
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, k, mid) >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* Lanczos with full (modified Gram-Schmidt) reorthogonalisation; returns the
 * smallest Ritz value after `steps` steps (or at breakdown). */
double or_lanczos_min(int n, const int *rp, const int *ci, const double *v, int steps, uint64_t seed) {
  ocsr Q = {n, n, rp[n], (int *)rp, (int *)ci, (double *)v};
  if (n == 0) return 0.0;
  int k = steps < n ? steps : n;
  double *V = dvec((size_t)(k + 1) * (size_t)n);
  double *al = dvec((size_t)k + 1), *be = dvec((size_t)k + 1);
  double *w = dvec((size_t)n);
  double nrm = 0.0;
  for (int i = 0; i < n; ++i) { V[i] = splitmix_uniform(seed, (uint64_t)i); nrm += V[i] * V[i]; }
  nrm = sqrt(nrm);
  for (int i = 0; i < n; ++i) V[i] /= nrm;
  int used = 0;
  for (int j = 0; j < k; ++j) {
    double *vj = V + (size_t)j * n;
    ocsr_mv(&Q, vj, w);
    al[j] = dot(w, vj, n);
    used = j + 1;
    for (int i = 0; i < n; ++i) w[i] -= al[j] * vj[i];
    if (j > 0) {
      double *vp = V + (size_t)(j - 1) * n;
      for (int i = 0; i < n; ++i) w[i] -= be[j - 1] * vp[i];
    }
    for (int p = 0; p <= j; ++p) {
      double *vpp = V + (size_t)p * n;
      double h = dot(w, vpp, n);
      for (int i = 0; i < n; ++i) w[i] -= h * vpp[i];
    }
    double b = sqrt(dot(w, w, n));
    be[j] = b;
    if (j == k - 1) break;
    if (b <= 1e-12 * (fabs(al[j]) + (j > 0 ? be[j - 1] : 0.0) + 1e-300)) break;
    double *vn = V + (size_t)(j + 1) * n;
    for (int i = 0; i < n; ++i) vn[i] = w[i] / b;
  }
  double lam = or_tridiag_min_eig(al, be, used);
  free(V); free(al); free(be); free(w);
  return lam;
}

/* Eq. R-choice with two independent Lanczos starts (the smaller estimate is
 * used), the FP64 proximal-shift stability check. */
static double choose_gamma(const sqp_t *S, const or_params *prm, double *lam_out) {
  double l1 = or_lanczos_min(S->n, S->Q.rp, S->Q.ci, S->Q.v, prm->lanczos_steps, 1ULL);
  double l2 = or_lanczos_min(S->n, S->Q.rp, S->Q.ci, S->Q.v, prm->lanczos_steps, 2ULL);
  double lam = dmin(l1, l2);
  *lam_out = lam;
  if (prm->gamma_override > 0.0) return prm->gamma_override;
  return 1.0 / (dmax(0.0, -lam) + prm->delta_gamma * dmax(1.0, S->qnorm));
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: the inner QP of Eq. inner-qp, formed explicitly.               */
/* w = (x, s_I, r_E, r_I);  B = [[A_E, 0, -I, 0], [A_I, -I, 0, -I]]         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n, m, mE, mI, dw;
  ocsr H, B, Bt;               /* Eq. inner-qp (outer-scaled) */
  double *q, *h, *lo, *hi;
  ocsr Hs, Bs, Bst;            /* penalty + Ruiz scaled (Sec. 3.3.2) */
  double *qs, *hs, *los, *his;
  double *ew, *dy;             /* w = ew .* w_scaled,  y = dy .* y_scaled */
  double *sig_row;             /* raw row penalties sigma_j (Eq. diagonal-scales) */
  double *mw, *my;
} iqp_t;

static int col_r(const iqp_t *I, int row) { return I->n + I->mI + row; } /* r_E then r_I */
static int col_s(const iqp_t *I, int row) { return I->n + (row - I->mE); }

static void iqp_form(const sqp_t *S, const double *z, const double *lam, const double *sig,
                     double gamma, iqp_t *I) {
  int n = S->n, m = S->m;
  memset(I, 0, sizeof(*I));
  I->n = n; I->m = m; I->mE = S->mE; I->mI = S->mI;
  I->dw = n + S->mI + m;
  int dw = I->dw;
  /* H_k = diag(Q + gamma^-1 I, 0, sigma_E I, sigma_I I); the diagonal of the
   * x block is stored explicitly (zero entries of Q included). */
  int nnzH = 0;
  for (int i = 0; i < n; ++i) {
    int hasd = 0;
    for (int k = S->Q.rp[i]; k < S->Q.rp[i + 1]; ++k) if (S->Q.ci[k] == i) hasd = 1;
    nnzH += S->Q.rp[i + 1] - S->Q.rp[i] + (hasd ? 0 : 1);
  }
  nnzH += m;
  ocsr_init(&I->H, dw, dw, nnzH);
  int pos = 0;
  for (int i = 0; i < n; ++i) {
    int hasd = 0;
    for (int k = S->Q.rp[i]; k < S->Q.rp[i + 1]; ++k) {
      I->H.ci[pos] = S->Q.ci[k];
      I->H.v[pos] = S->Q.v[k] + (S->Q.ci[k] == i ? 1.0 / gamma : 0.0);
      if (S->Q.ci[k] == i) hasd = 1;
      ++pos;
    }
    if (!hasd) { I->H.ci[pos] = i; I->H.v[pos] = 1.0 / gamma; ++pos; }
    I->H.rp[i + 1] = pos;
  }
  for (int i = n; i < n + S->mI; ++i) I->H.rp[i + 1] = pos; /* s block: zero rows */
  for (int j = 0; j < m; ++j) {                              /* r block */
    I->H.ci[pos] = col_r(I, j);
    I->H.v[pos] = sig[j];
    ++pos;
    I->H.rp[n + S->mI + j + 1] = pos;
  }
  /* B */
  int nnzB = S->A.nnz + S->mI + m;
  ocsr_init(&I->B, m, dw, nnzB);
  pos = 0;
  for (int j = 0; j < m; ++j) {
    for (int k = S->A.rp[j]; k < S->A.rp[j + 1]; ++k) {
      I->B.ci[pos] = S->A.ci[k]; I->B.v[pos] = S->A.v[k]; ++pos;
    }
    if (j >= S->mE) { I->B.ci[pos] = col_s(I, j); I->B.v[pos] = -1.0; ++pos; }
    I->B.ci[pos] = col_r(I, j); I->B.v[pos] = -1.0; ++pos;
    I->B.rp[j + 1] = pos;
  }
  ocsr_transpose(&I->B, &I->Bt);
  /* q_k = (c - gamma^-1 z, 0, lambda_E, lambda_I), h = (b_E, 0), Eq. inner-bounds. */
  I->q = dvec((size_t)dw); I->h = dvec((size_t)m); I->lo = dvec((size_t)dw); I->hi = dvec((size_t)dw);
  for (int i = 0; i < n; ++i) {
    I->q[i] = S->c[i] - z[i] / gamma;
    I->lo[i] = S->lx[i]; I->hi[i] = S->ux[i];
  }
  for (int j = S->mE; j < m; ++j) {
    int cs = col_s(I, j);
    I->q[cs] = 0.0; I->lo[cs] = S->lc[j]; I->hi[cs] = S->uc[j];
  }
  for (int j = 0; j < m; ++j) {
    int cr = col_r(I, j);
    I->q[cr] = lam[j]; I->lo[cr] = -HUGE_VAL; I->hi[cr] = HUGE_VAL;
    I->h[j] = j < S->mE ? S->lc[j] : 0.0;
  }
  I->sig_row = dvec((size_t)m);
  for (int j = 0; j < m; ++j) I->sig_row[j] = sig[j];
}

static void iqp_free(iqp_t *I) {
  ocsr_free(&I->H); ocsr_free(&I->B); ocsr_free(&I->Bt);
  ocsr_free(&I->Hs); ocsr_free(&I->Bs); ocsr_free(&I->Bst);
  free(I->q); free(I->h); free(I->lo); free(I->hi);
  free(I->qs); free(I->hs); free(I->los); free(I->his);
  free(I->ew); free(I->dy); free(I->sig_row); free(I->mw); free(I->my);
  memset(I, 0, sizeof(*I));
}

/* Apply w = diag(f) w', y = diag(g) y' to the working scaled copy. */
static void scale_inner(iqp_t *I, const double *f, const double *g) {
  for (int i = 0; i < I->Hs.nr; ++i)
    for (int k = I->Hs.rp[i]; k < I->Hs.rp[i + 1]; ++k) I->Hs.v[k] = f[i] * I->Hs.v[k] * f[I->Hs.ci[k]];
  for (int j = 0; j < I->Bs.nr; ++j)
    for (int k = I->Bs.rp[j]; k < I->Bs.rp[j + 1]; ++k) I->Bs.v[k] = g[j] * I->Bs.v[k] * f[I->Bs.ci[k]];
  for (int i = 0; i < I->dw; ++i) I->ew[i] *= f[i];
  for (int j = 0; j < I->m; ++j) I->dy[j] *= g[j];
}

/* Eq. inner-penalty-scaling, then inner Ruiz on [[H, B^T], [B, 0]] (Sec. 3.3.2),
 * then Eq. diagonal-scales on the scaled H, B. */
static void iqp_scale(iqp_t *I, int sweeps) {
  int dw = I->dw, m = I->m;
  ocsr_copy(&I->Hs, &I->H);
  ocsr_copy(&I->Bs, &I->B);
  I->ew = dvec((size_t)dw); I->dy = dvec((size_t)m);
  for (int i = 0; i < dw; ++i) I->ew[i] = 1.0;
  for (int j = 0; j < m; ++j) I->dy[j] = 1.0;
  double *f = dvec((size_t)dw), *g = dvec((size_t)m);
  /* r_i <- sqrt(sigma_i) r_i  is the change of variable r = r_hat / sqrt(sigma). */
  for (int i = 0; i < dw; ++i) f[i] = 1.0;
  for (int j = 0; j < m; ++j) { f[col_r(I, j)] = 1.0 / sqrt(I->sig_row[j]); g[j] = 1.0; }
  scale_inner(I, f, g);
  for (int s = 0; s < sweeps; ++s) {
    for (int i = 0; i < dw; ++i) f[i] = 0.0;
    for (int j = 0; j < m; ++j) g[j] = 0.0;
    for (int i = 0; i < dw; ++i)
      for (int k = I->Hs.rp[i]; k < I->Hs.rp[i + 1]; ++k) {
        double a = fabs(I->Hs.v[k]);
        if (a > f[I->Hs.ci[k]]) f[I->Hs.ci[k]] = a;
      }
    for (int j = 0; j < m; ++j)
      for (int k = I->Bs.rp[j]; k < I->Bs.rp[j + 1]; ++k) {
        double a = fabs(I->Bs.v[k]);
        if (a > f[I->Bs.ci[k]]) f[I->Bs.ci[k]] = a;
        if (a > g[j]) g[j] = a;
      }
    for (int i = 0; i < dw; ++i) f[i] = f[i] > 0.0 ? 1.0 / sqrt(f[i]) : 1.0;
    for (int j = 0; j < m; ++j) g[j] = g[j] > 0.0 ? 1.0 / sqrt(g[j]) : 1.0;
    scale_inner(I, f, g);
  }
  free(f); free(g);
  ocsr_transpose(&I->Bs, &I->Bst);
  I->qs = dvec((size_t)dw); I->hs = dvec((size_t)m); I->los = dvec((size_t)dw); I->his = dvec((size_t)dw);
  for (int i = 0; i < dw; ++i) {
    I->qs[i] = I->ew[i] * I->q[i];
    I->los[i] = I->lo[i] / I->ew[i];
    I->his[i] = I->hi[i] / I->ew[i];
  }
  for (int j = 0; j < m; ++j) I->hs[j] = I->dy[j] * I->h[j];
  /* Eq. diagonal-scales. */
  I->mw = dvec((size_t)dw); I->my = dvec((size_t)m);
  for (int i = 0; i < dw; ++i) {
    double h1 = 0.0, b1 = 0.0, b2 = 0.0;
    for (int k = I->Hs.rp[i]; k < I->Hs.rp[i + 1]; ++k) h1 += fabs(I->Hs.v[k]); /* H symmetric */
    for (int k = I->Bst.rp[i]; k < I->Bst.rp[i + 1]; ++k) {
      double b = I->Bst.v[k];
      b1 += fabs(b);
      b2 += I->sig_row[I->Bst.ci[k]] * b * b;
    }
    int is_xs = i < I->n + I->mI;
    I->mw[i] = h1 + (is_xs ? dmax(b1, sqrt(b2)) : b1);
  }
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int k = I->Bs.rp[j]; k < I->Bs.rp[j + 1]; ++k)
      if (I->mw[I->Bs.ci[k]] > 0.0) s += I->Bs.v[k] * I->Bs.v[k] / I->mw[I->Bs.ci[k]];
    I->my[j] = s;
  }
}

/* Eq. diagonal-steps with the common rejection factor kappa. */
static void make_steps(const iqp_t *I, double omega, double kappa, double *tau, double *eta) {
  for (int i = 0; i < I->dw; ++i) tau[i] = kappa * 0.99 / (omega * I->mw[i]);
  for (int j = 0; j < I->m; ++j) eta[j] = kappa * 0.99 * omega / I->my[j];
}

/* Eq. inner-residuals / inner-scales / inner-termination on the unscaled inner QP. */
typedef struct { double rp, rd, sp, sd; } inres_t;
static inres_t inner_residuals(const iqp_t *I, const double *wsc, const double *ysc, double *tmp_w,
                               double *tmp_y, double *Hw, double *Btu, double *Bw) {
  int dw = I->dw, m = I->m;
  for (int i = 0; i < dw; ++i) tmp_w[i] = I->ew[i] * wsc[i];
  for (int j = 0; j < m; ++j) tmp_y[j] = I->dy[j] * ysc[j];
  ocsr_mv(&I->B, tmp_w, Bw);
  ocsr_mv(&I->H, tmp_w, Hw);
  ocsr_mv(&I->Bt, tmp_y, Btu);
  inres_t R = {0, 0, 1.0, 1.0};
  for (int j = 0; j < m; ++j) {
    R.rp = dmax(R.rp, fabs(Bw[j] - I->h[j]));
    R.sp = dmax(R.sp, dmax(fabs(Bw[j]), fabs(I->h[j])));
  }
  for (int i = 0; i < dw; ++i) {
    double g = Hw[i] + I->q[i] - Btu[i];
    R.rd = dmax(R.rd, fabs(tmp_w[i] - proj(tmp_w[i] - g, I->lo[i], I->hi[i])));
    R.sd = dmax(R.sd, dmax(fabs(Hw[i]), dmax(fabs(I->q[i]), fabs(Btu[i]))));
  }
  return R;
}

/* Restart metric in the scaled inner space (reading of Sec. 3.3.7). */
static double kkt_metric(const iqp_t *I, const double *w, const double *y, double omega, double *Hw,
                         double *Btu, double *Bw) {
  ocsr_mv(&I->Bs, w, Bw);
  ocsr_mv(&I->Hs, w, Hw);
  ocsr_mv(&I->Bst, y, Btu);
  double p = 0.0, d = 0.0;
  for (int j = 0; j < I->m; ++j) { double e = Bw[j] - I->hs[j]; p += e * e; }
  for (int i = 0; i < I->dw; ++i) {
    double g = Hw[i] + I->qs[i] - Btu[i];
    double e = w[i] - proj(w[i] - g, I->los[i], I->his[i]);
    d += e * e;
  }
  return sqrt(omega * p + d / omega);
}

typedef struct {
  /* debug snapshots */
  int n_ckpt;
  const long long *ckpt;
  double *snap;
  int next_ckpt;
  int ignore_convergence;
  double *times; /* optional: wall-clock seconds at each snapshot */
  /* optional trace of the periodic checks (or_debug_checks): one row of
   * CHK_COLS scalars and the vectors w, y, wbar, ybar, w_start, y_start
   * (inner-unscaled coordinates) as they stand before the restart decision */
  int chk_max, chk_n;
  double *chk_rows, *chk_vecs;
} dbg_t;

#define CHK_COLS 22

typedef struct {
  long long trials, accepted, restarts;
  double sd_in; /* s_d^in (Eq. inner-scales) of the candidate an inner solve returned */
} ctr_t;

static double now_seconds(void);

static void take_snapshot(const iqp_t *I, dbg_t *D, const double *w, const double *y, const double *wb,
                          const double *yb, double omega, double kappa, long long t, long long ttot,
                          long long trials, long long restarts, double krest, double klast) {
  int dw = I->dw, m = I->m;
  size_t len = 2 * (size_t)(dw + m) + SNAP_SCALARS;
  double *o = D->snap + (size_t)D->next_ckpt * len;
  for (int i = 0; i < dw; ++i) o[i] = I->ew[i] * w[i];
  for (int j = 0; j < m; ++j) o[dw + j] = I->dy[j] * y[j];
  for (int i = 0; i < dw; ++i) o[dw + m + i] = I->ew[i] * wb[i];
  for (int j = 0; j < m; ++j) o[2 * dw + m + j] = I->dy[j] * yb[j];
  double *sc = o + 2 * (size_t)(dw + m);
  sc[0] = omega; sc[1] = kappa; sc[2] = (double)t; sc[3] = (double)ttot;
  sc[4] = (double)trials; sc[5] = (double)restarts; sc[6] = krest; sc[7] = klast;
  if (D->times) D->times[D->next_ckpt] = now_seconds();
  D->next_ckpt++;
}

/*
 * Algorithm 4 on the explicit inner QP.  x (outer-scaled, n) and y (inner
 * dual, outer-scaled, m) are read as the warm start and overwritten with the
 * returned candidate.  omega persists across calls.
 */
static int inner_solve(const sqp_t *S, const or_params *prm, const double *z, const double *lam,
                       const double *sig, double gamma, double dta, double dtr, double *x, double *y,
                       double *omega_io, ctr_t *C, dbg_t *D) {
  int n = S->n, m = S->m;
  iqp_t I;
  iqp_form(S, z, lam, sig, gamma, &I);
  int dw = I.dw;
  /* Eq. inner-warm-start (in inner-unscaled coordinates). */
  double *w0 = dvec((size_t)dw), *ax = dvec((size_t)m);
  ocsr_mv(&S->A, x, ax);
  for (int i = 0; i < n; ++i) w0[i] = x[i];
  for (int j = 0; j < m; ++j) {
    if (j < S->mE) {
      w0[col_r(&I, j)] = ax[j] - S->lc[j];
    } else {
      double s = proj(ax[j] + lam[j] / sig[j], S->lc[j], S->uc[j]);
      w0[col_s(&I, j)] = s;
      w0[col_r(&I, j)] = ax[j] - s;
    }
  }
  iqp_scale(&I, prm->ruiz_inner);
  double *w = dvec((size_t)dw), *yy = dvec((size_t)m);
  for (int i = 0; i < dw; ++i) w[i] = w0[i] / I.ew[i];
  for (int j = 0; j < m; ++j) yy[j] = y[j] / I.dy[j];
  double *wb = dvec((size_t)dw), *yb = dvec((size_t)m);
  double *wst = dvec((size_t)dw), *yst = dvec((size_t)m); /* epoch start */
  double *tau = dvec((size_t)dw), *eta = dvec((size_t)m);
  double *wmd = dvec((size_t)dw), *g = dvec((size_t)dw), *wtr = dvec((size_t)dw), *ytr = dvec((size_t)m);
  double *Bwtr = dvec((size_t)m), *Bw = dvec((size_t)m), *Bty = dvec((size_t)dw);
  double *dwv = dvec((size_t)dw), *dyv = dvec((size_t)m), *Hd = dvec((size_t)dw), *Btd = dvec((size_t)dw);
  double *t1 = dvec((size_t)dw), *t2 = dvec((size_t)m), *t3 = dvec((size_t)dw), *t4 = dvec((size_t)dw),
         *t5 = dvec((size_t)m);
  double omega = *omega_io, kappa = 1.0;
  make_steps(&I, omega, kappa, tau, eta);
  memcpy(wb, w, sizeof(double) * dw); memcpy(yb, yy, sizeof(double) * m);
  memcpy(wst, w, sizeof(double) * dw); memcpy(yst, yy, sizeof(double) * m);
  long long t = 0, ttot = 0;
  double k_restart = kkt_metric(&I, w, yy, omega, t3, t4, t5);
  double k_last = HUGE_VAL;
  int status = IN_ITER_LIMIT;
  const double *ret_w = w, *ret_y = yy;
  long long kin = D ? (long long)9e18 : prm->k_in;
  for (;;) {
    if (D && D->next_ckpt >= D->n_ckpt) break;
    if (ttot >= kin) break;
    int rej = 0, accepted = 0;
    while (!accepted) {
      double alpha = 2.0 / ((double)t + 2.0), beta = (double)t / ((double)t + 1.0);
      /* Eq. pdqp-trial, with H w_md computed from its definition. */
      for (int i = 0; i < dw; ++i) wmd[i] = (1.0 - alpha) * wb[i] + alpha * w[i];
      ocsr_mv(&I.Hs, wmd, g);
      ocsr_mv(&I.Bst, yy, Bty);
      for (int i = 0; i < dw; ++i)
        wtr[i] = proj(w[i] - tau[i] * (I.qs[i] + g[i] - Bty[i]), I.los[i], I.his[i]);
      ocsr_mv(&I.Bs, wtr, Bwtr);
      ocsr_mv(&I.Bs, w, Bw);
      for (int j = 0; j < m; ++j)
        ytr[j] = yy[j] + eta[j] * (I.hs[j] - Bwtr[j] - beta * (Bwtr[j] - Bw[j]));
      /* Eq. adaptive-condition. */
      for (int i = 0; i < dw; ++i) dwv[i] = wtr[i] - w[i];
      for (int j = 0; j < m; ++j) dyv[j] = ytr[j] - yy[j];
      ocsr_mv(&I.Hs, dwv, Hd);
      ocsr_mv(&I.Bst, dyv, Btd);
      double lhs = 0.0, rhs_h = 0.0, rhs_b = 0.0;
      for (int i = 0; i < dw; ++i) lhs += dwv[i] * dwv[i] / tau[i];
      for (int j = 0; j < m; ++j) lhs += dyv[j] * dyv[j] / eta[j];
      for (int i = 0; i < dw; ++i) rhs_h += fabs(dwv[i] * Hd[i]);
      for (int i = 0; i < dw; ++i) rhs_b += fabs(dwv[i] * Btd[i]);
      C->trials++;
      if (!isfinite(lhs) || !isfinite(rhs_h) || !isfinite(rhs_b)) { status = IN_NUMERICAL_ERROR; goto done; }
      if (0.5 * lhs >= 0.5 * rhs_h + rhs_b) {
        memcpy(w, wtr, sizeof(double) * dw);
        memcpy(yy, ytr, sizeof(double) * m);
        for (int i = 0; i < dw; ++i) wb[i] = (1.0 - alpha) * wb[i] + alpha * w[i];
        for (int j = 0; j < m; ++j) yb[j] = (1.0 - alpha) * yb[j] + alpha * yy[j];
        ++t; ++ttot; C->accepted++;
        accepted = 1;
      } else {
        kappa *= prm->kappa_shrink;
        make_steps(&I, omega, kappa, tau, eta);
        if (++rej >= prm->rej_limit) { status = IN_NUMERICAL_ERROR; goto done; }
      }
    }
    if ((prm->k_chk > 0 && ttot % prm->k_chk == 0) || (!D && ttot == kin)) {
      /* Sec. 3.3.3: stopping check of the current and averaged candidates. */
      inres_t Rc = inner_residuals(&I, w, yy, t1, t2, t3, t4, t5);
      inres_t Ra = inner_residuals(&I, wb, yb, t1, t2, t3, t4, t5);
      int okc = Rc.rp <= dta + dtr * Rc.sp && Rc.rd <= dta + dtr * Rc.sd;
      int oka = Ra.rp <= dta + dtr * Ra.sp && Ra.rd <= dta + dtr * Ra.sd;
      if (!(D && D->ignore_convergence)) {
        if (okc) { status = IN_CONVERGED; ret_w = w; ret_y = yy; C->sd_in = Rc.sd; goto done; }
        if (oka) { status = IN_CONVERGED; ret_w = wb; ret_y = yb; C->sd_in = Ra.sd; goto done; }
      }
      if (!D && ttot == kin) break;
      /* Restart test (reading of Sec. 3.3.7) and primal weight (Eq. primal-weight-update). */
      double kc = kkt_metric(&I, w, yy, omega, t3, t4, t5);
      double ka = kkt_metric(&I, wb, yb, omega, t3, t4, t5);
      int use_avg = ka < kc;
      double kcand = use_avg ? ka : kc;
      int do_restart = kcand <= prm->beta_suff * k_restart ||
                       (kcand <= prm->beta_nec * k_restart && kcand > k_last) ||
                       (double)t >= prm->beta_art * (double)ttot;
      double *crow = NULL;
      if (D && D->chk_rows && D->chk_n < D->chk_max) {
        crow = D->chk_rows + (size_t)D->chk_n * CHK_COLS;
        crow[0] = (double)ttot; crow[1] = (double)t; crow[2] = kc; crow[3] = ka; crow[4] = k_restart;
        crow[5] = k_last; crow[6] = use_avg; crow[7] = do_restart; crow[8] = omega; crow[10] = kappa;
        crow[14] = Rc.rp; crow[15] = Rc.rd; crow[16] = Rc.sp; crow[17] = Rc.sd;
        crow[18] = Ra.rp; crow[19] = Ra.rd; crow[20] = Ra.sp; crow[21] = Ra.sd;
        double *cv = D->chk_vecs + (size_t)D->chk_n * 3 * (size_t)(dw + m);
        for (int i = 0; i < dw; ++i) { cv[i] = I.ew[i] * w[i]; cv[dw + m + i] = I.ew[i] * wb[i];
                                        cv[2 * (dw + m) + i] = I.ew[i] * wst[i]; }
        for (int j = 0; j < m; ++j) { cv[dw + j] = I.dy[j] * yy[j]; cv[2 * dw + m + j] = I.dy[j] * yb[j];
                                       cv[3 * dw + 2 * m + j] = I.dy[j] * yst[j]; }
        D->chk_n++;
      }
      k_last = kcand;
      if (do_restart) {
        if (use_avg) { memcpy(w, wb, sizeof(double) * dw); memcpy(yy, yb, sizeof(double) * m); }
        double dW = 0.0, dY = 0.0;
        for (int i = 0; i < dw; ++i) dW += (w[i] - wst[i]) * (w[i] - wst[i]);
        for (int j = 0; j < m; ++j) dY += (yy[j] - yst[j]) * (yy[j] - yst[j]);
        dW = sqrt(dW); dY = sqrt(dY);
        if (dW > 0.0 && dY > 0.0) omega = exp(0.25 * log(dY / dW) + 0.75 * log(omega));
        kappa = 1.0;
        make_steps(&I, omega, kappa, tau, eta);
        memcpy(wst, w, sizeof(double) * dw); memcpy(yst, yy, sizeof(double) * m);
        memcpy(wb, w, sizeof(double) * dw); memcpy(yb, yy, sizeof(double) * m);
        t = 0;
        k_restart = kcand;
        k_last = HUGE_VAL;
        C->restarts++;
      }
      if (crow) { crow[9] = omega; crow[11] = kappa; crow[12] = (double)t; crow[13] = k_restart; }
    }
    if (D && D->next_ckpt < D->n_ckpt && ttot == D->ckpt[D->next_ckpt])
      take_snapshot(&I, D, w, yy, wb, yb, omega, kappa, t, ttot, C->trials, C->restarts, k_restart, k_last);
  }
done:
  if (status != IN_NUMERICAL_ERROR) {
    for (int i = 0; i < n; ++i) x[i] = I.ew[i] * ret_w[i];
    for (int j = 0; j < m; ++j) y[j] = I.dy[j] * ret_y[j];
  }
  *omega_io = omega;
  free(w0); free(ax); free(w); free(yy); free(wb); free(yb); free(wst); free(yst); free(tau); free(eta);
  free(wmd); free(g); free(wtr); free(ytr); free(Bwtr); free(Bw); free(Bty); free(dwv); free(dyv);
  free(Hd); free(Btd); free(t1); free(t2); free(t3); free(t4); free(t5);
  iqp_free(&I);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3: practical outer iteration.                                  */
/* ------------------------------------------------------------------------ */
typedef struct { double rp, rd, sp, sd; } ores_t;

/* Eq. outer-residuals / outer-scales evaluated (a) in the scaled space and
 * (b) on the original data (x = Dx xbar, lambda = Dc lambdabar / c_s), the
 * latter also counting bound violations as in the external test (Sec. 4.1). */
static void outer_residuals(const sqp_t *S, const double *x, const double *lam, ores_t *sc, ores_t *un) {
  int n = S->n, m = S->m;
  double *ax = dvec((size_t)m), *qx = dvec((size_t)n), *atl = dvec((size_t)n);
  ocsr_mv(&S->A, x, ax);
  ocsr_mv(&S->Q, x, qx);
  ocsr_mv(&S->At, lam, atl);
  ores_t a = {0, 0, 1, 1}, b = {0, 0, 1, 1};
  for (int j = 0; j < m; ++j) {
    double v = ax[j], lo = S->lc[j], hi = S->uc[j];
    double viol = v < lo ? lo - v : (v > hi ? v - hi : 0.0);
    a.rp = rmax(a.rp, viol);
    a.sp = smax(a.sp, fabs(v));
    if (isfinite(lo)) a.sp = smax(a.sp, fabs(lo));
    if (isfinite(hi)) a.sp = smax(a.sp, fabs(hi));
    double d = S->Dc[j];
    b.rp = rmax(b.rp, viol / d);
    b.sp = smax(b.sp, fabs(v) / d);
    if (isfinite(lo)) b.sp = smax(b.sp, fabs(lo) / d);
    if (isfinite(hi)) b.sp = smax(b.sp, fabs(hi) / d);
  }
  for (int i = 0; i < n; ++i) {
    double gsc = qx[i] + S->c[i] + atl[i];
    a.rd = rmax(a.rd, fabs(x[i] - proj(x[i] - gsc, S->lx[i], S->ux[i])));
    a.sd = smax(a.sd, smax(smax(fabs(qx[i]), fabs(S->c[i])), fabs(atl[i])));
    double f = 1.0 / (S->cs * S->Dx[i]);
    double xo = S->Dx[i] * x[i];
    double lo = S->lx[i] * S->Dx[i], hi = S->ux[i] * S->Dx[i];
    double go = gsc * f;
    b.rd = rmax(b.rd, fabs(xo - proj(xo - go, lo, hi)));
    b.rp = rmax(b.rp, xo < lo ? lo - xo : (xo > hi ? xo - hi : 0.0));
    b.sd = smax(b.sd, smax(smax(fabs(qx[i] * f), fabs(S->c[i] * f)), fabs(atl[i] * f)));
  }
  *sc = a; *un = b;
  free(ax); free(qx); free(atl);
}

/* Sec. "Infeasibility detection", on the scaled problem (reading: the
 * QPALM-style certificate tests with l_inf-normalised directions and one
 * tolerance eps).
 * Primal: y = lambda^{k+1} - lambda^k is an approximate Farkas certificate of
 *   {x in [l_x, u_x] : A x in [l_c, u_c]}: the support function
 *   sigma_C(y) + sigma_X(-A'y) (sigma_S(v) = sup over S of v's) is below
 *   -eps ||y||, where every term that would need an infinite bound (the sign
 *   and stationarity conditions) is at most eps ||y|| in size.
 * Dual: d = x^{k+1} - x^k is an approximate recession direction (A d in the
 *   recession cone of [l_c, u_c], d in that of [l_x, u_x], each within
 *   eps ||d||) along which the objective decreases: d'Qd < -eps ||d||^2, or
 *   ||Q d|| <= eps ||d|| and c'd < -eps ||d||.
 * Returns OR_PRIMAL_INFEASIBLE, OR_DUAL_INFEASIBLE or -1. */
static int infeasibility(const sqp_t *S, const double *dlam, const double *dx, double eps) {
  const int n = S->n, m = S->m;
  const double nl = norm_inf(dlam, m), nx = norm_inf(dx, n);
  if (nl > 0.0) {
    double *v = dvec((size_t)n);
    for (int i = 0; i < m; ++i)
      for (int k = S->A.rp[i]; k < S->A.rp[i + 1]; ++k) v[S->A.ci[k]] -= S->A.v[k] * dlam[i];
    double sgn = 0.0, sep = 0.0;
    for (int i = 0; i < m; ++i) {
      const double y = dlam[i];
      if (y > 0.0) {
        if (isinf(S->uc[i])) sgn = dmax(sgn, y); else sep += S->uc[i] * y;
      } else if (y < 0.0) {
        if (isinf(S->lc[i])) sgn = dmax(sgn, -y); else sep += S->lc[i] * y;
      }
    }
    for (int j = 0; j < n; ++j) {
      const double w = v[j];
      if (w > 0.0) {
        if (isinf(S->ux[j])) sgn = dmax(sgn, w); else sep += S->ux[j] * w;
      } else if (w < 0.0) {
        if (isinf(S->lx[j])) sgn = dmax(sgn, -w); else sep += S->lx[j] * w;
      }
    }
    free(v);
    if (sgn <= eps * nl && sep < -eps * nl) return OR_PRIMAL_INFEASIBLE;
  }
  if (nx > 0.0) {
    double *ad = dvec((size_t)m), *qd = dvec((size_t)n);
    ocsr_mv(&S->A, dx, ad);
    ocsr_mv(&S->Q, dx, qd);
    double rec = 0.0;
    for (int i = 0; i < m; ++i) {
      if (!isinf(S->lc[i]) && ad[i] < 0.0) rec = dmax(rec, -ad[i]);
      if (!isinf(S->uc[i]) && ad[i] > 0.0) rec = dmax(rec, ad[i]);
    }
    for (int j = 0; j < n; ++j) {
      if (!isinf(S->lx[j]) && dx[j] < 0.0) rec = dmax(rec, -dx[j]);
      if (!isinf(S->ux[j]) && dx[j] > 0.0) rec = dmax(rec, dx[j]);
    }
    const double curv = dot(dx, qd, n), lin = dot(S->c, dx, n), qn = norm_inf(qd, n);
    free(ad);
    free(qd);
    if (rec <= eps * nx && (curv < -eps * nx * nx || (qn <= eps * nx && lin < -eps * nx))) return OR_DUAL_INFEASIBLE;
  }
  return -1;
}

/* Sec. "Anderson acceleration": classical Type-II Anderson acceleration of the
 * outer fixed-point map G: u^k = (lambda^k, z^k) -> (lambda^{k+1}, z^{k+1}).
 * The memory holds the last m_A pairs (u_i, G(u_i)); with residuals
 * f_i = G(u_i) - u_i and the difference columns dF_a = f_{a+1} - f_a,
 * dG_a = G(u_{a+1}) - G(u_a) (a over the stored pairs), the coefficients
 * solve min_g ||f_k - dF g||_2 through the normal equations (dF'dF + mu I) g =
 * dF' f_k with mu = 1e-12 trace(dF'dF) (plain Gaussian elimination), and the
 * next point is G(u_k) - dG g. */
typedef struct {
  int cap, len, dim;
  double *u, *g; /* cap x dim each, oldest first */
} anderson_t;

static void aa_init(anderson_t *A, int cap, int dim) {
  A->cap = cap < 1 ? 1 : cap;
  A->len = 0;
  A->dim = dim;
  A->u = dvec((size_t)A->cap * dim);
  A->g = dvec((size_t)A->cap * dim);
}
static void aa_free(anderson_t *A) { free(A->u); free(A->g); }
static void aa_push(anderson_t *A, const double *u, const double *g) {
  if (A->len == A->cap) {
    memmove(A->u, A->u + A->dim, sizeof(double) * (size_t)(A->cap - 1) * A->dim);
    memmove(A->g, A->g + A->dim, sizeof(double) * (size_t)(A->cap - 1) * A->dim);
    A->len--;
  }
  memcpy(A->u + (size_t)A->len * A->dim, u, sizeof(double) * A->dim);
  memcpy(A->g + (size_t)A->len * A->dim, g, sizeof(double) * A->dim);
  A->len++;
}
/* Writes the extrapolated point to out; returns 0, or -1 without a step. */
static int aa_step(const anderson_t *A, double *out) {
  const int L = A->len, D = A->dim, nc = L - 1;
  if (nc < 1) return -1;
  double M[16], rhs[4], gam[4];
  const double *fk_u = A->u + (size_t)(L - 1) * D, *fk_g = A->g + (size_t)(L - 1) * D;
  for (int a = 0; a < nc; ++a) {
    rhs[a] = 0.0;
    for (int b = 0; b < nc; ++b) M[a * nc + b] = 0.0;
  }
  for (int i = 0; i < D; ++i) {
    double df[4];
    for (int a = 0; a < nc; ++a) {
      const double f1 = A->g[(size_t)(a + 1) * D + i] - A->u[(size_t)(a + 1) * D + i];
      const double f0 = A->g[(size_t)a * D + i] - A->u[(size_t)a * D + i];
      df[a] = f1 - f0;
    }
    const double fk = fk_g[i] - fk_u[i];
    for (int a = 0; a < nc; ++a) {
      rhs[a] += df[a] * fk;
      for (int b = 0; b < nc; ++b) M[a * nc + b] += df[a] * df[b];
    }
  }
  double tr = 0.0;
  for (int a = 0; a < nc; ++a) tr += M[a * nc + a];
  if (!(tr > 0.0) || !isfinite(tr)) return -1;
  for (int a = 0; a < nc; ++a) M[a * nc + a] += 1e-12 * tr;
  /* Gaussian elimination without pivoting (symmetric positive definite). */
  for (int c = 0; c < nc; ++c) {
    const double piv = M[c * nc + c];
    if (!(piv > 0.0)) return -1;
    for (int r = c + 1; r < nc; ++r) {
      const double f = M[r * nc + c] / piv;
      for (int k = c; k < nc; ++k) M[r * nc + k] -= f * M[c * nc + k];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int c = nc - 1; c >= 0; --c) {
    double v = rhs[c];
    for (int k = c + 1; k < nc; ++k) v -= M[c * nc + k] * gam[k];
    gam[c] = v / M[c * nc + c];
  }
  /* Safeguard (reading): no step when the extrapolation moves G(u_k) by more
   * than 10 ||f_k||_2. */
  double fn = 0.0, sn = 0.0;
  for (int i = 0; i < D; ++i) {
    double v = 0.0;
    for (int a = 0; a < nc; ++a) v += gam[a] * (A->g[(size_t)(a + 1) * D + i] - A->g[(size_t)a * D + i]);
    const double fk = fk_g[i] - fk_u[i];
    fn += fk * fk;
    sn += v * v;
    out[i] = fk_g[i] - v;
  }
  if (!(sn <= 100.0 * fn)) return -1;
  return 0;
}

/* Test entry: one Anderson step from len stored pairs (rows of U and G, oldest
 * first, len <= 5); returns 0 and writes out (dim), or -1 without a step. */
int or_anderson_step(int len, int dim, const double *U, const double *G, double *out) {
  if (len < 1 || len > 5 || dim < 1) return -1;
  anderson_t A;
  aa_init(&A, len, dim);
  for (int i = 0; i < len; ++i) aa_push(&A, U + (size_t)i * dim, G + (size_t)i * dim);
  const int rc = aa_step(&A, out);
  aa_free(&A);
  return rc;
}

static double now_seconds(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Shared setup (Sec. 3.1 and 3.2.1): scaled problem, gamma, x0, lambda0, sigma0. */
typedef struct {
  sqp_t S;
  double gamma, lam_min;
  double *x, *lam, *z, *sig, *rprev, *yin;
} state_t;

static void setup(const or_problem *P, const or_params *prm, state_t *T) {
  memset(T, 0, sizeof(*T));
  sqp_build(P, prm, &T->S);
  sqp_t *S = &T->S;
  int n = S->n, m = S->m;
  T->gamma = choose_gamma(S, prm, &T->lam_min);
  T->x = dvec((size_t)n); T->z = dvec((size_t)n);
  T->lam = dvec((size_t)m); T->sig = dvec((size_t)m); T->rprev = dvec((size_t)m); T->yin = dvec((size_t)m);
  for (int i = 0; i < n; ++i) {
    double x0 = P->x0 ? P->x0[i] / S->Dx[i] : 0.0;
    T->x[i] = proj(x0, S->lx[i], S->ux[i]);
    T->z[i] = T->x[i];
  }
  for (int r = 0; r < m; ++r) T->lam[r] = P->lam0 ? S->cs * P->lam0[S->perm[r]] / S->Dc[r] : 0.0;
  /* Initial row penalties as in QPALM: sigma_init max(1,|f(x0)|) / max(1, ||dist||^2/2). */
  double *ax = dvec((size_t)m), *qx = dvec((size_t)n);
  ocsr_mv(&S->A, T->x, ax);
  ocsr_mv(&S->Q, T->x, qx);
  double f0 = 0.5 * dot(T->x, qx, n) + dot(S->c, T->x, n);
  double dist2 = 0.0;
  for (int j = 0; j < m; ++j) { double e = ax[j] - proj(ax[j], S->lc[j], S->uc[j]); dist2 += e * e; }
  double s0 = prm->sigma_init * dmax(1.0, fabs(f0)) / dmax(1.0, 0.5 * dist2);
  s0 = dmin(1e4, dmax(1e-4, s0));
  for (int j = 0; j < m; ++j) {
    T->sig[j] = s0;
    double s = j < S->mE ? S->lc[j] : proj(ax[j] + T->lam[j] / s0, S->lc[j], S->uc[j]);
    T->rprev[j] = ax[j] - s;
    T->yin[j] = -T->lam[j];
  }
  free(ax); free(qx);
}

static void state_free(state_t *T) {
  sqp_free(&T->S);
  free(T->x); free(T->lam); free(T->z); free(T->sig); free(T->rprev); free(T->yin);
}

/* Optional per-outer-iteration trace (or_solve_traced), for the pins of the
 * outer rules: one row of OTR_COLS scalars per outer iteration that reached
 * the tolerance update,
 *   [0] k, [1] primal part of the termination test met, [2] ||r||_inf,
 *   [3] ||x^{k+1} - z^k||_inf, [4..7] scaled r_p, r_d, s_p, s_d,
 *   [8..11] the same on the original data, [12] gamma, [13] the ratio of Eq.
 *   inner-tolerance-factor, [14] rho_in, [15..16] delta_a, delta_r before,
 *   [17..18] after, [19..20] eps_a,k, eps_r,k before, [21..22] after,
 *   [23] center moved, [24] s_d^in of the candidate the inner solve returned
 * and the vectors [x^{k+1} | z^k | z after the center update | lambda^{k+1} |
 * sigma before | sigma after | r | r of the previous iteration] (n, n, n, m,
 * m, m, m, m entries) in the scaled internal coordinates (rows E then I). */
#define OTR_COLS 25
typedef struct {
  int max_rows, n_rows;
  double *rows, *vecs;
} otrace_t;

static int solve_impl(const or_problem *P, const or_params *prm, double *x_out, double *y_out, or_result *res,
                      otrace_t *TR);

int or_solve(const or_problem *P, const or_params *prm, double *x_out, double *y_out, or_result *res) {
  return solve_impl(P, prm, x_out, y_out, res, NULL);
}

/* or_solve with the outer trace; returns the status, rows written in *n_rows. */
int or_solve_traced(const or_problem *P, const or_params *prm, double *x_out, double *y_out, or_result *res,
                    int max_rows, double *rows, double *vecs, int *n_rows) {
  otrace_t tr = {max_rows, 0, rows, vecs};
  int st = solve_impl(P, prm, x_out, y_out, res, &tr);
  *n_rows = tr.n_rows;
  return st;
}

static int solve_impl(const or_problem *P, const or_params *prm, double *x_out, double *y_out, or_result *res,
                      otrace_t *TR) {
  double t0 = now_seconds();
  state_t T;
  setup(P, prm, &T);
  sqp_t *S = &T.S;
  int n = S->n, m = S->m;
  double omega = 1.0;
  double dta = 1.0, dtr = 1.0, eak = 1.0, erk = 1.0;
  ctr_t C = {0, 0, 0};
  memset(res, 0, sizeof(*res));
  res->gamma = T.gamma; res->lambda_min = T.lam_min;
  int status = OR_ITER_LIMIT;
  double *ax = dvec((size_t)m), *r = dvec((size_t)m), *xold = dvec((size_t)n);
  double *lold = dvec((size_t)m), *dl = dvec((size_t)m), *dxv = dvec((size_t)n);
  const double eps_inf = prm->eps_inf > 0.0 ? prm->eps_inf : 1e-5;
  /* Anderson state: u^k = (lambda^k, z^k) at the start of iteration k. */
  anderson_t AA;
  aa_init(&AA, prm->anderson_mem, m + n);
  double *u0 = dvec((size_t)(m + n)), *gu = dvec((size_t)(m + n)), *ue = dvec((size_t)(m + n));
  int primal_ok_prev = 0, aa_applied = 0, aa_cool = 0;
  double rel_prev = INFINITY;
  long long k;
  ores_t sc = {0, 0, 1, 1}, un = {0, 0, 1, 1};
  for (k = 0; k < prm->k_out; ++k) {
    if (now_seconds() - t0 > prm->time_limit) { status = OR_TIME_LIMIT; break; }
    memcpy(xold, T.x, sizeof(double) * n);
    memcpy(u0, T.lam, sizeof(double) * m);
    memcpy(u0 + m, T.z, sizeof(double) * n);
    int ist = inner_solve(S, prm, T.z, T.lam, T.sig, T.gamma, dta, dtr, T.x, T.yin, &omega, &C, NULL);
    if (ist == IN_NUMERICAL_ERROR) { status = OR_NUMERICAL_ERROR; ++k; break; }
    if (ist == IN_ITER_LIMIT) continue;
    /* Eq. practical-multiplier-update (two-sided reading for I rows). */
    memcpy(lold, T.lam, sizeof(double) * m);
    ocsr_mv(&S->A, T.x, ax);
    for (int j = 0; j < m; ++j) {
      if (j < S->mE) {
        r[j] = ax[j] - S->lc[j];
        T.lam[j] = T.lam[j] + T.sig[j] * r[j];
      } else {
        double s = proj(ax[j] + T.lam[j] / T.sig[j], S->lc[j], S->uc[j]);
        r[j] = ax[j] - s;
        T.lam[j] = T.lam[j] + T.sig[j] * r[j];
      }
    }
    /* Eq. outer-residuals / outer-scales / outer-termination. */
    outer_residuals(S, T.x, T.lam, &sc, &un);
    if (un.rp <= prm->eps_abs + prm->eps_rel * un.sp && un.rd <= prm->eps_abs + prm->eps_rel * un.sd) {
      status = OR_SOLVED; ++k; break;
    }
    /* Sec. "Infeasibility detection". */
    for (int j = 0; j < m; ++j) dl[j] = T.lam[j] - lold[j];
    for (int i = 0; i < n; ++i) dxv[i] = T.x[i] - xold[i];
    {
      const int inf = infeasibility(S, dl, dxv, eps_inf);
      if (inf >= 0) { status = inf; ++k; break; }
    }
    /* Eq. penalty-trigger-eq: row-wise increase when the residual did not drop enough,
     * as long as the primal part of Eq. outer-termination is not met yet. */
    double rn = norm_inf(r, m);
    int primal_ok = un.rp <= prm->eps_abs + prm->eps_rel * un.sp && sc.rp <= prm->eps_abs + prm->eps_rel * sc.sp;
    double *trow = NULL, *tvec = NULL;
    if (TR && TR->n_rows < TR->max_rows) {
      trow = TR->rows + (size_t)TR->n_rows * OTR_COLS;
      tvec = TR->vecs + (size_t)TR->n_rows * (3 * (size_t)n + 5 * (size_t)m);
      TR->n_rows++;
      trow[0] = (double)k; trow[1] = primal_ok; trow[2] = rn;
      trow[4] = sc.rp; trow[5] = sc.rd; trow[6] = sc.sp; trow[7] = sc.sd;
      trow[8] = un.rp; trow[9] = un.rd; trow[10] = un.sp; trow[11] = un.sd; trow[12] = T.gamma;
      trow[15] = dta; trow[16] = dtr; trow[19] = eak; trow[20] = erk;
      memcpy(tvec, T.x, sizeof(double) * n);
      memcpy(tvec + n, T.z, sizeof(double) * n);
      memcpy(tvec + 3 * (size_t)n, T.lam, sizeof(double) * m);
      memcpy(tvec + 3 * (size_t)n + m, T.sig, sizeof(double) * m);
      memcpy(tvec + 3 * (size_t)n + 3 * (size_t)m, r, sizeof(double) * m);
      memcpy(tvec + 3 * (size_t)n + 4 * (size_t)m, T.rprev, sizeof(double) * m);
    }
    for (int j = 0; j < m; ++j) {
      int active = j < S->mE || T.lam[j] != 0.0;
      if (active && !primal_ok && fabs(r[j]) > prm->theta_sigma * fabs(T.rprev[j]) && rn > 0.0)
        T.sig[j] = dmin(prm->sigma_max, T.sig[j] * dmax(1.0, prm->delta_sigma * fabs(r[j]) / rn));
      T.rprev[j] = r[j];
    }
    /* Eq. inner-tolerance-factor. */
    double dx = 0.0;
    for (int i = 0; i < n; ++i) dx = dmax(dx, fabs(T.x[i] - T.z[i]));
    double ratio = sc.rd > 0.0 ? dmin(1.0, (dx / T.gamma) / sc.rd) : 1.0;
    double rho = prm->rho_in_max - (prm->rho_in_max - prm->rho_in_min) * ratio;
    dta = dmax(dta * rho, prm->tol_floor * prm->eps_abs);
    dtr = dmax(dtr * rho, prm->tol_floor * prm->eps_rel);
    if (trow) {
      trow[3] = dx; trow[13] = ratio; trow[14] = rho; trow[17] = dta; trow[18] = dtr; trow[24] = C.sd_in;
      memcpy(tvec + 3 * (size_t)n + 2 * (size_t)m, T.sig, sizeof(double) * m);
    }
    if (prm->verbose) {
      double sig_hi = 0.0;
      for (int j = 0; j < m; ++j) sig_hi = dmax(sig_hi, T.sig[j]);
      fprintf(stderr, "k=%lld inner=%lld rp=%.3e rd=%.3e sp=%.3e sd=%.3e | un rp=%.3e rd=%.3e | dta=%.2e ratio=%.3f "
              "smax=%.2e eak=%.2e omega=%.3e\n", k, C.accepted, sc.rp, sc.rd, sc.sp, sc.sd, un.rp, un.rd, dta, ratio,
              sig_hi, eak, omega);
    }
    /* Eq. center-update / center-tolerance-update. */
    const int moved = sc.rp <= eak + erk * sc.sp;
    if (moved) {
      memcpy(T.z, T.x, sizeof(double) * n);
      eak = dmax(eak * prm->rho_z, prm->eps_abs);
      erk = dmax(erk * prm->rho_z, prm->eps_rel);
    }
    if (trow) {
      trow[21] = eak; trow[22] = erk; trow[23] = moved;
      memcpy(tvec + 2 * (size_t)n, T.z, sizeof(double) * n);
    }
    /* Sec. "Anderson acceleration" (reading: active while the primal part of
     * the termination test holds on this and the previous outer iteration,
     * i.e. once the penalties have stopped growing; the memory is cleared
     * otherwise, and an accelerated step that raised the relative KKT
     * residual pauses it for m_A iterations). */
    if (prm->anderson) {
      const double rel = dmax(un.rp / (1.0 + un.sp), un.rd / (1.0 + un.sd));
      /* A step that raised the relative KKT residual or lost primal
       * feasibility switches the acceleration off for the rest of the solve. */
      if (aa_applied && (rel > rel_prev || !primal_ok)) aa_cool = 1;
      const int active = primal_ok && primal_ok_prev && aa_cool == 0;
      if (!active) {
        AA.len = 0;
        aa_applied = 0;
      } else {
        memcpy(gu, T.lam, sizeof(double) * m);
        memcpy(gu + m, T.z, sizeof(double) * n);
        aa_push(&AA, u0, gu);
        aa_applied = 0;
        if (aa_step(&AA, ue) == 0) {
          memcpy(T.lam, ue, sizeof(double) * m);
          memcpy(T.z, ue + m, sizeof(double) * n);
          aa_applied = 1;
        }
      }
      rel_prev = rel;
    }
    primal_ok_prev = primal_ok;
  }
  /* Unscale and return (Algorithm 3). */
  for (int i = 0; i < n; ++i) x_out[i] = S->Dx[i] * T.x[i];
  for (int r2 = 0; r2 < m; ++r2) y_out[S->perm[r2]] = S->Dc[r2] * T.lam[r2] / S->cs;
  outer_residuals(S, T.x, T.lam, &sc, &un);
  res->status = status;
  res->outer_iters = k;
  res->inner_iters = C.accepted; res->trials = C.trials; res->restarts = C.restarts;
  res->r_p = un.rp; res->r_d = un.rd; res->s_p = un.sp; res->s_d = un.sd;
  res->rel_kkt = dmax(un.rp / (1.0 + un.sp), un.rd / (1.0 + un.sd));
  {
    /* objective in original coordinates */
    double *qx = dvec((size_t)n);
    ocsr Qo = {n, n, P->q_rp[n], (int *)P->q_rp, (int *)P->q_ci, (double *)P->q_v};
    ocsr_mv(&Qo, x_out, qx);
    res->obj = 0.5 * dot(x_out, qx, n) + dot(P->c, x_out, n);
    free(qx);
  }
  res->seconds = now_seconds() - t0;
  free(ax); free(r); free(xold); free(lold); free(dl); free(dxv);
  free(u0); free(gu); free(ue);
  aa_free(&AA);
  state_free(&T);
  return status;
}

/* Runs the inner solve of outer iteration 0 with convergence ignored and
 * writes snapshots after the listed accepted-iteration counts (increasing).
 * Snapshot layout: [w (dw) | y (m) | wbar (dw) | ybar (m) | 8 scalars] in the
 * outer-scaled, inner-unscaled coordinates of Eq. inner-qp, rows E then I. */
int or_debug_inner(const or_problem *P, const or_params *prm, int n_ckpt, const long long *ckpt,
                   double *snap, double *gamma_out) {
  state_t T;
  setup(P, prm, &T);
  double omega = 1.0;
  ctr_t C = {0, 0, 0};
  dbg_t D = {n_ckpt, ckpt, snap, 0, 1, NULL};
  int st = inner_solve(&T.S, prm, T.z, T.lam, T.sig, T.gamma, 1.0, 1.0, T.x, T.yin, &omega, &C, &D);
  if (gamma_out) *gamma_out = T.gamma;
  state_free(&T);
  return st == IN_NUMERICAL_ERROR ? -1 : D.next_ckpt;
}

/* Trace of the periodic checks of the first inner solve (convergence
 * ignored) for the restart pins: the first max_checks checks, each one row of
 * CHK_COLS scalars
 *   [0] accepted iterations so far, [1] epoch length t, [2] KKT_w of the
 *   current point, [3] of the average, [4] KKT_w at the last restart, [5] at
 *   the previous check, [6] average chosen, [7] restart, [8] omega before,
 *   [9] omega after, [10] kappa before, [11] kappa after, [12] t after,
 *   [13] KKT_w at the last restart after the decision, [14..17] r_p, r_d,
 *   s_p, s_d of Eqs. inner-residuals / inner-scales at the current point,
 *   [18..21] the same at the average
 * and the vectors [w | y | wbar | ybar | w_start | y_start] (dw and m
 * entries each, inner-unscaled coordinates, rows E then I) before the
 * decision.  Returns the number of rows written, or -1 on a numerical error. */
int or_debug_checks(const or_problem *P, const or_params *prm, int max_checks, double *rows, double *vecs) {
  state_t T;
  setup(P, prm, &T);
  double omega = 1.0;
  ctr_t C = {0, 0, 0};
  const long long stop = (long long)prm->k_chk * max_checks;
  int dw = T.S.n + T.S.mI + T.S.m;
  double *snap = dvec(2 * (size_t)(dw + T.S.m) + SNAP_SCALARS);
  dbg_t D = {1, &stop, snap, 0, 1, NULL, max_checks, 0, rows, vecs};
  int st = inner_solve(&T.S, prm, T.z, T.lam, T.sig, T.gamma, 1.0, 1.0, T.x, T.yin, &omega, &C, &D);
  free(snap);
  state_free(&T);
  return st == IN_NUMERICAL_ERROR ? -1 : D.chk_n;
}

/* Scaling data of the setup, for tests: Dc (internal row order), Dx, perm, c_s, gamma, sigma0. */
int or_setup_info(const or_problem *P, const or_params *prm, double *Dc, double *Dx, int *perm,
                  double *scalars /* cs, gamma, lambda_min, sigma0, mE, qnorm */) {
  state_t T;
  setup(P, prm, &T);
  sqp_t *S = &T.S;
  for (int j = 0; j < S->m; ++j) { Dc[j] = S->Dc[j]; perm[j] = S->perm[j]; }
  for (int i = 0; i < S->n; ++i) Dx[i] = S->Dx[i];
  scalars[0] = S->cs; scalars[1] = T.gamma; scalars[2] = T.lam_min;
  scalars[3] = S->m ? T.sig[0] : 0.0; scalars[4] = (double)S->mE; scalars[5] = S->qnorm;
  state_free(&T);
  return 0;
}

/* Dense form of the inner QP of Eq. inner-qp (no scaling), for tests on tiny
 * instances: H (dw x dw), q, B (m x dw), h, lo, hi.  Uses the problem's own
 * (unscaled, unpermuted-E-first) data when prm->no_scaling is set. */
int or_inner_qp_dense(const or_problem *P, const or_params *prm, const double *z, const double *lam,
                      const double *sig, double gamma, double *H, double *q, double *B, double *h,
                      double *lo, double *hi, int *dims /* n, m, mE, mI, dw */) {
  sqp_t S;
  sqp_build(P, prm, &S);
  iqp_t I;
  iqp_form(&S, z, lam, sig, gamma, &I);
  int dw = I.dw;
  memset(H, 0, sizeof(double) * (size_t)dw * dw);
  memset(B, 0, sizeof(double) * (size_t)S.m * dw);
  for (int i = 0; i < dw; ++i)
    for (int k = I.H.rp[i]; k < I.H.rp[i + 1]; ++k) H[(size_t)i * dw + I.H.ci[k]] += I.H.v[k];
  for (int j = 0; j < S.m; ++j)
    for (int k = I.B.rp[j]; k < I.B.rp[j + 1]; ++k) B[(size_t)j * dw + I.B.ci[k]] += I.B.v[k];
  memcpy(q, I.q, sizeof(double) * dw);
  memcpy(h, I.h, sizeof(double) * S.m);
  memcpy(lo, I.lo, sizeof(double) * dw);
  memcpy(hi, I.hi, sizeof(double) * dw);
  dims[0] = S.n; dims[1] = S.m; dims[2] = S.mE; dims[3] = S.mI; dims[4] = dw;
  iqp_free(&I);
  sqp_free(&S);
  return 0;
}

/* Diagonal step data of the first inner solve, for tests: mw (dw), my (m),
 * ew (dw), dy (m), in the scaled inner space of outer iteration 0. */
int or_inner_steps(const or_problem *P, const or_params *prm, double *mw, double *my, double *ew, double *dy) {
  state_t T;
  setup(P, prm, &T);
  iqp_t I;
  iqp_form(&T.S, T.z, T.lam, T.sig, T.gamma, &I);
  iqp_scale(&I, prm->ruiz_inner);
  memcpy(mw, I.mw, sizeof(double) * I.dw);
  memcpy(my, I.my, sizeof(double) * I.m);
  memcpy(ew, I.ew, sizeof(double) * I.dw);
  memcpy(dy, I.dy, sizeof(double) * I.m);
  iqp_free(&I);
  state_free(&T);
  return 0;
}

/* Solves one inner QP (Eq. inner-qp) with given z, lambda, sigma (internal row
 * order) and gamma to the tolerance tol from x, y; returns the status.  Used by
 * the brute-force pins.  Runs in the scaled space of the setup. */
int or_inner_solve_given(const or_problem *P, const or_params *prm, const double *z_orig, const double *lam_int,
                         const double *sig_int, double gamma, double tol, long long kin, double *x_io,
                         double *y_io, long long *iters) {
  or_params p2 = *prm;
  p2.k_in = kin;
  sqp_t S;
  sqp_build(P, &p2, &S);
  double *z = dvec((size_t)S.n), *x = dvec((size_t)S.n);
  for (int i = 0; i < S.n; ++i) { z[i] = z_orig[i] / S.Dx[i]; x[i] = x_io[i] / S.Dx[i]; }
  double omega = 1.0;
  ctr_t C = {0, 0, 0};
  int st = inner_solve(&S, &p2, z, lam_int, sig_int, gamma, tol, tol, x, y_io, &omega, &C, NULL);
  for (int i = 0; i < S.n; ++i) x_io[i] = S.Dx[i] * x[i];
  *iters = C.accepted;
  free(z); free(x);
  sqp_free(&S);
  return st;
}

/* External KKT test of Sec. 4.1 on the ORIGINAL problem: out = (r_p, r_d, s_p, s_d).
 * r_p includes variable-bound violations; lambda in the original row order. */
int or_kkt_check(const or_problem *P, const double *x, const double *lam, double *out) {
  int n = P->n, m = P->m;
  ocsr Q = {n, n, P->q_rp[n], (int *)P->q_rp, (int *)P->q_ci, (double *)P->q_v};
  ocsr A = {m, n, m ? P->a_rp[m] : 0, (int *)P->a_rp, (int *)P->a_ci, (double *)P->a_v};
  ocsr At;
  ocsr_transpose(&A, &At);
  double *ax = dvec((size_t)m), *qx = dvec((size_t)n), *atl = dvec((size_t)n);
  ocsr_mv(&A, x, ax);
  ocsr_mv(&Q, x, qx);
  ocsr_mv(&At, lam, atl);
  double rp = 0.0, rd = 0.0, sp = 1.0, sd = 1.0;
  for (int j = 0; j < m; ++j) {
    double lo = clean_bound(P->lc[j]), hi = clean_bound(P->uc[j]);
    double v = ax[j];
    rp = rmax(rp, v < lo ? lo - v : (v > hi ? v - hi : 0.0));
    sp = smax(sp, fabs(v));
    if (isfinite(lo)) sp = smax(sp, fabs(lo));
    if (isfinite(hi)) sp = smax(sp, fabs(hi));
  }
  for (int i = 0; i < n; ++i) {
    double lo = clean_bound(P->lx[i]), hi = clean_bound(P->ux[i]);
    rp = rmax(rp, x[i] < lo ? lo - x[i] : (x[i] > hi ? x[i] - hi : 0.0));
    double g = qx[i] + P->c[i] + atl[i];
    rd = rmax(rd, fabs(x[i] - proj(x[i] - g, lo, hi)));
    sd = smax(sd, smax(smax(fabs(qx[i]), fabs(P->c[i])), fabs(atl[i])));
  }
  out[0] = rp; out[1] = rd; out[2] = sp; out[3] = sd;
  free(ax); free(qx); free(atl);
  ocsr_free(&At);
  return 0;
}

/* Same as or_debug_inner, also returning the wall-clock time of each
 * snapshot relative to the start of the inner iterations (times[k]), for the
 * CPU baseline.  setup_seconds receives the time spent before the first
 * inner iteration. */
int or_debug_inner_timed(const or_problem *P, const or_params *prm, int n_ckpt, const long long *ckpt, double *snap,
                         double *times, double *setup_seconds) {
  double t0 = now_seconds();
  state_t T;
  setup(P, prm, &T);
  double omega = 1.0;
  ctr_t C = {0, 0, 0};
  dbg_t D = {n_ckpt, ckpt, snap, 0, 1, times};
  double t1 = now_seconds();
  int st = inner_solve(&T.S, prm, T.z, T.lam, T.sig, T.gamma, 1.0, 1.0, T.x, T.yin, &omega, &C, &D);
  for (int k = 0; k < D.next_ckpt; ++k) times[k] -= t1;
  *setup_seconds = t1 - t0;
  state_free(&T);
  return st == IN_NUMERICAL_ERROR ? -1 : D.next_ckpt;
}
