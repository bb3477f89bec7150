/*
 * tron_oracle.c -- CPU FP64 oracle of the batched trust-region Newton solve and of the
 * component ADMM of arXiv 2106.14995.
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark are the only users.  The product (CUDA) path never loads this code.
 *
 * Plain and slow on purpose: one problem at a time, textbook loops, sequential sums,
 * compiled with -ffp-contract=off.  Each routine cites the passage it restates.
 *
 *   Algorithm 1 (Sec. 3)       outer loop: evaluate, Cauchy point, free set, PCG, back
 *                              transform, projected search, convergence check
 *   Figure 2 (Sec. 3)          core operations axpy/copy/dot/gemv/nrm2/scal/trtrs/ccf/ccfs/
 *                              breakpt/gpstep/trqsol
 *   Sec. 4.3                   complete (dense) Cholesky of A + alpha*I, left-looking
 *   Sec. 4.4                   L^T kept explicitly in the upper triangle
 *   Sec. 5.1                   convergence test ||grad_[l,u] f||_inf <= eps
 *   Sec. 6.1, eq. exp-branch   branch objective, flows from eqs. pij-qji
 *   Sec. 6.1                   component ADMM: generator and branch, then bus, then
 *                              multipliers
 *   Sec. 4.2 footnote          hs45 variant f = 120 - prod x_i, x_i <= i
 *
 * Steps the paper leaves open (acceptance test, radius update, search constants,
 * Cholesky shift, CG tolerance, ADMM closed forms) follow the readings recorded in the
 * design notes; their constants are the fields of ot_opts.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

void ot_default_opts(ot_opts* o) {
  o->gtol = 1e-6;
  o->max_outer = 500;
  o->max_trials = 30;
  o->mu0 = 0.01;
  o->mu1 = 1.0;
  o->interpf = 0.1;
  o->extrapf = 10.0;
  o->proj_shrink = 0.5;
  o->eta0 = 1e-4;
  o->eta1 = 0.25;
  o->eta2 = 0.75;
  o->sigma1 = 0.25;
  o->sigma3 = 4.0;
  o->delta_max = 1e10;
  o->delta_min_rel = 1e-12;
  o->cg_rtol = 0.1;
  o->shift_frac = 1e-3;
  o->max_shift = 30;
  o->tr_norm = 0;
  o->ared_guard = 1e-13;
  o->cauchy_norm = 0;
  o->pad1 = 0;
}

/* ------------------------------------------------------------ Figure 2 core operations */

static double dot(int n, const double* x, const double* y, ot_counters* c) {
  double s = 0.0;
  for (int i = 0; i < n; i++) s += x[i] * y[i];
  if (c) c->flops += 2.0 * n;
  return s;
}

static double nrm2(int n, const double* x, ot_counters* c) {
  double s = dot(n, x, x, c);
  if (c) c->flops += 1.0;
  return sqrt(s);
}

/* y <- A x, A row-major n x n with leading dimension lda */
static void gemv(int n, const double* A, int lda, const double* x, double* y, ot_counters* c) {
  for (int i = 0; i < n; i++) {
    double s = 0.0;
    for (int j = 0; j < n; j++) s += A[(size_t)i * lda + j] * x[j];
    y[i] = s;
  }
  if (c) c->flops += 2.0 * n * n;
}

static double proj1(double v, double lo, double hi) {
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

/* gpstep: s <- P_[l,u](x + alpha w) - x */
static void gpstep(int n, const double* x, double alpha, const double* w, const double* l,
                   const double* u, double* s, ot_counters* c) {
  for (int i = 0; i < n; i++) s[i] = proj1(x[i] + alpha * w[i], l[i], u[i]) - x[i];
  if (c) c->flops += 3.0 * n;
}

/* breakpt: b_i = (u_i - x_i)/w_i if w_i > 0, (l_i - x_i)/w_i if w_i < 0, over the
 * variables that can still move in direction w. */
void ot_breakpt(int n, const double* x, const double* w, const double* l, const double* u,
                int* nbrpt, double* brptmin, double* brptmax) {
  int nb = 0;
  double bmin = 0.0, bmax = 0.0;
  for (int i = 0; i < n; i++) {
    double b;
    if (x[i] < u[i] && w[i] > 0.0) {
      b = (u[i] - x[i]) / w[i];
    } else if (x[i] > l[i] && w[i] < 0.0) {
      b = (l[i] - x[i]) / w[i];
    } else {
      continue;
    }
    if (nb == 0) {
      bmin = b;
      bmax = b;
    } else {
      if (b < bmin) bmin = b;
      if (b > bmax) bmax = b;
    }
    nb++;
  }
  *nbrpt = nb;
  *brptmin = bmin;
  *brptmax = bmax;
}

/* trqsol: sigma >= 0 with ||x + sigma p||_2 = delta (positive root of the quadratic) */
static double trqsol_c(int n, const double* x, const double* p, double delta, ot_counters* c) {
  double ptx = dot(n, p, x, c);
  double ptp = dot(n, p, p, c);
  double xtx = dot(n, x, x, c);
  double dsq = delta * delta;
  double rad = ptx * ptx + ptp * (dsq - xtx);
  if (rad < 0.0) rad = 0.0;
  rad = sqrt(rad);
  if (c) c->flops += 12.0;
  if (ptx >= 0.0) return (dsq - xtx) / (ptx + rad);
  return (rad - ptx) / ptp;
}

double ot_trqsol(int n, const double* x, const double* p, double delta) {
  return trqsol_c(n, x, p, delta, NULL);
}

/* trtrs with L: solve L y = b in place (L lower, row-major m x m), column oriented */
static void trsv_lower(int m, const double* L, double* b, ot_counters* c) {
  for (int j = 0; j < m; j++) {
    b[j] = b[j] / L[(size_t)j * m + j];
    for (int i = j + 1; i < m; i++) b[i] -= L[(size_t)i * m + j] * b[j];
  }
  if (c) c->flops += (double)m * m;
}

/* trtrs with L^T: solve L^T z = y in place, column oriented over the columns of L^T
 * (which are the rows of L) */
static void trsv_upper_t(int m, const double* L, double* z, ot_counters* c) {
  for (int j = m - 1; j >= 0; j--) {
    z[j] = z[j] / L[(size_t)j * m + j];
    for (int i = 0; i < j; i++) z[i] -= L[(size_t)j * m + i] * z[j];
  }
  if (c) c->flops += (double)m * m;
}

/* ccf: left-looking unblocked Cholesky (Sec. 4.3).  On entry the lower triangle of L
 * holds the matrix; on success it holds the factor and the strict upper triangle holds
 * L^T (Sec. 4.4).  Returns 0, or j+1 if pivot j is not positive. */
static int chol_left_c(int m, double* L, ot_counters* c) {
  for (int j = 0; j < m; j++) {
    for (int i = j; i < m; i++) {
      double v = L[(size_t)i * m + j];
      for (int k = 0; k < j; k++) v -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = v;
    }
    if (c) c->flops += 2.0 * j * (m - j);
    double piv = L[(size_t)j * m + j];
    if (!(piv > 0.0)) return j + 1;
    double d = sqrt(piv);
    L[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; i++) L[(size_t)i * m + j] = L[(size_t)i * m + j] / d;
    if (c) c->flops += 1.0 + (m - j - 1);
  }
  for (int i = 0; i < m; i++)
    for (int j = 0; j < i; j++) L[(size_t)j * m + i] = L[(size_t)i * m + j];
  return 0;
}

int ot_chol_left(int m, double* A, int lda) {
  /* dense helper for tests: factor the lower triangle of a row-major matrix in place */
  double* L = (double*)malloc(sizeof(double) * (size_t)m * m + 8);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) L[(size_t)i * m + j] = A[(size_t)i * lda + j];
  int r = chol_left_c(m, L, NULL);
  if (r == 0)
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) A[(size_t)i * lda + j] = L[(size_t)i * m + j];
  free(L);
  return r;
}

/* ccf + ccfs: factor A + alpha I = L L^T for the first alpha of the shift sequence
 * alpha_0 = 0 if min A_ii > 0 else beta - min A_ii, alpha <- max(2 alpha, beta), with
 * beta = shift_frac * max |A_ii| (Sec. 4.3: "for some alpha >= 0"). */
static int chol_shifted_c(int m, const double* A, double* L, double frac, int max_shift,
                          double* alpha_out, ot_counters* c) {
  double maxd = 0.0, mind = A[0];
  for (int i = 0; i < m; i++) {
    double a = A[(size_t)i * m + i];
    if (fabs(a) > maxd) maxd = fabs(a);
    if (a < mind) mind = a;
  }
  double beta = frac * maxd;
  if (beta == 0.0) beta = frac;
  double alpha = (mind > 0.0) ? 0.0 : beta - mind;
  for (int t = 0; t <= max_shift; t++) {
    if (c) c->chol_calls++;
    for (int i = 0; i < m; i++)
      for (int j = 0; j <= i; j++) L[(size_t)i * m + j] = A[(size_t)i * m + j];
    for (int i = 0; i < m; i++) L[(size_t)i * m + i] = A[(size_t)i * m + i] + alpha;
    if (c) c->flops += m;
    if (chol_left_c(m, L, c) == 0) {
      if (alpha_out) *alpha_out = alpha;
      return 0;
    }
    alpha = 2.0 * alpha;
    if (alpha < beta) alpha = beta;
  }
  return 1;
}

int ot_chol_shifted(int m, const double* A, double* L, double shift_frac, int max_shift,
                    double* alpha_out) {
  return chol_shifted_c(m, A, L, shift_frac, max_shift, alpha_out, NULL);
}

double ot_pgnorm(int n, const double* x, const double* g, const double* l, const double* u) {
  /* (grad_[l,u] f)_i = g_i inside, min(g_i,0) at l_i, max(g_i,0) at u_i (Sec. 5.1) */
  double m = 0.0;
  for (int i = 0; i < n; i++) {
    double p = g[i];
    if (x[i] <= l[i] && p > 0.0) p = 0.0;
    if (x[i] >= u[i] && p < 0.0) p = 0.0;
    double a = fabs(p);
    if (a > m) m = a;
  }
  return m;
}

/* Steihaug-Toint truncated CG on the preconditioned system (Algorithm 1, Sec. 3):
 * minimise 0.5 s'Ahat s + bhat's with Ahat = L^-1 A L^-T over the CG iterate s, whose
 * back transform w = L^-T s is accumulated along the iterations as
 * w += alpha L^-T p, the L^-T p being the backward solve that Ahat p needs anyway.
 * The trust region (norm == 0, the default) bounds the CG iterate itself, ||s||_2 <=
 * delta, as Algorithm 1 states; since s = L^T w this is ||L^T w||_2 <= delta on the step.
 * norm == 1 selects the other reading, ||w||_2 <= delta on the step in the original
 * variables.  trqsol (Figure 2) is applied to the vectors the bound is stated on.
 * Stops after m iterations, at the boundary, on negative curvature, or when the residual
 * norm drops to rtol*||bhat||.  Returns 0 converged, 1 iteration cap, 2 boundary,
 * 3 negative curvature; w receives the step L^-T s and *tr_len the length of the step
 * in the bounded norm (||s||_2 or ||w||_2). */
static int steihaug_c(int m, const double* A, const double* L, const double* bhat,
                      double delta, double rtol, int norm, double* w, int* iters,
                      double* tr_len, ot_counters* c) {
  double* res = (double*)malloc(sizeof(double) * (size_t)(7 * m + 8));
  double* p = res + m;
  double* q = p + m;
  double* z = q + m;
  double* wn = z + m;
  double* sv = wn + m;
  double* sn = sv + m;
  for (int i = 0; i < m; i++) {
    w[i] = 0.0;
    sv[i] = 0.0;
    res[i] = -bhat[i];
    p[i] = res[i];
  }
  double rr = dot(m, res, res, c);
  double tol = rtol * sqrt(rr);
  int info = 1, it = 0;
  while (it < m) {
    if (sqrt(rr) <= tol) {
      info = 0;
      break;
    }
    /* Ahat p = L^-1 (A (L^-T p)) : backward solve, gemv, forward solve (Sec. 4.4) */
    for (int i = 0; i < m; i++) z[i] = p[i];
    trsv_upper_t(m, L, z, c);
    gemv(m, A, m, z, q, c);
    trsv_lower(m, L, q, c);
    it++;
    if (c) c->cg_iters++;
    double kappa = dot(m, p, q, c);
    if (kappa <= 0.0) {
      double sigma = norm == 0 ? trqsol_c(m, sv, p, delta, c) : trqsol_c(m, w, z, delta, c);
      for (int i = 0; i < m; i++) {
        w[i] += sigma * z[i];
        sv[i] += sigma * p[i];
      }
      info = 3;
      break;
    }
    double alpha = rr / kappa;
    for (int i = 0; i < m; i++) {
      wn[i] = w[i] + alpha * z[i];
      sn[i] = sv[i] + alpha * p[i];
    }
    if (nrm2(m, norm == 0 ? sn : wn, c) >= delta) {
      double sigma = norm == 0 ? trqsol_c(m, sv, p, delta, c) : trqsol_c(m, w, z, delta, c);
      for (int i = 0; i < m; i++) {
        w[i] += sigma * z[i];
        sv[i] += sigma * p[i];
      }
      info = 2;
      break;
    }
    for (int i = 0; i < m; i++) {
      w[i] = wn[i];
      sv[i] = sn[i];
      res[i] -= alpha * q[i];
    }
    double rrn = dot(m, res, res, c);
    double beta = rrn / rr;
    rr = rrn;
    for (int i = 0; i < m; i++) p[i] = res[i] + beta * p[i];
    if (c) c->flops += (norm == 0 ? 8.0 : 6.0) * m + 2.0;
  }
  if (iters) *iters = it;
  if (tr_len) *tr_len = nrm2(m, norm == 0 ? sv : w, c);
  free(res);
  return info;
}

int ot_steihaug(int m, const double* A, const double* L, const double* bhat, double delta,
                double rtol, int norm, double* w, int* iters, double* tr_len) {
  return steihaug_c(m, A, L, bhat, delta, rtol, norm, w, iters, tr_len, NULL);
}

/* ------------------------------------------------------------------------ objectives */

/* Dense quartic family: params = [Q (n x n, row-major) | c (n) | d (n)],
 * f = 1/2 x'Qx + c'x + sum_i d_i x_i^4. */
static int eval_dense(int n, const double* P, const double* x, double* f, double* g,
                      double* H, ot_counters* c, double* fscale) {
  const double* Q = P;
  const double* cv = P + (size_t)n * n;
  const double* d = cv + n;
  double quad = 0.0, lin = 0.0, quart = 0.0, mag = 0.0;
  for (int i = 0; i < n; i++) {
    double qx = 0.0;
    for (int j = 0; j < n; j++) qx += Q[(size_t)i * n + j] * x[j];
    quad += x[i] * qx;
    lin += cv[i] * x[i];
    double x2 = x[i] * x[i];
    quart += d[i] * x2 * x2;
    mag += 0.5 * fabs(x[i] * qx) + fabs(cv[i] * x[i]) + fabs(d[i]) * x2 * x2;
    if (g) g[i] = qx + cv[i] + 4.0 * d[i] * x2 * x[i];
  }
  *f = 0.5 * quad + lin + quart;
  if (fscale) *fscale = mag;
  if (H) {
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) H[(size_t)i * n + j] = Q[(size_t)i * n + j];
    for (int i = 0; i < n; i++) H[(size_t)i * n + i] += 12.0 * d[i] * x[i] * x[i];
  }
  if (c) {
    c->flops += 2.0 * n * n + 9.0 * n + 2.0;
    if (g) c->flops += 5.0 * n;
    if (H) c->flops += 4.0 * n;
  }
  return 0;
}

/* hs45 variant (Sec. 4.2 footnote): f = 120 - prod_i x_i */
static int eval_hs45(int n, const double* x, double* f, double* g, double* H, ot_counters* c,
                     double* fscale) {
  double p = 1.0;
  for (int i = 0; i < n; i++) p *= x[i];
  *f = 120.0 - p;
  if (fscale) *fscale = 120.0 + fabs(p);
  if (g) {
    for (int i = 0; i < n; i++) {
      double q = 1.0;
      for (int j = 0; j < n; j++)
        if (j != i) q *= x[j];
      g[i] = -q;
    }
  }
  if (H) {
    for (int i = 0; i < n; i++) {
      for (int j = 0; j < n; j++) {
        if (i == j) {
          H[(size_t)i * n + j] = 0.0;
          continue;
        }
        double q = 1.0;
        for (int k = 0; k < n; k++)
          if (k != i && k != j) q *= x[k];
        H[(size_t)i * n + j] = -q;
      }
    }
  }
  if (c) {
    c->flops += n + 1.0;
    if (g) c->flops += (double)n * n;
    if (H) c->flops += (double)n * n * n;
  }
  return 0;
}

/* Branch record (36 doubles): [0:8] gc_ij bc_ij g_ij b_ij gc_ji bc_ji g_ji b_ji,
 * [8:16] multipliers, [16:24] targets, [24:32] penalties of the pairs
 * (p_ij q_ij p_ji q_ji w_i w_j th_i th_j), [32] smax^2, [33] line penalty. */

/* flows of eqs. pij-qji with w_i = v_i^2, w_j = v_j^2, wR = v_i v_j cos(th_i - th_j),
 * wI = v_i v_j sin(th_i - th_j) (Sec. 6.1) */
static void branch_pairs(const double* cf, const double* x, double cs, double sn, double* F) {
  double vi = x[0], vj = x[1];
  double wi = vi * vi, wj = vj * vj;
  double wR = vi * vj * cs, wI = vi * vj * sn;
  F[0] = cf[0] * wi - cf[2] * wR + cf[3] * wI;
  F[1] = cf[1] * wi - cf[3] * wR - cf[2] * wI;
  F[2] = cf[4] * wj - cf[6] * wR - cf[7] * wI;
  F[3] = cf[5] * wj - cf[7] * wR + cf[6] * wI;
  F[4] = wi;
  F[5] = wj;
  F[6] = x[2];
  F[7] = x[3];
}

/* eq. exp-branch plus the line-limit penalty (rho_l/2) max(0, p^2 + q^2 - smax^2)^2 for
 * both directions, with analytic gradient and Hessian */
static int eval_branch(const double* P, const double* x, double* f, double* g, double* H,
                       ot_counters* c, double* fscale) {
  const double* cf = P;
  const double* lam = P + 8;
  const double* tg = P + 16;
  const double* rh = P + 24;
  double smax2 = P[32], rhol = P[33];
  double vi = x[0], vj = x[1];
  double sn = sin(x[2] - x[3]);
  double cs = cos(x[2] - x[3]);
  if (c) c->sincos++;
  double wR = vi * vj * cs, wI = vi * vj * sn;
  double F[8];
  branch_pairs(cf, x, cs, sn, F);
  /* magnitudes of the terms of each pair quantity, for the rounding scale of f */
  double M[8];
  {
    const double wi = vi * vi, wj = vj * vj;
    M[0] = fabs(cf[0] * wi) + fabs(cf[2] * wR) + fabs(cf[3] * wI);
    M[1] = fabs(cf[1] * wi) + fabs(cf[3] * wR) + fabs(cf[2] * wI);
    M[2] = fabs(cf[4] * wj) + fabs(cf[6] * wR) + fabs(cf[7] * wI);
    M[3] = fabs(cf[5] * wj) + fabs(cf[7] * wR) + fabs(cf[6] * wI);
    M[4] = wi;
    M[5] = wj;
    M[6] = fabs(x[2]);
    M[7] = fabs(x[3]);
  }
  double val = 0.0, mag = 0.0;
  for (int k = 0; k < 8; k++) {
    double r = F[k] - tg[k];
    val += lam[k] * r + 0.5 * rh[k] * r * r;
    mag += fabs(lam[k] * r) + 0.5 * rh[k] * r * r + (fabs(lam[k]) + rh[k] * fabs(r)) * M[k];
  }
  for (int dir = 0; dir < 2; dir++) {
    double p = F[2 * dir], q = F[2 * dir + 1];
    double m = p * p + q * q - smax2;
    if (m > 0.0) {
      val += 0.5 * rhol * m * m;
      mag += 0.5 * rhol * m * m + rhol * m * (p * p + q * q + smax2);
    }
  }
  *f = val;
  if (fscale) *fscale = mag;
  if (c) c->flops += 30.0 + 8 * 5.0 + 2 * 9.0;
  if (!g && !H) return 0;

  /* first and second derivatives of w_i, w_j, wR, wI in the order (v_i, v_j, th_i, th_j) */
  double dwi[4] = {2.0 * vi, 0.0, 0.0, 0.0};
  double dwj[4] = {0.0, 2.0 * vj, 0.0, 0.0};
  double dwR[4] = {vj * cs, vi * cs, -wI, wI};
  double dwI[4] = {vj * sn, vi * sn, wR, -wR};
  double Hwi[16] = {0}, Hwj[16] = {0}, HwR[16] = {0}, HwI[16] = {0};
  Hwi[0] = 2.0;
  Hwj[5] = 2.0;
  /* wR = vi vj cos(ti - tj) */
  HwR[0 * 4 + 1] = cs;
  HwR[0 * 4 + 2] = -vj * sn;
  HwR[0 * 4 + 3] = vj * sn;
  HwR[1 * 4 + 2] = -vi * sn;
  HwR[1 * 4 + 3] = vi * sn;
  HwR[2 * 4 + 2] = -wR;
  HwR[2 * 4 + 3] = wR;
  HwR[3 * 4 + 3] = -wR;
  /* wI = vi vj sin(ti - tj) */
  HwI[0 * 4 + 1] = sn;
  HwI[0 * 4 + 2] = vj * cs;
  HwI[0 * 4 + 3] = -vj * cs;
  HwI[1 * 4 + 2] = vi * cs;
  HwI[1 * 4 + 3] = -vi * cs;
  HwI[2 * 4 + 2] = -wI;
  HwI[2 * 4 + 3] = wI;
  HwI[3 * 4 + 3] = -wI;
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < a; b++) {
      HwR[a * 4 + b] = HwR[b * 4 + a];
      HwI[a * 4 + b] = HwI[b * 4 + a];
    }
  /* each pair quantity F_k = ci*w_i + cj*w_j + cR*wR + cI*wI (+ theta for k = 6, 7) */
  double coefs[8][4] = {
      {cf[0], 0.0, -cf[2], cf[3]},  {cf[1], 0.0, -cf[3], -cf[2]}, {0.0, cf[4], -cf[6], -cf[7]},
      {0.0, cf[5], -cf[7], cf[6]},  {1.0, 0.0, 0.0, 0.0},         {0.0, 1.0, 0.0, 0.0},
      {0.0, 0.0, 0.0, 0.0},         {0.0, 0.0, 0.0, 0.0}};
  double dF[8][4], HF[8][16];
  for (int k = 0; k < 8; k++) {
    for (int a = 0; a < 4; a++)
      dF[k][a] = coefs[k][0] * dwi[a] + coefs[k][1] * dwj[a] + coefs[k][2] * dwR[a] +
                 coefs[k][3] * dwI[a];
    for (int e = 0; e < 16; e++)
      HF[k][e] = coefs[k][0] * Hwi[e] + coefs[k][1] * Hwj[e] + coefs[k][2] * HwR[e] +
                 coefs[k][3] * HwI[e];
  }
  dF[6][2] = 1.0;
  dF[7][3] = 1.0;
  double gg[4] = {0, 0, 0, 0}, HH[16];
  for (int e = 0; e < 16; e++) HH[e] = 0.0;
  for (int k = 0; k < 8; k++) {
    double r = F[k] - tg[k];
    double t = lam[k] + rh[k] * r;
    for (int a = 0; a < 4; a++) gg[a] += t * dF[k][a];
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) HH[a * 4 + b] += rh[k] * dF[k][a] * dF[k][b] + t * HF[k][a * 4 + b];
  }
  for (int dir = 0; dir < 2; dir++) {
    int kp = 2 * dir, kq = 2 * dir + 1;
    double p = F[kp], q = F[kq];
    double m = p * p + q * q - smax2;
    if (!(m > 0.0)) continue;
    double dm[4];
    for (int a = 0; a < 4; a++) dm[a] = 2.0 * p * dF[kp][a] + 2.0 * q * dF[kq][a];
    for (int a = 0; a < 4; a++) gg[a] += rhol * m * dm[a];
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) {
        double d2m = 2.0 * dF[kp][a] * dF[kp][b] + 2.0 * p * HF[kp][a * 4 + b] +
                     2.0 * dF[kq][a] * dF[kq][b] + 2.0 * q * HF[kq][a * 4 + b];
        HH[a * 4 + b] += rhol * (dm[a] * dm[b] + m * d2m);
      }
  }
  if (g)
    for (int a = 0; a < 4; a++) g[a] = gg[a];
  if (H)
    for (int e = 0; e < 16; e++) H[e] = HH[e];
  if (c) c->flops += 420.0;
  return 0;
}

/* Generator of the multi-period ADMM over its n periods (readings R16-R17), record
 * [c2 c1 rho rho_r R 0 0 0 | lambda[n] | target[n]]:
 *   f = sum_t c2 p_t^2 + c1 p_t + lambda_t (p_t - target_t) + rho/2 (p_t - target_t)^2
 *       + rho_r/2 sum_{t >= 1} max(0, |p_t - p_{t-1}| - R)^2
 * The ramp term's second derivative is rho_r on |d| > R and 0 below (as for the line
 * limit of the branch objective). */
static int eval_genramp(int n, const double* P, const double* x, double* f, double* g,
                        double* H, ot_counters* c, double* fscale) {
  double c2 = P[0], c1 = P[1], rho = P[2], rr = P[3], R = P[4];
  const double* lam = P + 8;
  const double* tgt = P + 8 + n;
  double val = 0.0, mag = 0.0;
  if (g)
    for (int t = 0; t < n; t++) g[t] = 0.0;
  if (H)
    for (int e = 0; e < n * n; e++) H[e] = 0.0;
  for (int t = 0; t < n; t++) {
    double p = x[t], r = p - tgt[t];
    val += c2 * p * p + c1 * p + lam[t] * r + 0.5 * rho * r * r;
    mag += fabs(c2) * p * p + fabs(c1 * p) + fabs(lam[t] * r) + 0.5 * rho * r * r +
           (fabs(lam[t]) + rho * fabs(r)) * (fabs(p) + fabs(tgt[t]));
    if (g) g[t] += 2.0 * c2 * p + c1 + lam[t] + rho * r;
    if (H) H[t * n + t] += 2.0 * c2 + rho;
  }
  for (int t = 1; t < n; t++) {
    double d = x[t] - x[t - 1];
    double e = fabs(d) - R;
    if (e > 0.0) {
      double s = d > 0.0 ? 1.0 : -1.0;
      val += 0.5 * rr * e * e;
      mag += 0.5 * rr * e * e + rr * e * (fabs(x[t]) + fabs(x[t - 1]) + R);
      if (g) {
        g[t] += rr * e * s;
        g[t - 1] -= rr * e * s;
      }
      if (H) {
        H[t * n + t] += rr;
        H[(t - 1) * n + (t - 1)] += rr;
        H[t * n + (t - 1)] -= rr;
        H[(t - 1) * n + t] -= rr;
      }
    }
  }
  *f = val;
  if (fscale) *fscale = mag;
  if (c) c->flops += 14.0 * n + 10.0 * (n - 1);
  return 0;
}

/* f, gradient, Hessian; *fscale receives the sum of the magnitudes of the terms f is
 * assembled from (including, for the branch, the first-order effect of the terms of
 * each flow), the scale of the rounding error of the computed f */
static int eval_c(int kind, int n, const double* P, const double* x, double* f, double* g,
                  double* H, ot_counters* c, double* fscale) {
  switch (kind) {
    case OT_OBJ_DENSE: return eval_dense(n, P, x, f, g, H, c, fscale);
    case OT_OBJ_HS45: return eval_hs45(n, x, f, g, H, c, fscale);
    case OT_OBJ_BRANCH:
      if (n != 4) return -1;
      return eval_branch(P, x, f, g, H, c, fscale);
    case OT_OBJ_GENRAMP: return eval_genramp(n, P, x, f, g, H, c, fscale);
    default: return -1;
  }
}

int ot_eval(int kind, int n, const double* params, const double* x, double* f, double* g,
            double* H) {
  return eval_c(kind, n, params, x, f, g, H, NULL, NULL);
}

double ot_fscale(int kind, int n, const double* params, const double* x) {
  double f, S = NAN;
  if (eval_c(kind, n, params, x, &f, NULL, NULL, NULL, &S) != 0) return NAN;
  return S;
}

/* length of a Cauchy trial s for its trust-region test: ||s||_2, or (cauchy_norm 1) the
 * norm of the model's Hessian, (s'Hs)^(1/2), where s'Hs > 0; Hs = H s is given */
static double cauchy_len(int n, const double* s, const double* Hs, const ot_opts* o,
                         ot_counters* c) {
  if (o->cauchy_norm == 1) {
    double h = dot(n, s, Hs, NULL);  /* s'Hs: the model value's product, already counted */
    if (c) c->flops += 1.0;
    if (h > 0.0) return sqrt(h);
  }
  return nrm2(n, s, c);
}

static int all_finite(int n, const double* v) {
  for (int i = 0; i < n; i++)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/* ----------------------------------------------------------------- Algorithm 1 (TRON) */

int ot_tron_solve(int kind, int n, const double* params, const double* l, const double* u,
                  double* x, double* delta_io, const ot_opts* o, double* f_out, double* pg_out,
                  int32_t* iters_out, ot_counters* cnt) {
  ot_counters local;
  memset(&local, 0, sizeof(local));
  ot_counters* c = cnt ? cnt : &local;
  size_t nn = (size_t)n * n;
  double* W = (double*)malloc(sizeof(double) * (3 * nn + 16 * (size_t)n + 16));
  int* F = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  double* H = W;
  double* A = H + nn;
  double* L = A + nn;
  double* g = L + nn;
  double* y = g + n;
  double* s = y + n;
  double* r = s + n;
  double* w = r + n;
  double* Hd = w + n;
  double* d = Hd + n;
  double* yt = d + n;
  double* rF = yt + n;
  double* bh = rF + n;
  double* sh = bh + n;
  double* mg = sh + n;
  int status = OT_MAX_ITER;
  int k = 0;
  double f = NAN;
  double delta = *delta_io;

  for (int i = 0; i < n; i++) {
    if (!(l[i] <= u[i])) {
      status = OT_BAD_BOUNDS;
      goto out_nopg;
    }
  }
  /* Alg. 1 REQUIRE: x0 in [l,u]; project it */
  for (int i = 0; i < n; i++) x[i] = proj1(x[i], l[i], u[i]);
  double fs = 0.0;
  if (eval_c(kind, n, params, x, &f, g, H, c, &fs) != 0) {
    status = OT_NONFINITE;
    goto out_nopg;
  }
  c->f_evals++;
  c->gh_evals++;
  if (!isfinite(f) || !all_finite(n, g) || !all_finite((int)nn, H)) {
    status = OT_NONFINITE;
    goto out;
  }
  if (!(delta > 0.0)) {
    /* automatic initial radius: ||P[x - g] - x||, or 1 when that is zero */
    for (int i = 0; i < n; i++) mg[i] = -g[i];
    gpstep(n, x, 1.0, mg, l, u, s, c);
    delta = nrm2(n, s, c);
    if (delta == 0.0) delta = 1.0;
  }
  double alpha_c = 1.0;

  for (;;) {
    /* Algorithm 1: convergence at x^k (Sec. 5.1) */
    double pg = ot_pgnorm(n, x, g, l, u);
    if (pg <= o->gtol) {
      status = OT_CONVERGED;
      break;
    }
    if (k >= o->max_outer) {
      status = OT_MAX_ITER;
      break;
    }
    k++;
    c->outer++;

    /* ---- Algorithm 1, Cauchy point: x_c = P[x - alpha g] with a sufficient-decrease
     * search on q(s) = g's + 1/2 s'Hs: q(s) <= mu0 g's and ||s|| <= mu1 delta. */
    for (int i = 0; i < n; i++) mg[i] = -g[i];
    double alpha = alpha_c;
    int ok;
    {
      gpstep(n, x, alpha, mg, l, u, s, c);
      gemv(n, H, n, s, Hd, c);
      double gts = dot(n, g, s, c);
      double q = gts + 0.5 * dot(n, s, Hd, c);
      ok = (q <= o->mu0 * gts) && (cauchy_len(n, s, Hd, o, c) <= o->mu1 * delta);
      c->cauchy_trials++;
    }
    if (ok) {
      int nb;
      double bmin, bmax;
      ot_breakpt(n, x, mg, l, u, &nb, &bmin, &bmax);
      c->flops += 2.0 * n;
      for (int t = 0; t < o->max_trials; t++) {
        if (!(alpha < bmax)) break;
        double a2 = alpha * o->extrapf;
        gpstep(n, x, a2, mg, l, u, s, c);
        gemv(n, H, n, s, Hd, c);
        double gts = dot(n, g, s, c);
        double q = gts + 0.5 * dot(n, s, Hd, c);
        c->cauchy_trials++;
        if (!((q <= o->mu0 * gts) && (cauchy_len(n, s, Hd, o, c) <= o->mu1 * delta))) break;
        alpha = a2;
      }
    } else {
      for (int t = 0; t < o->max_trials; t++) {
        alpha = alpha * o->interpf;
        gpstep(n, x, alpha, mg, l, u, s, c);
        gemv(n, H, n, s, Hd, c);
        double gts = dot(n, g, s, c);
        double q = gts + 0.5 * dot(n, s, Hd, c);
        c->cauchy_trials++;
        if ((q <= o->mu0 * gts) && (cauchy_len(n, s, Hd, o, c) <= o->mu1 * delta)) break;
      }
    }
    alpha_c = alpha;
    for (int i = 0; i < n; i++) y[i] = proj1(x[i] - alpha * g[i], l[i], u[i]);
    c->flops += 2.0 * n;
    /* length of the step in the norms of the trust regions that bound its pieces: the
     * Cauchy step in ||.||_2 here, each subspace pass's search step beta*w below in the
     * PCG's norm (used by the radius update when tr_norm == 0) */
    double nu = 0.0;
    if (o->tr_norm == 0) {
      for (int i = 0; i < n; i++) d[i] = y[i] - x[i];
      if (o->cauchy_norm == 1) gemv(n, H, n, d, yt, NULL);  /* H s of the accepted trial */
      nu = cauchy_len(n, d, yt, o, c);
    }

    /* ---- Algorithm 1's subspace step, repeated on the current face: free set, shifted complete
     * Cholesky, Steihaug PCG, back transform, projected search.  r is the model gradient
     * g + H (y - x) at the current point y. */
    for (int i = 0; i < n; i++) s[i] = y[i] - x[i];
    gemv(n, H, n, s, Hd, c);
    for (int i = 0; i < n; i++) r[i] = g[i] + Hd[i];
    c->flops += 2.0 * n;
    double rF0 = 0.0;
    for (int pass = 0; pass < n; pass++) {
      int m = 0;
      for (int i = 0; i < n; i++)
        if (l[i] < y[i] && y[i] < u[i]) F[m++] = i;
      if (m == 0) break;
      c->subspace_passes++;
      for (int a = 0; a < m; a++) rF[a] = r[F[a]];
      if (pass == 0) rF0 = nrm2(m, rF, c);
      /* A = H_FF (Sec. 5.3 gather) */
      for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++) A[(size_t)a * m + b] = H[(size_t)F[a] * n + F[b]];
      double shift;
      if (chol_shifted_c(m, A, L, o->shift_frac, o->max_shift, &shift, c) != 0) {
        status = OT_CHOL_FAIL;
        goto out;
      }
      /* bhat = L^-1 r_F */
      for (int a = 0; a < m; a++) bh[a] = rF[a];
      trsv_lower(m, L, bh, c);
      int cgit;
      /* Algorithm 1, PCG and back transform: sh receives w_F = L^-T s */
      double trlen;
      int info = steihaug_c(m, A, L, bh, delta, o->cg_rtol, o->tr_norm == 1 ? 1 : 0, sh, &cgit, &trlen, c);
      for (int i = 0; i < n; i++) w[i] = 0.0;
      for (int a = 0; a < m; a++) w[F[a]] = sh[a];
      /* Algorithm 1, projected search: y+ = P[y + beta w], sufficient decrease of the
       * model: r'd + 1/2 d'Hd <= mu0 r'd with d = y+ - y, beta halved on failure */
      double beta = 1.0;
      int found = 0;
      for (int t = 0; t < o->max_trials; t++) {
        c->proj_trials++;
        gpstep(n, y, beta, w, l, u, d, c);
        for (int i = 0; i < n; i++) yt[i] = proj1(y[i] + beta * w[i], l[i], u[i]);
        gemv(n, H, n, d, Hd, c);
        double rtd = dot(n, r, d, c);
        double dHd = dot(n, d, Hd, c);
        c->flops += 3.0;
        if (rtd + 0.5 * dHd <= o->mu0 * rtd) {
          found = 1;
          break;
        }
        beta = beta * o->proj_shrink;
      }
      if (!found) break;
      if (beta * trlen > nu) nu = beta * trlen;
      int newly_active = 0;
      for (int a = 0; a < m; a++) {
        int i = F[a];
        if (!(l[i] < yt[i] && yt[i] < u[i])) newly_active = 1;
      }
      for (int i = 0; i < n; i++) {
        y[i] = yt[i];
        r[i] = r[i] + Hd[i];
      }
      c->flops += n;
      for (int a = 0; a < m; a++) rF[a] = r[F[a]];
      double rFn = nrm2(m, rF, c);
      if (info == 2 || info == 3 || newly_active || rFn <= o->cg_rtol * rF0) break;
    }

    /* ---- acceptance and radius update on rho = (f(x) - f(y)) / (-q(y - x)) */
    for (int i = 0; i < n; i++) s[i] = y[i] - x[i];
    gemv(n, H, n, s, Hd, c);
    double qs = dot(n, g, s, c) + 0.5 * dot(n, s, Hd, c);
    double fy, fsy = 0.0;
    eval_c(kind, n, params, y, &fy, NULL, NULL, c, &fsy);
    c->f_evals++;
    /* rho = ared / pred, both shifted by the rounding level of f (Conn, Gould and
     * Toint, Trust-Region Methods, Sec. 17.4.2) so that reductions below the
     * precision of f do not decide the step; the level is taken from the magnitude
     * of the terms f is assembled from, not from |f|, which cancellation can make
     * much smaller */
    double pred = -qs;
    double ared = f - fy;
    double fl = o->ared_guard * (fs > 1.0 ? fs : 1.0);
    double rho = (pred > 0.0 && isfinite(fy)) ? (ared + fl) / (pred + fl) : -INFINITY;
    double snorm = o->tr_norm == 0 ? nu : nrm2(n, s, c);
    c->flops += 5.0 + n;
    if (rho > o->eta0) {
      for (int i = 0; i < n; i++) x[i] = y[i];
      f = fy;
      fs = fsy;
      eval_c(kind, n, params, x, &fy, g, H, c, NULL);
      c->gh_evals++;
      c->accepted++;
      if (!all_finite(n, g) || !all_finite((int)nn, H)) {
        status = OT_NONFINITE;
        break;
      }
    }
    if (rho < o->eta1) {
      delta = o->sigma1 * (snorm < delta ? snorm : delta);
    } else if (rho > o->eta2 && snorm >= 0.99 * delta) {
      delta = o->sigma3 * delta;
      if (delta > o->delta_max) delta = o->delta_max;
    }
    if (delta < o->delta_min_rel * (1.0 + nrm2(n, x, c))) {
      status = OT_TR_TOO_SMALL;
      break;
    }
  }
out:
  if (pg_out) *pg_out = isfinite(f) ? ot_pgnorm(n, x, g, l, u) : NAN;
  goto done;
out_nopg:
  if (pg_out) *pg_out = NAN;
done:
  if (f_out) *f_out = f;
  if (iters_out) *iters_out = k;
  *delta_io = delta;
  free(W);
  free(F);
  return status;
}

/* ------------------------------------------------------------------ batch, threaded */

typedef struct batch_job {
  int kind;
  const int32_t* n;
  const int64_t* poff;
  const int64_t* voff;
  const double *params, *l, *u;
  double *x, *delta, *f, *pg;
  int32_t *iters, *status;
  const ot_opts* o;
  int64_t begin, end;
  ot_counters cnt;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* j = (batch_job*)arg;
  memset(&j->cnt, 0, sizeof(j->cnt));
  for (int64_t p = j->begin; p < j->end; p++) {
    int64_t vo = j->voff[p];
    j->status[p] = ot_tron_solve(j->kind, j->n[p], j->params + j->poff[p], j->l + vo, j->u + vo,
                                 j->x + vo, j->delta + p, j->o, j->f + p, j->pg + p,
                                 j->iters + p, &j->cnt);
  }
  return NULL;
}

static void add_counters(ot_counters* a, const ot_counters* b) {
  a->outer += b->outer;
  a->accepted += b->accepted;
  a->f_evals += b->f_evals;
  a->gh_evals += b->gh_evals;
  a->cauchy_trials += b->cauchy_trials;
  a->proj_trials += b->proj_trials;
  a->cg_iters += b->cg_iters;
  a->chol_calls += b->chol_calls;
  a->subspace_passes += b->subspace_passes;
  a->sincos += b->sincos;
  a->flops += b->flops;
}

void ot_tron_batch(int kind, int64_t nprob, const int32_t* n, const int64_t* poff,
                   const int64_t* voff, const double* params, const double* l, const double* u,
                   double* x, double* delta, const ot_opts* o, double* f, double* pg,
                   int32_t* iters, int32_t* status, int nthreads, ot_counters* total) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > nprob) nthreads = (int)(nprob > 0 ? nprob : 1);
  batch_job* jobs = (batch_job*)calloc((size_t)nthreads, sizeof(batch_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  int64_t chunk = (nprob + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; t++) {
    batch_job* j = &jobs[t];
    j->kind = kind;
    j->n = n;
    j->poff = poff;
    j->voff = voff;
    j->params = params;
    j->l = l;
    j->u = u;
    j->x = x;
    j->delta = delta;
    j->f = f;
    j->pg = pg;
    j->iters = iters;
    j->status = status;
    j->o = o;
    j->begin = t * chunk < nprob ? t * chunk : nprob;
    j->end = (t + 1) * chunk < nprob ? (t + 1) * chunk : nprob;
  }
  if (nthreads == 1) {
    batch_worker(&jobs[0]);
  } else {
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  }
  if (total)
    for (int t = 0; t < nthreads; t++) add_counters(total, &jobs[t].cnt);
  free(jobs);
  free(th);
}

/* --------------------------------------------------------------- component ADMM (6.1) */

void ot_admm_branch_record(const ot_net* net, const ot_state* st, int k, double* rec) {
  int i = net->br_from[k], j = net->br_to[k];
  for (int a = 0; a < 8; a++) rec[a] = net->br_coef[8 * (size_t)k + a];
  for (int a = 0; a < 8; a++) rec[8 + a] = st->br_lam[8 * (size_t)k + a];
  for (int a = 0; a < 4; a++) rec[16 + a] = st->br_tilde[4 * (size_t)k + a];
  rec[20] = st->bus_w[i];
  rec[21] = st->bus_w[j];
  rec[22] = st->bus_th[i];
  rec[23] = st->bus_th[j];
  for (int a = 0; a < 8; a++) rec[24 + a] = net->rho;
  rec[32] = net->br_smax2[k];
  rec[33] = net->rho_line;
  rec[34] = 0.0;
  rec[35] = 0.0;
}

static void branch_values_at(const double* cf, const double* x, double* val) {
  double sn = sin(x[2] - x[3]);
  double cs = cos(x[2] - x[3]);
  branch_pairs(cf, x, cs, sn, val);
}

void ot_admm_init(const ot_net* net, ot_state* st) {
  for (int k = 0; k < net->nbranch; k++) {
    double* x = st->br_x + 4 * (size_t)k;
    x[0] = 1.0;
    x[1] = 1.0;
    x[2] = 0.0;
    x[3] = 0.0;
    st->br_delta[k] = 1.0;
    double* val = st->br_val + 8 * (size_t)k;
    branch_values_at(net->br_coef + 8 * (size_t)k, x, val);
    for (int a = 0; a < 8; a++) st->br_lam[8 * (size_t)k + a] = 0.0;
    for (int a = 0; a < 4; a++) st->br_tilde[4 * (size_t)k + a] = val[a];
  }
  for (int b = 0; b < net->nbus; b++) {
    st->bus_w[b] = 1.0;
    st->bus_th[b] = 0.0;
  }
  for (int g = 0; g < net->ngen; g++) {
    st->gen_pq[2 * g] = 0.5 * (net->gen_pmin[g] + net->gen_pmax[g]);
    st->gen_pq[2 * g + 1] = 0.5 * (net->gen_qmin[g] + net->gen_qmax[g]);
    st->gen_lam[2 * g] = 0.0;
    st->gen_lam[2 * g + 1] = 0.0;
    st->gen_tilde[2 * g] = st->gen_pq[2 * g];
    st->gen_tilde[2 * g + 1] = st->gen_pq[2 * g + 1];
  }
}

/* value of the bus-side copy of pair a of branch k */
static double pair_tilde(const ot_net* net, const ot_state* st, int k, int a) {
  switch (a) {
    case 4: return st->bus_w[net->br_from[k]];
    case 5: return st->bus_w[net->br_to[k]];
    case 6: return st->bus_th[net->br_from[k]];
    case 7: return st->bus_th[net->br_to[k]];
    default: return st->br_tilde[4 * (size_t)k + a];
  }
}

/* incidence lists and branch-solve buffers of one network (ADMM workspace) */
typedef struct admm_ws {
  int *ep, *gp, *el, *gl;
  int32_t* n4;
  int64_t *poff, *voff;
  double *recs, *bl, *bu, *bf, *bpg, *tprev;
  int32_t *bit, *bst;
} admm_ws;

static void admm_ws_init(const ot_net* net, admm_ws* w) {
  int nb = net->nbus, nl = net->nbranch, ng = net->ngen;
  /* bus incidence, ends and generators listed in increasing id (end id = 2 k + side) */
  w->ep = (int*)calloc((size_t)nb + 1, sizeof(int));
  w->gp = (int*)calloc((size_t)nb + 1, sizeof(int));
  w->el = (int*)malloc(sizeof(int) * (size_t)(2 * nl + 1));
  w->gl = (int*)malloc(sizeof(int) * (size_t)(ng + 1));
  int *ep = w->ep, *gp = w->gp, *el = w->el, *gl = w->gl;
  for (int k = 0; k < nl; k++) {
    ep[net->br_from[k] + 1]++;
    ep[net->br_to[k] + 1]++;
  }
  for (int g = 0; g < ng; g++) gp[net->gen_bus[g] + 1]++;
  for (int b = 0; b < nb; b++) {
    ep[b + 1] += ep[b];
    gp[b + 1] += gp[b];
  }
  {
    int* fill = (int*)calloc((size_t)nb + 1, sizeof(int));
    for (int e = 0; e < 2 * nl; e++) {
      int k = e / 2;
      int bus = (e % 2 == 0) ? net->br_from[k] : net->br_to[k];
      el[ep[bus] + fill[bus]++] = e;
    }
    memset(fill, 0, sizeof(int) * ((size_t)nb + 1));
    for (int g = 0; g < ng; g++) {
      int bus = net->gen_bus[g];
      gl[gp[bus] + fill[bus]++] = g;
    }
    free(fill);
  }
  w->n4 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl + 1));
  w->poff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nl + 1));
  w->voff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nl + 1));
  w->recs = (double*)malloc(sizeof(double) * 36 * (size_t)(nl + 1));
  w->bl = (double*)malloc(sizeof(double) * 4 * (size_t)(nl + 1));
  w->bu = (double*)malloc(sizeof(double) * 4 * (size_t)(nl + 1));
  w->bf = (double*)malloc(sizeof(double) * (size_t)(nl + 1));
  w->bpg = (double*)malloc(sizeof(double) * (size_t)(nl + 1));
  w->bit = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl + 1));
  w->bst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl + 1));
  w->tprev = (double*)malloc(sizeof(double) * (size_t)(8 * nl + 2 * ng + 1));
  const double twopi = 6.283185307179586476925286766559;
  for (int k = 0; k < nl; k++) {
    w->n4[k] = 4;
    w->poff[k] = 36 * (int64_t)k;
    w->voff[k] = 4 * (int64_t)k;
    w->bl[4 * k + 0] = net->vmin;
    w->bl[4 * k + 1] = net->vmin;
    w->bl[4 * k + 2] = -twopi;
    w->bl[4 * k + 3] = -twopi;
    w->bu[4 * k + 0] = net->vmax;
    w->bu[4 * k + 1] = net->vmax;
    w->bu[4 * k + 2] = twopi;
    w->bu[4 * k + 3] = twopi;
  }
}

static void admm_ws_free(admm_ws* w) {
  free(w->ep);
  free(w->gp);
  free(w->el);
  free(w->gl);
  free(w->n4);
  free(w->poff);
  free(w->voff);
  free(w->recs);
  free(w->bl);
  free(w->bu);
  free(w->bf);
  free(w->bpg);
  free(w->bit);
  free(w->bst);
  free(w->tprev);
}

/* closed-form generator update of generator g: minimiser of the box-clipped scalar
 * quadratics; only q when active_power is 0 (the multi-period update sets p) */
static void gen_update_one(const ot_net* net, ot_state* st, int g, int active_power) {
  double rho = net->rho;
  double pt = st->gen_tilde[2 * g], qt = st->gen_tilde[2 * g + 1];
  double lp = st->gen_lam[2 * g], lq = st->gen_lam[2 * g + 1];
  double p = (rho * pt - lp - net->gen_c1[g]) / (2.0 * net->gen_c2[g] + rho);
  double q = qt - lq / rho;
  if (active_power) st->gen_pq[2 * g] = proj1(p, net->gen_pmin[g], net->gen_pmax[g]);
  st->gen_pq[2 * g + 1] = proj1(q, net->gen_qmin[g], net->gen_qmax[g]);
}

static void admm_gen_update(const ot_net* net, ot_state* st, int active_power) {
  for (int g = 0; g < net->ngen; g++) gen_update_one(net, st, g, active_power);
}

/* bus update of bus b: minimise sum rho/2 (xt - a)^2 with a = x + lambda/rho subject to
 * the bus balance equations (eqs. PowerBalanceReal/Reactive); x = a - D^-1 A' mu with
 * (A D^-1 A') mu = A a - (p_d, q_d); writes the bus-side copies of its generators and
 * incident branch ends and its w, theta */
static void bus_update_one(const ot_net* net, ot_state* st, const admm_ws* w, int b) {
  double rho = net->rho;
  const int *ep = w->ep, *gp = w->gp, *el = w->el, *gl = w->gl;
  double rhsP = -net->bus_pd[b], rhsQ = -net->bus_qd[b];
  double sinv = 0.0, Dw = 0.0, awn = 0.0, athn = 0.0;
  for (int t = gp[b]; t < gp[b + 1]; t++) {
    int g = gl[t];
    rhsP += st->gen_pq[2 * g] + st->gen_lam[2 * g] / rho;
    rhsQ += st->gen_pq[2 * g + 1] + st->gen_lam[2 * g + 1] / rho;
    sinv += 1.0 / rho;
  }
  for (int t = ep[b]; t < ep[b + 1]; t++) {
    int e = el[t], k = e / 2, side = e % 2;
    const double* val = st->br_val + 8 * (size_t)k;
    const double* lam = st->br_lam + 8 * (size_t)k;
    int kp = side ? 2 : 0, kq = kp + 1, kw = side ? 5 : 4, kt = side ? 7 : 6;
    rhsP -= val[kp] + lam[kp] / rho;
    rhsQ -= val[kq] + lam[kq] / rho;
    sinv += 1.0 / rho;
    Dw += rho;
    awn += rho * (val[kw] + lam[kw] / rho);
    athn += rho * (val[kt] + lam[kt] / rho);
  }
  double gsh = net->bus_gsh[b], bsh = net->bus_bsh[b];
  double aw = Dw > 0.0 ? awn / Dw : st->bus_w[b];
  rhsP -= gsh * aw;
  rhsQ += bsh * aw;
  double M11 = sinv, M22 = sinv, M12 = 0.0;
  if (Dw > 0.0) {
    M11 += gsh * gsh / Dw;
    M22 += bsh * bsh / Dw;
    M12 = -gsh * bsh / Dw;
  }
  double det = M11 * M22 - M12 * M12;
  double mu1 = 0.0, mu2 = 0.0;
  if (det != 0.0) {
    mu1 = (M22 * rhsP - M12 * rhsQ) / det;
    mu2 = (M11 * rhsQ - M12 * rhsP) / det;
  }
  for (int t = gp[b]; t < gp[b + 1]; t++) {
    int g = gl[t];
    st->gen_tilde[2 * g] = st->gen_pq[2 * g] + st->gen_lam[2 * g] / rho - mu1 / rho;
    st->gen_tilde[2 * g + 1] =
        st->gen_pq[2 * g + 1] + st->gen_lam[2 * g + 1] / rho - mu2 / rho;
  }
  for (int t = ep[b]; t < ep[b + 1]; t++) {
    int e = el[t], k = e / 2, side = e % 2;
    const double* val = st->br_val + 8 * (size_t)k;
    const double* lam = st->br_lam + 8 * (size_t)k;
    int kp = side ? 2 : 0, kq = kp + 1;
    st->br_tilde[4 * (size_t)k + kp] = val[kp] + lam[kp] / rho + mu1 / rho;
    st->br_tilde[4 * (size_t)k + kq] = val[kq] + lam[kq] / rho + mu2 / rho;
  }
  if (Dw > 0.0) {
    st->bus_w[b] = aw - (-gsh * mu1 + bsh * mu2) / Dw;
    st->bus_th[b] = athn / Dw;
  }
}

/* multiplier update lambda += rho (x - xt) of one pair, and its squared primal and
 * (unscaled) dual residual terms */
static void pair_update(double* lam, double xv, double xt, double prev, double rho,
                        double* pr2, double* du2) {
  *lam += rho * (xv - xt);
  *pr2 += (xv - xt) * (xv - xt);
  double dd = xt - prev;
  *du2 += dd * dd;
}

/* one ADMM iteration after the generator update: branch updates, bus updates,
 * multipliers; returns the squared primal and (unscaled) dual residual sums */
static void admm_after_gens(const ot_net* net, ot_state* st, const ot_opts* o, int nthreads,
                            admm_ws* w, int64_t* status_counts, ot_counters* total,
                            double* pr2_out, double* du2_out) {
  int nb = net->nbus, nl = net->nbranch, ng = net->ngen;
  double rho = net->rho;
  double* tprev = w->tprev;
  /* branch update: TRON on eq. exp-branch, warm started from the previous x, delta */
  for (int k = 0; k < nl; k++) ot_admm_branch_record(net, st, k, w->recs + 36 * (size_t)k);
  ot_tron_batch(OT_OBJ_BRANCH, nl, w->n4, w->poff, w->voff, w->recs, w->bl, w->bu, st->br_x,
                st->br_delta, o, w->bf, w->bpg, w->bit, w->bst, nthreads, total);
  if (status_counts)
    for (int k = 0; k < nl; k++)
      if (w->bst[k] >= 0 && w->bst[k] < 6) status_counts[w->bst[k]]++;
  for (int k = 0; k < nl; k++)
    branch_values_at(net->br_coef + 8 * (size_t)k, st->br_x + 4 * (size_t)k,
                     st->br_val + 8 * (size_t)k);
  /* remember the bus-side copies for the dual residual */
  for (int g = 0; g < ng; g++) {
    tprev[2 * g] = st->gen_tilde[2 * g];
    tprev[2 * g + 1] = st->gen_tilde[2 * g + 1];
  }
  for (int k = 0; k < nl; k++)
    for (int a = 0; a < 8; a++) tprev[2 * ng + 8 * k + a] = pair_tilde(net, st, k, a);
  /* bus updates, then the multipliers and residuals of every pair */
  for (int b = 0; b < nb; b++) bus_update_one(net, st, w, b);
  double pr2 = 0.0, du2 = 0.0;
  for (int g = 0; g < ng; g++)
    for (int a = 0; a < 2; a++)
      pair_update(&st->gen_lam[2 * g + a], st->gen_pq[2 * g + a], st->gen_tilde[2 * g + a],
                  tprev[2 * g + a], rho, &pr2, &du2);
  for (int k = 0; k < nl; k++)
    for (int a = 0; a < 8; a++)
      pair_update(&st->br_lam[8 * (size_t)k + a], st->br_val[8 * (size_t)k + a],
                  pair_tilde(net, st, k, a), tprev[2 * ng + 8 * k + a], rho, &pr2, &du2);
  *pr2_out = pr2;
  *du2_out = du2;
}

void ot_admm_run(const ot_net* net, ot_state* st, const ot_opts* o, int niters, int nthreads,
                 double* hist_primal, double* hist_dual, int64_t* status_counts,
                 ot_counters* total) {
  admm_ws w;
  admm_ws_init(net, &w);
  for (int it = 0; it < niters; it++) {
    admm_gen_update(net, st, 1);
    double pr2, du2;
    admm_after_gens(net, st, o, nthreads, &w, status_counts, total, &pr2, &du2);
    if (hist_primal) hist_primal[it] = sqrt(pr2);
    if (hist_dual) hist_dual[it] = net->rho * sqrt(du2);
  }
  admm_ws_free(&w);
}

/* ------------------------------------------ the same iteration in phases, on a subset
 * A partitioned run (buses split between ranks, Sec. 6.3) performs the iteration above in
 * three phases, each on the components a rank owns, with exchanges in between:
 *   1. components: generators (closed form) and branches (TRON) of the masks;
 *   2. buses of the mask: the bus QP, then the multipliers and the residual terms of
 *      every pair whose bus-side copy the bus holds (its generators and incident branch
 *      ends).  A pair's multiplier is used only by its own bus and, in the next
 *      iteration, by its component, so updating it right after its bus gives the values
 *      of the undivided iteration; only the order of the residual sums differs. */
void ot_admm_phase_components(const ot_net* net, ot_state* st, const ot_opts* o,
                              int nthreads, const uint8_t* gen_mask,
                              const uint8_t* br_mask, ot_counters* total) {
  for (int g = 0; g < net->ngen; g++)
    if (gen_mask[g]) gen_update_one(net, st, g, 1);
  int nl = net->nbranch, m = 0;
  int* ids = (int*)malloc(sizeof(int) * (size_t)(nl + 1));
  for (int k = 0; k < nl; k++)
    if (br_mask[k]) ids[m++] = k;
  int32_t* n4 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  int64_t* poff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int64_t* voff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
  double* recs = (double*)malloc(sizeof(double) * 36 * (size_t)(m + 1));
  double* bx = (double*)malloc(sizeof(double) * 4 * (size_t)(m + 1));
  double* bl = (double*)malloc(sizeof(double) * 4 * (size_t)(m + 1));
  double* bu = (double*)malloc(sizeof(double) * 4 * (size_t)(m + 1));
  double* bd = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* bf = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* bpg = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  int32_t* bit = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  int32_t* bst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  const double twopi = 6.283185307179586476925286766559;
  for (int t = 0; t < m; t++) {
    int k = ids[t];
    n4[t] = 4;
    poff[t] = 36 * (int64_t)t;
    voff[t] = 4 * (int64_t)t;
    ot_admm_branch_record(net, st, k, recs + 36 * (size_t)t);
    for (int a = 0; a < 4; a++) bx[4 * t + a] = st->br_x[4 * (size_t)k + a];
    bd[t] = st->br_delta[k];
    bl[4 * t + 0] = net->vmin;
    bl[4 * t + 1] = net->vmin;
    bl[4 * t + 2] = -twopi;
    bl[4 * t + 3] = -twopi;
    bu[4 * t + 0] = net->vmax;
    bu[4 * t + 1] = net->vmax;
    bu[4 * t + 2] = twopi;
    bu[4 * t + 3] = twopi;
  }
  if (m > 0)
    ot_tron_batch(OT_OBJ_BRANCH, m, n4, poff, voff, recs, bl, bu, bx, bd, o, bf, bpg, bit,
                  bst, nthreads, total);
  for (int t = 0; t < m; t++) {
    int k = ids[t];
    for (int a = 0; a < 4; a++) st->br_x[4 * (size_t)k + a] = bx[4 * t + a];
    st->br_delta[k] = bd[t];
    branch_values_at(net->br_coef + 8 * (size_t)k, st->br_x + 4 * (size_t)k,
                     st->br_val + 8 * (size_t)k);
  }
  free(ids);
  free(n4);
  free(poff);
  free(voff);
  free(recs);
  free(bx);
  free(bl);
  free(bu);
  free(bd);
  free(bf);
  free(bpg);
  free(bit);
  free(bst);
}

void ot_admm_phase_buses(const ot_net* net, ot_state* st, const uint8_t* bus_mask,
                         double* pr2_out, double* du2_out) {
  admm_ws w;
  admm_ws_init(net, &w);
  double rho = net->rho;
  double pr2 = 0.0, du2 = 0.0;
  for (int b = 0; b < net->nbus; b++) {
    if (!bus_mask[b]) continue;
    /* the bus-side copies before the update (dual residual) */
    double prev_w = st->bus_w[b], prev_th = st->bus_th[b];
    for (int t = w.gp[b]; t < w.gp[b + 1]; t++) {
      int g = w.gl[t];
      w.tprev[2 * g] = st->gen_tilde[2 * g];
      w.tprev[2 * g + 1] = st->gen_tilde[2 * g + 1];
    }
    for (int t = w.ep[b]; t < w.ep[b + 1]; t++) {
      int e = w.el[t], k = e / 2, kp = (e % 2) ? 2 : 0;
      w.tprev[2 * net->ngen + 8 * k + kp] = st->br_tilde[4 * (size_t)k + kp];
      w.tprev[2 * net->ngen + 8 * k + kp + 1] = st->br_tilde[4 * (size_t)k + kp + 1];
    }
    bus_update_one(net, st, &w, b);
    /* multipliers and residual terms of the pairs whose copies this bus holds */
    for (int t = w.gp[b]; t < w.gp[b + 1]; t++) {
      int g = w.gl[t];
      for (int a = 0; a < 2; a++)
        pair_update(&st->gen_lam[2 * g + a], st->gen_pq[2 * g + a], st->gen_tilde[2 * g + a],
                    w.tprev[2 * g + a], rho, &pr2, &du2);
    }
    for (int t = w.ep[b]; t < w.ep[b + 1]; t++) {
      int e = w.el[t], k = e / 2, side = e % 2;
      int kp = side ? 2 : 0;
      int as[4] = {kp, kp + 1, side ? 5 : 4, side ? 7 : 6};
      for (int q = 0; q < 4; q++) {
        int a = as[q];
        double prev = q < 2 ? w.tprev[2 * net->ngen + 8 * k + a] : (q == 2 ? prev_w : prev_th);
        pair_update(&st->br_lam[8 * (size_t)k + a], st->br_val[8 * (size_t)k + a],
                    pair_tilde(net, st, k, a), prev, rho, &pr2, &du2);
      }
    }
  }
  admm_ws_free(&w);
  *pr2_out = pr2;
  *du2_out = du2;
}

/* ------------------------------------------------- multi-period ADMM (Sec. 7, readings)
 * The generator component spans the periods: its T active-power outputs are one NLP
 * (OT_OBJ_GENRAMP) with the ramp penalty, solved by the same TRON; everything else is
 * the single-period iteration, period by period. */
void ot_genramp_record(const ot_mp* mp, int g, double* rec) {
  int T = mp->T;
  const ot_net* n0 = &mp->nets[0];
  rec[0] = n0->gen_c2[g];
  rec[1] = n0->gen_c1[g];
  rec[2] = n0->rho;
  rec[3] = mp->rho_ramp;
  rec[4] = mp->ramp[g];
  rec[5] = 0.0;
  rec[6] = 0.0;
  rec[7] = 0.0;
  for (int t = 0; t < T; t++) {
    rec[8 + t] = mp->states[t].gen_lam[2 * g];
    rec[8 + T + t] = mp->states[t].gen_tilde[2 * g];
  }
}

void ot_admm_mp_init(ot_mp* mp) {
  for (int t = 0; t < mp->T; t++) ot_admm_init(&mp->nets[t], &mp->states[t]);
  for (int g = 0; g < mp->nets[0].ngen; g++) mp->gen_delta[g] = 1.0;
}

void ot_admm_mp_run(ot_mp* mp, const ot_opts* o, int niters, int nthreads,
                    double* hist_primal, double* hist_dual, ot_counters* total) {
  int T = mp->T, ng = mp->nets[0].ngen;
  const ot_net* n0 = &mp->nets[0];
  admm_ws w;
  admm_ws_init(n0, &w);  /* the periods share the topology */
  int rs = 8 + 2 * T;
  int32_t* nT = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ng + 1));
  int64_t* poff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ng + 1));
  int64_t* voff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ng + 1));
  double* recs = (double*)malloc(sizeof(double) * (size_t)rs * (size_t)(ng + 1));
  double* gl = (double*)malloc(sizeof(double) * (size_t)T * (size_t)(ng + 1));
  double* gu = (double*)malloc(sizeof(double) * (size_t)T * (size_t)(ng + 1));
  double* gx = (double*)malloc(sizeof(double) * (size_t)T * (size_t)(ng + 1));
  double* gf = (double*)malloc(sizeof(double) * (size_t)(ng + 1));
  double* gpg = (double*)malloc(sizeof(double) * (size_t)(ng + 1));
  int32_t* git = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ng + 1));
  int32_t* gst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ng + 1));
  for (int g = 0; g < ng; g++) {
    nT[g] = T;
    poff[g] = (int64_t)rs * g;
    voff[g] = (int64_t)T * g;
    for (int t = 0; t < T; t++) {
      gl[(size_t)T * g + t] = n0->gen_pmin[g];
      gu[(size_t)T * g + t] = n0->gen_pmax[g];
    }
  }
  for (int it = 0; it < niters; it++) {
    /* generator update: the T periods' p jointly (warm started), q per period */
    for (int g = 0; g < ng; g++) {
      ot_genramp_record(mp, g, recs + (size_t)rs * g);
      for (int t = 0; t < T; t++) gx[(size_t)T * g + t] = mp->states[t].gen_pq[2 * g];
    }
    ot_tron_batch(OT_OBJ_GENRAMP, ng, nT, poff, voff, recs, gl, gu, gx, mp->gen_delta, o, gf,
                  gpg, git, gst, nthreads, total);
    for (int t = 0; t < T; t++) {
      for (int g = 0; g < ng; g++) mp->states[t].gen_pq[2 * g] = gx[(size_t)T * g + t];
      admm_gen_update(&mp->nets[t], &mp->states[t], 0);
    }
    /* branches and buses, period by period */
    double pr2 = 0.0, du2 = 0.0;
    for (int t = 0; t < T; t++) {
      double p2, d2;
      admm_after_gens(&mp->nets[t], &mp->states[t], o, nthreads, &w, NULL, total, &p2, &d2);
      pr2 += p2;
      du2 += d2;
    }
    if (hist_primal) hist_primal[it] = sqrt(pr2);
    if (hist_dual) hist_dual[it] = n0->rho * sqrt(du2);
  }
  admm_ws_free(&w);
  free(nT);
  free(poff);
  free(voff);
  free(recs);
  free(gl);
  free(gu);
  free(gx);
  free(gf);
  free(gpg);
  free(git);
  free(gst);
}
