/*
 * oracle.h -- declarations of the CPU FP64 oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This header belongs to the oracle and is included by
 * nothing outside oracle/.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load the oracle library.  It shares no code, header,
 * constant or helper with the CUDA product path.
 *
 * The oracle is a plain, slow, step-by-step restatement of the trust-region Newton
 * method of Algorithm 1 (Section 3) with the core operations of Figure 2, the
 * objectives of Section 6.1 (eq. exp-branch with eqs. pij-qji), the dense quartic test
 * family and the hs45 variant of the Section 4.2 footnote, and the component ADMM of
 * Section 6.1.  Constants the paper leaves open are fields of ot_opts; their default
 * values are the readings listed in the design notes.
 */
#ifndef EXATRON_ORACLE_H
#define EXATRON_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* objective kinds (same numbering as the public C-ABI, defined independently) */
enum { OT_OBJ_BRANCH = 1, OT_OBJ_DENSE = 2, OT_OBJ_HS45 = 3, OT_OBJ_GENRAMP = 4 };

/* per-problem status */
enum {
  OT_CONVERGED = 0, OT_MAX_ITER = 1, OT_TR_TOO_SMALL = 2, OT_CHOL_FAIL = 3,
  OT_NONFINITE = 4, OT_BAD_BOUNDS = 5
};

typedef struct ot_opts {
  double gtol;          /* projected-gradient max-norm tolerance (Section 5.1) */
  int32_t max_outer;    /* outer iteration cap */
  int32_t max_trials;   /* cap on Cauchy and projected-search trials */
  double mu0;           /* sufficient-decrease constant */
  double mu1;           /* Cauchy step length bound, ||s|| <= mu1 * delta */
  double interpf;       /* Cauchy interpolation factor */
  double extrapf;       /* Cauchy extrapolation factor */
  double proj_shrink;   /* projected-search step shrink factor */
  double eta0, eta1, eta2;      /* acceptance / radius thresholds */
  double sigma1, sigma3;        /* radius shrink / expand factors */
  double delta_max;             /* radius cap */
  double delta_min_rel;         /* TR_TOO_SMALL threshold relative to 1+||x|| */
  double cg_rtol;               /* CG relative residual tolerance (footnote of Sec. 4.3) */
  double shift_frac;            /* Cholesky shift base, times max |A_ii| */
  int32_t max_shift;            /* Cholesky shift retries */
  int32_t tr_norm;              /* trust-region norm of the PCG step: 0 = the CG iterate s
                                   of the preconditioned system, ||s|| = ||L^T w|| (Algorithm 1),
                                   1 = the step itself, ||w|| */
  double ared_guard;            /* rounding guard of the ratio, times max(1, magnitude of the terms of f) */
  int32_t cauchy_norm;          /* norm of the Cauchy step's trust-region test: 0 = ||s||_2,
                                   1 = ||s||_H = (s'Hs)^(1/2) where s'Hs > 0, else ||s||_2 */
  int32_t pad1;
} ot_opts;

typedef struct ot_counters {
  int64_t outer;        /* outer iterations (trial steps) */
  int64_t accepted;
  int64_t f_evals;      /* objective values */
  int64_t gh_evals;     /* gradient + Hessian evaluations */
  int64_t cauchy_trials;
  int64_t proj_trials;
  int64_t cg_iters;     /* preconditioned-matrix products */
  int64_t chol_calls;   /* factorization attempts (including shift retries) */
  int64_t subspace_passes;
  int64_t sincos;       /* sin/cos pairs evaluated (not counted as flops) */
  double flops;         /* arithmetic operations: +,-,*,/,sqrt each count 1 */
} ot_counters;

void ot_default_opts(ot_opts* o);

/* One problem.  x: in x0, out x*.  delta: in delta0 (<=0 selects the automatic
 * initial radius), out final radius.  cnt may be NULL. */
int ot_tron_solve(int kind, int n, const double* params, const double* l, const double* u,
                  double* x, double* delta, const ot_opts* o, double* f_out, double* pg_out,
                  int32_t* iters_out, ot_counters* cnt);

/* A batch.  Problem p has n[p] variables, parameters at params + poff[p] and vectors at
 * offset voff[p] of l, u, x.  Uses up to nthreads host threads (static split). */
void ot_tron_batch(int kind, int64_t nprob, const int32_t* n, const int64_t* poff,
                   const int64_t* voff, const double* params, const double* l, const double* u,
                   double* x, double* delta, const ot_opts* o, double* f, double* pg,
                   int32_t* iters, int32_t* status, int nthreads, ot_counters* total);

/* objective value, gradient and Hessian (row-major n x n); g or H may be NULL */
int ot_eval(int kind, int n, const double* params, const double* x, double* f, double* g,
            double* H);

/* the rounding scale S of f at x used by the ratio's guard (reading R6): the sum of the
 * magnitudes of the terms f is assembled from */
double ot_fscale(int kind, int n, const double* params, const double* x);

/* core operations exposed for unit tests */
int ot_chol_left(int m, double* A, int lda);           /* in place, lower; 0 = ok */
int ot_chol_shifted(int m, const double* A, double* L, double shift_frac, int max_shift,
                    double* alpha_out);                 /* L (m x m) lower + mirrored upper */
double ot_trqsol(int n, const double* x, const double* p, double delta);
double ot_pgnorm(int n, const double* x, const double* g, const double* l, const double* u);
void ot_breakpt(int n, const double* x, const double* w, const double* l, const double* u,
                int* nbrpt, double* brptmin, double* brptmax);
int ot_steihaug(int m, const double* A, const double* L, const double* bhat, double delta,
                double rtol, int norm, double* w, int* iters,
                double* tr_len);  /* w = L^-T s; tr_len = ||s|| (norm 0) or ||w|| (1) */

/* ---------------------------------------------------------------- ADMM (Sec. 6.1) */
typedef struct ot_net {
  int32_t nbus, nbranch, ngen;
  const int32_t* br_from;     /* [nbranch] */
  const int32_t* br_to;       /* [nbranch] */
  const double* br_coef;      /* [nbranch][8] gc_ij bc_ij g_ij b_ij gc_ji bc_ji g_ji b_ji */
  const double* br_smax2;     /* [nbranch] squared apparent-power limit */
  const int32_t* gen_bus;     /* [ngen] */
  const double* gen_c2;       /* [ngen] */
  const double* gen_c1;       /* [ngen] */
  const double* gen_pmin, *gen_pmax, *gen_qmin, *gen_qmax;  /* [ngen] */
  const double* bus_pd, *bus_qd, *bus_gsh, *bus_bsh;        /* [nbus] */
  double rho;                 /* penalty of every coupling pair */
  double rho_line;            /* line-limit penalty */
  double vmin, vmax;          /* voltage magnitude bounds */
} ot_net;

typedef struct ot_state {
  double* br_x;       /* [nbranch][4] v_i v_j th_i th_j */
  double* br_delta;   /* [nbranch] */
  double* br_lam;     /* [nbranch][8] pairs p_ij q_ij p_ji q_ji w_i w_j th_i th_j */
  double* br_val;     /* [nbranch][8] branch-side values of the pairs */
  double* br_tilde;   /* [nbranch][4] bus-side flow copies p_ij q_ij p_ji q_ji */
  double* bus_w;      /* [nbus] */
  double* bus_th;     /* [nbus] */
  double* gen_pq;     /* [ngen][2] */
  double* gen_lam;    /* [ngen][2] */
  double* gen_tilde;  /* [ngen][2] */
} ot_state;

void ot_admm_init(const ot_net* net, ot_state* st);
/* runs niters iterations; hist_primal/hist_dual [niters] may be NULL */
void ot_admm_run(const ot_net* net, ot_state* st, const ot_opts* o, int niters, int nthreads,
                 double* hist_primal, double* hist_dual, int64_t* status_counts /*[6] or NULL*/,
                 ot_counters* total);
/* build the 36-entry branch record of branch k from the current state */
void ot_admm_branch_record(const ot_net* net, const ot_state* st, int k, double* rec);

/* The same iteration in phases on subsets (for partitioned runs, Sec. 6.3): generators
 * and branches of the masks; then buses of the mask, each followed by the multiplier
 * updates and squared residual terms of the pairs whose bus-side copies it holds
 * (their sums are returned in *pr2_out and, unscaled by rho, *du2_out). */
void ot_admm_phase_components(const ot_net* net, ot_state* st, const ot_opts* o,
                              int nthreads, const uint8_t* gen_mask,
                              const uint8_t* br_mask, ot_counters* total);
void ot_admm_phase_buses(const ot_net* net, ot_state* st, const uint8_t* bus_mask,
                         double* pr2_out, double* du2_out);

/* --------------------------------------- multi-period ADMM (future work of Sec. 7)
 * T periods of one network (nets[t] differ only in their loads); the generator
 * component spans the periods: its T active-power outputs are one NLP of kind
 * OT_OBJ_GENRAMP with the ramp penalty rho_ramp/2 max(0, |p_t - p_{t-1}| - ramp[g])^2,
 * solved by TRON warm started from the previous iteration; everything else is the
 * single-period iteration, period by period.  Residuals combine all periods. */
typedef struct ot_mp {
  int32_t T;
  const ot_net* nets;   /* [T] */
  ot_state* states;     /* [T] */
  const double* ramp;   /* [ngen] ramp limit between consecutive periods */
  double rho_ramp;
  double* gen_delta;    /* [ngen] trust radius carried between iterations */
} ot_mp;

void ot_admm_mp_init(ot_mp* mp);
void ot_admm_mp_run(ot_mp* mp, const ot_opts* o, int niters, int nthreads,
                    double* hist_primal, double* hist_dual, ot_counters* total);
/* the (8 + 2T)-entry record of generator g from the current states */
void ot_genramp_record(const ot_mp* mp, int g, double* rec);

#ifdef __cplusplus
}
#endif
#endif
