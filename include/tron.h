/*
 * tron.h -- C ABI of the GB300 batched trust-region Newton solver (libexatron_gb300.so).
 *
 * Solves many small bound-constrained problems  min f(x)  s.t.  l <= x <= u  (eq. prob,
 * Sec. 1) with the trust-region Newton method of Algorithm 1 (Sec. 3): Cauchy point,
 * free-set identification, a complete Cholesky preconditioner with diagonal shift
 * (Sec. 4.3), Steihaug PCG on the free variables, back transform and projected search,
 * stopping when the projected-gradient max-norm is below gtol (Sec. 5.1).  Every step
 * runs on the GPU (Sec. 3: no host/device traffic during a solve); one launch solves a
 * whole batch, one problem per thread group (Sec. 4.1, Sec. 4.2).
 *
 * Conventions
 *  - Pointers named d_* are DEVICE pointers owned by the caller.  The library owns only
 *    its own workspace, allocated in *_create and released in *_destroy; no call made
 *    after *_create allocates device memory.
 *  - All doubles are IEEE binary64.  Arrays are C-contiguous.
 *  - Calls enqueue work on `stream` (a cudaStream_t, NULL = legacy default stream) and
 *    return without synchronising unless stated otherwise.
 *  - Errors are returned as tron_err_t; tron_last_error() gives a thread-local message.
 *    Nothing throws across this ABI.  A problem that fails numerically is NOT a call
 *    error: its code goes to d_status (tron_status_t).
 *  - A handle may be used from one host thread at a time.
 */
#ifndef EXATRON_GB300_TRON_H
#define EXATRON_GB300_TRON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tron_err {
  TRON_OK = 0,
  TRON_EINVAL = 1,        /* bad argument (null pointer, size, kind, option)          */
  TRON_ENOMEM = 2,        /* workspace allocation failed in *_create                 */
  TRON_ECUDA = 3,         /* a CUDA runtime call failed (message in tron_last_error)  */
  TRON_EUNSUPPORTED = 4   /* valid request this build does not implement (e.g. size)  */
} tron_err_t;

/* Objective families and the packed per-problem parameter record of each.
 *
 * TRON_OBJ_ACOPF_BRANCH (n = 4, x = (v_i, v_j, theta_i, theta_j)): the branch
 *   subproblem of the component ADMM, eq. exp-branch (Sec. 6.1) with the flows of
 *   eqs. pij-qji, w_i = v_i^2, w_j = v_j^2, wR = v_i v_j cos(theta_i - theta_j),
 *   wI = v_i v_j sin(theta_i - theta_j), plus the line-limit penalty
 *   (rho_l / 2) max(0, p^2 + q^2 - smax^2)^2 for both directions.
 *   Record of 36 doubles:
 *     [0:8]   gc_ij bc_ij g_ij b_ij gc_ji bc_ji g_ji b_ji
 *     [8:16]  multipliers of the pairs (p_ij q_ij p_ji q_ji w_i w_j theta_i theta_j)
 *     [16:24] targets (bus-side copies) of the same pairs
 *     [24:32] penalties rho of the same pairs
 *     [32]    smax^2        [33] rho_l        [34:36] unused
 * TRON_OBJ_DENSE_QUARTIC (any n <= 128): f = 1/2 x'Qx + c'x + sum_i d_i x_i^4.
 *   Record of n*n + 2n doubles: Q (row-major, symmetric), c, d.
 * TRON_OBJ_HS45 (n <= 8): the hs45 variant of Sec. 4.2, f = 120 - prod_i x_i.
 *   No record (d_params may be NULL); bounds are the caller's.
 * TRON_OBJ_GEN_RAMP (n <= 32): one generator of the multi-period ADMM (the paper's
 *   future work, Sec. 7) over its n periods,
 *     f = sum_t c2 p_t^2 + c1 p_t + lambda_t (p_t - target_t) + rho/2 (p_t - target_t)^2
 *         + rho_r/2 sum_{t>=1} max(0, |p_t - p_{t-1}| - R)^2.
 *   Record of 8 + 2n doubles: [c2, c1, rho, rho_r, R, 0, 0, 0], lambda[n], target[n].
 */
typedef enum tron_obj {
  TRON_OBJ_ACOPF_BRANCH = 1,
  TRON_OBJ_DENSE_QUARTIC = 2,
  TRON_OBJ_HS45 = 3,
  TRON_OBJ_GEN_RAMP = 4
} tron_obj_t;

/* Per-problem outcome written to d_status. */
typedef enum tron_status {
  TRON_CONVERGED = 0,     /* ||grad_[l,u] f(x)||_inf <= gtol                           */
  TRON_MAX_ITER = 1,      /* max_outer iterations without convergence                  */
  TRON_TR_TOO_SMALL = 2,  /* radius fell below delta_min_rel * (1 + ||x||)             */
  TRON_CHOL_FAIL = 3,     /* no shift of the sequence made H_FF + alpha I factorizable */
  TRON_NONFINITE = 4,     /* f, gradient or Hessian not finite at an accepted point    */
  TRON_BAD_BOUNDS = 5     /* some l_i > u_i (or NaN); x is left as given               */
} tron_status_t;

/* How a batch is scheduled on the GPU. */
typedef enum tron_schedule {
  TRON_SCHED_PLAIN = 0,       /* one launch, one thread group per problem (Sec. 4.1)   */
  TRON_SCHED_PERSISTENT = 1   /* one launch of resident groups that pull problems from
                                 a device work counter until the batch is exhausted    */
} tron_schedule_t;

/* Solver constants.  The paper fixes none of the search and radius constants; the
 * defaults are the readings recorded in the design notes. */
typedef struct tron_options {
  double gtol;            /* 1e-6   projected-gradient max-norm tolerance (Sec. 5.1)     */
  int32_t max_outer;      /* 500    outer iterations                                     */
  int32_t max_trials;     /* 30     trials in each Cauchy and projected search           */
  double mu0;             /* 0.01   sufficient-decrease constant                         */
  double mu1;             /* 1.0    Cauchy step bound ||s|| <= mu1 * delta               */
  double interpf;         /* 0.1    Cauchy interpolation factor                          */
  double extrapf;         /* 10.0   Cauchy extrapolation factor                          */
  double proj_shrink;     /* 0.5    projected-search step factor                         */
  double eta0;            /* 1e-4   accept when rho > eta0                               */
  double eta1;            /* 0.25   shrink when rho < eta1                               */
  double eta2;            /* 0.75   expand when rho > eta2 and the step reached 0.99 delta */
  double sigma1;          /* 0.25   shrink factor, delta = sigma1 * min(||s||, delta)
                                    (||s|| as measured by tr_norm)                       */
  double sigma3;          /* 4.0    expansion factor                                     */
  double delta_max;       /* 1e10   radius cap                                           */
  double delta_min_rel;   /* 1e-12  TR_TOO_SMALL threshold, times (1 + ||x||)            */
  double cg_rtol;         /* 0.1    CG stops at ||residual|| <= cg_rtol * ||bhat||       */
  double shift_frac;      /* 1e-3   Cholesky shift base, times max |A_ii|                */
  int32_t max_shift;      /* 30     shift retries before TRON_CHOL_FAIL                  */
  int32_t group;          /* 0      threads per problem: 0 = library's table, or
                                    1, 2, 4, 8, 16, 32 (must divide the size class); the
                                    table's choice for the branch problems is 4 up to 96
                                    problems per SM sub-partition, 2 beyond            */
  double ared_guard;      /* 1e-13  rounding guard of the reduction ratio,
                                    rho = (ared + e) / (pred + e), e = ared_guard * max(1, S)
                                    with S the sum of the magnitudes of the terms of f */
  int32_t schedule;       /* TRON_SCHED_PLAIN                                            */
  int32_t warps_per_block;/* 0      CTA size in warps (0 = library's choice)             */
  int32_t layout;         /* 0      kernel storage variant: 0 = library's choice, else
                                    1 + bits (bit 0: packed factor, bit 1: Q in global,
                                    bit 2: Q as wrapped diagonals, n <= 32 only)         */
  int32_t cholesky;       /* 0      factorization form: 0 = the library's choice (right-
                                    looking, or the autotuner's per size class), 1 = left-
                                    looking (Sec. 4.3), 2 = right-looking with the trailing
                                    update spread over all lanes (two columns per pass for
                                    one problem per CTA); both factor the same matrix as
                                    Lu D Lu^T and agree to rounding                       */
  int32_t ctas_per_sm;    /* 0      persistent schedule: resident CTAs per SM (0 = as many
                                    as fit); fewer shorten each problem's time and so the
                                    launch's last-wave tail                                */
  int32_t tr_norm;        /* 0      trust-region norm of the PCG step (Algorithm 1):
                                    0 = the CG iterate s of the preconditioned system,
                                    ||s||_2 = ||L^T w||_2 <= delta, as Algorithm 1 states; the
                                    radius update then measures each piece of the step in
                                    the norm that bounded it (the Cauchy step in ||.||_2,
                                    each subspace search step beta w in ||L^T .||_2);
                                    1 = the step itself, ||w||_2 <= delta, with the radius
                                    update on ||x+ - x||_2                                 */
  int32_t cauchy_norm;    /* 0      norm of the Cauchy step's trust-region test: 0 = ||s||_2;
                                    1 = the model Hessian's norm (s'Hs)^(1/2) where s'Hs > 0
                                    (else ||s||_2), the norm in which the PCG's bound
                                    ||L^T w|| is nearly stated, so one radius suits both
                                    steps (with tr_norm 0)                                */
  int32_t split_outer;    /* 0      ADMM branch solves on one lane per problem (the pool's
                                    mapping for many branches per SM sub-partition): K > 0
                                    = the TRON iteration after which a solve that has not
                                    finished continues on four lanes, in a second launch
                                    over the unfinished solves only; <= 0 = never.  The
                                    continuation resumes Algorithm 1 at the same x, radius
                                    and Cauchy step, so it is the same iteration up to
                                    rounding.  Ignored by tron_batch_* and four-lane pools */
  int32_t reserved[2];    /* must be zero                                                */
} tron_options_t;

typedef struct tron_batch tron_batch_t;

/* Fill *opt with the defaults above.  Returns TRON_EINVAL if opt is NULL. */
tron_err_t tron_options_default(tron_options_t* opt);

/* Create a batch handle for nprob problems of one objective family.
 *   n_host:     host array [nprob] of per-problem sizes, or NULL when all problems have
 *               n_uniform variables.  With n_host, records and vectors of consecutive
 *               problems are concatenated (problem p starts after problems 0..p-1).
 *   opt:        NULL selects the defaults; copied into the handle.
 *   stream:     stream for the workspace uploads made here (the call synchronises it).
 * Allocates the handle's device workspace (size tables and work counters); fails with
 * TRON_EUNSUPPORTED for sizes outside the family's range and TRON_ENOMEM when the
 * allocation fails. */
tron_err_t tron_batch_create(tron_batch_t** out, tron_obj_t kind, int64_t nprob,
                             const int32_t* n_host, int32_t n_uniform,
                             const tron_options_t* opt, void* stream);

/* Replace the options of a handle (e.g. the schedule or the group size). */
tron_err_t tron_batch_set_options(tron_batch_t* b, const tron_options_t* opt);

/* Solve the batch.  Device arrays (caller-owned):
 *   d_params  packed records of the objective family (see tron_obj_t)
 *   d_lower, d_upper   bounds, [sum n]
 *   d_x       in: x0 (projected onto [l,u] first), out: final iterate, [sum n]
 *   d_delta   in: initial radius (<= 0 selects ||P[x0 - g0] - x0||, or 1), out: final
 *             radius, [nprob]
 *   d_f, d_pgnorm   out: objective and projected-gradient max-norm at x, [nprob]
 *   d_iters   out: outer iterations taken, [nprob]
 *   d_status  out: tron_status_t, [nprob]
 * Enqueues one launch per size class on `stream` (with the persistent schedule and
 * several classes, on streams forked from it and joined back).  Successive calls take
 * the handle's four sets of work counters and forked streams in turn, so up to four
 * solves of independent arrays may run at once on different streams (the last wave of
 * one overlapping the start of the next); a fifth call reuses the first call's set and
 * must be ordered after it (for example on the same stream). */
tron_err_t tron_batch_solve(tron_batch_t* b, const double* d_params, const double* d_lower,
                            const double* d_upper, double* d_x, double* d_delta,
                            double* d_f, double* d_pgnorm, int32_t* d_iters,
                            int32_t* d_status, void* stream);

/* Solve a batch of mixed sizes without allocating device memory.  (The paper has no
 * counterpart.)  It exists for callers that must not allocate device memory from a
 * library call: hosts whose device memory is all handed to their own pool allocator (a
 * framework's caching allocator or a fixed arena), where a cudaMalloc beside the pool
 * fails or fragments it, and processes run under a device-memory budget that library
 * allocations would break.
 *
 * Same problem layout and device arrays as tron_batch_solve with per-problem sizes
 * n_host (host array [nprob]); opt may be NULL; the persistent schedule is always used.
 * The library keeps the size/offset tables, per-class problem lists and work counters
 * in one fixed device array of about 24 * TRON_NOALLOC_MAX_PROBLEMS bytes (6 MiB)
 * that every GPU loading the library reserves until the process exits; no call
 * allocates device memory.
 *  - nprob > TRON_NOALLOC_MAX_PROBLEMS is rejected with TRON_EINVAL.
 *  - The first call on a device looks up the array's device address once for that
 *    device (cudaGetSymbolAddress) and keeps it; make that first call before any stream
 *    capture begins.  The kept address does not survive cudaDeviceReset of that device.
 *  - The tables are built in host memory and copied in from pageable memory on
 *    `stream`: such copies wait for the work already queued on the stream, so the call
 *    returns only after that work has finished.
 *  - The size classes are launched one after another on `stream` (tron_batch_solve
 *    runs them concurrently on forked streams), so a batch of several classes takes
 *    longer through this entry point.
 *  - Every call uses the same array: the counters are cleared and the tables rewritten
 *    by each call on `stream`, so calls on one stream are ordered, but calls that
 *    overlap on the GPU (other streams, other host threads) race and give wrong
 *    results. */
#define TRON_NOALLOC_MAX_PROBLEMS 262144
tron_err_t tron_solve_mixed_noalloc(tron_obj_t kind, int64_t nprob, const int32_t* n_host,
                                    const tron_options_t* opt, const double* d_params,
                                    const double* d_lower, const double* d_upper, double* d_x,
                                    double* d_delta, double* d_f, double* d_pgnorm,
                                    int32_t* d_iters, int32_t* d_status, void* stream);

/* Autotuner: for every size class of the batch, time each compiled kernel variant
 * (group size, storage layout) with 1, 2, 4 and 8 warps per CTA on the first `sample`
 * problems of the class (plain schedule, inputs read from d_params, d_lower, d_upper,
 * d_x0, d_delta0, which are not modified) and keep the fastest for later solves with
 * options.group == 0.  A setup-time call: it allocates and frees temporary device
 * buffers and synchronises the stream. */
tron_err_t tron_batch_autotune(tron_batch_t* b, const double* d_params, const double* d_lower,
                               const double* d_upper, const double* d_x0,
                               const double* d_delta0, int32_t sample, void* stream);

/* Size classes of the batch and the variant each will run with. layout bits: 1 = packed
 * factor, 2 = Q read from global memory, 4 = Q as wrapped diagonals in shared memory;
 * bits 3-4: the options.cholesky value used. */
int32_t tron_batch_buckets(const tron_batch_t* b);
tron_err_t tron_batch_get_choice(const tron_batch_t* b, int32_t bucket, int32_t* N, int32_t* G,
                                 int32_t* layout, int32_t* warps_per_block, int64_t* count);

/* Number of GPU kernel launches the last tron_batch_solve on this handle enqueued. */
int32_t tron_batch_last_launches(const tron_batch_t* b);

/* ---- Host-buffer path (a batch whose arrays live in host memory).
 * The same solve as tron_batch_solve (Sec. 4.1), with the copies to and from the device
 * made by the library.  The paper's solver works on device arrays only; this path lets
 * a stream of batches keep the GPU busy while the next batch is copied in and the
 * previous one's results are copied out.
 *
 * tron_batch_host_enable: setup-time call that allocates two device buffer sets (each
 * the size of one batch: records, l, u, x, delta, f, pgnorm, iters, status) and three
 * streams (copy in, solve, copy out).  Idempotent.  TRON_ENOMEM when the buffers do not
 * fit.
 *
 * tron_batch_solve_host: enqueues, for the next buffer set in turn, the copy of h_params,
 * h_lower, h_upper, h_x0, h_delta0 (layouts as in tron_batch_solve) to the device, the
 * solve, and the copy of x*, the final radius, f*, ||grad_P f||_inf, the iteration
 * counts and the statuses to h_x, h_delta, h_f, h_pgnorm, h_iters, h_status; returns
 * without waiting.  A set is reused only after its previous results have been copied
 * out, so two calls can be in flight: the inputs of one are copied while the other
 * solves.  The host arrays belong to the caller and must stay valid and unchanged until
 * tron_batch_host_sync returns; the inputs (const) may be shared by calls in flight, and
 * results are copied out in call order, so calls that share output arrays leave the
 * last call's results there.  Copies overlap with compute only from
 * page-locked host memory (pageable memory works, serialised).  The two sets solve on
 * two streams, so one call's solve may overlap the previous one's last wave.  h_params
 * may be NULL for TRON_OBJ_HS45.  TRON_EINVAL without tron_batch_host_enable or for
 * NULL arrays; TRON_ECUDA on a CUDA error.  Counts toward the four solves in flight of
 * tron_batch_solve.
 *
 * tron_batch_host_sync: waits until every call's results are in host memory. */
tron_err_t tron_batch_host_enable(tron_batch_t* b);
tron_err_t tron_batch_solve_host(tron_batch_t* b, const double* h_params, const double* h_lower,
                                 const double* h_upper, const double* h_x0,
                                 const double* h_delta0, double* h_x, double* h_delta,
                                 double* h_f, double* h_pgnorm, int32_t* h_iters,
                                 int32_t* h_status);
tron_err_t tron_batch_host_sync(tron_batch_t* b);

/* Release the handle and its workspace (NULL is ignored).  Synchronises nothing; the
 * caller must not destroy a handle whose solve is still running on the GPU. */
void tron_batch_destroy(tron_batch_t* b);

/* Message of the last error raised on this host thread ("" if none). */
const char* tron_last_error(void);

/* Library version string. */
const char* tron_version(void);

/* Measurement hook (the paper has no counterpart): the cost of one kind of dependent
 * operation.  One CTA of `lanes` threads (1..1024) runs a chain of
 * tron_bench_op_chain() operations, each on the previous result, between two clock64
 * reads; d_cycles[0] (caller-owned device int64) receives the SM cycles of the chain.
 * op: 0 FP64 fma, 1 FP64 add, 2 FP64 max, 3 FP64 compare and select, 4 int64 compare
 * and select, 5 the solver's quotient, 6 IEEE division, 7 the solver's square root,
 * 8 IEEE sqrt, 9 the library's sin, 10 the branch objective's sine series, 11 the
 * hardware reciprocal estimate, 12 a 64-bit shuffle, 13 the library's cos, 14 its sincos,
 * 15 an FP32 fma.  Enqueued on `stream`; TRON_EINVAL
 * for another op, a lane count out of range or a NULL d_cycles. */
tron_err_t tron_bench_op_latency(int32_t op, int32_t lanes, int64_t* d_cycles, void* stream);
/* Length of the chain tron_bench_op_latency times (2,048). */
int32_t tron_bench_op_chain(void);

/* Test hook of the factorization's pivot reciprocal (Sec. 4.3's factorization, computed
 * here square-root free as Lu D Lu^T with one reciprocal per pivot): d_out[i] = the
 * reciprocal of d_a[i] as the factorization forms it -- the hardware estimate refined by
 * one Newton-Raphson step, IEEE division from 2^1022 up.  d_a, d_out: caller-owned
 * device arrays of n doubles (n >= 0; positive normal values are the pivots it is made
 * for).  Enqueued on `stream`; TRON_EINVAL for a null array with n > 0. */
tron_err_t tron_test_pivot_rcp(const double* d_a, double* d_out, int64_t n, void* stream);

/* Test hook of the solver's own arithmetic: op 1, d_out[i] = d_a[i] / d_b[i]; op 2,
 * sqrt(d_a[i]) -- the CG step lengths alpha and beta, trqsol's root and the radius update
 * of Algorithm 1, by refinement of the hardware reciprocal (square-root) estimate, IEEE
 * division (sqrt) outside its range; op 3, sin(d_a[i]), op 4, cos(d_a[i]) -- the branch
 * objective's sine and cosine of theta_i - theta_j (eq. exp-branch), a Taylor series for
 * |x| <= pi/4, the library's sin and cos outside.  Each result is within one ulp of the
 * correctly rounded one.  d_b is read for op 1 only (may be NULL otherwise).  d_a, d_b,
 * d_out: caller-owned device arrays of n doubles (n >= 0).  Enqueued on `stream`;
 * TRON_EINVAL for another op, or a null array with n > 0. */
tron_err_t tron_test_arith(int32_t op, const double* d_a, const double* d_b, double* d_out,
                           int64_t n, void* stream);

/* Measurement hook (the paper has no counterpart): FP64 fused multiply-add throughput.
 * Launches `blocks` CTAs of `threads` threads; every thread runs 8 independent chains of
 * `iters` dependent FMAs and writes its result to d_out[thread] (caller-owned device
 * array of blocks * threads doubles), so one launch performs 16 * iters * blocks *
 * threads floating-point operations; the caller times it (CUDA events on `stream`).
 * TRON_EINVAL for non-positive sizes, threads > 1024 or threads not a multiple of 32. */
tron_err_t tron_bench_fp64_fma(double* d_out, int32_t blocks, int32_t threads, int64_t iters,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EXATRON_GB300_TRON_H */
