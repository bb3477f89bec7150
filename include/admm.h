/*
 * admm.h -- C ABI of the GPU component ADMM for AC optimal power flow (Sec. 6.1).
 *
 * The ACOPF of eq. ac-rectangular is split into generator, branch and bus components
 * with duplicated linking variables (Sec. 6.1).  Every iteration runs, on the GPU:
 *   1. generator updates (closed form) in parallel with the branch updates (the
 *      4-variable NLP of eq. exp-branch with a line-limit penalty, solved by the
 *      batched trust-region Newton solver of tron.h, warm started), one launch;
 *   2. bus updates (closed-form equality-constrained QP over the bus copies with the
 *      power-balance equations), the multiplier update lambda += rho (x - xt) and the
 *      primal/dual residuals, one launch.
 * Iterations are captured once into a CUDA graph and replayed.
 *
 * Two levels:
 *  - admm_* : one network (a pool holding exactly one instance).
 *  - admm_pool_* : a resident pool of many independent instances (continuous
 *    batching): instances are admitted into free slot ranges while others run, their
 *    state stays on the device between steps, every step advances all live instances
 *    with shared launches, and results do not depend on the other residents.
 *
 * Conventions as in tron.h: host pointers unless named d_*, errors as tron_err_t with
 * tron_last_error(), no allocation after *_create, work enqueued on `stream`.
 *
 * Pair order of a branch k (from bus i, to bus j), used by every per-branch array of 8:
 *   p_ij q_ij p_ji q_ji  w_i w_j  theta_i theta_j
 * branch x = (v_i, v_j, theta_i, theta_j); bus-side flow copies (4): p_ij q_ij p_ji q_ji.
 */
#ifndef EXATRON_GB300_ADMM_H
#define EXATRON_GB300_ADMM_H

#include <stdint.h>

#include "tron.h"

#ifdef __cplusplus
extern "C" {
#endif

/* A network, host arrays (copied at create/add). */
typedef struct admm_network {
  int32_t nbus, nbranch, ngen;
  const int32_t* br_from;   /* [nbranch] bus index of the from end                   */
  const int32_t* br_to;     /* [nbranch] bus index of the to end                     */
  const double* br_coef;    /* [nbranch][8] gc_ij bc_ij g_ij b_ij gc_ji bc_ji g_ji b_ji */
  const double* br_smax2;   /* [nbranch] squared apparent-power limit                */
  const int32_t* gen_bus;   /* [ngen] */
  const double* gen_c2;     /* [ngen] cost c2 p^2 + c1 p                             */
  const double* gen_c1;
  const double* gen_pmin, *gen_pmax, *gen_qmin, *gen_qmax;  /* [ngen] */
  const double* bus_pd, *bus_qd;     /* [nbus] loads                                 */
  const double* bus_gsh, *bus_bsh;   /* [nbus] shunts                                */
  double rho;        /* penalty of every coupling pair (400 in the workloads)         */
  double rho_line;   /* line-limit penalty                                            */
  double vmin, vmax; /* voltage magnitude bounds (theta is bounded by +-2 pi)          */
} admm_network_t;

/* Host buffers for state transfer (checkpoint / resume).  Sizes as in admm_network_t:
 * br_x [nbranch][4], br_delta [nbranch], br_lam [nbranch][8], br_val [nbranch][8],
 * br_tilde [nbranch][4], bus_w [nbus], bus_th [nbus], gen_pq [ngen][2],
 * gen_lam [ngen][2], gen_tilde [ngen][2]; iteration = iterations completed. */
typedef struct admm_state_view {
  double* br_x;
  double* br_delta;
  double* br_lam;
  double* br_val;
  double* br_tilde;
  double* bus_w;
  double* bus_th;
  double* gen_pq;
  double* gen_lam;
  double* gen_tilde;
  int64_t iteration;
} admm_state_view_t;

typedef struct admm_pool admm_pool_t;
typedef admm_pool_t admm_t;

/* ---------------------------------------------------------------- single network */

/* Create the device state of one network (initial point: v = 1, theta = 0, generators
 * at box midpoints, bus copies equal to the component values, lambda = 0, delta = 1).
 * opt: TRON options of the branch solves (NULL = defaults).  options.group is the number
 * of lanes per branch problem in the branch launch: 1, 4, or 0 = chosen by the branch
 * slots per SM sub-partition (4 up to 24 slots per sub-partition: the launch is then as
 * long as its slowest problem, whose serial chain four lanes shorten; 1 beyond, where
 * the FP64 issue rate over all problems decides); any other value is TRON_EINVAL.  The
 * choice is fixed for the life of the handle or pool. */
tron_err_t admm_create(admm_t** out, const admm_network_t* net, const tron_options_t* opt,
                       void* stream);

/* Run n_iters iterations; when h_primal / h_dual are not NULL, synchronise the stream
 * and return the residuals of the last iteration:
 *   primal = ||x - xt||_2 over all coupling pairs, dual = rho ||xt - xt_prev||_2. */
tron_err_t admm_step(admm_t* a, int32_t n_iters, double* h_primal, double* h_dual,
                     void* stream);

/* Residuals of iterations [first, first + count) (they must be among the last
 * admm_history_capacity() iterations).  Synchronises the stream. */
tron_err_t admm_residual_history(admm_t* a, int64_t first, int64_t count, double* h_primal,
                                 double* h_dual, void* stream);

/* Copy the whole state to / from host buffers (synchronises the stream).  Resuming
 * from a saved state reproduces the uninterrupted run bit for bit. */
tron_err_t admm_get_state(admm_t* a, admm_state_view_t* host, void* stream);
tron_err_t admm_set_state(admm_t* a, const admm_state_view_t* host, void* stream);

/* Status counts (tron_status_t, [6]) of the branch solves of the last iteration. */
tron_err_t admm_branch_status_counts(admm_t* a, int64_t* h_counts6, void* stream);

int64_t admm_iterations(const admm_t* a);
int64_t admm_history_capacity(const admm_t* a);
/* GPU kernel launches one iteration performs (inside the replayed graph) with four
 * lanes per branch: 2.  A pool with one lane per branch that finishes its slow solves
 * on four lanes (options.split_outer) performs 3: admm_pool_launches_per_iteration. */
int32_t admm_launches_per_iteration(void);
void admm_destroy(admm_t* a);

/* ------------------------------------------------- resident pool (continuous batching) */

/* Capacities in slots; instances are placed in contiguous, 128-aligned ranges.  opt as
 * for admm_create: with options.group = 0 the branch mapping follows the pool's branch
 * slots per SM sub-partition (its capacity, not the instances live at a time), fixed for
 * the pool's life, so an instance's results do not depend on its co-residents. */
tron_err_t admm_pool_create(admm_pool_t** out, int32_t cap_bus, int32_t cap_branch,
                            int32_t cap_gen, int32_t cap_instances, int32_t history_len,
                            const tron_options_t* opt, void* stream);

/* GPU kernel launches of one iteration of this pool (or of an admm_t, which is one):
 * 3 with one lane per branch and options.split_outer > 0, else 2; 0 for NULL. */
int32_t admm_pool_launches_per_iteration(const admm_pool_t* p);

/* Admit an instance: returns TRON_ENOMEM (and *id = -1) when no free ranges can hold
 * it — nothing is allocated here, the pool's slots are reused.  The new instance
 * starts at the initial point and advances with every later admm_pool_step. */
tron_err_t admm_pool_add(admm_pool_t* p, const admm_network_t* net, int32_t* id,
                         void* stream);

/* Retire an instance and free its slots (its results should be read first). */
tron_err_t admm_pool_remove(admm_pool_t* p, int32_t id, void* stream);

/* Advance every live instance by n_iters iterations (shared launches). */
tron_err_t admm_pool_step(admm_pool_t* p, int32_t n_iters, void* stream);

/* Latest residuals and iteration counts of all instance slots ([cap_instances] each,
 * iteration = -1 for a free slot).  Synchronises the stream. */
tron_err_t admm_pool_residuals(admm_pool_t* p, int64_t* h_iter, double* h_primal,
                               double* h_dual, void* stream);

/* Residual history of one instance, as admm_residual_history. */
tron_err_t admm_pool_history(admm_pool_t* p, int32_t id, int64_t first, int64_t count,
                             double* h_primal, double* h_dual, void* stream);

tron_err_t admm_pool_get_state(admm_pool_t* p, int32_t id, admm_state_view_t* host,
                               void* stream);
tron_err_t admm_pool_set_state(admm_pool_t* p, int32_t id, const admm_state_view_t* host,
                               void* stream);
int32_t admm_pool_live(const admm_pool_t* p);
/* Lanes per branch problem the pool's branch launch uses (1, 2 or 4); 0 for NULL. */
int32_t admm_pool_branch_group(const admm_pool_t* p);
void admm_pool_destroy(admm_pool_t* p);

/* --------------------------------------- multi-period ADMM (the paper's future work)
 * Sec. 7 names multi-period optimal power flow as the next use of the ADMM with the
 * batched solver and gives no formulation; this is one reading of it.  T periods of one
 * network: period t's loads are h_load_scale[t] times the network's; the periods are
 * coupled by the generators' ramp limits |p_t - p_{t-1}| <= h_ramp[g], enforced by the
 * penalty rho_ramp/2 max(0, |p_t - p_{t-1}| - h_ramp[g])^2 in the generator component.
 * That component spans the periods: every iteration solves each generator's T
 * active-power outputs as one bound-constrained NLP (TRON_OBJ_GEN_RAMP, one batched
 * TRON launch over all generators, warm started), its reactive powers in closed form;
 * branches and buses are the single-period components of each period (the periods
 * live as instances of one resident pool and share its launches).  Residuals combine
 * all periods: primal sqrt(sum_t primal_t^2), dual sqrt(sum_t dual_t^2).  With
 * rho_ramp = 0 the periods are independent load scenarios of the network (each
 * generator's T outputs are then T separate problems).  The branch launch takes each
 * line's T period copies side by side, so the lanes of a warp solve one line under
 * neighbouring loads.
 *
 * admm_mp_create: copies the network and allocates everything (T <= 32, loads > 0,
 *   rho_ramp >= 0, h_ramp[g] >= 0; TRON_EINVAL otherwise).
 * admm_mp_step: runs n_iters iterations (five launches each); when h_primal / h_dual
 *   are not NULL, synchronises and writes the last iteration's combined residuals.
 * admm_mp_get_state: state of one period, as admm_get_state.
 * admm_mp_gen_status_counts: tron_status_t counts ([6]) of the last generator solves. */
typedef struct admm_mp admm_mp_t;
tron_err_t admm_mp_create(admm_mp_t** out, const admm_network_t* net, int32_t T,
                          const double* h_load_scale, const double* h_ramp, double rho_ramp,
                          const tron_options_t* opt, void* stream);
tron_err_t admm_mp_step(admm_mp_t* mp, int32_t n_iters, double* h_primal, double* h_dual,
                        void* stream);

/* GPU kernel launches of one admm_mp_step iteration: the pool's branch launch (3 with
 * the four-lane continuation of one-lane pools, else 2, counting the bus launch) plus the
 * generator chains' gather, solve and scatter when there are generators; 0 for NULL. */
int32_t admm_mp_launches_per_iteration(const admm_mp_t* mp);
tron_err_t admm_mp_get_state(admm_mp_t* mp, int32_t period, admm_state_view_t* host,
                             void* stream);
tron_err_t admm_mp_gen_status_counts(admm_mp_t* mp, int64_t* h_counts6, void* stream);
void admm_mp_destroy(admm_mp_t* mp);

#ifdef __cplusplus
}
#endif
#endif /* EXATRON_GB300_ADMM_H */
