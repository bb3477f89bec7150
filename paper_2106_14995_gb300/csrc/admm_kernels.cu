// admm_kernels.cu -- component ADMM (Sec. 6.1) on the GPU: kernels, resident instance
// pool and the admm_* / admm_pool_* C ABI.
//
// One iteration = two launches, both over the pool's whole capacity:
//   k_admm_branch_gen : generator updates (closed form) alongside the branch updates
//                       (the branch NLP of eq. exp-branch solved by the TRON solver of
//                       tron_solver.cuh, one, two or four lanes per branch, warm
//                       started; the branch record is gathered on the fly from the
//                       multipliers and the bus copies, the pair values at the new
//                       point are written back)
//   (k_admm_branch_tail: with one lane per branch, a third launch between the two that
//                       finishes on four lanes the solves still running after a few
//                       TRON iterations)
//   k_admm_bus        : per bus, the closed-form equality-constrained QP over its copies
//                       (power balance, eqs. PowerBalanceReal/Reactive), the multiplier
//                       update of every pair it owns and the residual partial sums; the
//                       last CTA to finish reduces each instance's partials in a fixed
//                       order and appends to its residual history.
// Slots of free or retired instances carry instance id -1 and are skipped, so the
// iteration can be captured once into a CUDA graph and replayed while instances come
// and go.  Every instance occupies 128-aligned slot ranges, so its reductions are
// identical whether it runs alone or next to others.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/admm.h"
#include "capi_common.h"
#include "tron_solver.cuh"

namespace xt {

constexpr int kAlign = 128;      // slot alignment of every instance range
constexpr int kBusThreads = 128; // = kAlign: one bus block never spans two instances
constexpr int kGraphChunk = 8;   // iterations per replayed graph
// lanes per branch problem when options.group is 0: four while the pool holds at most
// this many branch slots per SM sub-partition (the launch is then as long as its slowest
// problem's serial chain, which four lanes shorten), one beyond (the FP64 issue rate over
// all problems decides, and one lane per problem needs the fewest instructions)
constexpr int kG4BranchesPerSmsp = 24;
constexpr double kTwoPi = 6.283185307179586;

struct PoolDev {
  // branch slots
  int32_t* br_from;
  int32_t* br_to;
  int32_t* br_inst;
  double* br_coef;
  double* br_smax2;
  double* br_x;
  double* br_delta;
  double* br_lam;
  double* br_val;
  double* br_tilde;
  int32_t* br_status;
  int32_t* br_iters;
  double* br_alpc;          // Cauchy step of a solve paused after the one-lane launch
  int32_t* split_list;      // slots of the paused solves, in no particular order
  unsigned int* split_cnt;  // their number (reset by the bus kernel)
  const int32_t* br_order;  // slot solved by each lane of the branch launch (null: slot order)
  // generator slots
  int32_t* gen_bus;
  int32_t* gen_inst;
  double* gen_c2;
  double* gen_c1;
  double* gen_pmin;
  double* gen_pmax;
  double* gen_qmin;
  double* gen_qmax;
  double* gen_pq;
  double* gen_lam;
  double* gen_tilde;
  // bus slots
  int32_t* bus_inst;
  int32_t* bus_eoff;
  int32_t* bus_ecnt;
  int32_t* bus_goff;
  int32_t* bus_gcnt;
  double* bus_pd;
  double* bus_qd;
  double* bus_gsh;
  double* bus_bsh;
  double* bus_w;
  double* bus_th;
  int32_t* end_list;  // end id 2 * branch_slot + side, grouped per bus
  int32_t* gen_list;  // generator slots grouped per bus
  // instances
  double* inst_param;  // [cap_inst][4] rho, rho_line, vmin, vmax
  int32_t* inst_active;
  int32_t* inst_flags; // bit 0: the generators are updated outside the pool's launches
  int32_t* inst_blk;   // [cap_inst][2] bus-block range
  int64_t* inst_iter;
  double* hist;        // [cap_inst][H][2] primal, dual
  // reduction scratch
  double* part;        // [bus blocks][2]
  unsigned int* done;
  int64_t* lat_iter;   // latest residuals gathered for the host
  double* lat_res;
  int32_t cap_br, cap_gen, cap_bus, cap_inst, H;
};

struct AdmmArgs {
  PoolDev d;
  tron_options_t opt;
  int32_t nbb;       // branch CTAs (warps_per_block warps of 32 / G branches each)
  int32_t ngb;       // generator CTAs
  int32_t pause_at;  // one-lane branch solves stop after this many TRON iterations and
                     // are finished by k_admm_branch_tail (INT_MAX: no split)
};

template <int G>
using BranchSolver = Solver<BranchObj<G>, 4, G>;

// the branch update of slot k by a group of G lanes (G = 1: one branch per lane; G = 4:
// lane t owns variable t, flow t and the pair terms t and t + 4)
template <int G>
__device__ __forceinline__ void branch_update(const PoolDev& d, const tron_options_t& opt,
                                              double* wsm, int k, int pause_at, bool resume) {
  using S = BranchSolver<G>;
  const int inst = d.br_inst[k];
  if (inst < 0 || !d.inst_active[inst]) return;
  const double rho = d.inst_param[4 * inst + 0];
  const double rhol = d.inst_param[4 * inst + 1];
  const double vmin = d.inst_param[4 * inst + 2];
  const double vmax = d.inst_param[4 * inst + 3];
  S sv(opt, wsm);
  sv.n = 4;
  sv.obj.n = 4;
  const int i = d.br_from[k], j = d.br_to[k];
  bool fin = true;
  if constexpr (G == 1) {
    sv.l[0] = vmin;
    sv.l[1] = vmin;
    sv.l[2] = -kTwoPi;
    sv.l[3] = -kTwoPi;
    sv.u[0] = vmax;
    sv.u[1] = vmax;
    sv.u[2] = kTwoPi;
    sv.u[3] = kTwoPi;
    // the branch record: coefficients, multipliers, bus-side copies as targets
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double c = d.br_coef[8 * (size_t)k + q];
      const double l = d.br_lam[8 * (size_t)k + q];
      fin = fin && finite_bits(c) && finite_bits(l);
      sv.obj.rec[q] = c;
      sv.obj.rec[8 + q] = l;
      sv.obj.rec[24 + q] = rho;
    }
    double tg[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) tg[q] = d.br_tilde[4 * (size_t)k + q];
    tg[4] = d.bus_w[i];
    tg[5] = d.bus_w[j];
    tg[6] = d.bus_th[i];
    tg[7] = d.bus_th[j];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      fin = fin && finite_bits(tg[q]);
      sv.obj.rec[16 + q] = tg[q];
    }
    sv.obj.rec[32] = d.br_smax2[k];
    sv.obj.rec[33] = rhol;
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = d.br_x[4 * (size_t)k + q];
    double delta = d.br_delta[k];
    double f, pg;
    int it;
    sv.pause_at = pause_at;
    const int st = sv.run(x, delta, f, pg, it, fin);
    if (st == kTronPaused) {
      // unfinished after pause_at iterations: the state for the four-lane continuation,
      // and the slot on the list of k_admm_branch_tail
#pragma unroll
      for (int q = 0; q < 4; ++q) d.br_x[4 * (size_t)k + q] = x[q];
      d.br_delta[k] = delta;
      d.br_alpc[k] = sv.alpha_out;
      d.br_iters[k] = it;
      d.split_list[atomicAdd(d.split_cnt, 1u)] = k;
      return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d.br_x[4 * (size_t)k + q] = x[q];
      d.br_val[8 * (size_t)k + q] = sv.obj.Fx[q];
    }
    d.br_val[8 * (size_t)k + 4] = x[0] * x[0];
    d.br_val[8 * (size_t)k + 5] = x[1] * x[1];
    d.br_val[8 * (size_t)k + 6] = x[2];
    d.br_val[8 * (size_t)k + 7] = x[3];
    d.br_delta[k] = delta;
    d.br_status[k] = st;
    d.br_iters[k] = it;
  } else if constexpr (G == 2) {
    // rank t: bus t of the branch, variables (v, theta) of that bus; it stages entries
    // t, t + 2, t + 4, t + 6 of the coefficients, multipliers, penalties and targets
    const int t = sv.gp.t;
    sv.l[0] = vmin;
    sv.u[0] = vmax;
    sv.l[1] = -kTwoPi;
    sv.u[1] = kTwoPi;
    const int bus = t ? j : i;
#pragma unroll
    for (int q = t; q < 8; q += 2) {
      const double c = d.br_coef[8 * (size_t)k + q];
      const double l = d.br_lam[8 * (size_t)k + q];
      fin = fin && finite_bits(c) && finite_bits(l);
      sv.obj.rec[q] = c;
      sv.obj.rec[8 + q] = l;
      sv.obj.rec[24 + q] = rho;
    }
    // targets: flows t, t + 2 (branch-side copies), then w and theta of bus t
    const double tg0 = d.br_tilde[4 * (size_t)k + t], tg1 = d.br_tilde[4 * (size_t)k + t + 2];
    const double tgw = d.bus_w[bus], tgt = d.bus_th[bus];
    fin = fin && finite_bits(tg0) && finite_bits(tg1) && finite_bits(tgw) && finite_bits(tgt);
    sv.obj.rec[16 + t] = tg0;
    sv.obj.rec[18 + t] = tg1;
    sv.obj.rec[20 + t] = tgw;
    sv.obj.rec[22 + t] = tgt;
    if (t == 0) sv.obj.rec[32] = d.br_smax2[k];
    if (t == 1) sv.obj.rec[33] = rhol;
    sv.gp.sync();
    sv.obj.prepare(t);
    fin = !sv.gp.any(!fin);
    double x[2] = {d.br_x[4 * (size_t)k + t], d.br_x[4 * (size_t)k + 2 + t]};
    double delta = d.br_delta[k];
    double f, pg;
    int it;
    const int st = sv.run(x, delta, f, pg, it, fin);
    d.br_x[4 * (size_t)k + t] = x[0];
    d.br_x[4 * (size_t)k + 2 + t] = x[1];
    d.br_val[8 * (size_t)k + 2 * t] = sv.obj.Fx[0];
    d.br_val[8 * (size_t)k + 2 * t + 1] = sv.obj.Fx[1];
    d.br_val[8 * (size_t)k + 4 + t] = x[0] * x[0];
    d.br_val[8 * (size_t)k + 6 + t] = x[1];
    if (t == 0) {
      d.br_delta[k] = delta;
      d.br_status[k] = st;
      d.br_iters[k] = it;
    }
  } else {
    const int t = sv.gp.t;
    sv.l[0] = t < 2 ? vmin : -kTwoPi;
    sv.u[0] = t < 2 ? vmax : kTwoPi;
    // rank t stages entries t and t + 4 of the coefficients, multipliers and penalties,
    // and the targets of the pair terms t (flow) and t + 4 (w_i, w_j, theta_i, theta_j)
#pragma unroll
    for (int q = t; q < 8; q += 4) {
      const double c = d.br_coef[8 * (size_t)k + q];
      const double l = d.br_lam[8 * (size_t)k + q];
      fin = fin && finite_bits(c) && finite_bits(l);
      sv.obj.rec[q] = c;
      sv.obj.rec[8 + q] = l;
      sv.obj.rec[24 + q] = rho;
    }
    const int bus = (t & 1) ? j : i;
    const double tg1 = d.br_tilde[4 * (size_t)k + t];
    const double tg2 = t < 2 ? d.bus_w[bus] : d.bus_th[bus];
    fin = fin && finite_bits(tg1) && finite_bits(tg2);
    sv.obj.rec[16 + t] = tg1;
    sv.obj.rec[20 + t] = tg2;
    if (t == 0) sv.obj.rec[32] = d.br_smax2[k];
    if (t == 1) sv.obj.rec[33] = rhol;
    sv.gp.sync();
    sv.obj.prepare(t);
    fin = !sv.gp.any(!fin);
    double x[1] = {d.br_x[4 * (size_t)k + t]};
    double delta = d.br_delta[k];
    if (resume) {  // the continuation of a paused one-lane solve
      sv.k_start = d.br_iters[k];
      sv.alpha0 = d.br_alpc[k];
    }
    double f, pg;
    int it;
    const int st = sv.run(x, delta, f, pg, it, fin);
    d.br_x[4 * (size_t)k + t] = x[0];
    d.br_val[8 * (size_t)k + t] = sv.obj.Fx;
    d.br_val[8 * (size_t)k + 4 + t] = t < 2 ? x[0] * x[0] : x[0];
    if (t == 0) {
      d.br_delta[k] = delta;
      d.br_status[k] = st;
      d.br_iters[k] = it;
    }
  }
}

template <int G>
__global__ void __launch_bounds__(256) k_admm_branch_gen(const AdmmArgs a) {
  const PoolDev& d = a.d;
  if ((int)blockIdx.x < a.nbb) {
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int k = ((int)blockIdx.x * (int)(blockDim.x >> 5) + warp) * (32 / G) + lane / G;
    if (k >= d.cap_br) return;
    if (d.br_order) {
      k = d.br_order[k];
      if (k < 0) return;
    }
    branch_update<G>(d, a.opt, smem + (size_t)warp * BranchSolver<G>::WARP_DOUBLES, k,
                     G == 1 ? a.pause_at : 0x7FFFFFFF, false);
  } else {
    const int g = ((int)blockIdx.x - a.nbb) * (int)blockDim.x + (int)threadIdx.x;
    if (g >= d.cap_gen) return;
    const int inst = d.gen_inst[g];
    if (inst < 0 || !d.inst_active[inst] || (d.inst_flags[inst] & 1)) return;
    const double rho = d.inst_param[4 * inst];
    const double pt = d.gen_tilde[2 * g], qt = d.gen_tilde[2 * g + 1];
    const double lp = d.gen_lam[2 * g], lq = d.gen_lam[2 * g + 1];
    // minimiser of c2 p^2 + c1 p + lp (p - pt) + rho/2 (p - pt)^2 on [pmin, pmax],
    // and of lq (q - qt) + rho/2 (q - qt)^2 on [qmin, qmax]
    double p = (rho * pt - lp - d.gen_c1[g]) / (2.0 * d.gen_c2[g] + rho);
    double q = qt - lq / rho;
    p = p < d.gen_pmin[g] ? d.gen_pmin[g] : (p > d.gen_pmax[g] ? d.gen_pmax[g] : p);
    q = q < d.gen_qmin[g] ? d.gen_qmin[g] : (q > d.gen_qmax[g] ? d.gen_qmax[g] : q);
    d.gen_pq[2 * g] = p;
    d.gen_pq[2 * g + 1] = q;
  }
}

// The continuation of the one-lane solves that k_admm_branch_gen<1> paused: four lanes
// per solve (each TRON iteration about half as long as on one lane), the paused slots
// taken from the list in order by the groups of a grid of one-warp CTAs.  Only the few
// slow solves of an iteration get here, so they no longer hold one-lane warps (and their
// SMs) to the end of the branch launch.
__global__ void __launch_bounds__(32) k_admm_branch_tail(const AdmmArgs a) {
  const PoolDev& d = a.d;
  extern __shared__ double smem[];
  const unsigned cnt = *d.split_cnt;  // written by the previous launch
  const unsigned ng = gridDim.x * 8u;
  for (unsigned e = blockIdx.x * 8u + (threadIdx.x >> 2); e < cnt; e += ng)
    branch_update<4>(d, a.opt, smem, d.split_list[e], 0x7FFFFFFF, true);
}

// the branch kernel and its shared memory per warp for branch group size G (1, 2 or 4)
static const void* branch_kernel(int G) {
  return G == 4 ? (const void*)k_admm_branch_gen<4>
                : (G == 2 ? (const void*)k_admm_branch_gen<2> : (const void*)k_admm_branch_gen<1>);
}
static size_t branch_warp_bytes(int G) {
  return sizeof(double) * (size_t)(G == 4 ? BranchSolver<4>::WARP_DOUBLES
                                          : (G == 2 ? BranchSolver<2>::WARP_DOUBLES
                                                    : BranchSolver<1>::WARP_DOUBLES));
}

__global__ void __launch_bounds__(kBusThreads) k_admm_bus(const AdmmArgs a) {
  const PoolDev& d = a.d;
  const int b = (int)blockIdx.x * kBusThreads + (int)threadIdx.x;
  double pr2 = 0.0, du2 = 0.0;
  if (b < d.cap_bus) {
    const int inst = d.bus_inst[b];
    if (inst >= 0 && d.inst_active[inst]) {
      // one thread per bus, so a hub bus's chain sets the launch: every division by rho
      // or by a per-bus quantity is one reciprocal, and the incidence loops are unrolled
      // so that their gathers are in flight together
      const double rho = d.inst_param[4 * inst];
      const double irho = 1.0 / rho;
      const int g0 = d.bus_goff[b], gn = d.bus_gcnt[b];
      const int e0 = d.bus_eoff[b], en = d.bus_ecnt[b];
      // a = x + lambda / rho for every copy; balance rows A a - (p_d, q_d)
      double rhsP = -d.bus_pd[b], rhsQ = -d.bus_qd[b];
      double awn = 0.0, athn = 0.0;
#pragma unroll 2
      for (int t = 0; t < gn; ++t) {
        const int g = d.gen_list[g0 + t];
        rhsP += fma(d.gen_lam[2 * g], irho, d.gen_pq[2 * g]);
        rhsQ += fma(d.gen_lam[2 * g + 1], irho, d.gen_pq[2 * g + 1]);
      }
#pragma unroll 4
      for (int t = 0; t < en; ++t) {
        const int e = d.end_list[e0 + t];
        const size_t k = (size_t)(e >> 1);
        const int side = e & 1;
        const int kp = side ? 2 : 0, kq = kp + 1, kw = side ? 5 : 4, kt = side ? 7 : 6;
        const double* val = d.br_val + 8 * k;
        const double* lam = d.br_lam + 8 * k;
        rhsP -= fma(lam[kp], irho, val[kp]);
        rhsQ -= fma(lam[kq], irho, val[kq]);
        awn += fma(rho, val[kw], lam[kw]);    // rho (x + lambda / rho)
        athn += fma(rho, val[kt], lam[kt]);
      }
      const double sinv = (double)(gn + en) * irho;  // sum of 1/rho over the copies
      const double Dw = (double)en * rho;
      const double iDw = en > 0 ? 1.0 / Dw : 0.0;
      const double gsh = d.bus_gsh[b], bsh = d.bus_bsh[b];
      const double w_old = d.bus_w[b], th_old = d.bus_th[b];
      const double aw = en > 0 ? awn * iDw : w_old;
      rhsP -= gsh * aw;
      rhsQ += bsh * aw;
      double M11 = sinv, M22 = sinv, M12 = 0.0;
      if (en > 0) {
        M11 += gsh * gsh * iDw;
        M22 += bsh * bsh * iDw;
        M12 = -gsh * bsh * iDw;
      }
      const double det = M11 * M22 - M12 * M12;
      double mu1 = 0.0, mu2 = 0.0;
      if (det != 0.0) {
        const double idet = 1.0 / det;
        mu1 = (M22 * rhsP - M12 * rhsQ) * idet;
        mu2 = (M11 * rhsQ - M12 * rhsP) * idet;
      }
      const double w_new = en > 0 ? aw - (-gsh * mu1 + bsh * mu2) * iDw : w_old;
      const double th_new = en > 0 ? athn * iDw : th_old;
      const double m1r = mu1 * irho, m2r = mu2 * irho;
      // new copies, multipliers lambda += rho (x - xt), residual sums; every copy's
      // loads are issued before its stores, so they travel together
#pragma unroll 2
      for (int t = 0; t < gn; ++t) {
        const int g = d.gen_list[g0 + t];
        const double xv0 = d.gen_pq[2 * g], xv1 = d.gen_pq[2 * g + 1];
        const double l0 = d.gen_lam[2 * g], l1 = d.gen_lam[2 * g + 1];
        const double o0 = d.gen_tilde[2 * g], o1 = d.gen_tilde[2 * g + 1];
        const double xt0 = fma(l0, irho, xv0) - m1r;
        const double xt1 = fma(l1, irho, xv1) - m2r;
        d.gen_tilde[2 * g] = xt0;
        d.gen_tilde[2 * g + 1] = xt1;
        d.gen_lam[2 * g] = fma(rho, xv0 - xt0, l0);
        d.gen_lam[2 * g + 1] = fma(rho, xv1 - xt1, l1);
        pr2 = fma(xv0 - xt0, xv0 - xt0, pr2);
        du2 = fma(xt0 - o0, xt0 - o0, du2);
        pr2 = fma(xv1 - xt1, xv1 - xt1, pr2);
        du2 = fma(xt1 - o1, xt1 - o1, du2);
      }
      const double dw2 = (w_new - w_old) * (w_new - w_old);
      const double dt2 = (th_new - th_old) * (th_new - th_old);
      // the branch ends in batches of four: the four copies' loads first, then their
      // updates and stores (a store may alias the next copy's loads as far as the
      // compiler knows, so one copy at a time would wait out a memory latency per copy);
      // the residual sums accumulate in the same order as one at a time
      constexpr int kEB = 4;
      for (int t0 = 0; t0 < en; t0 += kEB) {
        size_t kk[kEB];
        int kp[kEB];
        double vp[kEB], vq[kEB], vw[kEB], vt[kEB], lp[kEB], lq[kEB], lw[kEB], lt[kEB];
        double op[kEB], oq[kEB];
#pragma unroll
        for (int u = 0; u < kEB; ++u) {
          if (t0 + u < en) {
            const int e = d.end_list[e0 + t0 + u];
            const size_t k = (size_t)(e >> 1);
            const int side = e & 1;
            const int p0 = side ? 2 : 0, kw = side ? 5 : 4, kt = side ? 7 : 6;
            const double* val = d.br_val + 8 * k;
            const double* lam = d.br_lam + 8 * k;
            const double* tl = d.br_tilde + 4 * k;
            kk[u] = k;
            kp[u] = p0;
            vp[u] = val[p0];
            vq[u] = val[p0 + 1];
            vw[u] = val[kw];
            vt[u] = val[kt];
            lp[u] = lam[p0];
            lq[u] = lam[p0 + 1];
            lw[u] = lam[kw];
            lt[u] = lam[kt];
            op[u] = tl[p0];
            oq[u] = tl[p0 + 1];
          }
        }
#pragma unroll
        for (int u = 0; u < kEB; ++u) {
          if (t0 + u < en) {
            const int p0 = kp[u], kw = p0 ? 5 : 4, kt = p0 ? 7 : 6;
            double* lam = d.br_lam + 8 * kk[u];
            double* tl = d.br_tilde + 4 * kk[u];
            const double xp = fma(lp[u], irho, vp[u]) + m1r;
            const double xq = fma(lq[u], irho, vq[u]) + m2r;
            tl[p0] = xp;
            tl[p0 + 1] = xq;
            lam[p0] = fma(rho, vp[u] - xp, lp[u]);
            lam[p0 + 1] = fma(rho, vq[u] - xq, lq[u]);
            lam[kw] = fma(rho, vw[u] - w_new, lw[u]);
            lam[kt] = fma(rho, vt[u] - th_new, lt[u]);
            pr2 = fma(vp[u] - xp, vp[u] - xp, pr2);
            du2 = fma(xp - op[u], xp - op[u], du2);
            pr2 = fma(vq[u] - xq, vq[u] - xq, pr2);
            du2 = fma(xq - oq[u], xq - oq[u], du2);
            pr2 = fma(vw[u] - w_new, vw[u] - w_new, pr2);
            du2 += dw2;
            pr2 = fma(vt[u] - th_new, vt[u] - th_new, pr2);
            du2 += dt2;
          }
        }
      }
      d.bus_w[b] = w_new;
      d.bus_th[b] = th_new;
    }
  }
  // block sums in a fixed order: butterfly in each warp, then warp 0..3 in order
  __shared__ double sp[kBusThreads / 32], sd[kBusThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pr2 += __shfl_xor_sync(0xffffffffu, pr2, o);
    du2 += __shfl_xor_sync(0xffffffffu, du2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sp[threadIdx.x >> 5] = pr2;
    sd[threadIdx.x >> 5] = du2;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double p = 0.0, q = 0.0;
    for (int w = 0; w < kBusThreads / 32; ++w) {
      p += sp[w];
      q += sd[w];
    }
    d.part[2 * blockIdx.x] = p;
    d.part[2 * blockIdx.x + 1] = q;
    __threadfence();
    const unsigned ticket = atomicAdd(d.done, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // last CTA: each warp reduces whole instances, its lanes summing the instance's block
  // partials strided by 32 and then combining them in a fixed butterfly; the result
  // depends only on the instance's own blocks (the same bits alone or in a mix)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < d.cap_inst; i += kBusThreads / 32) {
    if (!d.inst_active[i]) continue;
    double p = 0.0, q = 0.0;
    const int b0 = d.inst_blk[2 * i], b1 = d.inst_blk[2 * i + 1];
    for (int bk = b0 + lane; bk < b1; bk += 32) {
      p += __ldcg(d.part + 2 * bk);
      q += __ldcg(d.part + 2 * bk + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p += __shfl_xor_sync(0xffffffffu, p, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (lane == 0) {
      const int64_t it = d.inst_iter[i];
      const size_t slot = ((size_t)i * d.H + (size_t)(it % d.H)) * 2;
      d.hist[slot] = sqrt(p);
      d.hist[slot + 1] = d.inst_param[4 * i] * sqrt(q);
      d.inst_iter[i] = it + 1;
    }
  }
  if (threadIdx.x == 0) {
    *d.done = 0u;
    *d.split_cnt = 0u;
  }
}

// initial point of a newly admitted instance (v = 1, theta = 0, generators at box
// midpoints, bus copies equal to the component values, lambda = 0, delta = 1)
__global__ void k_admm_init(const AdmmArgs a, int l0, int l1, int g0, int g1, int b0, int b1) {
  const PoolDev& d = a.d;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = l0 + t;
  if (k < l1 && d.br_inst[k] >= 0) {
    const double* cf = d.br_coef + 8 * (size_t)k;
    double sn, cs;
    sincos(0.0, &sn, &cs);
    const double F[4] = {cf[0] - cf[2] * cs + cf[3] * sn, cf[1] - cf[3] * cs - cf[2] * sn,
                         cf[4] - cf[6] * cs - cf[7] * sn, cf[5] - cf[7] * cs + cf[6] * sn};
    const double x0[4] = {1.0, 1.0, 0.0, 0.0};
    for (int q = 0; q < 4; ++q) {
      d.br_x[4 * (size_t)k + q] = x0[q];
      d.br_val[8 * (size_t)k + q] = F[q];
      d.br_tilde[4 * (size_t)k + q] = F[q];
    }
    d.br_val[8 * (size_t)k + 4] = 1.0;
    d.br_val[8 * (size_t)k + 5] = 1.0;
    d.br_val[8 * (size_t)k + 6] = 0.0;
    d.br_val[8 * (size_t)k + 7] = 0.0;
    for (int q = 0; q < 8; ++q) d.br_lam[8 * (size_t)k + q] = 0.0;
    d.br_delta[k] = 1.0;
    d.br_status[k] = 0;
    d.br_iters[k] = 0;
  }
  const int g = g0 + t;
  if (g < g1 && d.gen_inst[g] >= 0) {
    const double p = 0.5 * (d.gen_pmin[g] + d.gen_pmax[g]);
    const double q = 0.5 * (d.gen_qmin[g] + d.gen_qmax[g]);
    d.gen_pq[2 * g] = p;
    d.gen_pq[2 * g + 1] = q;
    d.gen_tilde[2 * g] = p;
    d.gen_tilde[2 * g + 1] = q;
    d.gen_lam[2 * g] = 0.0;
    d.gen_lam[2 * g + 1] = 0.0;
  }
  const int b = b0 + t;
  if (b < b1 && d.bus_inst[b] >= 0) {
    d.bus_w[b] = 1.0;
    d.bus_th[b] = 0.0;
  }
}

__global__ void k_admm_latest(const PoolDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.cap_inst) return;
  if (!d.inst_active[i] || d.inst_iter[i] == 0) {
    d.lat_iter[i] = d.inst_active[i] ? 0 : -1;
    d.lat_res[2 * i] = CUDART_NAN;
    d.lat_res[2 * i + 1] = CUDART_NAN;
    return;
  }
  const int64_t it = d.inst_iter[i];
  const size_t slot = ((size_t)i * d.H + (size_t)((it - 1) % d.H)) * 2;
  d.lat_iter[i] = it;
  d.lat_res[2 * i] = d.hist[slot];
  d.lat_res[2 * i + 1] = d.hist[slot + 1];
}

// ---- multi-period ADMM: the generator component spanning the periods.  Period t of
// generator g sits in pool slot g0[t] + g.  Gather: the chain records (multipliers and
// bus-side copies of p over the periods) and the warm start; reactive power per period
// in closed form (minimiser of lq (q - qt) + rho/2 (q - qt)^2 on [qmin, qmax]).
__global__ void k_mp_gather(const PoolDev d, const int32_t* __restrict__ g0, int T, int ngen,
                            double* __restrict__ rec, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ngen * T) return;
  const int g = i / T, t = i - g * T;
  const int s = g0[t] + g;
  const size_t rs = 8 + 2 * (size_t)T;
  rec[(size_t)g * rs + 8 + t] = d.gen_lam[2 * s];
  rec[(size_t)g * rs + 8 + T + t] = d.gen_tilde[2 * s];
  x[i] = d.gen_pq[2 * s];
  const double rho = d.inst_param[4 * d.gen_inst[s]];
  double q = d.gen_tilde[2 * s + 1] - d.gen_lam[2 * s + 1] / rho;
  q = q < d.gen_qmin[s] ? d.gen_qmin[s] : (q > d.gen_qmax[s] ? d.gen_qmax[s] : q);
  d.gen_pq[2 * s + 1] = q;
}

// the solved active powers back into the periods' generator slots
__global__ void k_mp_scatter(const PoolDev d, const int32_t* __restrict__ g0, int T, int ngen,
                             const double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ngen * T) return;
  const int g = i / T, t = i - g * T;
  d.gen_pq[2 * (g0[t] + g)] = x[i];
}

// first-fit allocator of aligned slot ranges
struct RangeAlloc {
  std::vector<std::pair<int, int>> free_;  // sorted, disjoint [start, end)
  void init(int cap) {
    free_.clear();
    if (cap > 0) free_.push_back({0, cap});
  }
  int take(int n) {  // returns start or -1
    if (n == 0) return 0;
    for (size_t i = 0; i < free_.size(); ++i) {
      if (free_[i].second - free_[i].first >= n) {
        const int s = free_[i].first;
        free_[i].first += n;
        if (free_[i].first == free_[i].second) free_.erase(free_.begin() + i);
        return s;
      }
    }
    return -1;
  }
  void give(int s, int n) {
    if (n == 0) return;
    free_.push_back({s, s + n});
    std::sort(free_.begin(), free_.end());
    std::vector<std::pair<int, int>> m;
    for (auto& r : free_) {
      if (!m.empty() && m.back().second == r.first) m.back().second = r.second;
      else m.push_back(r);
    }
    free_ = m;
  }
};

static int align_up(int v) { return (v + kAlign - 1) / kAlign * kAlign; }

}  // namespace xt

using namespace xt;

struct admm_pool {
  PoolDev d;
  tron_options_t opt;
  int nbb, ngb, nbusb;
  int bw;   // warps per branch CTA
  int grp;  // lanes per branch problem (1, 2 or 4)
  int split;  // one-lane pools: TRON iterations before a solve moves to four lanes (0: never)
  int ntb;    // CTAs of k_admm_branch_tail
  RangeAlloc ab, al, ag;
  struct Inst {
    bool live;
    int b0, nb, l0, nl, g0, ng;  // slot starts and sizes (sizes aligned)
    int nbus, nbranch, ngen;      // true sizes
  };
  std::vector<Inst> inst;
  int live;
  cudaStream_t cap_stream;
  cudaGraphExec_t g1, gc;  // 1-iteration and chunk graphs
  std::vector<void*> allocs;
};

static tron_err_t pool_alloc(admm_pool* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 8;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    set_error("admm: cudaMalloc of %zu bytes failed", bytes);
    return TRON_ENOMEM;
  }
  p->allocs.push_back(*ptr);
  return TRON_OK;
}

#define PA(field, count)                                                                  \
  do {                                                                                    \
    tron_err_t e_ = pool_alloc(p, (void**)&p->d.field, sizeof(*p->d.field) * (size_t)(count)); \
    if (e_ != TRON_OK) {                                                                  \
      admm_pool_destroy(p);                                                               \
      return e_;                                                                          \
    }                                                                                     \
  } while (0)

static AdmmArgs make_args(const admm_pool* p) {
  AdmmArgs a;
  memset(&a, 0, sizeof(a));
  a.d = p->d;
  a.opt = p->opt;
  a.nbb = p->nbb;
  a.ngb = p->ngb;
  a.pause_at = p->split > 0 ? p->split : 0x7FFFFFFF;
  return a;
}

static tron_err_t launch_iteration(admm_pool* p, cudaStream_t st) {
  AdmmArgs a = make_args(p);
  const size_t smem = (size_t)p->bw * branch_warp_bytes(p->grp);
  void* args[] = {&a};
  // every CTA has bw warps: a branch CTA solves 32 / grp branches per warp (each warp
  // owns its slice of the shared memory), a generator CTA updates one generator per thread
  XT_CUDA(cudaLaunchKernel(branch_kernel(p->grp), dim3(p->nbb + p->ngb),
                           dim3(p->bw * 32), args, smem, st));
  if (p->split > 0)
    XT_CUDA(cudaLaunchKernel((const void*)k_admm_branch_tail, dim3(p->ntb), dim3(32), args,
                             branch_warp_bytes(4), st));
  XT_CUDA(cudaLaunchKernel((const void*)k_admm_bus, dim3(p->nbusb), dim3(kBusThreads), args, 0,
                           st));
  return TRON_OK;
}

static tron_err_t capture(admm_pool* p, int iters, cudaGraphExec_t* out) {
  cudaGraph_t g;
  XT_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  tron_err_t e = TRON_OK;
  for (int i = 0; i < iters && e == TRON_OK; ++i) e = launch_iteration(p, p->cap_stream);
  cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
  if (e != TRON_OK) return e;
  if (ce != cudaSuccess) {
    set_error("admm: graph capture failed: %s", cudaGetErrorString(ce));
    return TRON_ECUDA;
  }
  ce = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) {
    set_error("admm: graph instantiation failed: %s", cudaGetErrorString(ce));
    return TRON_ECUDA;
  }
  return TRON_OK;
}

extern "C" {

int32_t admm_launches_per_iteration(void) { return 2; }

int32_t admm_pool_launches_per_iteration(const admm_pool_t* p) {
  return p ? (p->split > 0 ? 3 : 2) : 0;
}

tron_err_t admm_pool_create(admm_pool_t** out, int32_t cap_bus, int32_t cap_branch,
                            int32_t cap_gen, int32_t cap_instances, int32_t history_len,
                            const tron_options_t* opt, void* stream) {
  clear_error();
  XT_REQUIRE(out != nullptr, TRON_EINVAL, "admm_pool_create: out is NULL");
  *out = nullptr;
  XT_REQUIRE(cap_bus >= 0 && cap_branch >= 0 && cap_gen >= 0 && cap_instances > 0 &&
                 history_len > 0,
             TRON_EINVAL, "admm_pool_create: bad capacities");
  XT_REQUIRE(!opt || opt->group == 0 || opt->group == 1 || opt->group == 2 || opt->group == 4,
             TRON_EINVAL, "admm: options.group must be 0, 1, 2 or 4");
  XT_REQUIRE(!opt || opt->tr_norm == 0 || opt->tr_norm == 1, TRON_EINVAL,
             "admm: options.tr_norm must be 0 or 1");
  XT_REQUIRE(!opt || opt->cauchy_norm == 0 || opt->cauchy_norm == 1, TRON_EINVAL,
             "admm: options.cauchy_norm must be 0 or 1");
  admm_pool* p = new admm_pool();
  memset(&p->d, 0, sizeof(p->d));
  p->cap_stream = nullptr;
  p->g1 = nullptr;
  p->gc = nullptr;
  p->live = 0;
  if (opt) p->opt = *opt;
  else tron_options_default(&p->opt);
  const int cb = align_up(cap_bus), cl = align_up(cap_branch), cg = align_up(cap_gen);
  // lanes per branch problem: options.group 1 or 4, or (0) chosen by the branch slots
  // per SM sub-partition; fixed for the pool's life, so an instance's results do not
  // depend on its co-residents
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    nsm = 0;
  if (p->opt.group == 0) {
    p->grp = (nsm > 0 && (long long)cl <= (long long)kG4BranchesPerSmsp * 4 * nsm) ? 4 : 1;
  } else {
    p->grp = p->opt.group;
  }
  p->opt.group = p->grp;
  // with options.split_outer = K > 0, one-lane pools finish the solves still running
  // after K iterations on four lanes, in a grid of one-warp CTAs that holds the usual
  // number of them with one group each (16 resident per SM); more paused solves are
  // taken in turn
  p->split = (p->grp == 1 && p->opt.split_outer > 0) ? p->opt.split_outer : 0;
  p->ntb = std::max(1, std::min((cl + 7) / 8, 16 * std::max(nsm, 1)));
  p->d.cap_bus = cb;
  p->d.cap_br = cl;
  p->d.cap_gen = cg;
  p->d.cap_inst = cap_instances;
  p->d.H = history_len;
  // branch CTA size: options.warps_per_block (default 1: spread the branch warps over
  // every SM); 32 / grp branches per CTA warp
  p->bw = p->opt.warps_per_block > 0 ? std::min(p->opt.warps_per_block, 8) : 1;
  const int bpw = 32 / p->grp;
  p->nbb = (cl + p->bw * bpw - 1) / (p->bw * bpw);
  p->ngb = (cg + p->bw * 32 - 1) / (p->bw * 32);
  p->nbusb = std::max(1, (cb + kBusThreads - 1) / kBusThreads);
  PA(br_from, cl);
  PA(br_to, cl);
  PA(br_inst, cl);
  PA(br_coef, 8 * (size_t)cl);
  PA(br_smax2, cl);
  PA(br_x, 4 * (size_t)cl);
  PA(br_delta, cl);
  PA(br_lam, 8 * (size_t)cl);
  PA(br_val, 8 * (size_t)cl);
  PA(br_tilde, 4 * (size_t)cl);
  PA(br_status, cl);
  PA(br_iters, cl);
  PA(br_alpc, cl);
  PA(split_list, cl);
  PA(split_cnt, 1);
  PA(gen_bus, cg);
  PA(gen_inst, cg);
  PA(gen_c2, cg);
  PA(gen_c1, cg);
  PA(gen_pmin, cg);
  PA(gen_pmax, cg);
  PA(gen_qmin, cg);
  PA(gen_qmax, cg);
  PA(gen_pq, 2 * (size_t)cg);
  PA(gen_lam, 2 * (size_t)cg);
  PA(gen_tilde, 2 * (size_t)cg);
  PA(bus_inst, cb);
  PA(bus_eoff, cb);
  PA(bus_ecnt, cb);
  PA(bus_goff, cb);
  PA(bus_gcnt, cb);
  PA(bus_pd, cb);
  PA(bus_qd, cb);
  PA(bus_gsh, cb);
  PA(bus_bsh, cb);
  PA(bus_w, cb);
  PA(bus_th, cb);
  PA(end_list, 2 * (size_t)cl);
  PA(gen_list, cg);
  PA(inst_param, 4 * (size_t)cap_instances);
  PA(inst_active, cap_instances);
  PA(inst_flags, cap_instances);
  PA(inst_blk, 2 * (size_t)cap_instances);
  PA(inst_iter, cap_instances);
  PA(hist, 2 * (size_t)cap_instances * history_len);
  PA(part, 2 * (size_t)p->nbusb);
  PA(done, 1);
  PA(lat_iter, cap_instances);
  PA(lat_res, 2 * (size_t)cap_instances);
  cudaStream_t st = (cudaStream_t)stream;
  auto fail = [&](const char* what) {
    set_error("admm_pool_create: %s failed", what);
    admm_pool_destroy(p);
    return TRON_ECUDA;
  };
  if (cudaMemsetAsync(p->d.br_inst, 0xFF, sizeof(int32_t) * cl, st) ||
      cudaMemsetAsync(p->d.gen_inst, 0xFF, sizeof(int32_t) * cg, st) ||
      cudaMemsetAsync(p->d.bus_inst, 0xFF, sizeof(int32_t) * cb, st) ||
      cudaMemsetAsync(p->d.bus_ecnt, 0, sizeof(int32_t) * cb, st) ||
      cudaMemsetAsync(p->d.bus_gcnt, 0, sizeof(int32_t) * cb, st) ||
      cudaMemsetAsync(p->d.bus_eoff, 0, sizeof(int32_t) * cb, st) ||
      cudaMemsetAsync(p->d.bus_goff, 0, sizeof(int32_t) * cb, st) ||
      cudaMemsetAsync(p->d.inst_active, 0, sizeof(int32_t) * cap_instances, st) ||
      cudaMemsetAsync(p->d.inst_flags, 0, sizeof(int32_t) * cap_instances, st) ||
      cudaMemsetAsync(p->d.inst_blk, 0, sizeof(int32_t) * 2 * cap_instances, st) ||
      cudaMemsetAsync(p->d.inst_iter, 0, sizeof(int64_t) * cap_instances, st) ||
      cudaMemsetAsync(p->d.inst_param, 0, sizeof(double) * 4 * cap_instances, st) ||
      cudaMemsetAsync(p->d.done, 0, sizeof(unsigned int), st) ||
      cudaMemsetAsync(p->d.split_cnt, 0, sizeof(unsigned int), st) ||
      cudaMemsetAsync(p->d.part, 0, sizeof(double) * 2 * p->nbusb, st))
    return fail("workspace initialisation");
  const size_t smem = (size_t)p->bw * branch_warp_bytes(p->grp);
  if (cudaFuncSetAttribute(branch_kernel(p->grp),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
    return fail("cudaFuncSetAttribute");
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking)) return fail("stream");
  if (cudaStreamSynchronize(st)) return fail("synchronisation");
  tron_err_t e = capture(p, 1, &p->g1);
  if (e == TRON_OK) e = capture(p, kGraphChunk, &p->gc);
  if (e != TRON_OK) {
    admm_pool_destroy(p);
    return e;
  }
  p->ab.init(cb);
  p->al.init(cl);
  p->ag.init(cg);
  p->inst.assign(cap_instances, admm_pool::Inst{false, 0, 0, 0, 0, 0, 0, 0, 0, 0});
  *out = p;
  return TRON_OK;
}

tron_err_t admm_pool_add(admm_pool_t* p, const admm_network_t* net, int32_t* id, void* stream) {
  clear_error();
  XT_REQUIRE(p && net && id, TRON_EINVAL, "admm_pool_add: null argument");
  *id = -1;
  const int nb = net->nbus, nl = net->nbranch, ng = net->ngen;
  XT_REQUIRE(nb > 0 && nl >= 0 && ng >= 0, TRON_EINVAL, "admm_pool_add: bad sizes");
  XT_REQUIRE(net->rho > 0.0 && net->vmin <= net->vmax, TRON_EINVAL,
             "admm_pool_add: need rho > 0 and vmin <= vmax");
  for (int k = 0; k < nl; ++k)
    XT_REQUIRE(net->br_from[k] >= 0 && net->br_from[k] < nb && net->br_to[k] >= 0 &&
                   net->br_to[k] < nb && net->br_from[k] != net->br_to[k],
               TRON_EINVAL, "admm_pool_add: branch %d has bad end buses", k);
  for (int g = 0; g < ng; ++g)
    XT_REQUIRE(net->gen_bus[g] >= 0 && net->gen_bus[g] < nb, TRON_EINVAL,
               "admm_pool_add: generator %d has a bad bus", g);
  int slot = -1;
  for (int i = 0; i < (int)p->inst.size(); ++i)
    if (!p->inst[i].live) {
      slot = i;
      break;
    }
  if (slot < 0) {
    set_error("admm_pool_add: all %d instance slots are live", (int)p->inst.size());
    return TRON_ENOMEM;
  }
  const int anb = align_up(nb), anl = align_up(nl), ang = align_up(ng);
  const int b0 = p->ab.take(anb);
  const int l0 = b0 < 0 ? -1 : p->al.take(anl);
  const int g0 = l0 < 0 ? -1 : p->ag.take(ang);
  if (b0 < 0 || l0 < 0 || g0 < 0) {
    if (b0 >= 0) p->ab.give(b0, anb);
    if (l0 >= 0) p->al.give(l0, anl);
    set_error("admm_pool_add: no free slot ranges for %d buses, %d branches, %d generators",
              nb, nl, ng);
    return TRON_ENOMEM;
  }
  // host images of the instance's slot ranges (global slot indices)
  std::vector<int32_t> bfrom(anl, 0), bto(anl, 0), binst(anl, -1);
  std::vector<double> coef(8 * (size_t)anl, 0.0), smax2(anl, 0.0);
  for (int k = 0; k < nl; ++k) {
    bfrom[k] = b0 + net->br_from[k];
    bto[k] = b0 + net->br_to[k];
    binst[k] = slot;
    for (int q = 0; q < 8; ++q) coef[8 * (size_t)k + q] = net->br_coef[8 * (size_t)k + q];
    smax2[k] = net->br_smax2[k];
  }
  std::vector<int32_t> gbus(ang, 0), ginst(ang, -1);
  std::vector<double> gc2(ang, 0.0), gc1(ang, 0.0), gpmin(ang, 0.0), gpmax(ang, 0.0),
      gqmin(ang, 0.0), gqmax(ang, 0.0);
  for (int g = 0; g < ng; ++g) {
    gbus[g] = b0 + net->gen_bus[g];
    ginst[g] = slot;
    gc2[g] = net->gen_c2[g];
    gc1[g] = net->gen_c1[g];
    gpmin[g] = net->gen_pmin[g];
    gpmax[g] = net->gen_pmax[g];
    gqmin[g] = net->gen_qmin[g];
    gqmax[g] = net->gen_qmax[g];
  }
  // incidence lists, ends and generators in increasing id per bus
  std::vector<int32_t> ecnt(anb, 0), gcnt(anb, 0), eoff(anb, 0), goff(anb, 0);
  for (int k = 0; k < nl; ++k) {
    ecnt[net->br_from[k]]++;
    ecnt[net->br_to[k]]++;
  }
  for (int g = 0; g < ng; ++g) gcnt[net->gen_bus[g]]++;
  {
    int ae = 2 * l0, ag = g0;
    for (int b = 0; b < anb; ++b) {
      eoff[b] = ae;
      goff[b] = ag;
      ae += ecnt[b];
      ag += gcnt[b];
    }
  }
  std::vector<int32_t> elist(2 * (size_t)anl, 0), glist(ang, 0);
  {
    std::vector<int32_t> fill(anb, 0);
    for (int e = 0; e < 2 * nl; ++e) {
      const int k = e / 2;
      const int bus = (e % 2 == 0) ? net->br_from[k] : net->br_to[k];
      elist[eoff[bus] - 2 * l0 + fill[bus]++] = 2 * (l0 + k) + (e % 2);
    }
    std::fill(fill.begin(), fill.end(), 0);
    for (int g = 0; g < ng; ++g) {
      const int bus = net->gen_bus[g];
      glist[goff[bus] - g0 + fill[bus]++] = g0 + g;
    }
  }
  std::vector<int32_t> binst_bus(anb, -1);
  std::vector<double> pd(anb, 0.0), qd(anb, 0.0), gsh(anb, 0.0), bsh(anb, 0.0);
  for (int b = 0; b < nb; ++b) {
    binst_bus[b] = slot;
    pd[b] = net->bus_pd[b];
    qd[b] = net->bus_qd[b];
    gsh[b] = net->bus_gsh[b];
    bsh[b] = net->bus_bsh[b];
  }
  cudaStream_t st = (cudaStream_t)stream;
  auto up = [&](void* dst, const void* src, size_t bytes) -> bool {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = true;
  ok = ok && up(p->d.br_from + l0, bfrom.data(), 4 * (size_t)anl);
  ok = ok && up(p->d.br_to + l0, bto.data(), 4 * (size_t)anl);
  ok = ok && up(p->d.br_coef + 8 * (size_t)l0, coef.data(), 64 * (size_t)anl);
  ok = ok && up(p->d.br_smax2 + l0, smax2.data(), 8 * (size_t)anl);
  ok = ok && up(p->d.gen_bus + g0, gbus.data(), 4 * (size_t)ang);
  ok = ok && up(p->d.gen_c2 + g0, gc2.data(), 8 * (size_t)ang);
  ok = ok && up(p->d.gen_c1 + g0, gc1.data(), 8 * (size_t)ang);
  ok = ok && up(p->d.gen_pmin + g0, gpmin.data(), 8 * (size_t)ang);
  ok = ok && up(p->d.gen_pmax + g0, gpmax.data(), 8 * (size_t)ang);
  ok = ok && up(p->d.gen_qmin + g0, gqmin.data(), 8 * (size_t)ang);
  ok = ok && up(p->d.gen_qmax + g0, gqmax.data(), 8 * (size_t)ang);
  ok = ok && up(p->d.bus_eoff + b0, eoff.data(), 4 * (size_t)anb);
  ok = ok && up(p->d.bus_ecnt + b0, ecnt.data(), 4 * (size_t)anb);
  ok = ok && up(p->d.bus_goff + b0, goff.data(), 4 * (size_t)anb);
  ok = ok && up(p->d.bus_gcnt + b0, gcnt.data(), 4 * (size_t)anb);
  ok = ok && up(p->d.bus_pd + b0, pd.data(), 8 * (size_t)anb);
  ok = ok && up(p->d.bus_qd + b0, qd.data(), 8 * (size_t)anb);
  ok = ok && up(p->d.bus_gsh + b0, gsh.data(), 8 * (size_t)anb);
  ok = ok && up(p->d.bus_bsh + b0, bsh.data(), 8 * (size_t)anb);
  ok = ok && up(p->d.end_list + 2 * (size_t)l0, elist.data(), 8 * (size_t)anl);
  ok = ok && up(p->d.gen_list + g0, glist.data(), 4 * (size_t)ang);
  // membership last: the slots join the iteration once everything else is in place
  ok = ok && up(p->d.br_inst + l0, binst.data(), 4 * (size_t)anl);
  ok = ok && up(p->d.gen_inst + g0, ginst.data(), 4 * (size_t)ang);
  ok = ok && up(p->d.bus_inst + b0, binst_bus.data(), 4 * (size_t)anb);
  const double param[4] = {net->rho, net->rho_line, net->vmin, net->vmax};
  const int32_t blk[2] = {b0 / kBusThreads, (b0 + anb) / kBusThreads};
  const int64_t zero64 = 0;
  ok = ok && up(p->d.inst_param + 4 * (size_t)slot, param, sizeof(param));
  ok = ok && up(p->d.inst_blk + 2 * (size_t)slot, blk, sizeof(blk));
  ok = ok && up(p->d.inst_iter + slot, &zero64, sizeof(zero64));
  const int32_t zero32 = 0;
  ok = ok && up(p->d.inst_flags + slot, &zero32, sizeof(zero32));
  if (ok) {
    AdmmArgs a = make_args(p);
    const int m = std::max(anl, std::max(ang, anb));
    k_admm_init<<<(m + 127) / 128, 128, 0, st>>>(a, l0, l0 + anl, g0, g0 + ang, b0, b0 + anb);
    ok = cudaGetLastError() == cudaSuccess;
  }
  const int32_t one = 1;
  ok = ok && up(p->d.inst_active + slot, &one, sizeof(one));
  if (!ok) {
    p->ab.give(b0, anb);
    p->al.give(l0, anl);
    p->ag.give(g0, ang);
    set_error("admm_pool_add: upload failed: %s", cudaGetErrorString(cudaGetLastError()));
    return TRON_ECUDA;
  }
  p->inst[slot] = admm_pool::Inst{true, b0, anb, l0, anl, g0, ang, nb, nl, ng};
  p->live++;
  *id = slot;
  return TRON_OK;
}

tron_err_t admm_pool_remove(admm_pool_t* p, int32_t id, void* stream) {
  clear_error();
  XT_REQUIRE(p && id >= 0 && id < (int)p->inst.size() && p->inst[id].live, TRON_EINVAL,
             "admm_pool_remove: %d is not a live instance", id);
  cudaStream_t st = (cudaStream_t)stream;
  auto& I = p->inst[id];
  const int32_t zero = 0;
  XT_CUDA(cudaMemcpyAsync(p->d.inst_active + id, &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
  XT_CUDA(cudaMemsetAsync(p->d.br_inst + I.l0, 0xFF, 4 * (size_t)I.nl, st));
  XT_CUDA(cudaMemsetAsync(p->d.gen_inst + I.g0, 0xFF, 4 * (size_t)I.ng, st));
  XT_CUDA(cudaMemsetAsync(p->d.bus_inst + I.b0, 0xFF, 4 * (size_t)I.nb, st));
  XT_CUDA(cudaMemsetAsync(p->d.bus_ecnt + I.b0, 0, 4 * (size_t)I.nb, st));
  XT_CUDA(cudaMemsetAsync(p->d.bus_gcnt + I.b0, 0, 4 * (size_t)I.nb, st));
  p->ab.give(I.b0, I.nb);
  p->al.give(I.l0, I.nl);
  p->ag.give(I.g0, I.ng);
  I.live = false;
  p->live--;
  return TRON_OK;
}

tron_err_t admm_pool_step(admm_pool_t* p, int32_t n_iters, void* stream) {
  clear_error();
  XT_REQUIRE(p && n_iters >= 0, TRON_EINVAL, "admm_pool_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  int left = n_iters;
  while (left >= kGraphChunk) {
    XT_CUDA(cudaGraphLaunch(p->gc, st));
    left -= kGraphChunk;
  }
  while (left-- > 0) XT_CUDA(cudaGraphLaunch(p->g1, st));
  return TRON_OK;
}

tron_err_t admm_pool_residuals(admm_pool_t* p, int64_t* h_iter, double* h_primal,
                               double* h_dual, void* stream) {
  clear_error();
  XT_REQUIRE(p && h_iter && h_primal && h_dual, TRON_EINVAL, "admm_pool_residuals: null");
  cudaStream_t st = (cudaStream_t)stream;
  const int ci = p->d.cap_inst;
  k_admm_latest<<<(ci + 127) / 128, 128, 0, st>>>(p->d);
  XT_CUDA(cudaGetLastError());
  std::vector<double> res(2 * (size_t)ci);
  XT_CUDA(cudaMemcpyAsync(h_iter, p->d.lat_iter, 8 * (size_t)ci, cudaMemcpyDeviceToHost, st));
  XT_CUDA(cudaMemcpyAsync(res.data(), p->d.lat_res, 16 * (size_t)ci, cudaMemcpyDeviceToHost, st));
  XT_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < ci; ++i) {
    h_primal[i] = res[2 * i];
    h_dual[i] = res[2 * i + 1];
  }
  return TRON_OK;
}

tron_err_t admm_pool_history(admm_pool_t* p, int32_t id, int64_t first, int64_t count,
                             double* h_primal, double* h_dual, void* stream) {
  clear_error();
  XT_REQUIRE(p && id >= 0 && id < (int)p->inst.size() && p->inst[id].live, TRON_EINVAL,
             "admm_pool_history: %d is not a live instance", id);
  XT_REQUIRE(count >= 0 && first >= 0 && h_primal && h_dual, TRON_EINVAL,
             "admm_pool_history: bad range");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t it = 0;
  XT_CUDA(cudaMemcpyAsync(&it, p->d.inst_iter + id, 8, cudaMemcpyDeviceToHost, st));
  XT_CUDA(cudaStreamSynchronize(st));
  XT_REQUIRE(first + count <= it && first >= it - p->d.H, TRON_EINVAL,
             "admm_pool_history: iterations [%lld, %lld) not in the last %d of %lld",
             (long long)first, (long long)(first + count), p->d.H, (long long)it);
  std::vector<double> buf(2 * (size_t)p->d.H);
  XT_CUDA(cudaMemcpy(buf.data(), p->d.hist + (size_t)id * p->d.H * 2, 16 * (size_t)p->d.H,
                     cudaMemcpyDeviceToHost));
  for (int64_t t = 0; t < count; ++t) {
    const size_t s = (size_t)((first + t) % p->d.H);
    h_primal[t] = buf[2 * s];
    h_dual[t] = buf[2 * s + 1];
  }
  return TRON_OK;
}

static tron_err_t state_xfer(admm_pool_t* p, int32_t id, admm_state_view_t* h, bool to_host,
                             cudaStream_t st) {
  XT_REQUIRE(p && h && id >= 0 && id < (int)p->inst.size() && p->inst[id].live, TRON_EINVAL,
             "admm state: %d is not a live instance", id);
  const auto& I = p->inst[id];
  const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
  auto x = [&](void* dev, void* host, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return to_host ? cudaMemcpyAsync(host, dev, bytes, kind, st)
                   : cudaMemcpyAsync(dev, host, bytes, kind, st);
  };
  const size_t L = I.nbranch, B = I.nbus, G = I.ngen;
  XT_CUDA(x(p->d.br_x + 4 * (size_t)I.l0, h->br_x, 32 * L));
  XT_CUDA(x(p->d.br_delta + I.l0, h->br_delta, 8 * L));
  XT_CUDA(x(p->d.br_lam + 8 * (size_t)I.l0, h->br_lam, 64 * L));
  XT_CUDA(x(p->d.br_val + 8 * (size_t)I.l0, h->br_val, 64 * L));
  XT_CUDA(x(p->d.br_tilde + 4 * (size_t)I.l0, h->br_tilde, 32 * L));
  XT_CUDA(x(p->d.bus_w + I.b0, h->bus_w, 8 * B));
  XT_CUDA(x(p->d.bus_th + I.b0, h->bus_th, 8 * B));
  XT_CUDA(x(p->d.gen_pq + 2 * (size_t)I.g0, h->gen_pq, 16 * G));
  XT_CUDA(x(p->d.gen_lam + 2 * (size_t)I.g0, h->gen_lam, 16 * G));
  XT_CUDA(x(p->d.gen_tilde + 2 * (size_t)I.g0, h->gen_tilde, 16 * G));
  XT_CUDA(x(p->d.inst_iter + id, &h->iteration, 8));
  XT_CUDA(cudaStreamSynchronize(st));
  return TRON_OK;
}

tron_err_t admm_pool_get_state(admm_pool_t* p, int32_t id, admm_state_view_t* host,
                               void* stream) {
  clear_error();
  return state_xfer(p, id, host, true, (cudaStream_t)stream);
}

tron_err_t admm_pool_set_state(admm_pool_t* p, int32_t id, const admm_state_view_t* host,
                               void* stream) {
  clear_error();
  return state_xfer(p, id, const_cast<admm_state_view_t*>(host), false, (cudaStream_t)stream);
}

int32_t admm_pool_live(const admm_pool_t* p) { return p ? p->live : 0; }

int32_t admm_pool_branch_group(const admm_pool_t* p) { return p ? p->grp : 0; }

void admm_pool_destroy(admm_pool_t* p) {
  if (!p) return;
  if (p->g1) cudaGraphExecDestroy(p->g1);
  if (p->gc) cudaGraphExecDestroy(p->gc);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (void* a : p->allocs) cudaFree(a);
  delete p;
}

// ------------------------------------------------------------------ single network
tron_err_t admm_create(admm_t** out, const admm_network_t* net, const tron_options_t* opt,
                       void* stream) {
  clear_error();
  XT_REQUIRE(out && net, TRON_EINVAL, "admm_create: null argument");
  *out = nullptr;
  admm_pool_t* p = nullptr;
  tron_err_t e = admm_pool_create(&p, net->nbus, net->nbranch, net->ngen, 1, 1 << 16, opt,
                                  stream);
  if (e != TRON_OK) return e;
  int32_t id = -1;
  e = admm_pool_add(p, net, &id, stream);
  if (e != TRON_OK) {
    admm_pool_destroy(p);
    return e;
  }
  *out = p;
  return TRON_OK;
}

tron_err_t admm_step(admm_t* a, int32_t n_iters, double* h_primal, double* h_dual,
                     void* stream) {
  tron_err_t e = admm_pool_step(a, n_iters, stream);
  if (e != TRON_OK || (!h_primal && !h_dual)) return e;
  int64_t it = 0;
  double pr = 0.0, du = 0.0;
  e = admm_pool_residuals(a, &it, &pr, &du, stream);
  if (e != TRON_OK) return e;
  if (h_primal) *h_primal = pr;
  if (h_dual) *h_dual = du;
  return TRON_OK;
}

tron_err_t admm_residual_history(admm_t* a, int64_t first, int64_t count, double* h_primal,
                                 double* h_dual, void* stream) {
  return admm_pool_history(a, 0, first, count, h_primal, h_dual, stream);
}

tron_err_t admm_get_state(admm_t* a, admm_state_view_t* host, void* stream) {
  return admm_pool_get_state(a, 0, host, stream);
}

tron_err_t admm_set_state(admm_t* a, const admm_state_view_t* host, void* stream) {
  return admm_pool_set_state(a, 0, host, stream);
}

// ---------------------------------------------------------------- multi-period
}  // extern "C"

struct admm_mp {
  admm_pool* pool;
  int T, ngen;
  std::vector<int32_t> inst;   // pool instance of each period
  int32_t* d_g0;               // [T] first generator slot of each period
  tron_batch_t* tb;            // the generator chains: ngen problems of T periods
  double *d_rec, *d_lo, *d_hi, *d_x, *d_delta, *d_f, *d_pg;
  int32_t *d_iters, *d_status;
  // the generator chains run on a side stream beside the branch launch (the two touch
  // disjoint data: the flagged periods' generators are skipped by the branch kernel), and
  // the bus kernel waits for both
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  std::vector<void*> allocs;
};

extern "C" {

void admm_mp_destroy(admm_mp_t* mp) {
  if (!mp) return;
  if (mp->tb) tron_batch_destroy(mp->tb);
  if (mp->pool) admm_pool_destroy(mp->pool);
  for (void* a : mp->allocs) cudaFree(a);
  if (mp->ev_fork) cudaEventDestroy(mp->ev_fork);
  if (mp->ev_join) cudaEventDestroy(mp->ev_join);
  if (mp->side) cudaStreamDestroy(mp->side);
  delete mp;
}

tron_err_t admm_mp_create(admm_mp_t** out, const admm_network_t* net, int32_t T,
                          const double* h_load_scale, const double* h_ramp, double rho_ramp,
                          const tron_options_t* opt, void* stream) {
  clear_error();
  XT_REQUIRE(out && net && h_load_scale && h_ramp, TRON_EINVAL, "admm_mp_create: null argument");
  *out = nullptr;
  XT_REQUIRE(T >= 1 && T <= 32, TRON_EINVAL, "admm_mp_create: T = %d not in [1, 32]", (int)T);
  XT_REQUIRE(rho_ramp >= 0.0, TRON_EINVAL, "admm_mp_create: rho_ramp < 0");
  for (int t = 0; t < T; ++t)
    XT_REQUIRE(h_load_scale[t] > 0.0 && isfinite(h_load_scale[t]), TRON_EINVAL,
               "admm_mp_create: load scale %d must be positive", t);
  const int ng = net->ngen;
  for (int g = 0; g < ng; ++g)
    XT_REQUIRE(h_ramp[g] >= 0.0, TRON_EINVAL, "admm_mp_create: ramp of generator %d < 0", g);
  cudaStream_t st = (cudaStream_t)stream;
  admm_mp* mp = new admm_mp();
  mp->pool = nullptr;
  mp->tb = nullptr;
  mp->side = nullptr;
  mp->ev_fork = nullptr;
  mp->ev_join = nullptr;
  mp->T = T;
  mp->ngen = ng;
  auto fail = [&](tron_err_t e) {
    admm_mp_destroy(mp);
    return e;
  };
  tron_err_t e = admm_pool_create(&mp->pool, T * align_up(net->nbus), T * align_up(net->nbranch),
                                  T * align_up(ng), T, 1 << 12, opt, stream);
  if (e != TRON_OK) return fail(e);
  std::vector<double> pd(net->nbus), qd(net->nbus);
  std::vector<int32_t> g0(T);
  for (int t = 0; t < T; ++t) {
    for (int b = 0; b < net->nbus; ++b) {
      pd[b] = net->bus_pd[b] * h_load_scale[t];
      qd[b] = net->bus_qd[b] * h_load_scale[t];
    }
    admm_network_t nt = *net;
    nt.bus_pd = pd.data();
    nt.bus_qd = qd.data();
    int32_t id = -1;
    e = admm_pool_add(mp->pool, &nt, &id, stream);
    if (e != TRON_OK) return fail(e);
    if (cudaStreamSynchronize(st) != cudaSuccess) {  // pd, qd are reused
      set_error("admm_mp_create: synchronisation failed");
      return fail(TRON_ECUDA);
    }
    mp->inst.push_back(id);
    g0[t] = mp->pool->inst[id].g0;
    const int32_t flag = 1;  // this period's generators are the chains' business
    if (cudaMemcpy(mp->pool->d.inst_flags + id, &flag, sizeof(flag), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      set_error("admm_mp_create: upload failed");
      return fail(TRON_ECUDA);
    }
  }
  // the chains' arrays: records with their constant header, bounds, warm radius 1
  const size_t rs = 8 + 2 * (size_t)T, ngs = (size_t)std::max(ng, 1);
  auto alloc = [&](void** ptr, size_t bytes) {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
    mp->allocs.push_back(*ptr);
    return true;
  };
  // launch order of the branch slots: the T period copies of each line side by side, so
  // that a warp's lanes hold the same line under neighbouring loads -- problems that take
  // nearly the same path through the solver, which the warp then runs together (each
  // problem's arithmetic, so its bits, do not depend on its lane)
  {
    const int cap = mp->pool->d.cap_br, nl = net->nbranch;
    std::vector<int32_t> ord(cap, -1);
    for (int r = 0; r < T * nl; ++r) ord[r] = mp->pool->inst[mp->inst[r % T]].l0 + r / T;
    int32_t* d_ord = nullptr;
    if (!alloc((void**)&d_ord, 4 * (size_t)cap)) {
      set_error("admm_mp_create: cudaMalloc failed");
      return fail(TRON_ENOMEM);
    }
    if (cudaMemcpy(d_ord, ord.data(), 4 * (size_t)cap, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("admm_mp_create: order upload failed");
      return fail(TRON_ECUDA);
    }
    mp->pool->d.br_order = d_ord;
  }
  if (!alloc((void**)&mp->d_g0, 4 * (size_t)T) || !alloc((void**)&mp->d_rec, 8 * rs * ngs) ||
      !alloc((void**)&mp->d_lo, 8 * (size_t)T * ngs) || !alloc((void**)&mp->d_hi, 8 * (size_t)T * ngs) ||
      !alloc((void**)&mp->d_x, 8 * (size_t)T * ngs) || !alloc((void**)&mp->d_delta, 8 * ngs) ||
      !alloc((void**)&mp->d_f, 8 * ngs) || !alloc((void**)&mp->d_pg, 8 * ngs) ||
      !alloc((void**)&mp->d_iters, 4 * ngs) || !alloc((void**)&mp->d_status, 4 * ngs)) {
    set_error("admm_mp_create: cudaMalloc failed");
    return fail(TRON_ENOMEM);
  }
  std::vector<double> rec(rs * ngs, 0.0), lo((size_t)T * ngs), hi((size_t)T * ngs), dl(ngs, 1.0);
  for (int g = 0; g < ng; ++g) {
    double* r = rec.data() + rs * g;
    r[0] = net->gen_c2[g];
    r[1] = net->gen_c1[g];
    r[2] = net->rho;
    r[3] = rho_ramp;
    r[4] = h_ramp[g];
    for (int t = 0; t < T; ++t) {
      lo[(size_t)T * g + t] = net->gen_pmin[g];
      hi[(size_t)T * g + t] = net->gen_pmax[g];
    }
  }
  std::vector<int32_t> status0(ngs, 0);
  if (cudaMemcpy(mp->d_g0, g0.data(), 4 * (size_t)T, cudaMemcpyHostToDevice) ||
      cudaMemcpy(mp->d_rec, rec.data(), 8 * rs * ngs, cudaMemcpyHostToDevice) ||
      cudaMemcpy(mp->d_lo, lo.data(), 8 * (size_t)T * ngs, cudaMemcpyHostToDevice) ||
      cudaMemcpy(mp->d_hi, hi.data(), 8 * (size_t)T * ngs, cudaMemcpyHostToDevice) ||
      cudaMemcpy(mp->d_delta, dl.data(), 8 * ngs, cudaMemcpyHostToDevice) ||
      cudaMemcpy(mp->d_status, status0.data(), 4 * ngs, cudaMemcpyHostToDevice)) {
    set_error("admm_mp_create: upload failed");
    return fail(TRON_ECUDA);
  }
  tron_options_t o;
  if (opt) o = *opt;
  else tron_options_default(&o);
  o.group = 0;
  o.layout = 0;
  o.schedule = TRON_SCHED_PERSISTENT;
  if (ng > 0) {
    e = tron_batch_create(&mp->tb, TRON_OBJ_GEN_RAMP, ng, nullptr, T, &o, stream);
    if (e != TRON_OK) return fail(e);
  }
  if (cudaStreamCreateWithFlags(&mp->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&mp->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&mp->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    set_error("admm_mp_create: stream or event creation failed");
    return fail(TRON_ECUDA);
  }
  *out = mp;
  return TRON_OK;
}

int32_t admm_mp_launches_per_iteration(const admm_mp_t* mp) {
  if (!mp) return 0;
  return admm_pool_launches_per_iteration(mp->pool) + (mp->ngen > 0 ? 3 : 0);
}

tron_err_t admm_mp_step(admm_mp_t* mp, int32_t n_iters, double* h_primal, double* h_dual,
                        void* stream) {
  clear_error();
  XT_REQUIRE(mp && n_iters >= 0, TRON_EINVAL, "admm_mp_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  admm_pool* p = mp->pool;
  AdmmArgs a = make_args(p);
  void* args[] = {&a};
  const size_t smem = (size_t)p->bw * branch_warp_bytes(p->grp);
  const int nthr = mp->ngen * mp->T;
  for (int it = 0; it < n_iters; ++it) {
    // the generator chains of all periods on the side stream ...
    if (nthr > 0) {
      XT_CUDA(cudaEventRecord(mp->ev_fork, st));
      XT_CUDA(cudaStreamWaitEvent(mp->side, mp->ev_fork, 0));
      k_mp_gather<<<(nthr + 127) / 128, 128, 0, mp->side>>>(p->d, mp->d_g0, mp->T, mp->ngen,
                                                            mp->d_rec, mp->d_x);
      XT_CUDA(cudaGetLastError());
      tron_err_t e = tron_batch_solve(mp->tb, mp->d_rec, mp->d_lo, mp->d_hi, mp->d_x,
                                      mp->d_delta, mp->d_f, mp->d_pg, mp->d_iters,
                                      mp->d_status, (void*)mp->side);
      if (e != TRON_OK) return e;
      k_mp_scatter<<<(nthr + 127) / 128, 128, 0, mp->side>>>(p->d, mp->d_g0, mp->T, mp->ngen,
                                                             mp->d_x);
      XT_CUDA(cudaGetLastError());
      XT_CUDA(cudaEventRecord(mp->ev_join, mp->side));
    }
    // ... beside the branches (the flagged periods' generators are skipped there) ...
    XT_CUDA(cudaLaunchKernel(branch_kernel(p->grp), dim3(p->nbb + p->ngb),
                             dim3(p->bw * 32), args, smem, st));
    if (p->split > 0)
      XT_CUDA(cudaLaunchKernel((const void*)k_admm_branch_tail, dim3(p->ntb), dim3(32), args,
                               branch_warp_bytes(4), st));
    // ... then the buses, multipliers and residuals of every period, after both
    if (nthr > 0) XT_CUDA(cudaStreamWaitEvent(st, mp->ev_join, 0));
    XT_CUDA(cudaLaunchKernel((const void*)k_admm_bus, dim3(p->nbusb), dim3(kBusThreads), args,
                             0, st));
  }
  if (!h_primal && !h_dual) return TRON_OK;
  const int ci = p->d.cap_inst;
  std::vector<int64_t> its(ci);
  std::vector<double> pr(ci), du(ci);
  tron_err_t e = admm_pool_residuals(p, its.data(), pr.data(), du.data(), stream);
  if (e != TRON_OK) return e;
  double p2 = 0.0, d2 = 0.0;
  for (int t = 0; t < mp->T; ++t) {
    p2 += pr[mp->inst[t]] * pr[mp->inst[t]];
    d2 += du[mp->inst[t]] * du[mp->inst[t]];
  }
  if (h_primal) *h_primal = sqrt(p2);
  if (h_dual) *h_dual = sqrt(d2);
  return TRON_OK;
}

tron_err_t admm_mp_get_state(admm_mp_t* mp, int32_t period, admm_state_view_t* host,
                             void* stream) {
  clear_error();
  XT_REQUIRE(mp && period >= 0 && period < mp->T, TRON_EINVAL,
             "admm_mp_get_state: bad period");
  return admm_pool_get_state(mp->pool, mp->inst[period], host, stream);
}

tron_err_t admm_mp_gen_status_counts(admm_mp_t* mp, int64_t* h_counts6, void* stream) {
  clear_error();
  XT_REQUIRE(mp && h_counts6, TRON_EINVAL, "admm_mp_gen_status_counts: bad argument");
  std::vector<int32_t> st((size_t)std::max(mp->ngen, 1));
  cudaStream_t s = (cudaStream_t)stream;
  if (mp->ngen > 0)
    XT_CUDA(cudaMemcpyAsync(st.data(), mp->d_status, 4 * (size_t)mp->ngen,
                            cudaMemcpyDeviceToHost, s));
  XT_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 6; ++k) h_counts6[k] = 0;
  for (int g = 0; g < mp->ngen; ++g)
    if (st[g] >= 0 && st[g] < 6) h_counts6[st[g]]++;
  return TRON_OK;
}

tron_err_t admm_branch_status_counts(admm_t* a, int64_t* h_counts6, void* stream) {
  clear_error();
  XT_REQUIRE(a && h_counts6 && !a->inst.empty() && a->inst[0].live, TRON_EINVAL,
             "admm_branch_status_counts: bad argument");
  const auto& I = a->inst[0];
  std::vector<int32_t> st(I.nbranch > 0 ? I.nbranch : 1);
  cudaStream_t s = (cudaStream_t)stream;
  if (I.nbranch > 0) {
    XT_CUDA(cudaMemcpyAsync(st.data(), a->d.br_status + I.l0, 4 * (size_t)I.nbranch,
                            cudaMemcpyDeviceToHost, s));
  }
  XT_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 6; ++k) h_counts6[k] = 0;
  for (int k = 0; k < I.nbranch; ++k)
    if (st[k] >= 0 && st[k] < 6) h_counts6[st[k]]++;
  return TRON_OK;
}

int64_t admm_iterations(const admm_t* a) {
  if (!a) return 0;
  int64_t it = 0;
  if (cudaMemcpy(&it, a->d.inst_iter, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return it;
}

int64_t admm_history_capacity(const admm_t* a) { return a ? a->d.H : 0; }

void admm_destroy(admm_t* a) { admm_pool_destroy(a); }

}  // extern "C"
