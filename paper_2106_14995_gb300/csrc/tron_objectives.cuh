// tron_objectives.cuh -- device evaluators of f, grad f and the Hessian (Algorithm 1).
//
// Interface used by the solver (tron_solver.cuh):
//   SMEM                doubles of per-problem shared memory the evaluator needs
//   kHasHd              the Hessian is hq(i,j) + [i==j] hd(i)
//   load(gp, rec, n)    stage the packed record; returns false when an entry that enters
//                       f at every point is not finite (f is then not finite anywhere,
//                       so the solve stops as TRON_NONFINITE); entries that enter f only
//                       on part of the box (a penalty's limit and weight) are left to
//                       the evaluation, as f itself decides there
//   eval_f(gp, y)       f(y); caches what the gradient needs; sets fsc, the sum of the
//                       magnitudes of the terms f is assembled from (its rounding scale)
//   kStepEval           eval_f_step(gp, y, s, Hs) is available: f(y) at y = x + s from
//                       the product Hs = H(x) s the solver already holds
//   grad_hess(gp, x, g) gradient at the point of the last eval_f, Hessian made current
//   hq(i,j), hd(i)      Hessian entries at the current point
//   hess_finite(gp)     all Hessian entries finite
#pragma once

#include "tron_common.cuh"

namespace xt {

// ------------------------------------------------------------------ dense quartic
// f = 1/2 x'Qx + c'x + sum_i d_i x_i^4, record [Q (n x n) | c | d], Q symmetric.
// Storage of Q (QL):
//   kQShared: staged once in shared memory (odd stride, conflict-free columns).
//   kQGlobal: left in global memory (L2-resident while the problem runs) and read
//             column-wise -- Q(i, j) as Q[j][i] -- so the lanes of a group read
//             consecutive doubles; used where the factor alone fills the shared memory.
//   kQDiag:   (one variable per lane, G = N <= 32) the wrapped diagonals
//             D_k[i] = Q(i, (i + k) mod n), k = 0..n/2, in shared memory: about half of
//             kQShared, so more problems fit on an SM.  Q(i, j) for (j - i) mod n > n/2 is
//             D_{n-k}[j] by symmetry; a product walks the diagonals, and every access of
//             the group is a rotation of one diagonal (conflict free).
// The Hessian is Q + diag(12 d_i x_i^2), kept as Q plus a diagonal vector.
enum { kQShared = 0, kQGlobal = 1, kQDiag = 2 };

template <int N, int G, int QL = kQShared>
struct DenseObj {
  static_assert(QL != kQDiag || (G == N && N <= 32), "diagonal storage needs G = N <= 32");
  static constexpr int R = N / G;
  static constexpr int LDQ = (G == 1) ? N : N + 1;
  static constexpr int QSZ = QL == kQShared ? N * LDQ : (QL == kQDiag ? N * (N / 2 + 1) : 0);
  static constexpr int SMEM = QSZ + 2 * N;  // Q, hd, staging
  static constexpr bool kHasHd = true;
  static constexpr bool kStepEval = true;

  SV<G> Q, hdg, st;
  const double* __restrict__ qg;
  double c[R], d[R], qy[R];
  double qx[R];  // Q x at the current (accepted) point
  double fsc;
  int n;

  __device__ __forceinline__ void bind(SV<G> base) {
    Q = base;
    hdg = base.at(QSZ);
    st = base.at(QSZ + N);
  }

  template <class GP>
  __device__ __forceinline__ bool load(const GP& gp, const double* __restrict__ rec, int n_) {
    n = n_;
    qg = rec;
    bool fin = true;
    const int nn = n * n;
    if constexpr (QL == kQGlobal) {
      for (int e = gp.t; e < nn; e += G) fin = fin && finite_bits(__ldg(rec + e));
    } else if constexpr (QL == kQDiag) {
      // lane i gathers D_k[i] = Q(i, (i + k) mod n); entries outside n x n are zero
      for (int e = gp.t; e < nn; e += G) fin = fin && finite_bits(__ldg(rec + e));
      const int i = gp.t;
#pragma unroll 4
      for (int k = 0; k <= N / 2; ++k) {
        double v = 0.0;
        if (i < n && 2 * k <= n) {
          int j = i + k;
          if (j >= n) j -= n;
          v = __ldg(rec + i * n + j);
        }
        Q[k * N + i] = v;
      }
    } else {
      // zero the padding rows/columns, then copy Q (coalesced over the group)
      for (int e = gp.t; e < N * LDQ; e += G) Q[e] = 0.0;
      gp.sync();
      for (int e = gp.t; e < nn; e += G) {
        double v = __ldg(rec + e);
        fin = fin && finite_bits(v);
        int i = e / n, j = e - i * n;
        Q[i * LDQ + j] = v;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int i = r * G + gp.t;
      c[r] = (i < n) ? __ldg(rec + nn + i) : 0.0;
      d[r] = (i < n) ? __ldg(rec + nn + n + i) : 0.0;
      fin = fin && finite_bits(c[r]) && finite_bits(d[r]);
      hdg[i] = 0.0;
    }
    gp.sync();
    return !gp.any(!fin);
  }

  // sum_j Q(i, j) v[j] for row i of this lane (G >= 2; v staged in shared memory), two
  // independent FMA chains
  __device__ __forceinline__ double row_dot(int i, SV<G> v) const {
    double s0 = 0.0, s1 = 0.0;
    if constexpr (QL == kQDiag) {
      if (i < n) {
        // k = t <= n/2: D_t[i] v[(i + t) mod n]; k = t + n/2 + 1: Q(i, j) = D_{n-k}[j]
        const int h = n >> 1;
        int j0 = i, j1 = i + h + 1;
        if (j1 >= n) j1 -= n;
        for (int t = 0; t <= h; ++t) {
          s0 = fma(Q[t * N + i], v[j0], s0);
          if (t + h + 1 < n) s1 = fma(Q[(n - t - h - 1) * N + j1], v[j1], s1);
          j0 = (j0 + 1 == n) ? 0 : j0 + 1;
          j1 = (j1 + 1 == n) ? 0 : j1 + 1;
        }
      }
    } else {
      int j = 0;
      for (; j + 1 < n; j += 2) {
        s0 = fma(hq(i, j), v[j], s0);
        s1 = fma(hq(i, j + 1), v[j + 1], s1);
      }
      if (j < n) s0 = fma(hq(i, j), v[j], s0);
    }
    return s0 + s1;
  }

  // y_i = sum_j Q_ij v_j for the slots of this lane (v staged in st for G >= 2)
  template <class GP>
  __device__ __forceinline__ void qmul(const GP& gp, const double (&v)[R], double (&y)[R]) {
    if constexpr (G == 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(Q[i * LDQ + j], v[j], s);
        y[i] = s;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) st[r * G + gp.t] = v[r];
      gp.sync();
#pragma unroll
      for (int r = 0; r < R; ++r) y[r] = row_dot(r * G + gp.t, st);
      gp.sync();
    }
  }

  template <class GP>
  __device__ __forceinline__ double eval_f(const GP& gp, const double (&y)[R]) {
    qmul(gp, y, qy);
    return f_from_qy(gp, y);
  }

  // f(x + s) without a product with Q: Q (x + s) = Q x + H s - diag(hd) s, H and hd at x
  template <class GP>
  __device__ __forceinline__ double eval_f_step(const GP& gp, const double (&y)[R],
                                                const double (&s)[R], const double (&Hs)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) qy[r] = qx[r] + fma(-hdg[r * G + gp.t], s[r], Hs[r]);
    return f_from_qy(gp, y);
  }

  template <class GP>
  __device__ __forceinline__ double f_from_qy(const GP& gp, const double (&y)[R]) {
    double s = 0.0, m = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double y2 = y[r] * y[r];
      s += y[r] * (0.5 * qy[r] + c[r]) + d[r] * y2 * y2;
      m += 0.5 * fabs(y[r] * qy[r]) + fabs(c[r] * y[r]) + fabs(d[r]) * y2 * y2;
    }
    gp.sum2(s, m);
    fsc = m;
    return s;
  }

  template <class GP>
  __device__ __forceinline__ void grad_hess(const GP& gp, const double (&x)[R], double (&g)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double x2 = x[r] * x[r];
      qx[r] = qy[r];
      g[r] = qy[r] + c[r] + 4.0 * d[r] * x2 * x[r];
      hdg[r * G + gp.t] = 12.0 * d[r] * x[r] * x[r];
    }
    gp.sync();
  }

  __device__ __forceinline__ double hq(int i, int j) const {
    if constexpr (QL == kQGlobal) {
      return (i < n && j < n) ? __ldg(qg + (size_t)j * n + i) : 0.0;
    } else if constexpr (QL == kQDiag) {
      if (i >= n || j >= n) return 0.0;
      int k = j - i;
      if (k < 0) k += n;
      return (2 * k <= n) ? Q[k * N + i] : Q[(n - k) * N + j];
    } else {
      return Q[i * LDQ + j];
    }
  }
  __device__ __forceinline__ double hd(int i) const { return hdg[i]; }

  template <class GP>
  __device__ __forceinline__ bool hess_finite(const GP& gp) const {
    bool fin = true;
#pragma unroll
    for (int r = 0; r < R; ++r) fin = fin && finite_bits(hdg[r * G + gp.t]);
    return !gp.any(!fin);
  }
};

// -------------------------------------------------------------- ACOPF branch (n = 4)
// eq. exp-branch of Sec. 6.1 with the flows of eqs. pij-qji and the line-limit penalty,
// record [coefficients c[8] | lambda[8] | targets[8] | rho[8] | smax^2 | rho_line].
// Two mappings:
//   BranchObj<1>: one problem per lane; every lane evaluates its own branch, so the FP64
//                 pipe (including the sin/cos of theta_i - theta_j) runs with all 32
//                 lanes busy -- the most problems per FP64 instruction.
//   BranchObj<4>: one problem per four lanes; lane t owns variable t, flow t and the pair
//                 terms t and t + 4 and assembles row t of the Hessian.  A warp's
//                 duration is that of its slowest problem, and with one problem's work
//                 spread over four lanes that serial chain is much shorter: the mapping
//                 for launches with few problems per SM (an ADMM iteration's branches).
template <int G>
struct BranchObj;

template <>
struct BranchObj<1> {
  static constexpr int N = 4;
  static constexpr int R = 4;
  static constexpr int SMEM = 36 + 16;  // record, Hessian
  static constexpr bool kHasHd = false;
  static constexpr bool kStepEval = false;

  SV<1> rec, H;
  double cs, sn, F[4];
  double Fx[4];  // flows at the current (accepted) point
  double fsc;
  int n;

  __device__ __forceinline__ void bind(SV<1> base) {
    rec = base;
    H = base.at(36);
  }

  __device__ __forceinline__ bool load(const Grp<1>&, const double* __restrict__ src, int n_) {
    n = n_;
    bool fin = true;
#pragma unroll
    for (int k = 0; k < 34; ++k) {
      double v = __ldg(src + k);
      if (k < 32) fin = fin && finite_bits(v);  // smax^2, rho_line: only where a line is over
      rec[k] = v;
    }
    return fin;
  }

  __device__ __forceinline__ double eval_f(const Grp<1>&, const double (&y)[4]) {
    const double dth = y[2] - y[3];
    if (small_angle(dth)) {  // the usual case: the series (see sin_cos_small)
      sn = sin_cos_small(dth, false);
      cs = sin_cos_small(dth, true);
    } else {
      sincos(dth, &sn, &cs);
    }
    const double vi = y[0], vj = y[1];
    const double wi = vi * vi, wj = vj * vj;
    const double vv = vi * vj;
    const double wR = vv * cs, wI = vv * sn;
    F[0] = rec[0] * wi - rec[2] * wR + rec[3] * wI;
    F[1] = rec[1] * wi - rec[3] * wR - rec[2] * wI;
    F[2] = rec[4] * wj - rec[6] * wR - rec[7] * wI;
    F[3] = rec[5] * wj - rec[7] * wR + rec[6] * wI;
    const double P[8] = {F[0], F[1], F[2], F[3], wi, wj, y[2], y[3]};
    // magnitudes of the terms of each pair quantity (rounding scale of f)
    const double aR = fabs(wR), aI = fabs(wI);
    const double M[8] = {fabs(rec[0]) * wi + fabs(rec[2]) * aR + fabs(rec[3]) * aI,
                         fabs(rec[1]) * wi + fabs(rec[3]) * aR + fabs(rec[2]) * aI,
                         fabs(rec[4]) * wj + fabs(rec[6]) * aR + fabs(rec[7]) * aI,
                         fabs(rec[5]) * wj + fabs(rec[7]) * aR + fabs(rec[6]) * aI,
                         wi, wj, fabs(y[2]), fabs(y[3])};
    double val = 0.0, mag = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double r = P[k] - rec[16 + k];
      const double lam = rec[8 + k], rho = rec[24 + k];
      val += lam * r + 0.5 * rho * r * r;
      mag += fabs(lam * r) + 0.5 * rho * r * r + (fabs(lam) + rho * fabs(r)) * M[k];
    }
    const double smax2 = rec[32], rhol = rec[33];
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const double p2q2 = F[2 * dir] * F[2 * dir] + F[2 * dir + 1] * F[2 * dir + 1];
      const double m = p2q2 - smax2;
      if (positive_bits(m)) {
        val += 0.5 * rhol * m * m;
        mag += 0.5 * rhol * m * m + rhol * m * (p2q2 + smax2);
      }
    }
    fsc = mag;
    return val;
  }

  // gradient and Hessian at the point of the last eval_f.  Each pair quantity is
  // F_k = a_k w_i + b_k w_j + cR_k wR + cI_k wI (+ theta for k = 6, 7); the first-order
  // weights t_k = lambda_k + rho_k (F_k - target_k) are folded into four scalars that
  // multiply the second derivatives of w_i, w_j, wR, wI, and the Gauss-Newton part is
  // the sum of rho_k grad F_k grad F_k'.
  __device__ __forceinline__ void grad_hess(const Grp<1>&, const double (&x)[4], double (&g)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) Fx[k] = F[k];
    const double vi = x[0], vj = x[1];
    const double vv = vi * vj;
    const double wR = vv * cs, wI = vv * sn;
    const double wi = vi * vi, wj = vj * vj;
    // derivatives of wR, wI along (v_i, v_j, theta_i); along theta_j they are minus the
    // theta_i ones, and so are those of every flow
    const double dR[3] = {vj * cs, vi * cs, -wI};
    const double dI[3] = {vj * sn, vi * sn, wR};
    // coefficients (a, b, cR, cI) of the four flows
    const double co[4][4] = {{rec[0], 0.0, -rec[2], rec[3]},
                             {rec[1], 0.0, -rec[3], -rec[2]},
                             {0.0, rec[4], -rec[6], -rec[7]},
                             {0.0, rec[5], -rec[7], rec[6]}};
    double dF[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dF[k][0] = co[k][0] * (2.0 * vi) + co[k][2] * dR[0] + co[k][3] * dI[0];
      dF[k][1] = co[k][1] * (2.0 * vj) + co[k][2] * dR[1] + co[k][3] * dI[1];
      dF[k][2] = co[k][2] * dR[2] + co[k][3] * dI[2];
    }
    double t[8], W[4];
    {
      const double P[8] = {F[0], F[1], F[2], F[3], wi, wj, x[2], x[3]};
#pragma unroll
      for (int k = 0; k < 8; ++k) t[k] = rec[8 + k] + rec[24 + k] * (P[k] - rec[16 + k]);
#pragma unroll
      for (int k = 0; k < 4; ++k) W[k] = rec[24 + k];
    }
    // the six distinct entries (0,0) (0,1) (0,2) (1,1) (1,2) (2,2) of the Hessian without
    // the pair terms of the angles; the theta_j row follows by the sign rule above
    double E00 = 0.0, E01 = 0.0, E02 = 0.0, E11 = 0.0, E12 = 0.0, E22 = 0.0;
    const double smax2 = rec[32], rhol = rec[33];
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int kp = 2 * dir, kq = 2 * dir + 1;
      const double p = F[kp], q = F[kq];
      const double m = p * p + q * q - smax2;
      if (positive_bits(m)) {
        // (rho_l/2) m^2: first-order weight rho_l m grad m, grad m = 2p dp + 2q dq;
        // second order rho_l (grad m grad m' + m (2 dp dp' + 2p H_p + 2 dq dq' + 2q H_q))
        t[kp] += rhol * m * 2.0 * p;
        t[kq] += rhol * m * 2.0 * q;
        W[kp] += 2.0 * rhol * m;
        W[kq] += 2.0 * rhol * m;
        double gm[3], ug[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          gm[a] = 2.0 * p * dF[kp][a] + 2.0 * q * dF[kq][a];
          ug[a] = rhol * gm[a];
        }
        E00 = fma(gm[0], ug[0], E00);
        E01 = fma(gm[0], ug[1], E01);
        E02 = fma(gm[0], ug[2], E02);
        E11 = fma(gm[1], ug[1], E11);
        E12 = fma(gm[1], ug[2], E12);
        E22 = fma(gm[2], ug[2], E22);
      }
    }
    // scalars multiplying grad/Hessian of w_i, w_j, wR, wI
    double Aw = t[4], Bw = t[5], CR = 0.0, CI = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Aw += t[k] * co[k][0];
      Bw += t[k] * co[k][1];
      CR += t[k] * co[k][2];
      CI += t[k] * co[k][3];
    }
    g[0] = Aw * (2.0 * vi) + CR * dR[0] + CI * dI[0];
    g[1] = Bw * (2.0 * vj) + CR * dR[1] + CI * dI[1];
    const double c2 = CR * dR[2] + CI * dI[2];
    g[2] = c2 + t[6];
    g[3] = t[7] - c2;
    // Gauss-Newton part sum_k W_k dF_k dF_k'
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double u0 = W[k] * dF[k][0], u1 = W[k] * dF[k][1], u2 = W[k] * dF[k][2];
      E00 = fma(dF[k][0], u0, E00);
      E01 = fma(dF[k][0], u1, E01);
      E02 = fma(dF[k][0], u2, E02);
      E11 = fma(dF[k][1], u1, E11);
      E12 = fma(dF[k][1], u2, E12);
      E22 = fma(dF[k][2], u2, E22);
    }
    // pair terms of w_i, w_j (rho (2 v)^2) and the second derivatives of w_i, w_j, wR, wI
    E00 += rec[28] * (2.0 * vi) * (2.0 * vi) + 2.0 * Aw;
    E11 += rec[29] * (2.0 * vj) * (2.0 * vj) + 2.0 * Bw;
    E01 += CR * cs + CI * sn;
    const double gmm = CI * cs - CR * sn;
    E02 += vj * gmm;
    E12 += vi * gmm;
    E22 -= CR * wR + CI * wI;
    H[0] = E00;
    H[1] = E01;
    H[2] = E02;
    H[3] = -E02;
    H[4] = E01;
    H[5] = E11;
    H[6] = E12;
    H[7] = -E12;
    H[8] = E02;
    H[9] = E12;
    H[10] = E22 + rec[30];  // pair terms of the angles: rho on the diagonal
    H[11] = -E22;
    H[12] = -E02;
    H[13] = -E12;
    H[14] = -E22;
    H[15] = E22 + rec[31];
  }

  __device__ __forceinline__ double hq(int i, int j) const { return H[i * 4 + j]; }
  __device__ __forceinline__ double hd(int) const { return 0.0; }
  __device__ __forceinline__ bool hess_finite(const Grp<1>&) const {
    bool fin = true;
#pragma unroll
    for (int e = 0; e < 16; ++e) fin = fin && finite_bits(H[e]);
    return fin;
  }
};

template <>
struct BranchObj<4> {
  static constexpr int N = 4;
  static constexpr int R = 1;
  static constexpr int SMEM = 36 + 16;  // record, Hessian (row-major)
  static constexpr bool kHasHd = false;
  static constexpr bool kStepEval = false;

  SV<4> rec, H;
  double ca, cR, cI;  // flow t = ca w + cR wR + cI wI (w = w_i for t < 2, else w_j)
  double a0, a1;      // 2 ca where w is w_i (a0) or w_j (a1), else 0
  // at the point of the last eval_f; the first six are the same in the four lanes
  double vi, vj, sn, cs, wR, wI;
  double Ft, r1, r2;  // flow t, residuals of the pair terms t and t + 4
  double mx;          // p^2 + q^2 - smax^2 of the direction of flow t
  double Fx;          // flow t at the point of the last grad_hess
  double fsc;
  int n;

  __device__ __forceinline__ void bind(SV<4> base) {
    rec = base;
    H = base.at(36);
  }

  // per-lane coefficients from the staged record (after the group has synchronised):
  //   F0 = c0 w_i - c2 wR + c3 wI,  F1 = c1 w_i - c3 wR - c2 wI,
  //   F2 = c4 w_j - c6 wR - c7 wI,  F3 = c5 w_j - c7 wR + c6 wI
  __device__ __forceinline__ void prepare(int t) {
    ca = rec[t < 2 ? t : t + 2];
    cR = -rec[t == 0 ? 2 : (t == 1 ? 3 : (t == 2 ? 6 : 7))];
    const double c = rec[t == 0 ? 3 : (t == 1 ? 2 : (t == 2 ? 7 : 6))];
    cI = (t == 0 || t == 3) ? c : -c;
    a0 = t < 2 ? 2.0 * ca : 0.0;
    a1 = t < 2 ? 0.0 : 2.0 * ca;
  }

  template <class GP>
  __device__ __forceinline__ bool load(const GP& gp, const double* __restrict__ src, int n_) {
    n = n_;
    bool fin = true;
    for (int k = gp.t; k < 34; k += 4) {
      const double v = __ldg(src + k);
      if (k < 32) fin = fin && finite_bits(v);  // smax^2, rho_line: only where a line is over
      rec[k] = v;
    }
    gp.sync();
    prepare(gp.t);
    return !gp.any(!fin);
  }

  template <class GP>
  __device__ __forceinline__ double eval_f(const GP& gp, const double (&y)[1]) {
    const int t = gp.t;
    vi = gp.bcast(y[0], 0);
    vj = gp.bcast(y[0], 1);
    const double thi = gp.bcast(y[0], 2), thj = gp.bcast(y[0], 3);
    const double dth = thi - thj;
    // even ranks the sine, odd ranks the cosine of the angle difference: by the series
    // for |dth| <= pi/4 (one instruction stream for both), else as the library's sine
    // of the argument shifted by pi/2 on odd ranks (again one stream)
    const double sc = small_angle(dth) ? sin_cos_small(dth, (t & 1) != 0)
                                       : sin((t & 1) ? dth + 1.5707963267948966 : dth);
    sn = gp.bcast(sc, 0);
    cs = gp.bcast(sc, 1);
    const double vv = vi * vj;
    wR = vv * cs;
    wI = vv * sn;
    const double vf = t < 2 ? vi : vj;
    const double wf = vf * vf;
    const double yy = y[0] * y[0];
    Ft = ca * wf + cR * wR + cI * wI;
    // magnitudes of the terms of each pair quantity (rounding scale of f)
    const double Mt = fabs(ca) * wf + fabs(cR) * fabs(wR) + fabs(cI) * fabs(wI);
    // pair term t + 4: w_i, w_j, theta_i, theta_j
    const double P2 = t < 2 ? yy : y[0];
    const double M2 = t < 2 ? yy : fabs(y[0]);
    r1 = Ft - rec[16 + t];
    r2 = P2 - rec[20 + t];
    const double l1 = rec[8 + t], l2 = rec[12 + t];
    const double p1 = rec[24 + t], p2 = rec[28 + t];
    double val = l1 * r1 + 0.5 * p1 * r1 * r1;
    double mag = fabs(l1 * r1) + 0.5 * p1 * r1 * r1 + (fabs(l1) + p1 * fabs(r1)) * Mt;
    val += l2 * r2 + 0.5 * p2 * r2 * r2;
    mag += fabs(l2 * r2) + 0.5 * p2 * r2 * r2 + (fabs(l2) + p2 * fabs(r2)) * M2;
    // line limit of the direction of flow t (its flows on ranks 2d, 2d + 1): squares
    // added unfused, so both ranks of the pair hold the same bits and take the same branch
    const double sq = __dmul_rn(Ft, Ft);
    const double p2q2 = __dadd_rn(sq, gp.exch(sq, 1));
    const double smax2 = rec[32], rhol = rec[33];
    mx = p2q2 - smax2;
    if (positive_bits(mx) && (t & 1) == 0) {
      val += 0.5 * rhol * mx * mx;
      mag += 0.5 * rhol * mx * mx + rhol * mx * (p2q2 + smax2);
    }
    gp.sum2(val, mag);
    fsc = mag;
    return val;
  }

  // gradient and Hessian row t at the point of the last eval_f.  The sums over the four
  // flows -- the scalars (Aw, Bw, CR, CI) multiplying the derivatives of w_i, w_j, wR, wI
  // (with the weights of the pair terms of w_i, w_j) and the Gauss-Newton entries of
  // sum_k W_k dF_k dF_k' -- are one reduce-scatter butterfly over the group.
  template <class GP>
  __device__ __forceinline__ void grad_hess(const GP& gp, const double (&x)[1], double (&g)[1]) {
    const int t = gp.t;
    Fx = Ft;
    const double p1 = rec[24 + t], rhol = rec[33];
    double tw = rec[8 + t] + p1 * r1;                   // first-order weight of flow t
    const double tw2 = rec[12 + t] + rec[28 + t] * r2;  // of the pair term t + 4
    double W = p1;                                      // Gauss-Newton weight of flow t
    const bool act = positive_bits(mx);
    if (act) {
      // (rho_l/2) m^2, m = p^2 + q^2 - smax^2: first-order weight 2 rho_l m F_t, and
      // 2 rho_l m on dF_t dF_t' (the rest, rho_l grad m grad m', below)
      tw += rhol * mx * 2.0 * Ft;
      W += 2.0 * rhol * mx;
    }
    // row t of dF = d(flows)/d(v_i, v_j, theta_i, theta_j); the theta_j entry is -d2
    const double h = cR * cs + cI * sn;
    const double d0 = fma(a0, vi, vj * h);
    const double d1 = fma(a1, vj, vi * h);
    const double d2 = cI * wR - cR * wI;
    const double twc = tw * ca, tws = twc + tw2;
    const double u0 = W * d0, u1 = W * d1, u2 = W * d2;
    double v[10];
    v[0] = t == 0 ? tws : (t == 1 ? twc : 0.0);  // Aw: flows 0, 1 and the term of w_i
    v[1] = t == 1 ? tw2 : (t >= 2 ? twc : 0.0);  // Bw: flows 2, 3 and the term of w_j
    v[2] = tw * cR;
    v[3] = tw * cI;
    v[4] = d0 * u0;
    v[5] = d0 * u1;
    v[6] = d0 * u2;
    v[7] = d1 * u1;
    v[8] = d1 * u2;
    v[9] = d2 * u2;
    if (gp.any(act)) {
      // rho_l grad m grad m' of each exceeded direction, grad m = 2p dF_p + 2q dF_q,
      // added once per direction (by its even rank)
      const double f2 = 2.0 * Ft;
      const double c0 = f2 * d0, c1 = f2 * d1, c2 = f2 * d2;
      const double m0 = c0 + gp.exch(c0, 1), m1 = c1 + gp.exch(c1, 1), m2 = c2 + gp.exch(c2, 1);
      if (act && (t & 1) == 0) {
        const double q0 = rhol * m0, q1 = rhol * m1, q2 = rhol * m2;
        v[4] = fma(m0, q0, v[4]);
        v[5] = fma(m0, q1, v[5]);
        v[6] = fma(m0, q2, v[6]);
        v[7] = fma(m1, q1, v[7]);
        v[8] = fma(m1, q2, v[8]);
        v[9] = fma(m2, q2, v[9]);
      }
    }
    // reduce-scatter: after the exchange across rank bit 1, ranks 0, 1 hold partial sums
    // of v[0..4] and ranks 2, 3 of v[5..9]; after the one across bit 0 rank 0 holds the
    // sums of v[0..2], rank 1 of v[3..4], rank 2 of v[5..7], rank 3 of v[8..9]
    const bool h2 = (t & 2) != 0, h1 = (t & 1) != 0;
    double k5[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const double keep = h2 ? v[5 + s] : v[s];
      const double send = h2 ? v[s] : v[5 + s];
      k5[s] = keep + gp.exch(send, 2);
    }
    double k3[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const double hi = s < 2 ? k5[3 + s] : 0.0;
      const double keep = h1 ? hi : k5[s];
      const double send = h1 ? k5[s] : hi;
      k3[s] = keep + gp.exch(send, 1);
    }
    const double Aw = gp.bcast(k3[0], 0), Bw = gp.bcast(k3[1], 0), CR = gp.bcast(k3[2], 0);
    const double CI = gp.bcast(k3[0], 1), e00 = gp.bcast(k3[1], 1);
    const double e01 = gp.bcast(k3[0], 2), e02 = gp.bcast(k3[1], 2), e11 = gp.bcast(k3[2], 2);
    const double e12 = gp.bcast(k3[0], 3), e22 = gp.bcast(k3[1], 3);
    // g_t = [t=0] 2 v_i Aw + [t=1] 2 v_j Bw + [t>=2] (weight of term t + 4)
    //       + CR dwR/dx_t + CI dwI/dx_t,
    // dwR/dx = (v_j cs, v_i cs, -wI, wI), dwI/dx = (v_j sn, v_i sn, wR, -wR)
    const double vo = t == 0 ? vj : vi;
    const double dRv = vo * cs, dIv = vo * sn;
    const double dRt = t < 2 ? dRv : (t == 2 ? -wI : wI);
    const double dIt = t < 2 ? dIv : (t == 2 ? wR : -wR);
    const double ab = t == 0 ? Aw : Bw;
    const double x2 = 2.0 * x[0];
    const double base = t < 2 ? x2 * ab : tw2;
    g[0] = base + CR * dRt + CI * dIt;
    // second derivatives of w_i, w_j, wR, wI times (Aw, Bw, CR, CI):
    //   (0,0) 2 Aw, (1,1) 2 Bw, (0,1) CR cs + CI sn,
    //   (0,2) = -(0,3) = v_j gm, (1,2) = -(1,3) = v_i gm with gm = CI cs - CR sn,
    //   (2,2) = (3,3) = -(2,3) = -(CR wR + CI wI)
    const double q01 = CR * cs + CI * sn;
    const double gm = CI * cs - CR * sn;
    const double aj = vj * gm, ai = vi * gm;
    const double bb = CR * wR + CI * wI;
    // diagonal: the Gauss-Newton part of the pair terms t + 4 (rho (2 v)^2 for w_i, w_j;
    // rho for the angles) plus the second-derivative entry
    const double dterm = t < 2 ? rec[28 + t] * (x2 * x2) : rec[28 + t];
    const double sdiag = (t < 2 ? 2.0 * ab : -bb) + dterm;
    double gn[4], s2[4];
    if (t == 0) {
      gn[0] = e00; gn[1] = e01; gn[2] = e02; gn[3] = -e02;
      s2[0] = sdiag; s2[1] = q01; s2[2] = aj; s2[3] = -aj;
    } else if (t == 1) {
      gn[0] = e01; gn[1] = e11; gn[2] = e12; gn[3] = -e12;
      s2[0] = q01; s2[1] = sdiag; s2[2] = ai; s2[3] = -ai;
    } else if (t == 2) {
      gn[0] = e02; gn[1] = e12; gn[2] = e22; gn[3] = -e22;
      s2[0] = aj; s2[1] = ai; s2[2] = sdiag; s2[3] = bb;
    } else {
      gn[0] = -e02; gn[1] = -e12; gn[2] = -e22; gn[3] = e22;
      s2[0] = -aj; s2[1] = -ai; s2[2] = bb; s2[3] = sdiag;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) H[4 * t + b] = gn[b] + s2[b];
    gp.sync();
  }

  __device__ __forceinline__ double hq(int i, int j) const { return H[4 * i + j]; }
  __device__ __forceinline__ double hd(int) const { return 0.0; }
  // row i of H times v (v staged in shared memory)
  __device__ __forceinline__ double row_dot(int i, SV<4> v) const {
    double s = H[4 * i] * v[0];
    s = fma(H[4 * i + 1], v[1], s);
    s = fma(H[4 * i + 2], v[2], s);
    return fma(H[4 * i + 3], v[3], s);
  }

  template <class GP>
  __device__ __forceinline__ bool hess_finite(const GP& gp) const {
    const int t = gp.t;
    const bool fin = finite_bits(H[4 * t]) && finite_bits(H[4 * t + 1]) && finite_bits(H[4 * t + 2]) &&
                     finite_bits(H[4 * t + 3]);
    return !gp.any(!fin);
  }
};

// Two lanes per problem: rank t holds bus t's variables of the branch, x = (v, theta)
// of bus i (t = 0) or bus j (t = 1) -- the solver's variables t and t + 2 -- and owns
// the two flows of its end (p_ij, q_ij or p_ji, q_ji: both use its own w = v^2), its
// line-limit direction, and the pair terms of those flows and of its w and theta.  The
// sums over all four flows (the scalars CR, CI and the six distinct Gauss-Newton
// entries) take one exchange between the two ranks; each rank writes the Hessian rows
// of its two variables.
template <>
struct BranchObj<2> {
  static constexpr int N = 4;
  static constexpr int R = 2;
  static constexpr int SMEM = 36 + 16;  // record, Hessian (row-major)
  static constexpr bool kHasHd = false;
  static constexpr bool kStepEval = false;

  SV<2> rec, H;
  double ca[2], cR[2], cI[2];  // flows 2t, 2t + 1 = ca w + cR wR + cI wI (w: own bus)
  // at the point of the last eval_f; the first six are the same on both ranks
  double vi, vj, sn, cs, wR, wI;
  double F[2], rf[2], rw, rth;  // own flows; residuals of their pair terms, of w, theta
  double mx;                    // p^2 + q^2 - smax^2 of the own direction
  double Fx[2];                 // own flows at the point of the last grad_hess
  double fsc;
  int n;

  __device__ __forceinline__ void bind(SV<2> base) {
    rec = base;
    H = base.at(36);
  }

  // coefficients of flow f (0..3) as for four lanes:
  //   F0 = c0 w_i - c2 wR + c3 wI,  F1 = c1 w_i - c3 wR - c2 wI,
  //   F2 = c4 w_j - c6 wR - c7 wI,  F3 = c5 w_j - c7 wR + c6 wI
  __device__ __forceinline__ void prepare(int t) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int f = 2 * t + e;
      ca[e] = rec[f < 2 ? f : f + 2];
      cR[e] = -rec[f == 0 ? 2 : (f == 1 ? 3 : (f == 2 ? 6 : 7))];
      const double c = rec[f == 0 ? 3 : (f == 1 ? 2 : (f == 2 ? 7 : 6))];
      cI[e] = (f == 0 || f == 3) ? c : -c;
    }
  }

  template <class GP>
  __device__ __forceinline__ bool load(const GP& gp, const double* __restrict__ src, int n_) {
    n = n_;
    bool fin = true;
    for (int k = gp.t; k < 34; k += 2) {
      const double v = __ldg(src + k);
      if (k < 32) fin = fin && finite_bits(v);  // smax^2, rho_line: only where a line is over
      rec[k] = v;
    }
    gp.sync();
    prepare(gp.t);
    return !gp.any(!fin);
  }

  template <class GP>
  __device__ __forceinline__ double eval_f(const GP& gp, const double (&y)[2]) {
    const int t = gp.t;
    const double vo = y[0], tho = y[1];
    const double vp = gp.exch(vo, 1), thp = gp.exch(tho, 1);
    vi = t == 0 ? vo : vp;
    vj = t == 0 ? vp : vo;
    const double thi = t == 0 ? tho : thp, thj = t == 0 ? thp : tho;
    const double dth = thi - thj;
    // rank 0 the sine, rank 1 the cosine of the angle difference (one stream)
    const double sc = small_angle(dth) ? sin_cos_small(dth, t == 1)
                                       : sin(t == 1 ? dth + 1.5707963267948966 : dth);
    sn = gp.bcast(sc, 0);
    cs = gp.bcast(sc, 1);
    const double vv = vi * vj;
    wR = vv * cs;
    wI = vv * sn;
    const double wo = vo * vo;
    const double aR = fabs(wR), aI = fabs(wI);
    double val = 0.0, mag = 0.0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      F[e] = ca[e] * wo + cR[e] * wR + cI[e] * wI;
      const double M = fabs(ca[e]) * wo + fabs(cR[e]) * aR + fabs(cI[e]) * aI;
      const int k = 2 * t + e;
      const double r = F[e] - rec[16 + k];
      rf[e] = r;
      const double l = rec[8 + k], p = rec[24 + k];
      val += l * r + 0.5 * p * r * r;
      mag += fabs(l * r) + 0.5 * p * r * r + (fabs(l) + p * fabs(r)) * M;
    }
    {  // pair terms of the own w (k = 4 + t) and theta (k = 6 + t)
      rw = wo - rec[20 + t];
      rth = tho - rec[22 + t];
      const double lw = rec[12 + t], pw = rec[28 + t];
      const double lt = rec[14 + t], pt = rec[30 + t];
      val += lw * rw + 0.5 * pw * rw * rw;
      mag += fabs(lw * rw) + 0.5 * pw * rw * rw + (fabs(lw) + pw * fabs(rw)) * wo;
      val += lt * rth + 0.5 * pt * rth * rth;
      mag += fabs(lt * rth) + 0.5 * pt * rth * rth + (fabs(lt) + pt * fabs(rth)) * fabs(tho);
    }
    // line limit of the own direction (both of its flows are this rank's)
    const double p2q2 = F[0] * F[0] + F[1] * F[1];
    const double smax2 = rec[32], rhol = rec[33];
    mx = p2q2 - smax2;
    if (positive_bits(mx)) {
      val += 0.5 * rhol * mx * mx;
      mag += 0.5 * rhol * mx * mx + rhol * mx * (p2q2 + smax2);
    }
    gp.sum2(val, mag);
    fsc = mag;
    return val;
  }

  // gradient and Hessian rows of the own variables at the point of the last eval_f
  template <class GP>
  __device__ __forceinline__ void grad_hess(const GP& gp, const double (&x)[2], double (&g)[2]) {
    const int t = gp.t;
    Fx[0] = F[0];
    Fx[1] = F[1];
    const double rhol = rec[33];
    const bool act = positive_bits(mx);
    const double h2 = act ? 2.0 * rhol * mx : 0.0;  // line term: 2 rho_l m on F and on W
    const double vo = x[0];
    // flows: first-order weights tw, Gauss-Newton weights W, derivative rows
    // (d0, d1, d2) along (v_i, v_j, theta_i) (theta_j: -d2)
    double CR = 0.0, CI = 0.0, ab = 0.0;
    double e00 = 0.0, e01 = 0.0, e02 = 0.0, e11 = 0.0, e12 = 0.0, e22 = 0.0;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;  // grad m / 2 of the own direction
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 2 * t + e;
      double tw = rec[8 + k] + rec[24 + k] * rf[e];
      double W = rec[24 + k];
      if (act) {
        tw += h2 * F[e];
        W += h2;
      }
      const double h = cR[e] * cs + cI[e] * sn;
      const double a2 = 2.0 * ca[e];
      const double d0 = t == 0 ? fma(a2, vi, vj * h) : vj * h;
      const double d1 = t == 0 ? vi * h : fma(a2, vj, vi * h);
      const double d2 = cI[e] * wR - cR[e] * wI;
      ab = fma(tw, ca[e], ab);
      CR = fma(tw, cR[e], CR);
      CI = fma(tw, cI[e], CI);
      const double u0 = W * d0, u1 = W * d1, u2 = W * d2;
      e00 = fma(d0, u0, e00);
      e01 = fma(d0, u1, e01);
      e02 = fma(d0, u2, e02);
      e11 = fma(d1, u1, e11);
      e12 = fma(d1, u2, e12);
      e22 = fma(d2, u2, e22);
      m0 = fma(F[e], d0, m0);
      m1 = fma(F[e], d1, m1);
      m2 = fma(F[e], d2, m2);
    }
    if (act) {  // rho_l grad m grad m', grad m = 2 (p dF_p + q dF_q)
      const double q0 = 2.0 * m0, q1 = 2.0 * m1, q2 = 2.0 * m2;
      const double r0 = rhol * q0, r1 = rhol * q1, r2 = rhol * q2;
      e00 = fma(q0, r0, e00);
      e01 = fma(q0, r1, e01);
      e02 = fma(q0, r2, e02);
      e11 = fma(q1, r1, e11);
      e12 = fma(q1, r2, e12);
      e22 = fma(q2, r2, e22);
    }
    const double tww = rec[12 + t] + rec[28 + t] * rw;  // weight of the own w term
    const double twt = rec[14 + t] + rec[30 + t] * rth; // of the own theta term
    ab += tww;  // Aw on rank 0, Bw on rank 1
    // the other rank's flows
    CR += gp.exch(CR, 1);
    CI += gp.exch(CI, 1);
    e00 += gp.exch(e00, 1);
    e01 += gp.exch(e01, 1);
    e02 += gp.exch(e02, 1);
    e11 += gp.exch(e11, 1);
    e12 += gp.exch(e12, 1);
    e22 += gp.exch(e22, 1);
    // gradient: g_v = 2 v ab + CR dwR/dv + CI dwI/dv (dwR/dv_i = v_j cs, dwI/dv_i =
    // v_j sn, and i <-> j), g_theta = tw_theta + CR dwR/dtheta + CI dwI/dtheta
    // (dwR/dtheta_i = -wI, dwI/dtheta_i = wR; theta_j: the opposite)
    const double vq = t == 0 ? vj : vi;
    const double x2 = 2.0 * vo;
    g[0] = x2 * ab + CR * (vq * cs) + CI * (vq * sn);
    const double dRt = t == 0 ? -wI : wI, dIt = t == 0 ? wR : -wR;
    g[1] = twt + CR * dRt + CI * dIt;
    // second derivatives of w_i, w_j, wR, wI times the aggregates (as for four lanes)
    const double q01 = CR * cs + CI * sn;
    const double gm = CI * cs - CR * sn;
    const double aj = vj * gm, ai = vi * gm;
    const double bb = CR * wR + CI * wI;
    const double sdv = 2.0 * ab + rec[28 + t] * (x2 * x2);
    const double sdt = -bb + rec[30 + t];
    // row of v_own (variable t) and of theta_own (variable t + 2)
    double rv[4], rt[4];
    if (t == 0) {
      rv[0] = e00 + sdv; rv[1] = e01 + q01; rv[2] = e02 + aj; rv[3] = -e02 - aj;
      rt[0] = e02 + aj;  rt[1] = e12 + ai;  rt[2] = e22 + sdt; rt[3] = -e22 + bb;
    } else {
      rv[0] = e01 + q01; rv[1] = e11 + sdv; rv[2] = e12 + ai; rv[3] = -e12 - ai;
      rt[0] = -e02 - aj; rt[1] = -e12 - ai; rt[2] = -e22 + bb; rt[3] = e22 + sdt;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      H[4 * t + b] = rv[b];
      H[4 * (t + 2) + b] = rt[b];
    }
    gp.sync();
  }

  __device__ __forceinline__ double hq(int i, int j) const { return H[4 * i + j]; }
  __device__ __forceinline__ double hd(int) const { return 0.0; }
  __device__ __forceinline__ double row_dot(int i, SV<2> v) const {
    double s = H[4 * i] * v[0];
    s = fma(H[4 * i + 1], v[1], s);
    s = fma(H[4 * i + 2], v[2], s);
    return fma(H[4 * i + 3], v[3], s);
  }
  template <class GP>
  __device__ __forceinline__ bool hess_finite(const GP& gp) const {
    const int t = gp.t;
    bool fin = true;
#pragma unroll
    for (int b = 0; b < 4; ++b) fin = fin && finite_bits(H[4 * t + b]) && finite_bits(H[4 * (t + 2) + b]);
    return !gp.any(!fin);
  }
};

// --------------------------------------------- multi-period generator (n <= 32 periods)
// The generator component of the multi-period ADMM: its active power over the periods,
// f = sum_t c2 p_t^2 + c1 p_t + lambda_t (p_t - target_t) + rho/2 (p_t - target_t)^2
//     + rho_r/2 sum_{t>=1} max(0, |p_t - p_{t-1}| - R)^2,
// record [c2 c1 rho rho_r R 0 0 0 | lambda[n] | target[n]].  One period per lane (G = N):
// the ramp term of the pair (t-1, t) lives on lane t and reaches its neighbours by
// shuffles; the Hessian is tridiagonal, kept as its diagonal and subdiagonal.
template <int N, int G>
struct GenRampObj {
  static_assert(G == N && N <= 32, "one period per lane");
  static constexpr int R = 1;
  static constexpr int SMEM = 2 * N;  // diagonal, subdiagonal H(t, t-1) at t
  static constexpr bool kHasHd = false;
  static constexpr bool kStepEval = false;

  SV<G> dg, sd;
  double c2, c1, rho, rr, ramp, lam, tgt;
  double ex, sg;  // ramp excess |d| - R and sign of d of the pair (t-1, t), last eval_f
  double fsc;
  int n;

  __device__ __forceinline__ void bind(SV<G> base) {
    dg = base;
    sd = base.at(N);
  }

  template <class GP>
  __device__ __forceinline__ bool load(const GP& gp, const double* __restrict__ rec, int n_) {
    n = n_;
    c2 = __ldg(rec + 0);
    c1 = __ldg(rec + 1);
    rho = __ldg(rec + 2);
    rr = __ldg(rec + 3);
    ramp = __ldg(rec + 4);
    const int t = gp.t;
    lam = t < n ? __ldg(rec + 8 + t) : 0.0;
    tgt = t < n ? __ldg(rec + 8 + n + t) : 0.0;
    // rho_r and R enter f only where a ramp limit is exceeded
    const bool fin = finite_bits(c2) && finite_bits(c1) && finite_bits(rho) &&
                     finite_bits(lam) && finite_bits(tgt);
    dg[t] = 0.0;
    sd[t] = 0.0;
    gp.sync();
    return !gp.any(!fin);
  }

  template <class GP>
  __device__ __forceinline__ double eval_f(const GP& gp, const double (&y)[R]) {
    const int t = gp.t;
    const double p = y[0];
    const double pp = gp.from_prev(p);
    double val = 0.0, mag = 0.0;
    ex = -1.0;
    sg = 0.0;
    if (t < n) {
      const double r = p - tgt;
      val = c2 * p * p + c1 * p + lam * r + 0.5 * rho * r * r;
      mag = fabs(c2) * p * p + fabs(c1 * p) + fabs(lam * r) + 0.5 * rho * r * r +
            (fabs(lam) + rho * fabs(r)) * (fabs(p) + fabs(tgt));
      if (t >= 1) {
        const double d = p - pp;
        ex = fabs(d) - ramp;
        sg = positive_bits(d) ? 1.0 : -1.0;
        if (positive_bits(ex)) {
          val += 0.5 * rr * ex * ex;
          mag += 0.5 * rr * ex * ex + rr * ex * (fabs(p) + fabs(pp) + ramp);
        }
      }
    }
    gp.sum2(val, mag);
    fsc = mag;
    return val;
  }

  // gradient and Hessian at the point of the last eval_f
  template <class GP>
  __device__ __forceinline__ void grad_hess(const GP& gp, const double (&x)[R], double (&g)[R]) {
    const int t = gp.t;
    const bool act = positive_bits(ex);
    const double w = act ? rr * ex * sg : 0.0;  // d/dp_t of the pair (t-1, t)
    const double wn = gp.from_next(w);          // the pair (t, t+1), from lane t+1
    const double an = gp.from_next(act ? 1.0 : 0.0);
    const bool has_next = t + 1 < n;
    double gt = 0.0, dt = 0.0;
    if (t < n) {
      const double p = x[0], r = p - tgt;
      gt = 2.0 * c2 * p + c1 + lam + rho * r + w - (has_next ? wn : 0.0);
      dt = 2.0 * c2 + rho + (act ? rr : 0.0) + (has_next && nonzero_bits(an) ? rr : 0.0);
    }
    g[0] = gt;
    dg[t] = dt;
    sd[t] = (t < n && act) ? -rr : 0.0;
    gp.sync();
  }

  __device__ __forceinline__ double hq(int i, int j) const {
    if (i == j) return dg[i];
    if (j == i - 1) return sd[i];
    if (j == i + 1) return sd[j];
    return 0.0;
  }
  __device__ __forceinline__ double hd(int) const { return 0.0; }

  // row i of the tridiagonal Hessian times v (v staged in shared memory)
  __device__ __forceinline__ double row_dot(int i, SV<G> v) const {
    double s = dg[i] * v[i];
    if (i >= 1) s = fma(sd[i], v[i - 1], s);
    if (i + 1 < N) s = fma(sd[i + 1], v[i + 1], s);
    return s;
  }

  template <class GP>
  __device__ __forceinline__ bool hess_finite(const GP& gp) const {
    const bool fin = finite_bits(dg[gp.t]) && finite_bits(sd[gp.t]);
    return !gp.any(!fin);
  }
};

// ------------------------------------------------------------------ hs45 variant
// f = 120 - prod_i x_i (Sec. 4.2 footnote), one problem per lane, n <= N.
template <int N>
struct Hs45Obj {
  static constexpr int R = N;
  static constexpr int SMEM = N * N;
  static constexpr bool kHasHd = false;
  static constexpr bool kStepEval = false;

  SV<1> H;
  double xc[N];
  double fsc;
  int n;

  __device__ __forceinline__ void bind(SV<1> base) { H = base; }
  __device__ __forceinline__ bool load(const Grp<1>&, const double*, int n_) {
    n = n_;
    return true;
  }
  __device__ __forceinline__ double eval_f(const Grp<1>&, const double (&y)[N]) {
    double p = 1.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      xc[i] = y[i];
      if (i < n) p *= y[i];
    }
    fsc = 120.0 + fabs(p);
    return 120.0 - p;
  }
  __device__ __forceinline__ void grad_hess(const Grp<1>&, const double (&)[N], double (&g)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double q = 1.0;
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (j != i && j < n) q *= xc[j];
      g[i] = (i < n) ? -q : 0.0;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) {
        double q = 1.0;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k != i && k != j && k < n) q *= xc[k];
        H[i * N + j] = (i == j || i >= n || j >= n) ? 0.0 : -q;
      }
  }
  __device__ __forceinline__ double hq(int i, int j) const { return H[i * N + j]; }
  __device__ __forceinline__ double hd(int) const { return 0.0; }
  __device__ __forceinline__ bool hess_finite(const Grp<1>&) const {
    bool fin = true;
    for (int e = 0; e < n * N; ++e) fin = fin && finite_bits(H[e]);
    return fin;
  }
};

}  // namespace xt
