// tron_solver.cuh -- Algorithm 1 (Sec. 3) on one thread group of G lanes.
//
// Per outer iteration, all on the device (Sec. 4.1: single kernel, no host traffic):
//   projected-gradient max-norm test (Sec. 5.1) -> Cauchy point with the
//   interpolation/extrapolation search -> free set of the current point and
//   gather of H_FF (Sec. 5.3) -> shifted complete factorization, left- or
//   right-looking, with the factor mirrored into the upper triangle (Sec. 4.3,
//   4.4) -> Steihaug PCG with the CG iterate s = L^T w of the
//   preconditioned system kept inside ||s||_2 <= delta -> back transform -> projected
//   search -> reduction ratio, acceptance and radius update.
//
// Storage: the vectors of a problem are register arrays spread over the group (slot r
// of lane t holds variable r*G + t); the factor (with its transpose mirrored) and the
// objective data sit in the problem's shared-memory slice; the free-set indices are an
// int list in shared memory.  Triangular solves read rows of the lower part (backward)
// or rows of the mirrored upper part (forward), so every shared-memory access of a
// solve is contiguous across the group (Sec. 4.4).
//
// FP64 economy on this GPU (a warp FP64 instruction costs the same issue slot with one
// active lane or 32): the factorization is the square-root-free form A = Lu D Lu^T of
// the paper's L L^T, one reciprocal per pivot (hardware approximation + one Newton
// step); the right-looking form spreads the trailing update over all lanes (the
// paper's left-looking form remains as options.cholesky = 1); the PCG runs in the step
// itself, where only M^-1 = Lu^-T D^-1 Lu^-1 is needed, and takes the exact-
// preconditioner step directly when no shift was needed; norms are compared squared;
// dot products needed together are reduced in one fused butterfly.
#pragma once

#include "../../include/tron.h"
#include "tron_common.cuh"
#include "tron_objectives.cuh"

namespace xt {

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// status of a run stopped by Solver::pause_at (never reported: the run is resumed)
constexpr int kTronPaused = 64;

// PK selects the storage of the factor: false = full N x (N+1) array with L^T mirrored
// into the upper triangle (Sec. 4.4); true = packed lower triangle, row c at c(c+1)/2,
// half the shared memory.  Both keep every warp access conflict free: in the packed
// layout the rows c(c+1)/2 of 16 consecutive c fall on 16 distinct 8-byte banks.
template <class Obj, int N, int G, bool PK = false>
struct Solver {
  static constexpr int R = N / G;
  static_assert(N % G == 0, "size class must be a multiple of the group size");
  static constexpr int LD = (G == 1) ? N : N + 1;
  static constexpr int LSZ = PK ? N * (N + 1) / 2 : N * LD;
  // per-problem shared-memory slice, offsets in doubles
  static constexpr int OFF_L = 0;
  static constexpr int OFF_VB = OFF_L + LSZ;
  static constexpr int OFF_DINV = OFF_VB + N;
  static constexpr int OFF_FI = OFF_DINV + N;  // N ints (in N double slots)
  // a second staging vector for the two-column factorization pass of CTA groups
  static constexpr int NVB2 = (G > 32) ? N : 0;
  static constexpr int OFF_VB2 = OFF_FI + N;
  static constexpr int OFF_OBJ = OFF_VB2 + NVB2;
  static constexpr int S_RAW = OFF_OBJ + Obj::SMEM;
  // problems of one warp start at banks that differ by G doubles (conflict-free when
  // several problems share a warp)
  static constexpr int S = (G == 1 || G >= 16) ? round_up(S_RAW, 2)
                                               : S_RAW + ((G - S_RAW % 16) % 16 + 16) % 16;
  // problems per warp (warp groups) and shared memory per warp; a CTA group (G > 32)
  // holds one problem per CTA and S doubles per CTA
  static constexpr int PROBS_PER_WARP = (G > 32) ? 0 : 32 / G;
  static constexpr int WARP_DOUBLES = (G == 1) ? S * 32 : (G > 32 ? S : S * PROBS_PER_WARP);

  GroupOf<G> gp;
  const tron_options_t& o;
  Obj obj;
  int n;
  SV<G> Lm, vb, dinv, vb2;
  SV<G, int> Fi;
  double l[R], u[R];
  long long kl[R], ku[R];  // integer keys of the bounds
  // a run split in two launches: the first stops after pause_at iterations with
  // kTronPaused (x, delta, the iteration count and the Cauchy step alpha_c are then the
  // whole state of Algorithm 1 between iterations; f, g and H follow from x), and the
  // second resumes from them with k_start and alpha0
  int pause_at = 0x7FFFFFFF;
  int k_start = 0;
  double alpha0 = 1.0;
  double alpha_out = 1.0;

  __device__ __forceinline__ Solver(const tron_options_t& opt, double* warp_smem) : o(opt) {
    double* base = (G == 1) ? warp_smem + gp.lane
                            : (G > 32 ? warp_smem : warp_smem + (gp.lane / G) * S);
    SV<G> sv{base};
    Lm = sv.at(OFF_L);
    vb = sv.at(OFF_VB);
    dinv = sv.at(OFF_DINV);
    vb2 = sv.at(OFF_VB2);
    Fi = SV<G, int>{(G == 1) ? reinterpret_cast<int*>(warp_smem + OFF_FI * 32) + gp.lane
                             : reinterpret_cast<int*>(base + OFF_FI)};
    obj.bind(sv.at(OFF_OBJ));
  }

  // L(c, j), c >= j, in the lower storage
  __device__ __forceinline__ double& lo(int c, int j) const {
    return PK ? Lm[c * (c + 1) / 2 + j] : Lm[c * LD + j];
  }
  // L(c, j), c >= j, read through the transposed copy (row j of L^T); the same element
  // as lo(c, j) in the packed layout
  __device__ __forceinline__ double& mt(int j, int c) const {
    return PK ? Lm[c * (c + 1) / 2 + j] : Lm[j * LD + c];
  }

  // ------------------------------------------------------------------ vector helpers
  // order-preserving integer key of a double: the two's-complement order of the keys is
  // the numeric order, and -0 takes the key of +0, so for non-NaN values every
  // comparison of keys gives the IEEE comparison's answer without an FP64 instruction
  // (projections, bound and sign tests)
  __device__ __forceinline__ static long long okey(double v) {
    long long b = __double_as_longlong(v);
    if (b == (long long)0x8000000000000000ULL) b = 0;
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
  }
  // a <= b and a < b for non-NaN doubles, on the integer keys (no FP64 instruction)
  __device__ __forceinline__ static bool le(double a, double b) { return okey(a) <= okey(b); }
  __device__ __forceinline__ static bool lt(double a, double b) { return okey(a) < okey(b); }
  // |v| > t for t >= 0 (magnitude bits compared as integers)
  __device__ __forceinline__ static bool abs_above(double v, long long tkey) {
    return (__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL) > tkey;
  }
  __device__ __forceinline__ double P(double v, int r) const {
    const long long k = okey(v);
    return k < kl[r] ? l[r] : (k > ku[r] ? u[r] : v);
  }
  __device__ __forceinline__ void key_bounds() {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      kl[r] = okey(l[r]);
      ku[r] = okey(u[r]);
    }
  }
  __device__ __forceinline__ double dotv(const double (&a)[R], const double (&b)[R]) const {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) s = fma(a[r], b[r], s);
    return gp.sum(s);
  }
  // (grad_P f)_i: g_i, or 0 where x_i sits on a bound that g_i pushes against
  __device__ __forceinline__ double pgi(double x, double g, int r) const {
    const long long kx = okey(x), kg = okey(g);
    return ((kx <= kl[r] && kg > 0) || (kx >= ku[r] && kg < 0)) ? 0.0 : g;
  }
  __device__ __forceinline__ double pgnorm(const double (&x)[R], const double (&g)[R]) const {
    double m = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) m = fmax(m, fabs(pgi(x[r], g[r], r)));
    return gp.max(m);
  }

  // some |(grad_P f)_i| > tol (tol >= 0), decided on integer keys
  __device__ __forceinline__ bool pg_above(const double (&x)[R], const double (&g)[R],
                                           double tol) const {
    const long long tk = __double_as_longlong(tol);
    bool above = false;
#pragma unroll
    for (int r = 0; r < R; ++r) above = above || abs_above(pgi(x[r], g[r], r), tk);
    return gp.any(above);
  }
  // l_i < v < u_i on integer keys
  __device__ __forceinline__ bool strictly_inside(double v, int r) const {
    const long long k = okey(v);
    return kl[r] < k && k < ku[r];
  }

  // y = H v over the full vector (H at the current accepted point)
  __device__ __forceinline__ void hv(const double (&v)[R], double (&y)[R]) {
    if constexpr (G == 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(obj.hq(i, j), v[j], s);
        if (Obj::kHasHd) s = fma(obj.hd(i), v[i], s);
        y[i] = s;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) vb[r * G + gp.t] = v[r];
      gp.sync();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = r * G + gp.t;
        double s = obj.row_dot(i, vb);
        if (Obj::kHasHd) s = fma(obj.hd(i), v[r], s);
        y[r] = s;
      }
      gp.sync();
    }
  }

  // q = H_FF z in compacted coordinates (slot r <-> free position r*G + t)
  __device__ __forceinline__ void hv_free(int m, const double (&z)[R], double (&q)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) vb[r * G + gp.t] = z[r];
    gp.sync();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = r * G + gp.t;
      double s = 0.0;
      if (c < m) {
        const int i = Fi[c];
        double s1 = 0.0;
        int d = 0;
        for (; d + 1 < m; d += 2) {
          s = fma(obj.hq(i, Fi[d]), vb[d], s);
          s1 = fma(obj.hq(i, Fi[d + 1]), vb[d + 1], s1);
        }
        if (d < m) s = fma(obj.hq(i, Fi[d]), vb[d], s);
        if (Obj::kHasHd) s = fma(obj.hd(i), z[r], s);
        s += s1;
      }
      q[r] = s;
    }
    gp.sync();
  }

  // y = H v for a v with few nonzero coordinates: one column of H per nonzero (lanes
  // read column j of Q across the group); false, with nothing computed, when more than
  // N/4 coordinates are nonzero or for groups wider than a warp or a single lane
  __device__ __forceinline__ bool hv_sparse(const double (&v)[R], double (&y)[R]) {
    if constexpr (G == 1 || G > 32) {
      return false;
    } else {
      unsigned msk[R];
      int cnt = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        msk[r] = gp.ballot(nonzero_bits(v[r]));
        cnt += __popc(msk[r]);
      }
      if (cnt > N / 4) return false;
#pragma unroll
      for (int r = 0; r < R; ++r) y[r] = 0.0;
#pragma unroll
      for (int rj = 0; rj < R; ++rj) {
        unsigned mm = msk[rj];
        while (mm) {
          const int tj = __ffs(mm) - 1;
          mm &= mm - 1u;
          const int j = rj * G + tj;
          const double vj = gp.bcast(v[rj], tj);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int i = r * G + gp.t;
            double hij = obj.hq(i, j);
            if (Obj::kHasHd && i == j) hij = hij + obj.hd(i);
            y[r] = fma(hij, vj, y[r]);
          }
        }
      }
      return true;
    }
  }

  // Along a projected path the trial steps scale with the step length wherever neither
  // trial is clipped by the box (sn = kap so there, up to rounding), so H sn is
  // kap H so plus the columns of the coordinates clipped in either trial (cl), with
  // the full product when those are many.  Hs holds H so on entry, H sn on exit.
  __device__ __forceinline__ void rescaled_product(const double (&sn)[R], double kap,
                                                   const double (&so)[R], const bool (&cl)[R],
                                                   double (&Hs)[R]) {
    if constexpr (G == 1 || G > 32) {
      hv(sn, Hs);
      return;
    }
    double dl[R], Hd[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dl[r] = cl[r] ? fma(-kap, so[r], sn[r]) : 0.0;
    if (hv_sparse(dl, Hd)) {
#pragma unroll
      for (int r = 0; r < R; ++r) Hs[r] = fma(kap, Hs[r], Hd[r]);
    } else {
      hv(sn, Hs);
    }
  }

  // pivot test on the bit pattern (no FP64 compare): a positive, normal, finite value;
  // a subnormal pivot counts as not positive, so the shift takes over
  __device__ __forceinline__ static bool positive(double piv) {
    const long long b = __double_as_longlong(piv);
    return b >= 0x0010000000000000LL && b < 0x7FF0000000000000LL;
  }

  __device__ __forceinline__ static double pivot_rcp(double a) { return xt::pivot_rcp(a); }

  // ------------------------------------------------ LDL^T factorization (Sec. 4.3)
  // A = Lu D Lu^T with Lu unit lower triangular: the strictly lower part of the factor
  // storage holds Lu (mirrored into the upper triangle in the full layout), the
  // diagonal holds D and dinv holds 1/D.  The paper's L L^T is Lu D^(1/2); the PCG
  // below needs only M^-1 = Lu^-T D^-1 Lu^-1, so no square root is ever taken and each
  // column costs one reciprocal.

  // left-looking: column j gathers the updates of columns 0..j-1 (read from the
  // mirrored rows of Lu^T) against row j of D Lu^T, which is formed first over the
  // group; the pivots sit in dinv until the end, when all are inverted at once.
  __device__ __forceinline__ bool chol_left(int m) {
    for (int j = 0; j < m; ++j) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = r * G + gp.t;
        if (k < j) vb[k] = lo(j, k) * dinv[k];
      }
      gp.sync();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * G + gp.t;
        if (c >= j && c < m) {
          double v = lo(c, j);
          for (int k = 0; k < j; ++k) v = fma(-mt(k, c), vb[k], v);
          mt(j, c) = v;
        }
      }
      gp.sync();
      const double piv = mt(j, j);
      if (!positive(piv)) {
        gp.sync();
        return false;
      }
      const double ri = pivot_rcp(piv);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * G + gp.t;
        if (c > j && c < m) {
          const double lcj = mt(j, c) * ri;
          mt(j, c) = lcj;
          if (!PK) lo(c, j) = lcj;
        }
      }
      if (gp.t == (j & (G - 1))) dinv[j] = piv;
      gp.sync();
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = r * G + gp.t;
      if (c < m) dinv[c] = pivot_rcp(dinv[c]);
    }
    gp.sync();
    return true;
  }

  // right-looking with the trailing update spread over the whole group: after the pivot
  // of column j is inverted, the (m-j-1)(m-j)/2 elements of the trailing triangle are
  // updated by all G lanes (element e of the triangle -> row cc, column ec), so no lane
  // waits on the triangle's shape.  The update a_cd -= Lu_cj (D_j Lu_dj) reads the scaled
  // column from vb and the still unscaled one from the factor storage, which takes the
  // scaled values once the update is done.
  __device__ __forceinline__ bool chol_right(int m) {
    // row/column of element gp.t of a trailing triangle (the same for every j); later
    // elements of this lane follow by stepping G positions along the rows
    int cc0 = (int)((sqrtf(8.0f * (float)gp.t + 1.0f) - 1.0f) * 0.5f);
    while (cc0 * (cc0 + 1) / 2 > gp.t) --cc0;
    while ((cc0 + 1) * (cc0 + 2) / 2 <= gp.t) ++cc0;
    const int ec0 = gp.t - cc0 * (cc0 + 1) / 2;
    for (int j = 0; j < m; ++j) {
      if constexpr (G > 32) {
        if (j + 1 < m) {
          if (!two_columns(j, m, cc0, ec0)) return false;
          ++j;
          continue;
        }
      }
      const double piv = lo(j, j);
      if (!positive(piv)) {
        gp.sync();
        return false;
      }
      const double ri = pivot_rcp(piv);
      double lc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * G + gp.t;
        lc[r] = 0.0;
        if (c > j && c < m) {
          lc[r] = lo(c, j) * ri;
          vb[c] = lc[r];
        }
      }
      if (gp.t == (j & (G - 1))) dinv[j] = ri;
      gp.sync();
      const int M = m - j - 1;
      const int T = M * (M + 1) / 2;
      int cc = cc0, ec = ec0;
      for (int e = gp.t; e < T; e += G) {
        const int c = j + 1 + cc, d = j + 1 + ec;
        lo(c, d) = fma(-vb[c], lo(d, j), lo(c, d));
        ec += G;
        while (ec > cc) {
          ec -= cc + 1;
          ++cc;
        }
      }
      gp.sync();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * G + gp.t;
        if (c > j && c < m) {
          lo(c, j) = lc[r];
          if (!PK) mt(j, c) = lc[r];
        }
      }
    }
    gp.sync();
    return true;
  }

  // columns j and j + 1 of chol_right in one pass, for CTA groups, where each pass costs
  // two CTA barriers: the owners of the rows below first apply column j to their entry
  // of column j + 1 (which needs only Lu_{j+1,j} D_j, final when the pass starts), every
  // lane forms the pivot of column j + 1 the same way, and one sweep over the trailing
  // triangle applies column j and then column j + 1 to each element -- the operations of
  // two one-column passes in the same order, so the factor is the same bit for bit
  __device__ __forceinline__ bool two_columns(int j, int m, int cc0, int ec0) {
    const double p0 = lo(j, j);
    if (!positive(p0)) {
      gp.sync();
      return false;
    }
    const double r0 = pivot_rcp(p0);
    const double a10 = lo(j + 1, j);
    const double p1 = fma(-(a10 * r0), a10, lo(j + 1, j + 1));
    if (!positive(p1)) {
      gp.sync();
      return false;
    }
    const double r1 = pivot_rcp(p1);
    double lc0[R], lc1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = r * G + gp.t;
      lc0[r] = 0.0;
      lc1[r] = 0.0;
      if (c > j && c < m) {
        lc0[r] = lo(c, j) * r0;
        vb[c] = lc0[r];
        if (c > j + 1) {
          const double a1 = fma(-lc0[r], a10, lo(c, j + 1));  // column j + 1 after column j
          lo(c, j + 1) = a1;
          lc1[r] = a1 * r1;
          vb2[c] = lc1[r];
        }
      }
    }
    if (gp.t == (j & (G - 1))) dinv[j] = r0;
    if (gp.t == ((j + 1) & (G - 1))) dinv[j + 1] = r1;
    gp.sync();
    const int M = m - j - 2;
    const int T = M * (M + 1) / 2;
    int cc = cc0, ec = ec0;
    for (int e = gp.t; e < T; e += G) {
      const int c = j + 2 + cc, d = j + 2 + ec;
      lo(c, d) = fma(-vb2[c], lo(d, j + 1), fma(-vb[c], lo(d, j), lo(c, d)));
      ec += G;
      while (ec > cc) {
        ec -= cc + 1;
        ++cc;
      }
    }
    gp.sync();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = r * G + gp.t;
      if (c > j && c < m) {
        lo(c, j) = lc0[r];
        if (!PK) mt(j, c) = lc0[r];
      }
      if (c > j + 1 && c < m) {
        lo(c, j + 1) = lc1[r];
        if (!PK) mt(j + 1, c) = lc1[r];
      }
      if (c == j + 1) lo(c, c) = p1;
    }
    return true;
  }

  // shifted factorization A + alpha I = Lu D Lu^T, alpha from the sequence
  // 0 (or beta - min A_ii), then max(2 alpha, beta), beta = shift_frac * max |A_ii|.
  // Returns 0 when every shift failed, 1 for a factor of A itself (alpha = 0), 2 for a
  // shifted one.
  __device__ __forceinline__ int factor(int m) {
    // the first shift is 0 when every diagonal entry is positive (decided by a vote);
    // the max/min reductions that set beta are paid only when a shift is needed
    bool nonpos = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = r * G + gp.t;
      if (c < m) {
        const int i = Fi[c];
        double a = obj.hq(i, i);
        if (Obj::kHasHd) a = a + obj.hd(i);
        nonpos = nonpos || !(okey(a) > 0);  // finite: a non-finite Hessian stops earlier
      }
    }
    const bool all_pos = !gp.any(nonpos);
    double beta = 0.0, alpha = 0.0;
    bool have_beta = false;
    auto shift_stats = [&]() {
      double dmax = 0.0, dmin = CUDART_INF;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * G + gp.t;
        if (c < m) {
          const int i = Fi[c];
          double a = obj.hq(i, i);
          if (Obj::kHasHd) a = a + obj.hd(i);
          dmax = fmax(dmax, fabs(a));
          dmin = fmin(dmin, a);
        }
      }
      dmax = gp.max(dmax);
      dmin = gp.min(dmin);
      beta = o.shift_frac * dmax;
      if (beta == 0.0) beta = o.shift_frac;
      have_beta = true;
      return dmin;
    };
    if (!all_pos) {
      const double dmin = shift_stats();  // sets beta
      alpha = beta - dmin;
    }
    for (int tr = 0; tr <= o.max_shift; ++tr) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * G + gp.t;
        if (c < m) {
          const int i = Fi[c];
          for (int d = 0; d < c; ++d) lo(c, d) = obj.hq(i, Fi[d]);
          double a = obj.hq(i, i);
          if (Obj::kHasHd) a = a + obj.hd(i);
          lo(c, c) = a + alpha;
        }
      }
      gp.sync();
      // options.cholesky: 1 left-looking, 2 right-looking, 0 the size class's default
      const bool right = o.cholesky != 1;
      if (right ? chol_right(m) : chol_left(m)) return nonzero_bits(alpha) ? 2 : 1;
      if (!have_beta) shift_stats();
      alpha = fmax(2.0 * alpha, beta);
    }
    return 0;
  }

  // v <- M^-1 v, M = Lu D Lu^T: unit forward substitution with Lu (column j of Lu is
  // row j of the mirrored upper part), v <- D^-1 v, unit backward substitution with
  // Lu^T (column j of Lu^T is row j of Lu); every shared-memory read of a column is
  // contiguous across the group (Sec. 4.4)
  __device__ __forceinline__ void precond(int m, double (&v)[R]) {
#pragma unroll
    for (int rj = 0; rj < R; ++rj) {
      for (int tj = 0; tj < G; ++tj) {
        const int j = rj * G + tj;
        if (j >= m) break;
        const double vj = gp.bcast(v[rj], tj);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int c = r * G + gp.t;
          if (c > j && c < m) v[r] = fma(-mt(j, c), vj, v[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = r * G + gp.t;
      if (c < m) v[r] = v[r] * dinv[c];
    }
#pragma unroll
    for (int rj = R - 1; rj >= 0; --rj) {
      for (int tj = G - 1; tj >= 0; --tj) {
        const int j = rj * G + tj;
        if (j >= m) continue;
        const double vj = gp.bcast(v[rj], tj);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int c = r * G + gp.t;
          if (c < j) v[r] = fma(-lo(j, c), vj, v[r]);
        }
      }
    }
  }

  // trqsol (Figure 2) from the three inner products of x and p in the trust-region
  // norm: sigma >= 0 with xx + 2 sigma xp + sigma^2 pp = delta^2 (the positive root,
  // in the form without cancellation)
  __device__ __forceinline__ static double trqsol3(double xp, double pp, double xx,
                                                   double delta) {
    const double dsq = delta * delta;
    double rad = xp * xp + pp * (dsq - xx);
    if (okey(rad) < 0) rad = 0.0;
    rad = square_root(rad);
    return (okey(xp) >= 0) ? quotient(dsq - xx, xp + rad) : quotient(rad - xp, pp);
  }
  // trqsol (Figure 2): sigma >= 0 with ||x + sigma p||_2 = delta
  __device__ __forceinline__ double trqsol(const double (&x)[R], const double (&p)[R],
                                           double delta) const {
    double ptx = 0.0, ptp = 0.0, xtx = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ptx = fma(p[r], x[r], ptx);
      ptp = fma(p[r], p[r], ptp);
      xtx = fma(x[r], x[r], xtx);
    }
    gp.sum3(ptx, ptp, xtx);
    return trqsol3(ptx, ptp, xtx, delta);
  }

  // Steihaug PCG of Algorithm 1 for min rF'w + 1/2 w'Aw inside the trust region, run in
  // the step w itself with the preconditioner M = A + alpha I = L L^T.  With
  // phat = L^T p and rhat = L^-1 res this is CG on Ahat = L^-1 A L^-T in s = L^T w step
  // for step: the same step lengths (rhat'rhat = res'M^-1 res, phat'Ahat phat = p'Ap)
  // and the same exits.  Algorithm 1's trust region bounds the CG iterate,
  // ||s||_2 = ||w||_M <= delta (options.tr_norm 0); its M-inner products come from the
  // recurrences of preconditioned CG, with no product by M (w1, p1, res1: the next
  // iterate, direction and residual):
  //   ||w1||_M^2 = ||w + alpha p||_M^2 = ww + 2 alpha wp + alpha^2 pp,
  //   <w1, p1>_M = beta (wp + alpha pp),   ||p1||_M^2 = res1' M^-1 res1 + beta^2 pp,
  // which hold because res1 is orthogonal to every earlier direction (w1 lies in their
  // span, and M p1 = res1 + beta M p).  tr_norm 1 bounds ||w||_2 instead.  When alpha = 0,
  // M = A and Ahat = I: the first step, of length 1 along M^-1 res, is the minimiser and
  // leaves a zero residual, so it is taken without forming A p; its length is
  // ||M^-1 res||_M^2 = res'M^-1 res.
  // Returns 0 converged, 1 iteration cap, 2 boundary, 3 negative curvature; wscale is
  // sigma > 0 when w was taken that way (then A w = -sigma rF), else 0; tl2 is the
  // squared length of w in the bounded norm (tr_norm 0; 0 with tr_norm 1).  With
  // tr_norm 1 the three inner products are formed from w and p before each step, and
  // the boundary test and trqsol use them as with tr_norm 0.
  __device__ __forceinline__ int steihaug(int m, double delta, bool exact,
                                          const double (&rF)[R], double (&w)[R],
                                          double& wscale, double& tl2) {
    wscale = 0.0;
    tl2 = 0.0;
    const bool pre = (o.tr_norm == 0);
    double res[R], z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      w[r] = 0.0;
      res[r] = -rF[r];
      z[r] = res[r];
    }
    precond(m, z);
    const double dsq = delta * delta;
    if (exact) {
      const double zz = pre ? dotv(res, z) : dotv(z, z);
      const bool bnd = le(dsq, zz);
      const double sg = bnd ? quotient(delta, square_root(zz)) : 1.0;
#pragma unroll
      for (int r = 0; r < R; ++r) w[r] = sg * z[r];
      wscale = sg;  // A w = -sg rF
      if (pre) tl2 = bnd ? dsq : zz;
      return bnd ? 2 : 0;
    }
    double p[R], q[R];
    double rz = dotv(res, z);
    const double tol2 = (o.cg_rtol * o.cg_rtol) * rz;  // ||rhat|| <= cg_rtol ||rhat_0||, squared
#pragma unroll
    for (int r = 0; r < R; ++r) p[r] = z[r];
    // inner products of w and p in the bounded norm: by the recurrences (tr_norm 0), or
    // formed from the vectors before each step (tr_norm 1)
    double ww = 0.0, wp = 0.0, pp = rz;
    int info = 1;
    for (int it = 0; it < m; ++it) {
      if (le(rz, tol2)) {
        info = 0;
        break;
      }
      if (!pre) {
        ww = 0.0;
        wp = 0.0;
        pp = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          ww = fma(w[r], w[r], ww);
          wp = fma(w[r], p[r], wp);
          pp = fma(p[r], p[r], pp);
        }
        gp.sum3(ww, wp, pp);
      }
      hv_free(m, p, q);
      const double kappa = dotv(p, q);
      const double alpha = quotient(rz, kappa);
      // negative curvature, or the step leaves the region: to the boundary along p
      const bool negc = !(okey(kappa) > 0);
      if (negc || le(dsq, fma(alpha, fma(alpha, pp, 2.0 * wp), ww))) {
        const double sg = trqsol3(wp, pp, ww, delta);
#pragma unroll
        for (int r = 0; r < R; ++r) w[r] = fma(sg, p[r], w[r]);
        info = negc ? 3 : 2;
        break;
      }
      ww = fma(alpha, fma(alpha, pp, 2.0 * wp), ww);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        w[r] = fma(alpha, p[r], w[r]);
        res[r] = fma(-alpha, q[r], res[r]);
        z[r] = res[r];
      }
      precond(m, z);
      const double rzn = dotv(res, z);
      const double beta = quotient(rzn, rz);
      rz = rzn;
      wp = beta * fma(alpha, pp, wp);
      pp = fma(beta * beta, pp, rz);
#pragma unroll
      for (int r = 0; r < R; ++r) p[r] = fma(beta, p[r], z[r]);
    }
    if (pre) tl2 = (info >= 2) ? dsq : ww;
    return info;
  }

  // Cauchy trial s(alpha) = P[x - alpha g] - x: q(s) <= mu0 g's and ||s|| <= mu1 delta
  // (||s||_2, or with options.cauchy_norm 1 the model Hessian's norm (s'Hs)^(1/2) where
  // s'Hs > 0).
  // kap = 0 for the first trial of a search (full product); otherwise alpha is kap times
  // the step length of the trial held in s, Hs, cl (clipped coordinates), and H s is
  // rescaled from it.  inside: alpha is below the largest breakpoint along -g (breakpt of
  // Figure 2), i.e. some coordinate that -g moves is still strictly inside its box at
  // x - alpha g: decided on the trial's own integer keys, without the breakpoints'
  // divisions.
  __device__ __forceinline__ bool cauchy_try(double alpha, const double (&x)[R],
                                             const double (&g)[R], double bound2,
                                             double (&s)[R], double (&Hs)[R], bool (&cl)[R],
                                             double kap, bool& inside, double& ssq) {
    double sn[R];
    bool cn[R];
    bool mv = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double v = fma(alpha, -g[r], x[r]);
      const long long k = okey(v);
      cn[r] = (k < kl[r]) || (k > ku[r]);
      mv = mv || (kl[r] < k && k < ku[r] && okey(g[r]) != 0);
      sn[r] = P(v, r) - x[r];
    }
    inside = gp.any(mv);
    if (nonzero_bits(kap)) {
      bool both[R];
#pragma unroll
      for (int r = 0; r < R; ++r) both[r] = cn[r] || cl[r];
      rescaled_product(sn, kap, s, both, Hs);
    } else {
      hv(sn, Hs);
    }
    double gts = 0.0, sHs = 0.0, ss = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      s[r] = sn[r];
      cl[r] = cn[r];
      gts = fma(g[r], s[r], gts);
      sHs = fma(s[r], Hs[r], sHs);
      ss = fma(s[r], s[r], ss);
    }
    gp.sum3(gts, sHs, ss);
    // squared length for the trust-region test: ||s||_2^2, or (cauchy_norm 1) s'Hs where
    // it is positive
    const double len2 = (o.cauchy_norm == 1 && okey(sHs) > 0) ? sHs : ss;
    ssq = len2;
    const double q = gts + 0.5 * sHs;
    return le(q, o.mu0 * gts) && le(len2, bound2);
  }

  __device__ __forceinline__ bool all_finite(const double (&v)[R]) const {
    bool fin = true;
#pragma unroll
    for (int r = 0; r < R; ++r) fin = fin && finite_bits(v[r]);
    return !gp.any(!fin);
  }

  // H d for the projected search's first trial d = P[y + w] - y when nothing is clipped
  // and w came from the exact-preconditioner step: on the free rows H_FF w_F = -sigma rF
  // (rF is rv there), so only the rows of the bound variables (at most 6, d = 0 on
  // them) need their dot products, reduced three at a time in fused butterflies.  One
  // variable per lane only; false, with nothing computed, otherwise.
  __device__ __forceinline__ bool first_trial_known(double wscale, const int (&cidx)[R],
                                                    const bool (&cn)[R], const double (&rv)[R],
                                                    const double (&d)[R], double (&Hd)[R]) {
    if constexpr (R != 1 || G == 1 || G > 32) {
      return false;
    } else {
      if (!nonzero_bits(wscale) || gp.any(cn[0])) return false;
      const bool bnd = cidx[0] < 0 && gp.t < n;
      unsigned mm = gp.ballot(bnd);
      if (__popc(mm) > 6) return false;
      double h = (cidx[0] >= 0) ? -wscale * rv[0] : 0.0;
      while (mm) {  // group-uniform: up to three bound rows per fused reduction
        int ib[3] = {-1, -1, -1};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (mm) {
            ib[q] = __ffs(mm) - 1;
            mm &= mm - 1u;
          }
        }
        double p0 = ib[0] >= 0 ? obj.hq(ib[0], gp.t) * d[0] : 0.0;
        double p1 = ib[1] >= 0 ? obj.hq(ib[1], gp.t) * d[0] : 0.0;
        double p2 = ib[2] >= 0 ? obj.hq(ib[2], gp.t) * d[0] : 0.0;
        gp.sum3(p0, p1, p2);
        if (gp.t == ib[0]) h = p0;
        if (gp.t == ib[1]) h = p1;
        if (gp.t == ib[2]) h = p2;
      }
      Hd[0] = h;
      return true;
    }
  }

  // ------------------------------------------------------------------- Algorithm 1
  __device__ int run(double (&x)[R], double& delta, double& f, double& pg, int& k,
                     bool params_finite) {
    k = k_start;
    {
      bool bad = false;
#pragma unroll
      for (int r = 0; r < R; ++r) bad = bad || !(l[r] <= u[r]);
      if (gp.any(bad)) {
        f = CUDART_NAN;
        pg = CUDART_NAN;
        return TRON_BAD_BOUNDS;
      }
    }
    key_bounds();
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = P(x[r], r);
    double g[R];
    f = obj.eval_f(gp, x);
    double fs = obj.fsc;  // rounding scale of f at x
    obj.grad_hess(gp, x, g);
    if (!params_finite || !finite_bits(f) || !all_finite(g) || !obj.hess_finite(gp)) {
      pg = finite_bits(f) ? pgnorm(x, g) : CUDART_NAN;
      return TRON_NONFINITE;
    }
    if (!(delta > 0.0)) {
      double s[R];
#pragma unroll
      for (int r = 0; r < R; ++r) s[r] = P(x[r] - g[r], r) - x[r];
      delta = sqrt(dotv(s, s));
      if (delta == 0.0) delta = 1.0;
    }
    double alpha_c = alpha0;
    int status = TRON_MAX_ITER;
    // ||x||^2 <= xb2 for every x in the box (infinite when a bound is)
    double xb2 = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      // max(|l_i|, |u_i|) on the magnitude bits (the bounds are not NaN past the test above)
      const long long ml = __double_as_longlong(l[r]) & 0x7FFFFFFFFFFFFFFFLL;
      const long long mu = __double_as_longlong(u[r]) & 0x7FFFFFFFFFFFFFFFLL;
      const double mb = __longlong_as_double(ml > mu ? ml : mu);
      xb2 = fma(mb, mb, xb2);
    }
    xb2 = gp.sum(xb2);

    for (;;) {
      // ||grad_P f||_inf <= gtol decided by a vote of the lanes; the norm itself is
      // reduced once, at exit
      if (!pg_above(x, g, o.gtol)) {
        status = TRON_CONVERGED;
        break;
      }
      if (k >= o.max_outer) {
        status = TRON_MAX_ITER;
        break;
      }
      if (k >= pause_at) {
        status = kTronPaused;
        break;
      }
      ++k;

      // ---- Cauchy point
      double s[R], Hs[R];
      bool cl[R];
      double alpha = alpha_c;
      const double bmu = o.mu1 * delta;
      const double bound2 = bmu * bmu;  // (mu1 delta)^2 of the trials' length test
      bool inside;
      double ssc;  // squared length of the accepted Cauchy step (in the test's norm)
      if (cauchy_try(alpha, x, g, bound2, s, Hs, cl, 0.0, inside, ssc)) {
        double sb[R], Hsb[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          sb[r] = s[r];
          Hsb[r] = Hs[r];
        }
        double ssb = ssc;
        for (int t = 0; t < o.max_trials; ++t) {
          if (!inside) break;  // alpha at or beyond the largest breakpoint
          const double a2 = alpha * o.extrapf;
          if (!cauchy_try(a2, x, g, bound2, s, Hs, cl, o.extrapf, inside, ssc)) break;
          alpha = a2;
          ssb = ssc;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            sb[r] = s[r];
            Hsb[r] = Hs[r];
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          s[r] = sb[r];
          Hs[r] = Hsb[r];
        }
        ssc = ssb;
      } else {
        for (int t = 0; t < o.max_trials; ++t) {
          alpha = alpha * o.interpf;
          if (cauchy_try(alpha, x, g, bound2, s, Hs, cl, o.interpf, inside, ssc)) break;
        }
      }
      // squared length of the step in the norms of the trust regions that bounded its
      // pieces (tr_norm 0): the Cauchy step in ||.||_2, each subspace pass's search step
      // beta w in the PCG's norm; the radius update measures the step by it
      double nu2 = ssc;
      alpha_c = alpha;
      double y[R], rv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // x_c = P[x - alpha g]; y - x equals the s of the accepted trial bit for bit,
        // so the model gradient at x_c is g + Hs without another product
        y[r] = P(fma(-alpha, g[r], x[r]), r);
        rv[r] = g[r] + Hs[r];
      }

      // ---- subspace passes: free set, factorization, PCG, back transform, search
      double rF0 = 0.0;
      for (int pass = 0; pass < n; ++pass) {
        int cidx[R];
        int m = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const bool fr = strictly_inside(y[r], r);
          int tot;
          const int pre = gp.prefix(fr, tot);
          cidx[r] = fr ? m + pre : -1;
          m += tot;
        }
        if (m == 0) break;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (cidx[r] >= 0) Fi[cidx[r]] = r * G + gp.t;
          vb[r * G + gp.t] = rv[r];
        }
        gp.sync();
        double rF[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int c = r * G + gp.t;
          rF[r] = (c < m) ? vb[Fi[c]] : 0.0;
        }
        gp.sync();
        const int fac = factor(m);
        if (fac == 0) {
          status = TRON_CHOL_FAIL;
          break;
        }
        double wF[R], wscale, tl2;
        const int info = steihaug(m, delta, fac == 1, rF, wF, wscale, tl2);
        // scatter w_F to the full direction w
#pragma unroll
        for (int r = 0; r < R; ++r) vb[r * G + gp.t] = 0.0;
        gp.sync();
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int c = r * G + gp.t;
          if (c < m) vb[Fi[c]] = wF[r];
        }
        gp.sync();
        double w[R];
#pragma unroll
        for (int r = 0; r < R; ++r) w[r] = vb[r * G + gp.t];
        gp.sync();
        // projected search from y along w
        double beta = 1.0;
        bool found = false;
        double yt[R], d[R], Hd[R];
        bool dcl[R];
        for (int t = 0; t < o.max_trials; ++t) {
          double dn[R];
          bool cn[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double v = fma(beta, w[r], y[r]);
            const long long k = okey(v);
            cn[r] = (k < kl[r]) || (k > ku[r]);
            yt[r] = P(v, r);
            dn[r] = yt[r] - y[r];
          }
          // after the first trial, H d is rescaled from the previous one (the step
          // length shrinks by proj_shrink)
          if (t == 0) {
            if (!first_trial_known(wscale, cidx, cn, rv, dn, Hd)) hv(dn, Hd);
          } else {
            bool both[R];
#pragma unroll
            for (int r = 0; r < R; ++r) both[r] = cn[r] || dcl[r];
            rescaled_product(dn, o.proj_shrink, d, both, Hd);
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            d[r] = dn[r];
            dcl[r] = cn[r];
          }
          double rtd = 0.0, dHd = 0.0;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            rtd = fma(rv[r], d[r], rtd);
            dHd = fma(d[r], Hd[r], dHd);
          }
          gp.sum2(rtd, dHd);
          if (le(fma(0.5, dHd, rtd), o.mu0 * rtd)) {
            found = true;
            break;
          }
          beta = beta * o.proj_shrink;
        }
        if (!found) break;
        {
          const double c = (beta * beta) * tl2;
          if (lt(nu2, c)) nu2 = c;
        }
        bool na = false;
        double ss = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (cidx[r] >= 0 && !strictly_inside(yt[r], r)) na = true;
          y[r] = yt[r];
          rv[r] = rv[r] + Hd[r];
          if (cidx[r] >= 0) ss = fma(rv[r], rv[r], ss);
        }
        const bool newly_active = gp.any(na);
        if (info == 2 || info == 3 || newly_active) break;
        // ||rF||^2 after the pass against cg_rtol^2 ||rF||^2 before the first pass (both
        // squared); the first pass reduces the two together, and neither is formed when
        // the pass already ended on the boundary, on negative curvature or a new bound
        double rFn2 = ss;
        if (pass == 0) {
          double r0 = 0.0;
#pragma unroll
          for (int r = 0; r < R; ++r) r0 = fma(rF[r], rF[r], r0);
          gp.sum2(rFn2, r0);
          rF0 = r0;
        } else {
          rFn2 = gp.sum(rFn2);
        }
        if (le(rFn2, (o.cg_rtol * o.cg_rtol) * rF0)) break;
      }
      if (status == TRON_CHOL_FAIL) break;

      // ---- reduction ratio, acceptance, radius
      // q(s) = g's + 1/2 s'Hs with s = y - x; the model gradient rv = g + H s was
      // accumulated along the steps, so H s = rv - g needs no further product
      double s2[R], hs2[R], gts = 0.0, sHs = 0.0, ss2 = 0.0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        s2[r] = y[r] - x[r];
        hs2[r] = rv[r] - g[r];
        gts = fma(g[r], s2[r], gts);
        sHs = fma(s2[r], hs2[r], sHs);
        ss2 = fma(s2[r], s2[r], ss2);
      }
      gp.sum3(gts, sHs, ss2);
      const double qs = gts + 0.5 * sHs;
      double fy;
      if constexpr (Obj::kStepEval) fy = obj.eval_f_step(gp, y, s2, hs2);
      else fy = obj.eval_f(gp, y);
      const double fsy = obj.fsc;
      // ratio guarded by the rounding level of f (Conn, Gould and Toint, Trust-Region
      // Methods, Sec. 17.4.2), measured on the magnitudes of the terms of f
      const double pred = -qs;
      const double ared = f - fy;
      const double fl = o.ared_guard * (le(fs, 1.0) ? 1.0 : fs);  // max(1, S), S >= 0
      // rho = (ared + fl) / (pred + fl) is compared with each eta as
      // ared + fl > eta (pred + fl), the denominator being positive: no division; an
      // invalid ratio (pred <= 0 or f(y) not finite) counts as -infinity
      const bool valid = (okey(pred) > 0) && finite_bits(fy) && finite_bits(pred);
      const double num = ared + fl, den = pred + fl;
      const bool above0 = valid && lt(o.eta0 * den, num);
      const bool below1 = !valid || lt(num, o.eta1 * den);
      const bool above2 = valid && lt(o.eta2 * den, num);
      if (above0) {
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = y[r];
        f = fy;
        fs = fsy;
        obj.grad_hess(gp, x, g);
        if (!all_finite(g) || !obj.hess_finite(gp)) {
          status = TRON_NONFINITE;
          break;
        }
      }
      // the step's length: in the norms that bounded its pieces (tr_norm 0), or
      // ||y - x||_2 (tr_norm 1); ||s|| >= 0.99 delta compared squared, the norm itself
      // formed only when it sets delta
      const double sl2 = (o.tr_norm == 0) ? nu2 : ss2;
      const double d99 = 0.99 * delta;
      if (below1) {
        const double sl = square_root(sl2);
        delta = o.sigma1 * (lt(sl, delta) ? sl : delta);
      } else if (above2 && le(d99 * d99, sl2)) {
        const double dg = o.sigma3 * delta;
        delta = lt(o.delta_max, dg) ? o.delta_max : dg;
      }
      // delta < c (1 + ||x||), decided without a square root:
      // delta - c < 0, or (delta - c)^2 < c^2 ||x||^2; ||x|| is reduced only when the
      // box bound xb2 cannot decide
      const double dc = delta - o.delta_min_rel;
      const double c2 = o.delta_min_rel * o.delta_min_rel;
      if (okey(dc) < 0 || (lt(dc * dc, c2 * xb2) && lt(dc * dc, c2 * dotv(x, x)))) {
        status = TRON_TR_TOO_SMALL;
        break;
      }
    }
    alpha_out = alpha_c;
    if (status == kTronPaused) return status;
    pg = pgnorm(x, g);
    return status;
  }
};

}  // namespace xt
