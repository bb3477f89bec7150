// tron_common.cuh -- thread-group primitives shared by the TRON device code.
//
// A problem is solved by a group of G lanes of one warp (G = 1, 2, 4, 8, 16, 32).
// Lane t of the group owns the variables i = r*G + t, r = 0..N/G-1 ("slots"), so every
// vector of a problem lives in registers spread over the group (data-level parallelism,
// Sec. 5.2).  Reductions use register shuffles inside the group with a butterfly, which
// leaves the result in every lane and needs no broadcast step (Sec. 5.1, Figure 4).
//
// FP64 on this GPU: a warp-wide FP64 instruction costs the same issue slot whether one
// lane or all 32 are active, so the mapping keeps lanes busy: G = 32 (one variable per
// lane) for n = 32; for the 4-variable branch problems G = 1 (one problem per lane, the
// fewest instructions) when they are many per SM, G = 4 when they are few (a launch then
// lasts as long as its slowest problem, whose serial chain four lanes shorten).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <type_traits>

namespace xt {

// tests on the IEEE bit pattern, so they take no FP64 instruction (the FP64 unit is the
// bottleneck of the solver), each the same predicate as its comparison for every input,
// NaN included: finite (exponent not all ones); nonzero (v != 0: any bit but the sign);
// positive (v > 0: sign clear, nonzero, at most +infinity)
__device__ __forceinline__ bool finite_bits(double v) {
  return (__double_as_longlong(v) & 0x7FF0000000000000LL) != 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool nonzero_bits(double v) {
  return (__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL) != 0;
}
__device__ __forceinline__ bool positive_bits(double v) {
  const long long b = __double_as_longlong(v);
  return b > 0 && b <= 0x7FF0000000000000LL;
}

template <int G>
struct Grp {
  static_assert(G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32 || G == 64 ||
                    G == 128,
                "group size");
  int lane;       // lane in the warp
  int t;          // rank in the group
  unsigned mask;  // lanes of this group

  __device__ __forceinline__ Grp() {
    lane = threadIdx.x & 31;
    t = lane & (G - 1);
    mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  }
  __device__ __forceinline__ void sync() const {
    if (G > 1) __syncwarp(mask);
  }
  __device__ __forceinline__ double sum(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
  }
  // two and three sums at once: the first butterfly level sends each lane the value
  // its partner does not keep, so both halves of the group reduce a different quantity
  // and the remaining levels cost one addition for all of them; the results are read
  // back from the owning lanes, identical in every lane
  __device__ __forceinline__ void sum2(double& a, double& b) const {
    if constexpr (G >= 2) {
      const bool hi = (t & (G / 2)) != 0;
      double keep = hi ? b : a, send = hi ? a : b;
      keep += __shfl_xor_sync(mask, send, G / 2, G);
#pragma unroll
      for (int o = G / 4; o > 0; o >>= 1) keep += __shfl_xor_sync(mask, keep, o, G);
      a = __shfl_sync(mask, keep, 0, G);
      b = __shfl_sync(mask, keep, G / 2, G);
    } else {
      a = sum(a);
      b = sum(b);
    }
  }
  __device__ __forceinline__ void sum3(double& a, double& b, double& c) const {
    if constexpr (G >= 4) {
      // level G/2: the low half keeps (a, b), the high half (c, 0)
      const bool hi = (t & (G / 2)) != 0;
      double k0 = hi ? c : a, k1 = hi ? 0.0 : b;
      const double s0 = hi ? a : c, s1 = hi ? b : 0.0;
      k0 += __shfl_xor_sync(mask, s0, G / 2, G);
      k1 += __shfl_xor_sync(mask, s1, G / 2, G);
      // level G/4: in each half, lanes with that bit clear keep k0, set keep k1
      const bool b2 = (t & (G / 4)) != 0;
      double keep = b2 ? k1 : k0;
      const double send = b2 ? k0 : k1;
      keep += __shfl_xor_sync(mask, send, G / 4, G);
#pragma unroll
      for (int o = G / 8; o > 0; o >>= 1) keep += __shfl_xor_sync(mask, keep, o, G);
      a = __shfl_sync(mask, keep, 0, G);
      b = __shfl_sync(mask, keep, G / 4, G);
      c = __shfl_sync(mask, keep, G / 2, G);
    } else {
      a = sum(a);
      sum2(b, c);
    }
  }
  __device__ __forceinline__ double max(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
  __device__ __forceinline__ double min(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
  // ballot restricted to the group, bit k = rank k
  __device__ __forceinline__ unsigned ballot(bool p) const {
    if (G == 1) return p ? 1u : 0u;
    unsigned b = __ballot_sync(mask, p) & mask;
    return b >> (lane & ~(G - 1));
  }
  __device__ __forceinline__ bool any(bool p) const { return ballot(p) != 0u; }
  // exclusive prefix count of p over the ranks below t, and the group total
  __device__ __forceinline__ int prefix(bool p, int& total) const {
    const unsigned b = ballot(p);
    total = __popc(b);
    return __popc(b & ((1u << t) - 1u));
  }
  __device__ __forceinline__ double bcast(double v, int src) const {
    if (G == 1) return v;
    return __shfl_sync(mask, v, src, G);
  }
  // value of rank t-1 (rank 0 gets its own) and of rank t+1 (the last rank its own)
  __device__ __forceinline__ double from_prev(double v) const {
    if (G == 1) return v;
    return __shfl_up_sync(mask, v, 1, G);
  }
  __device__ __forceinline__ double from_next(double v) const {
    if (G == 1) return v;
    return __shfl_down_sync(mask, v, 1, G);
  }
  __device__ __forceinline__ int bcast(int v, int src) const {
    if (G == 1) return v;
    return __shfl_sync(mask, v, src, G);
  }
  // value of rank t ^ o (0 < o < G)
  __device__ __forceinline__ double exch(double v, int o) const {
    if (G == 1) return v;
    return __shfl_xor_sync(mask, v, o, G);
  }
};

// A group spanning a whole CTA (G = 64 or 128 threads, one problem per CTA) for the
// large size classes: reductions combine warp butterflies with a fixed-order pass over
// the warps' partial results in shared memory, so every thread gets the same bits.
template <int G>
struct GrpCta {
  static_assert(G == 64 || G == 128, "CTA group size");
  static constexpr int W = G / 32;
  int lane;
  int t;
  unsigned mask;

  __device__ __forceinline__ GrpCta() {
    t = threadIdx.x;
    lane = t & 31;
    mask = 0xffffffffu;
  }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ double wsum(double v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
  __device__ __forceinline__ double sum(double v) const {
    __shared__ double red[W];
    v = wsum(v);
    if (lane == 0) red[t >> 5] = v;
    __syncthreads();
    double s = red[0];
#pragma unroll
    for (int w = 1; w < W; ++w) s += red[w];
    __syncthreads();
    return s;
  }
  __device__ __forceinline__ void sum2(double& a, double& b) const {
    __shared__ double red[2][W];
    a = wsum(a);
    b = wsum(b);
    if (lane == 0) {
      red[0][t >> 5] = a;
      red[1][t >> 5] = b;
    }
    __syncthreads();
    a = red[0][0];
    b = red[1][0];
#pragma unroll
    for (int w = 1; w < W; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    __syncthreads();
  }
  __device__ __forceinline__ void sum3(double& a, double& b, double& c) const {
    __shared__ double red[3][W];
    a = wsum(a);
    b = wsum(b);
    c = wsum(c);
    if (lane == 0) {
      red[0][t >> 5] = a;
      red[1][t >> 5] = b;
      red[2][t >> 5] = c;
    }
    __syncthreads();
    a = red[0][0];
    b = red[1][0];
    c = red[2][0];
#pragma unroll
    for (int w = 1; w < W; ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
    }
    __syncthreads();
  }
  __device__ __forceinline__ double max(double v) const {
    __shared__ double red[W];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[t >> 5] = v;
    __syncthreads();
    double s = red[0];
#pragma unroll
    for (int w = 1; w < W; ++w) s = fmax(s, red[w]);
    __syncthreads();
    return s;
  }
  __device__ __forceinline__ double min(double v) const {
    __shared__ double red[W];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[t >> 5] = v;
    __syncthreads();
    double s = red[0];
#pragma unroll
    for (int w = 1; w < W; ++w) s = fmin(s, red[w]);
    __syncthreads();
    return s;
  }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
  __device__ __forceinline__ int prefix(bool p, int& total) const {
    __shared__ int cnt[W];
    const unsigned b = __ballot_sync(0xffffffffu, p);
    if (lane == 0) cnt[t >> 5] = __popc(b);
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      if (w < (t >> 5)) before += cnt[w];
      total += cnt[w];
    }
    __syncthreads();
    return before + __popc(b & ((1u << lane) - 1u));
  }
  __device__ __forceinline__ double bcast(double v, int src) const {
    __shared__ double slot;
    if (t == src) slot = v;
    __syncthreads();
    const double r = slot;
    __syncthreads();
    return r;
  }
};

template <int G>
using GroupOf = typename std::conditional<(G > 32), GrpCta<G>, Grp<G>>::type;

// View of one problem's slice of shared memory.  With G = 1 the 32 problems of a warp
// are interleaved element by element (element k of lane q at k*32 + q), so a warp-wide
// access is always conflict free; with G >= 2 each problem owns a contiguous slice.
template <int G, typename T = double>
struct SV {
  T* p;
  __device__ __forceinline__ T& operator[](int k) const { return p[(G == 1) ? k * 32 : k]; }
  __device__ __forceinline__ SV at(int off) const { return SV{p + ((G == 1) ? off * 32 : off)}; }
};

// 1/d of a positive normal pivot d: the hardware reciprocal approximation refined by one
// Newton-Raphson step y <- y + y (1 - d y), which squares its relative error; two FP64
// instructions.  Pivots from 2^1022 up (whose reciprocal the approximation flushes to
// zero) divide.
__device__ __forceinline__ double pivot_rcp(double a) {
  if (__double_as_longlong(a) >= 0x7FD0000000000000LL) return 1.0 / a;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  return fma(y, fma(-a, y, 1.0), y);
}

// On this GPU an IEEE double division or square root is a sequence about nine FP64
// instructions deep, and every FP64 warp instruction holds the sub-partition's FP64 unit
// for a fixed time whatever the number of active lanes.  The two below take six or seven,
// from the hardware approximations.  Both are faithful (error below one ulp) and, with a
// seed accurate to 2^-20, round correctly in all but rare cases near a rounding midpoint;
// operands outside their range take the IEEE operation.
//
// a / b: Markstein's scheme (P. Markstein, IBM J. Res. Develop. 34(1), 1990): the
// reciprocal seed y0 with e = 1 - b y0 gives y = y0 (1 + e + e^2), relative error e^3;
// the remainder r = a - b q0 of the first quotient q0 = a y0 is exact up to its own
// rounding, and q0 + r y is the quotient.  Fast path: a and b normal, a away from the
// bottom of the range (r stays normal) and below 2^1023 (so a y0 cannot overflow through
// the seed's error), 1/b normal, the quotient's exponent within 1000 of zero; zeros
// (signed), subnormals, infinities and NaNs take a / b.
__device__ __forceinline__ double quotient(double a, double b) {
  const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
  const int ea = (int)((ba >> 52) & 0x7FF), eb = (int)((bb >> 52) & 0x7FF);
  const int dq = ea - eb;
  if (ea >= 64 && ea <= 2045 && eb >= 2 && eb <= 2044 && dq >= -1000 && dq <= 1000) {
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(b));
    const double e = fma(-b, y0, 1.0);
    const double q0 = a * y0;
    const double e2 = fma(e, e, e);
    const double r = fma(-b, q0, a);
    const double y = fma(y0, e2, y0);
    return fma(r, y, q0);
  }
  return a / b;
}

// sqrt(x): Goldschmidt's iteration from the reciprocal square-root seed y0 (s = x y0,
// h = y0 / 2, r = 1/2 - s h; s += s r, h += h r), then one Newton correction of s with
// the exact residual x - s^2 (Markstein, ibid.).  Fast path: x positive and normal with
// exponent field in [64, 1980) (so y0 / 2 is an exponent decrement); otherwise sqrt.
__device__ __forceinline__ double square_root(double x) {
  const long long bx = __double_as_longlong(x);
  if (bx >= (64LL << 52) && bx < (1980LL << 52)) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
    const double s0 = x * y0;
    const double h0 = __longlong_as_double(__double_as_longlong(y0) - (1LL << 52));
    const double r = fma(-s0, h0, 0.5);
    const double s1 = fma(s0, r, s0);
    const double h1 = fma(h0, r, h0);
    const double d = fma(-s1, s1, x);
    return fma(d, h1, s1);
  }
  return sqrt(x);
}

// sin x (cosine false) or cos x (cosine true) for |x| <= pi/4: the Taylor series to the
// x^19 (sine) or x^18 (cosine) term -- coefficients (-1)^k / (2k+1)! and (-1)^k / (2k)!,
// remainder below 4e-21 on that range -- evaluated as m + m z P(z), z = x^2, m = x
// (sine) or 1 (cosine), P by Horner's rule in z: eleven FP64 instructions against about
// twenty for the library's sin, and an error below one ulp (0.61 and 0.80 ulp at most in
// an exact-arithmetic check of this evaluation over 20,000 arguments).  The sine and the
// cosine share one instruction stream, so the lanes of a warp may take either without
// diverging.
__device__ __forceinline__ double sin_cos_small(double x, bool cosine) {
  constexpr double S[9] = {-0.16666666666666666,     0.008333333333333333,
                           -0.0001984126984126984,   2.7557319223985893e-06,
                           -2.505210838544172e-08,   1.6059043836821613e-10,
                           -7.647163731819816e-13,   2.8114572543455206e-15,
                           -8.22063524662433e-18};
  constexpr double C[9] = {-0.5,                     0.041666666666666664,
                           -0.001388888888888889,    2.48015873015873e-05,
                           -2.755731922398589e-07,   2.08767569878681e-09,
                           -1.1470745597729725e-11,  4.779477332387385e-14,
                           -1.5619206968586225e-16};
  const double m = cosine ? 1.0 : x;
  const double z = x * x;
  const double mz = m * z;
  double p = cosine ? C[8] : S[8];
#pragma unroll
  for (int k = 7; k >= 0; --k) p = fma(p, z, cosine ? C[k] : S[k]);
  // sin(+-0) = +-0 (the sum would give +0 for -0)
  return (cosine || nonzero_bits(x)) ? fma(mz, p, m) : x;
}
// |x| <= pi/4 (the double nearest pi/4), on the magnitude bits
__device__ __forceinline__ bool small_angle(double x) {
  return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL) <= 0x3FE921FB54442D18LL;
}

}  // namespace xt
