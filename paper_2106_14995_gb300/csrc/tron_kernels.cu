// tron_kernels.cu -- batched TRON kernels and the tron_batch_* C ABI.
//
// Plain schedule: one launch per size class, grid = problems / problems-per-CTA, each
// thread group solves one problem start to finish (single-kernel design, Sec. 4.1).
// Persistent schedule: one launch of resident CTAs; each warp pulls the next problems
// of its size class from a device work counter until the class is exhausted, so warps
// that drew quick problems take more of them instead of idling.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "capi_common.h"
#include "tron_solver.cuh"

namespace xt {

// ------------------------------------------------------------------ error plumbing
static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

int device_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return v;
}

// warps per CTA, reduced until the CTA's shared memory fits the device
static int fit_wpb(int wpb, int warp_doubles, int optin) {
  while (wpb > 1 && (size_t)wpb * warp_doubles * sizeof(double) > (size_t)optin) --wpb;
  return wpb;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// ------------------------------------------------------------------ kernel arguments
struct KArgs {
  const double* params;
  const double* lo;
  const double* hi;
  double* x;
  double* delta;
  double* f;
  double* pg;
  int32_t* iters;
  int32_t* status;
  const int32_t* nvec;   // per-problem sizes (NULL: uniform)
  const int64_t* poff;   // record offsets (NULL: p * pstride)
  const int64_t* voff;   // vector offsets (NULL: p * n_uniform)
  const int32_t* plist;  // problems of this launch (NULL: 0..count-1)
  int64_t count;
  int64_t pstride;
  int32_t n_uniform;
  int32_t ppw;  // problems per warp for groups of a warp or less (0: as many as it holds)
  unsigned long long* counter;  // persistent schedule work counter
  tron_options_t opt;
};

template <class Obj, int N, int G, bool PK>
__device__ __forceinline__ void solve_problem(const KArgs& a, int64_t idx, double* wsm) {
  using S = Solver<Obj, N, G, PK>;
  constexpr int R = S::R;
  S sv(a.opt, wsm);
  const int64_t q = a.plist ? (int64_t)a.plist[idx] : idx;
  const int n = a.nvec ? a.nvec[q] : a.n_uniform;
  const int64_t po = a.poff ? a.poff[q] : q * a.pstride;
  const int64_t vo = a.voff ? a.voff[q] : q * (int64_t)a.n_uniform;
  sv.n = n;
  double x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = r * G + sv.gp.t;
    if (i < n) {
      sv.l[r] = a.lo[vo + i];
      sv.u[r] = a.hi[vo + i];
      x[r] = a.x[vo + i];
    } else {
      sv.l[r] = 0.0;
      sv.u[r] = 0.0;
      x[r] = 0.0;
    }
  }
  const bool pf = sv.obj.load(sv.gp, a.params ? a.params + po : nullptr, n);
  double delta = a.delta[q];
  double f, pg;
  int k;
  const int st = sv.run(x, delta, f, pg, k, pf);
  if (st != TRON_BAD_BOUNDS) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = r * G + sv.gp.t;
      if (i < n) a.x[vo + i] = x[r];
    }
  }
  if (sv.gp.t == 0) {
    a.delta[q] = delta;
    a.f[q] = f;
    a.pg[q] = pg;
    a.iters[q] = k;
    a.status[q] = st;
  }
}

template <class Obj, int N, int G, bool PK>
__global__ void __launch_bounds__(256) k_tron_plain(const KArgs a) {
  using S = Solver<Obj, N, G, PK>;
  extern __shared__ double smem[];
  if constexpr (G > 32) {  // one problem per CTA
    const int64_t idx = blockIdx.x;
    if (idx >= a.count) return;
    solve_problem<Obj, N, G, PK>(a, idx, smem);
  } else {
    const int warp = threadIdx.x >> 5;
    double* wsm = smem + (size_t)warp * S::WARP_DOUBLES;
    const int ppw = a.ppw > 0 ? a.ppw : S::PROBS_PER_WARP;
    const int grp = (threadIdx.x & 31) / G;
    if (grp >= ppw) return;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t idx = gw * ppw + grp;
    if (idx >= a.count) return;
    solve_problem<Obj, N, G, PK>(a, idx, wsm);
  }
}

template <class Obj, int N, int G, bool PK>
__global__ void __launch_bounds__(256) k_tron_persistent(const KArgs a) {
  using S = Solver<Obj, N, G, PK>;
  extern __shared__ double smem[];
  if constexpr (G > 32) {  // the CTA pulls one problem at a time
    __shared__ unsigned long long next;
    for (;;) {
      if (threadIdx.x == 0) next = atomicAdd(a.counter, 1ull);
      __syncthreads();
      const int64_t idx = (int64_t)next;
      __syncthreads();
      if (idx >= a.count) break;
      solve_problem<Obj, N, G, PK>(a, idx, smem);
      __syncthreads();
    }
  } else {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double* wsm = smem + (size_t)warp * S::WARP_DOUBLES;
    const int ppw = a.ppw > 0 ? a.ppw : S::PROBS_PER_WARP;
    for (;;) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)ppw);
      base = __shfl_sync(0xffffffffu, base, 0);
      if ((int64_t)base >= a.count) break;
      const int64_t idx = (int64_t)base + lane / G;
      if (lane / G < ppw && idx < a.count) solve_problem<Obj, N, G, PK>(a, idx, wsm);
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------ dispatch table
// layout bits of a kernel variant: bit 0 = packed factor, bit 1 = Q read from global,
// bit 2 = Q as wrapped diagonals in shared memory
enum { kLayoutPacked = 1, kLayoutQGlobal = 2, kLayoutQDiag = 4 };

struct KernelEntry {
  int kind, N, G, layout;
  const void* plain;
  const void* persistent;
  int warp_doubles;    // shared memory per warp (per CTA for CTA groups)
  int probs_per_warp;  // 0 for CTA groups
  int occupancy[9];    // CTAs per SM by warps per block (cached, 0 = unknown)
};

// launch geometry of a variant for a requested number of warps per CTA
struct Geometry {
  int threads;
  size_t smem;
  int64_t per_cta;
  int wpb;
};
static Geometry geometry(const KernelEntry& e, int wpb) {
  Geometry g;
  if (e.G > 32) {  // one problem per CTA of G threads
    g.wpb = e.G / 32;
    g.threads = e.G;
    g.smem = (size_t)e.warp_doubles * sizeof(double);
    g.per_cta = 1;
  } else {
    g.wpb = wpb;
    g.threads = wpb * 32;
    g.smem = (size_t)wpb * e.warp_doubles * sizeof(double);
    g.per_cta = (int64_t)wpb * e.probs_per_warp;
  }
  return g;
}

template <class Obj, int N, int G, bool PK>
static KernelEntry make_entry(int kind, int layout) {
  using S = Solver<Obj, N, G, PK>;
  KernelEntry e;
  e.kind = kind;
  e.N = N;
  e.G = G;
  e.layout = layout;
  e.plain = (const void*)k_tron_plain<Obj, N, G, PK>;
  e.persistent = (const void*)k_tron_persistent<Obj, N, G, PK>;
  e.warp_doubles = S::WARP_DOUBLES;
  e.probs_per_warp = S::PROBS_PER_WARP;
  for (int i = 0; i < 9; ++i) e.occupancy[i] = 0;
  return e;
}

// every compiled variant; the first entry of a (kind, N) pair is its default
static std::vector<KernelEntry>& table() {
  static std::vector<KernelEntry> t = {
      make_entry<BranchObj<1>, 4, 1, false>(TRON_OBJ_ACOPF_BRANCH, 0),
      make_entry<BranchObj<4>, 4, 4, false>(TRON_OBJ_ACOPF_BRANCH, 0),
      make_entry<BranchObj<2>, 4, 2, false>(TRON_OBJ_ACOPF_BRANCH, 0),
      make_entry<DenseObj<4, 4>, 4, 4, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<4, 1>, 4, 1, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<8, 8>, 8, 8, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<8, 1>, 8, 1, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<16, 16>, 16, 16, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<16, 8>, 16, 8, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<32, 32>, 32, 32, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<32, 32>, 32, 32, true>(TRON_OBJ_DENSE_QUARTIC, kLayoutPacked),
      make_entry<DenseObj<32, 32, kQDiag>, 32, 32, true>(TRON_OBJ_DENSE_QUARTIC,
                                                        kLayoutPacked | kLayoutQDiag),
      make_entry<DenseObj<32, 32, kQGlobal>, 32, 32, true>(TRON_OBJ_DENSE_QUARTIC,
                                                      kLayoutPacked | kLayoutQGlobal),
      make_entry<DenseObj<32, 16>, 32, 16, false>(TRON_OBJ_DENSE_QUARTIC, 0),
      make_entry<DenseObj<64, 64, kQGlobal>, 64, 64, true>(TRON_OBJ_DENSE_QUARTIC,
                                                      kLayoutPacked | kLayoutQGlobal),
      make_entry<DenseObj<64, 64>, 64, 64, true>(TRON_OBJ_DENSE_QUARTIC, kLayoutPacked),
      make_entry<DenseObj<64, 32, kQGlobal>, 64, 32, true>(TRON_OBJ_DENSE_QUARTIC,
                                                      kLayoutPacked | kLayoutQGlobal),
      make_entry<DenseObj<64, 32>, 64, 32, true>(TRON_OBJ_DENSE_QUARTIC, kLayoutPacked),
      make_entry<DenseObj<128, 128, kQGlobal>, 128, 128, true>(TRON_OBJ_DENSE_QUARTIC,
                                                          kLayoutPacked | kLayoutQGlobal),
      make_entry<DenseObj<128, 32, kQGlobal>, 128, 32, true>(TRON_OBJ_DENSE_QUARTIC,
                                                        kLayoutPacked | kLayoutQGlobal),
      make_entry<Hs45Obj<8>, 8, 1, false>(TRON_OBJ_HS45, 0),
      make_entry<GenRampObj<8, 8>, 8, 8, false>(TRON_OBJ_GEN_RAMP, 0),
      make_entry<GenRampObj<16, 16>, 16, 16, false>(TRON_OBJ_GEN_RAMP, 0),
      make_entry<GenRampObj<32, 32>, 32, 32, true>(TRON_OBJ_GEN_RAMP, kLayoutPacked),
  };
  return t;
}
static std::mutex g_table_mu;

// size classes (largest last); a problem of size n runs in the smallest class >= n
static const int kClasses[] = {4, 8, 16, 32, 64, 128};
constexpr int kNumClasses = 6;

static int size_class(int kind, int n) {
  if (kind == TRON_OBJ_ACOPF_BRANCH) return n == 4 ? 4 : -1;
  if (kind == TRON_OBJ_HS45) return (n >= 1 && n <= 8) ? 8 : -1;
  if (kind == TRON_OBJ_GEN_RAMP) return n < 1 ? -1 : (n <= 8 ? 8 : (n <= 16 ? 16 : (n <= 32 ? 32 : -1)));
  if (kind == TRON_OBJ_DENSE_QUARTIC) {
    if (n < 1) return -1;
    for (int c : kClasses)
      if (n <= c) return c;
  }
  return -1;
}
static int class_slot(int c) {
  for (int s = 0; s < kNumClasses; ++s)
    if (kClasses[s] == c) return s;
  return -1;
}
// default variant of a class, or the first variant with group G when G != 0 and with
// the storage layout (options.layout - 1) when that option is not 0
static KernelEntry* find_entry(int kind, int N, int G, int layout_opt = 0) {
  for (auto& e : table())
    if (e.kind == kind && e.N == N && (G == 0 || e.G == G) &&
        (layout_opt == 0 || e.layout == layout_opt - 1))
      return &e;
  return nullptr;
}
// The default mapping of the branch problems follows the batch: four lanes per problem
// while the class holds at most this many problems per SM sub-partition (the launch then
// lasts as long as its slowest problem, whose serial chain four lanes shorten), two
// lanes beyond (half the instructions of four per problem, a chain still far shorter
// than on one lane).  Cold-started branch batches on 152 SMs, ms with 1 / 2 / 4 lanes:
// 32,768 problems 1.70 / 1.32 / 1.28, 49,152 2.41 / 1.82 / 1.75, 65,536 1.88 / 1.65 /
// 1.67, 131,072 3.13 / 2.87 / 2.98, 262,144 5.63 / 5.23 / 5.65; one lane is the slowest
// throughout (these solves take 5.5 TRON iterations on average, up to 29).
constexpr int64_t kG4BranchProblemsPerSmsp = 96;

static int default_group(int kind, int N, int64_t count, int sms) {
  if (kind == TRON_OBJ_ACOPF_BRANCH && N == 4)
    return (sms > 0 && count > 0 && count <= kG4BranchProblemsPerSmsp * 4 * sms) ? 4 : 2;
  KernelEntry* e = find_entry(kind, N, 0);
  return e ? e->G : 1;
}

}  // namespace xt

using namespace xt;

// ------------------------------------------------------------------------ handle
struct tron_batch {
  tron_obj_t kind;
  int64_t nprob;
  tron_options_t opt;
  int32_t n_uniform;  // > 0 when every problem has this size
  int32_t* d_n;
  int64_t* d_poff;
  int64_t* d_voff;
  struct Bucket {
    int N;
    int64_t count;
    int32_t* d_list;     // NULL when the bucket is the whole (uniform) batch
    KernelEntry* tuned;  // variant chosen by tron_batch_autotune (NULL: options/default)
    int tuned_wpb;
    int tuned_chol;
  };
  std::vector<Bucket> buckets;
  // Work counters (one per bucket), forked streams and events of the persistent
  // schedule, in kSolveSets sets taken in turn by successive solves, so that solves of
  // independent batches on different streams can run at the same time (one's last wave
  // overlapping the next one's start)
  static constexpr int kSolveSets = 4;
  unsigned long long* d_counter;  // [kSolveSets][8]
  cudaStream_t side[kSolveSets][kNumClasses];
  cudaEvent_t ev_fork[kSolveSets], ev_join[kSolveSets][kNumClasses];
  int next_set;
  int64_t total_n;     // length of the concatenated vectors
  int64_t params_len;  // doubles of the packed parameter records
  int last_launches;
  int sms;
  int smem_optin;
  // host-buffer path (tron_batch_host_enable): two device buffer sets used in turn, so
  // the copies of one call overlap the solve of the previous one
  struct HostSet {
    double *params, *lo, *hi, *x, *delta, *f, *pg;
    int32_t *iters, *status;
    cudaEvent_t in_done, solved, out_done;
  };
  HostSet hs[2];
  bool host_ready;
  int host_next;
  cudaStream_t s_in, s_run[2], s_out;  // copy in, solve (one per buffer set), copy out
};

static int64_t record_size(int kind, int n) {
  if (kind == TRON_OBJ_ACOPF_BRANCH) return 36;
  if (kind == TRON_OBJ_DENSE_QUARTIC) return (int64_t)n * n + 2 * n;
  if (kind == TRON_OBJ_GEN_RAMP) return 8 + 2 * (int64_t)n;
  return 0;
}

namespace xt {
__global__ void k_pivot_rcp(const double* a, double* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = pivot_rcp(a[i]);
}

__global__ void k_arith(int op, const double* a, const double* b, double* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = a[i];
  if (op == 1) out[i] = quotient(v, b[i]);
  else if (op == 2) out[i] = square_root(v);
  else if (op == 3) out[i] = small_angle(v) ? sin_cos_small(v, false) : sin(v);
  else out[i] = small_angle(v) ? sin_cos_small(v, true) : cos(v);
}

// FP64 FMA throughput: 8 independent dependent chains per thread (enough to cover the
// FMA latency with a few warps per SM sub-partition); the factor and increment keep the
// values bounded, and the result is written so nothing is eliminated
__global__ void k_fp64_fma(double* out, int64_t iters) {
  const double a = 0.9999999, b = 1e-7;
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (double)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// Dependent-operation cost: one CTA of `lanes` threads runs a chain of kOpChain
// operations of one kind, each on the previous result, between two clock64 reads;
// thread 0 writes the cycles.  The operands stay finite and in the fast ranges of the
// solver's own quotient, square root and sine.
constexpr int kOpChain = 2048;
template <int OP>
__global__ void k_op_latency(long long* cyc) {
  double v = 0.5 + 1e-3 * (double)threadIdx.x;
  const double a = 0.9999999, b = 1e-7;
  long long x = __double_as_longlong(v), xb = __double_as_longlong(b);
  float fv = (float)v;
  __syncwarp(__activemask());
  const long long t0 = clock64();
#pragma unroll 16
  for (int i = 0; i < kOpChain; ++i) {
    if (OP == 0) v = fma(v, a, b);
    if (OP == 1) asm volatile("add.f64 %0, %0, %1;" : "+d"(v) : "d"(b));
    if (OP == 2) asm volatile("max.f64 %0, %0, %1;" : "+d"(v) : "d"(b));
    if (OP == 3)
      asm volatile("{ .reg .pred p; setp.gt.f64 p, %0, %1; selp.f64 %0, %1, %0, p; }"
                   : "+d"(v) : "d"(b));
    if (OP == 4)
      asm volatile("{ .reg .pred p; setp.gt.s64 p, %0, %1; selp.b64 %0, %1, %0, p; }"
                   : "+l"(x) : "l"(xb));
    if (OP == 5) v = quotient(a, v);
    if (OP == 6) v = a / v;
    if (OP == 7) v = square_root(v);
    if (OP == 8) v = sqrt(v);
    if (OP == 9) v = sin(v);
    if (OP == 10) v = sin_cos_small(v, false);
    if (OP == 11) asm volatile("rcp.approx.ftz.f64 %0, %0;" : "+d"(v));
    if (OP == 12) x = __shfl_sync(__activemask(), x, threadIdx.x ^ (blockDim.x > 1 ? 1 : 0));
    if (OP == 13) v = cos(v);
    if (OP == 14) {
      double sn, cs;
      sincos(v, &sn, &cs);
      v = fma(cs, 1e-3, sn);
    }
    if (OP == 15) fv = fmaf(fv, 0.9999999f, 1e-7f);
  }
  const long long t1 = clock64();
  if (threadIdx.x == 0)
    cyc[0] = (t1 - t0) + (long long)(v == 12345.0) + (x == 12345 ? 1 : 0) + (fv == 12345.0f ? 1 : 0);
}
static const void* op_latency_kernel(int op) {
  switch (op) {
    case 0: return (const void*)k_op_latency<0>;
    case 1: return (const void*)k_op_latency<1>;
    case 2: return (const void*)k_op_latency<2>;
    case 3: return (const void*)k_op_latency<3>;
    case 4: return (const void*)k_op_latency<4>;
    case 5: return (const void*)k_op_latency<5>;
    case 6: return (const void*)k_op_latency<6>;
    case 7: return (const void*)k_op_latency<7>;
    case 8: return (const void*)k_op_latency<8>;
    case 9: return (const void*)k_op_latency<9>;
    case 10: return (const void*)k_op_latency<10>;
    case 11: return (const void*)k_op_latency<11>;
    case 12: return (const void*)k_op_latency<12>;
    case 13: return (const void*)k_op_latency<13>;
    case 14: return (const void*)k_op_latency<14>;
    case 15: return (const void*)k_op_latency<15>;
    default: return nullptr;
  }
}
}  // namespace xt

static tron_err_t check_options(const tron_options_t* o) {
  XT_REQUIRE(o->max_outer >= 0 && o->max_trials >= 0 && o->max_shift >= 0, TRON_EINVAL,
             "negative iteration cap in options");
  XT_REQUIRE(o->group == 0 || o->group == 1 || o->group == 2 || o->group == 4 ||
                 o->group == 8 || o->group == 16 || o->group == 32,
             TRON_EINVAL, "options.group must be 0, 1, 2, 4, 8, 16 or 32");
  XT_REQUIRE(o->schedule == TRON_SCHED_PLAIN || o->schedule == TRON_SCHED_PERSISTENT,
             TRON_EINVAL, "options.schedule must be TRON_SCHED_PLAIN or TRON_SCHED_PERSISTENT");
  XT_REQUIRE(o->warps_per_block >= 0 && o->warps_per_block <= 8, TRON_EINVAL,
             "options.warps_per_block must be in [0, 8]");
  XT_REQUIRE(o->layout >= 0 && o->layout <= 8, TRON_EINVAL, "options.layout must be in [0, 8]");
  XT_REQUIRE(o->cholesky >= 0 && o->cholesky <= 2, TRON_EINVAL,
             "options.cholesky must be 0, 1 or 2");
  XT_REQUIRE(o->ctas_per_sm >= 0, TRON_EINVAL, "options.ctas_per_sm must be >= 0");
  XT_REQUIRE(o->tr_norm == 0 || o->tr_norm == 1, TRON_EINVAL, "options.tr_norm must be 0 or 1");
  XT_REQUIRE(o->cauchy_norm == 0 || o->cauchy_norm == 1, TRON_EINVAL,
             "options.cauchy_norm must be 0 or 1");
  return TRON_OK;
}

extern "C" {

const char* tron_last_error(void) { return g_err.c_str(); }
const char* tron_version(void) { return "exatron-gb300 0.1 (sm_103a, FP64)"; }

tron_err_t tron_bench_fp64_fma(double* d_out, int32_t blocks, int32_t threads, int64_t iters,
                               void* stream) {
  clear_error();
  XT_REQUIRE(d_out != nullptr, TRON_EINVAL, "tron_bench_fp64_fma: d_out is NULL");
  XT_REQUIRE(blocks > 0 && threads > 0 && threads <= 1024 && threads % 32 == 0 && iters > 0,
             TRON_EINVAL, "tron_bench_fp64_fma: bad launch size");
  xt::k_fp64_fma<<<(unsigned)blocks, (unsigned)threads, 0, (cudaStream_t)stream>>>(d_out, iters);
  XT_CUDA(cudaGetLastError());
  return TRON_OK;
}

tron_err_t tron_bench_op_latency(int32_t op, int32_t lanes, int64_t* d_cycles, void* stream) {
  clear_error();
  XT_REQUIRE(d_cycles != nullptr, TRON_EINVAL, "tron_bench_op_latency: d_cycles is NULL");
  XT_REQUIRE(lanes >= 1 && lanes <= 1024, TRON_EINVAL, "tron_bench_op_latency: lanes not in [1, 1024]");
  const void* fn = xt::op_latency_kernel(op);
  XT_REQUIRE(fn != nullptr, TRON_EINVAL, "tron_bench_op_latency: op not in [0, 15]");
  long long* cyc = reinterpret_cast<long long*>(d_cycles);
  void* args[] = {&cyc};
  XT_CUDA(cudaLaunchKernel(fn, dim3(1), dim3((unsigned)lanes), args, 0, (cudaStream_t)stream));
  return TRON_OK;
}

int32_t tron_bench_op_chain(void) { return xt::kOpChain; }

tron_err_t tron_test_pivot_rcp(const double* d_a, double* d_out, int64_t n, void* stream) {
  clear_error();
  XT_REQUIRE(n >= 0, TRON_EINVAL, "tron_test_pivot_rcp: n < 0");
  if (n == 0) return TRON_OK;
  XT_REQUIRE(d_a && d_out, TRON_EINVAL, "tron_test_pivot_rcp: null device array");
  const int64_t blocks = (n + 255) / 256;
  XT_REQUIRE(blocks < (1ll << 31), TRON_EINVAL, "tron_test_pivot_rcp: n too large");
  xt::k_pivot_rcp<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_a, d_out, n);
  XT_CUDA(cudaGetLastError());
  return TRON_OK;
}

tron_err_t tron_test_arith(int32_t op, const double* d_a, const double* d_b, double* d_out,
                           int64_t n, void* stream) {
  clear_error();
  XT_REQUIRE(op >= 1 && op <= 4, TRON_EINVAL, "tron_test_arith: op must be 1, 2, 3 or 4");
  XT_REQUIRE(n >= 0, TRON_EINVAL, "tron_test_arith: n < 0");
  if (n == 0) return TRON_OK;
  XT_REQUIRE(d_a && d_out && (op != 1 || d_b), TRON_EINVAL, "tron_test_arith: null device array");
  const int64_t blocks = (n + 255) / 256;
  XT_REQUIRE(blocks < (1ll << 31), TRON_EINVAL, "tron_test_arith: n too large");
  xt::k_arith<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(op, d_a, d_b, d_out, n);
  XT_CUDA(cudaGetLastError());
  return TRON_OK;
}

tron_err_t tron_options_default(tron_options_t* o) {
  XT_REQUIRE(o != nullptr, TRON_EINVAL, "tron_options_default: null pointer");
  memset(o, 0, sizeof(*o));
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
  o->group = 0;
  o->ared_guard = 1e-13;
  o->schedule = TRON_SCHED_PLAIN;
  o->warps_per_block = 0;
  return TRON_OK;
}

tron_err_t tron_batch_create(tron_batch_t** out, tron_obj_t kind, int64_t nprob,
                             const int32_t* n_host, int32_t n_uniform,
                             const tron_options_t* opt, void* stream) {
  clear_error();
  XT_REQUIRE(out != nullptr, TRON_EINVAL, "tron_batch_create: out is NULL");
  *out = nullptr;
  XT_REQUIRE(kind == TRON_OBJ_ACOPF_BRANCH || kind == TRON_OBJ_DENSE_QUARTIC ||
                 kind == TRON_OBJ_HS45 || kind == TRON_OBJ_GEN_RAMP,
             TRON_EINVAL, "tron_batch_create: unknown objective kind %d", (int)kind);
  XT_REQUIRE(nprob >= 0 && nprob < (int64_t)1 << 31, TRON_EINVAL,
             "tron_batch_create: nprob %lld out of range", (long long)nprob);
  tron_options_t o;
  if (opt) o = *opt;
  else tron_options_default(&o);
  tron_err_t e = check_options(&o);
  if (e != TRON_OK) return e;
  cudaStream_t st = (cudaStream_t)stream;

  tron_batch* b = new tron_batch();
  b->kind = kind;
  b->nprob = nprob;
  b->opt = o;
  b->n_uniform = 0;
  b->d_n = nullptr;
  b->d_poff = nullptr;
  b->d_voff = nullptr;
  b->d_counter = nullptr;
  b->next_set = 0;
  for (int k = 0; k < tron_batch::kSolveSets; ++k) {
    b->ev_fork[k] = nullptr;
    for (int i = 0; i < kNumClasses; ++i) {
      b->side[k][i] = nullptr;
      b->ev_join[k][i] = nullptr;
    }
  }
  b->last_launches = 0;
  b->params_len = 0;
  memset(b->hs, 0, sizeof(b->hs));
  b->host_ready = false;
  b->host_next = 0;
  b->s_in = b->s_run[0] = b->s_run[1] = b->s_out = nullptr;
  b->sms = device_sm_count();
  b->smem_optin = device_smem_optin();
  auto fail = [&](tron_err_t code) {
    tron_batch_destroy(b);
    return code;
  };
  if (b->sms <= 0) {
    set_error("tron_batch_create: no CUDA device");
    return fail(TRON_ECUDA);
  }
  if (n_host == nullptr) {
    if (size_class(kind, n_uniform) < 0) {
      set_error("tron_batch_create: size n=%d not supported for kind %d", n_uniform, (int)kind);
      return fail(TRON_EUNSUPPORTED);
    }
    b->n_uniform = n_uniform;
    b->total_n = nprob * (int64_t)n_uniform;
    b->params_len = nprob * record_size(kind, n_uniform);
    b->buckets.push_back({size_class(kind, n_uniform), nprob, nullptr, nullptr, 0, 0});
  } else {
    std::vector<int64_t> poff(nprob), voff(nprob);
    std::vector<std::vector<int32_t>> lists(kNumClasses);
    int64_t pa = 0, va = 0;
    for (int64_t p = 0; p < nprob; ++p) {
      const int n = n_host[p];
      const int c = size_class(kind, n);
      if (c < 0) {
        set_error("tron_batch_create: problem %lld has unsupported size %d", (long long)p, n);
        return fail(TRON_EUNSUPPORTED);
      }
      poff[p] = pa;
      voff[p] = va;
      pa += record_size(kind, n);
      va += n;
      lists[class_slot(c)].push_back((int32_t)p);
    }
    b->total_n = va;
    b->params_len = pa;
    if (cudaMalloc(&b->d_n, sizeof(int32_t) * std::max<int64_t>(nprob, 1)) != cudaSuccess ||
        cudaMalloc(&b->d_poff, sizeof(int64_t) * std::max<int64_t>(nprob, 1)) != cudaSuccess ||
        cudaMalloc(&b->d_voff, sizeof(int64_t) * std::max<int64_t>(nprob, 1)) != cudaSuccess) {
      set_error("tron_batch_create: cudaMalloc of size tables failed");
      return fail(TRON_ENOMEM);
    }
    if (nprob > 0) {
      if (cudaMemcpyAsync(b->d_n, n_host, sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st) ||
          cudaMemcpyAsync(b->d_poff, poff.data(), sizeof(int64_t) * nprob,
                          cudaMemcpyHostToDevice, st) ||
          cudaMemcpyAsync(b->d_voff, voff.data(), sizeof(int64_t) * nprob,
                          cudaMemcpyHostToDevice, st)) {
        set_error("tron_batch_create: upload of size tables failed");
        return fail(TRON_ECUDA);
      }
    }
    // largest class first: the longest solves start earliest
    for (int slot = kNumClasses - 1; slot >= 0; --slot) {
      if (lists[slot].empty()) continue;
      tron_batch::Bucket bk{kClasses[slot], (int64_t)lists[slot].size(), nullptr, nullptr, 0, 0};
      if (cudaMalloc(&bk.d_list, sizeof(int32_t) * lists[slot].size()) != cudaSuccess) {
        set_error("tron_batch_create: cudaMalloc of a problem list failed");
        return fail(TRON_ENOMEM);
      }
      b->buckets.push_back(bk);
      if (cudaMemcpyAsync(bk.d_list, lists[slot].data(), sizeof(int32_t) * lists[slot].size(),
                          cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_error("tron_batch_create: upload of a problem list failed");
        return fail(TRON_ECUDA);
      }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("tron_batch_create: stream synchronisation failed");
      return fail(TRON_ECUDA);
    }
  }
  if (cudaMalloc(&b->d_counter, sizeof(unsigned long long) * 8 * tron_batch::kSolveSets) !=
      cudaSuccess) {
    set_error("tron_batch_create: cudaMalloc of work counters failed");
    return fail(TRON_ENOMEM);
  }
  for (int k = 0; k < tron_batch::kSolveSets; ++k) {
    if (cudaEventCreateWithFlags(&b->ev_fork[k], cudaEventDisableTiming) != cudaSuccess) {
      set_error("tron_batch_create: cudaEventCreate failed");
      return fail(TRON_ECUDA);
    }
    if (b->buckets.size() < 2) continue;  // one class: nothing to fork
    for (size_t i = 0; i < b->buckets.size(); ++i) {
      if (cudaStreamCreateWithFlags(&b->side[k][i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_join[k][i], cudaEventDisableTiming) != cudaSuccess) {
        set_error("tron_batch_create: stream/event creation failed");
        return fail(TRON_ECUDA);
      }
    }
  }
  // resolve the kernels now so that a bad group option fails here
  for (auto& bk : b->buckets) {
    const int G = o.group ? o.group : default_group(kind, bk.N, bk.count, b->sms);
    if (!find_entry(kind, bk.N, G, o.layout)) {
      set_error("tron_batch_create: no kernel for kind %d, size class %d, group %d", (int)kind,
                bk.N, G);
      return fail(TRON_EUNSUPPORTED);
    }
  }
  *out = b;
  return TRON_OK;
}

tron_err_t tron_batch_set_options(tron_batch_t* b, const tron_options_t* opt) {
  clear_error();
  XT_REQUIRE(b && opt, TRON_EINVAL, "tron_batch_set_options: null argument");
  tron_err_t e = check_options(opt);
  if (e != TRON_OK) return e;
  for (auto& bk : b->buckets) {
    const int G = opt->group ? opt->group : default_group(b->kind, bk.N, bk.count, b->sms);
    XT_REQUIRE(find_entry(b->kind, bk.N, G, opt->layout), TRON_EUNSUPPORTED,
               "no kernel for kind %d, size class %d, group %d", (int)b->kind, bk.N, G);
  }
  b->opt = *opt;
  return TRON_OK;
}

tron_err_t tron_batch_solve(tron_batch_t* b, const double* d_params, const double* d_lower,
                            const double* d_upper, double* d_x, double* d_delta, double* d_f,
                            double* d_pgnorm, int32_t* d_iters, int32_t* d_status,
                            void* stream) {
  clear_error();
  XT_REQUIRE(b != nullptr, TRON_EINVAL, "tron_batch_solve: null handle");
  b->last_launches = 0;
  if (b->nprob == 0) return TRON_OK;
  XT_REQUIRE(d_lower && d_upper && d_x && d_delta && d_f && d_pgnorm && d_iters && d_status,
             TRON_EINVAL, "tron_batch_solve: null device array");
  XT_REQUIRE(d_params || b->kind == TRON_OBJ_HS45, TRON_EINVAL,
             "tron_batch_solve: d_params is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const bool persistent = b->opt.schedule == TRON_SCHED_PERSISTENT;
  // persistent schedule with several size classes: every class on its own forked
  // stream, so all classes share the GPU in one pass
  const bool fork = persistent && b->buckets.size() > 1;
  const int cs = b->next_set;
  b->next_set = (cs + 1) % tron_batch::kSolveSets;
  if (fork) XT_CUDA(cudaEventRecord(b->ev_fork[cs], st));
  for (size_t bi = 0; bi < b->buckets.size(); ++bi) {
    const auto& bk = b->buckets[bi];
    if (bk.count == 0) continue;
    KernelEntry* ke = nullptr;
    int wpb = b->opt.warps_per_block ? b->opt.warps_per_block : 4;
    if (bk.tuned && b->opt.group == 0) {
      ke = bk.tuned;
      if (!b->opt.warps_per_block) wpb = bk.tuned_wpb;
    } else {
      const int G =
          b->opt.group ? b->opt.group : default_group(b->kind, bk.N, bk.count, b->sms);
      ke = find_entry(b->kind, bk.N, G, b->opt.layout);
    }
    XT_REQUIRE(ke, TRON_EUNSUPPORTED, "no kernel for size class %d", bk.N);
    wpb = fit_wpb(wpb, ke->warp_doubles, b->smem_optin);
    const Geometry geo = geometry(*ke, wpb);
    wpb = geo.wpb;
    cudaStream_t ls = st;
    if (fork) {
      ls = b->side[cs][bi];
      XT_CUDA(cudaStreamWaitEvent(ls, b->ev_fork[cs], 0));
    }
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.params = d_params;
    a.lo = d_lower;
    a.hi = d_upper;
    a.x = d_x;
    a.delta = d_delta;
    a.f = d_f;
    a.pg = d_pgnorm;
    a.iters = d_iters;
    a.status = d_status;
    a.nvec = b->d_n;
    a.poff = b->d_poff;
    a.voff = b->d_voff;
    a.plist = bk.d_list;
    a.count = bk.count;
    a.n_uniform = b->n_uniform;
    a.pstride = record_size(b->kind, b->n_uniform);
    a.counter = b->d_counter + 8 * cs + bi;
    a.opt = b->opt;
    if (bk.tuned && b->opt.group == 0 && b->opt.cholesky == 0) a.opt.cholesky = bk.tuned_chol;
    // a class too small to give every SM sub-partition a warp holds fewer problems per
    // warp (as few as one): each FP64 warp instruction costs the same whatever its active
    // lanes, so the warps stay one per sub-partition while the problems sharing a warp,
    // whose divergent paths that warp runs one after another, become fewer
    int64_t per_cta = geo.per_cta;
    if (ke->G <= 32 && ke->probs_per_warp > 1) {
      const int64_t smsp = 4 * (int64_t)b->sms;
      const int64_t want = (bk.count + smsp - 1) / smsp;
      if (want < ke->probs_per_warp) {
        a.ppw = (int32_t)std::max<int64_t>(1, want);
        per_cta = (int64_t)geo.wpb * a.ppw;
      }
    }
    const size_t smem = geo.smem;
    const void* fn = persistent ? ke->persistent : ke->plain;
    {
      std::lock_guard<std::mutex> lk(g_table_mu);
      XT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    int64_t grid;
    if (persistent) {
      int occ = 0;
      {
        std::lock_guard<std::mutex> lk(g_table_mu);
        occ = ke->occupancy[wpb];
        if (occ == 0) {
          XT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, geo.threads, smem));
          ke->occupancy[wpb] = occ;
        }
      }
      XT_REQUIRE(occ > 0, TRON_EUNSUPPORTED, "kernel does not fit on an SM (smem %zu)", smem);
      if (b->opt.ctas_per_sm > 0) occ = std::min(occ, (int)b->opt.ctas_per_sm);
      grid = std::min<int64_t>((int64_t)occ * b->sms, (bk.count + per_cta - 1) / per_cta);
      XT_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), ls));
    } else {
      grid = (bk.count + per_cta - 1) / per_cta;
    }
    void* args[] = {&a};
    XT_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(geo.threads), args, smem, ls));
    b->last_launches++;
    if (fork) {
      XT_CUDA(cudaEventRecord(b->ev_join[cs][bi], ls));
      XT_CUDA(cudaStreamWaitEvent(st, b->ev_join[cs][bi], 0));
    }
  }
  return TRON_OK;
}

int32_t tron_batch_last_launches(const tron_batch_t* b) { return b ? b->last_launches : 0; }

int32_t tron_batch_buckets(const tron_batch_t* b) { return b ? (int32_t)b->buckets.size() : 0; }

tron_err_t tron_batch_get_choice(const tron_batch_t* b, int32_t bucket, int32_t* N, int32_t* G,
                                 int32_t* layout, int32_t* warps_per_block, int64_t* count) {
  clear_error();
  XT_REQUIRE(b && bucket >= 0 && bucket < (int)b->buckets.size(), TRON_EINVAL,
             "tron_batch_get_choice: bad bucket");
  const auto& bk = b->buckets[bucket];
  KernelEntry* ke = nullptr;
  int wpb = b->opt.warps_per_block ? b->opt.warps_per_block : 4;
  if (bk.tuned && b->opt.group == 0) {
    ke = bk.tuned;
    if (!b->opt.warps_per_block) wpb = bk.tuned_wpb;
  } else {
    ke = find_entry(b->kind, bk.N,
                    b->opt.group ? b->opt.group
                                 : default_group(b->kind, bk.N, bk.count, b->sms),
                    b->opt.layout);
  }
  XT_REQUIRE(ke, TRON_EUNSUPPORTED, "no kernel for size class %d", bk.N);
  wpb = geometry(*ke, fit_wpb(wpb, ke->warp_doubles, b->smem_optin)).wpb;
  if (N) *N = ke->N;
  if (G) *G = ke->G;
  if (layout) {
    const int chol = (bk.tuned && b->opt.group == 0 && b->opt.cholesky == 0) ? bk.tuned_chol
                                                                             : b->opt.cholesky;
    *layout = ke->layout | (chol << 3);
  }
  if (warps_per_block) *warps_per_block = wpb;
  if (count) *count = bk.count;
  return TRON_OK;
}

tron_err_t tron_batch_autotune(tron_batch_t* b, const double* d_params, const double* d_lower,
                               const double* d_upper, const double* d_x0,
                               const double* d_delta0, int32_t sample, void* stream) {
  clear_error();
  XT_REQUIRE(b && d_lower && d_upper && d_x0 && d_delta0 && sample > 0, TRON_EINVAL,
             "tron_batch_autotune: bad argument");
  XT_REQUIRE(d_params || b->kind == TRON_OBJ_HS45, TRON_EINVAL,
             "tron_batch_autotune: d_params is NULL");
  if (b->nprob == 0) return TRON_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // scratch outputs for the trial solves (freed before returning)
  double *xt = nullptr, *dt = nullptr, *ft = nullptr, *pt = nullptr;
  int32_t *it = nullptr, *stt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tron_err_t err = TRON_OK;
  const size_t nx = (size_t)std::max<int64_t>(b->total_n, 1);
  const size_t np = (size_t)b->nprob;
  if (cudaMalloc(&xt, 8 * nx) || cudaMalloc(&dt, 8 * np) || cudaMalloc(&ft, 8 * np) ||
      cudaMalloc(&pt, 8 * np) || cudaMalloc(&it, 4 * np) || cudaMalloc(&stt, 4 * np) ||
      cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
    set_error("tron_batch_autotune: scratch allocation failed");
    err = TRON_ENOMEM;
  }
  int dev = 0;
  cudaDeviceProp prop;
  if (err == TRON_OK && (cudaGetDevice(&dev) || cudaGetDeviceProperties(&prop, dev))) {
    set_error("tron_batch_autotune: device query failed");
    err = TRON_ECUDA;
  }
  for (size_t bi = 0; err == TRON_OK && bi < b->buckets.size(); ++bi) {
    auto& bk = b->buckets[bi];
    const int64_t cs = std::min<int64_t>(bk.count, sample);
    float best = 1e30f;
    KernelEntry* best_e = nullptr;
    int best_w = 4, best_c = 0;
    for (auto& ke : table()) {
      if (ke.kind != b->kind || ke.N != bk.N) continue;
      for (int trial = 0; trial < 8; ++trial) {
        const int wpb = 1 << (trial & 3);
        const int chol = 1 + (trial >> 2);  // 1 left-looking, 2 right-looking
        if (wpb > 8) continue;
        if (ke.G > 32 && wpb != 1) continue;  // CTA groups have one geometry
        const Geometry geo = geometry(ke, wpb);
        const size_t smem = geo.smem;
        if (smem > prop.sharedMemPerBlockOptin) continue;
        KArgs a;
        memset(&a, 0, sizeof(a));
        a.params = d_params;
        a.lo = d_lower;
        a.hi = d_upper;
        a.x = xt;
        a.delta = dt;
        a.f = ft;
        a.pg = pt;
        a.iters = it;
        a.status = stt;
        a.nvec = b->d_n;
        a.poff = b->d_poff;
        a.voff = b->d_voff;
        a.plist = bk.d_list;
        a.count = cs;
        a.n_uniform = b->n_uniform;
        a.pstride = record_size(b->kind, b->n_uniform);
        a.opt = b->opt;
        a.opt.cholesky = chol;
        const int64_t grid = (cs + geo.per_cta - 1) / geo.per_cta;
        void* args[] = {&a};
        float ms = 1e30f;
        bool ok = cudaFuncSetAttribute(ke.plain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem) == cudaSuccess;
        for (int rep = 0; ok && rep < 2; ++rep) {
          ok = cudaMemcpyAsync(xt, d_x0, 8 * (size_t)b->total_n, cudaMemcpyDeviceToDevice,
                               st) == cudaSuccess &&
               cudaMemcpyAsync(dt, d_delta0, 8 * np, cudaMemcpyDeviceToDevice, st) ==
                   cudaSuccess &&
               cudaEventRecord(e0, st) == cudaSuccess &&
               cudaLaunchKernel(ke.plain, dim3((unsigned)grid), dim3(geo.threads), args, smem,
                                st) == cudaSuccess &&
               cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
          if (ok && rep == 1) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        }
        if (!ok) {
          cudaGetLastError();  // a variant that cannot launch is skipped
          continue;
        }
        if (ms < best) {
          best = ms;
          best_e = &ke;
          best_w = geo.wpb;
          best_c = chol;
        }
      }
    }
    if (best_e) {
      bk.tuned = best_e;
      bk.tuned_wpb = best_w;
      bk.tuned_chol = best_c;
    }
  }
  if (err == TRON_OK && cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("tron_batch_autotune: synchronisation failed");
    err = TRON_ECUDA;
  }
  cudaFree(xt);
  cudaFree(dt);
  cudaFree(ft);
  cudaFree(pt);
  cudaFree(it);
  cudaFree(stt);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return err;
}

static void host_release(tron_batch* b);

void tron_batch_destroy(tron_batch_t* b) {
  if (!b) return;
  for (int k = 0; k < tron_batch::kSolveSets; ++k) {
    for (int i = 0; i < kNumClasses; ++i) {
      if (b->side[k][i]) cudaStreamDestroy(b->side[k][i]);
      if (b->ev_join[k][i]) cudaEventDestroy(b->ev_join[k][i]);
    }
    if (b->ev_fork[k]) cudaEventDestroy(b->ev_fork[k]);
  }
  cudaFree(b->d_n);
  cudaFree(b->d_poff);
  cudaFree(b->d_voff);
  cudaFree(b->d_counter);
  for (auto& bk : b->buckets) cudaFree(bk.d_list);
  host_release(b);
  delete b;
}

// ------------------------------------------------------------------- host buffers
static void host_release(tron_batch* b) {
  for (auto& h : b->hs) {
    cudaFree(h.params);
    cudaFree(h.lo);
    cudaFree(h.hi);
    cudaFree(h.x);
    cudaFree(h.delta);
    cudaFree(h.f);
    cudaFree(h.pg);
    cudaFree(h.iters);
    cudaFree(h.status);
    if (h.in_done) cudaEventDestroy(h.in_done);
    if (h.solved) cudaEventDestroy(h.solved);
    if (h.out_done) cudaEventDestroy(h.out_done);
  }
  memset(b->hs, 0, sizeof(b->hs));
  if (b->s_in) cudaStreamDestroy(b->s_in);
  if (b->s_run[0]) cudaStreamDestroy(b->s_run[0]);
  if (b->s_run[1]) cudaStreamDestroy(b->s_run[1]);
  if (b->s_out) cudaStreamDestroy(b->s_out);
  b->s_in = b->s_run[0] = b->s_run[1] = b->s_out = nullptr;
  b->host_ready = false;
}

static tron_err_t host_setup(tron_batch* b);

tron_err_t tron_batch_host_enable(tron_batch_t* b) {
  clear_error();
  XT_REQUIRE(b != nullptr, TRON_EINVAL, "tron_batch_host_enable: null handle");
  if (b->host_ready) return TRON_OK;
  const tron_err_t e = host_setup(b);
  if (e != TRON_OK) host_release(b);  // nothing half-made stays behind
  return e;
}

static tron_err_t host_setup(tron_batch* b) {
  const size_t np = (size_t)std::max<int64_t>(b->nprob, 1);
  const size_t nv = (size_t)std::max<int64_t>(b->total_n, 1);
  const size_t npar = (size_t)std::max<int64_t>(b->params_len, 1);
  for (auto& h : b->hs) {
    if (cudaMalloc(&h.params, npar * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.lo, nv * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.hi, nv * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.x, nv * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.delta, np * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.f, np * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.pg, np * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h.iters, np * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&h.status, np * sizeof(int32_t)) != cudaSuccess) {
      set_error("tron_batch_host_enable: cudaMalloc of the device buffer sets failed");
      return TRON_ENOMEM;
    }
    XT_CUDA(cudaEventCreateWithFlags(&h.in_done, cudaEventDisableTiming));
    XT_CUDA(cudaEventCreateWithFlags(&h.solved, cudaEventDisableTiming));
    XT_CUDA(cudaEventCreateWithFlags(&h.out_done, cudaEventDisableTiming));
  }
  XT_CUDA(cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking));
  XT_CUDA(cudaStreamCreateWithFlags(&b->s_run[0], cudaStreamNonBlocking));
  XT_CUDA(cudaStreamCreateWithFlags(&b->s_run[1], cudaStreamNonBlocking));
  XT_CUDA(cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking));
  b->host_ready = true;
  return TRON_OK;
}

tron_err_t tron_batch_solve_host(tron_batch_t* b, const double* h_params, const double* h_lower,
                                 const double* h_upper, const double* h_x0,
                                 const double* h_delta0, double* h_x, double* h_delta,
                                 double* h_f, double* h_pgnorm, int32_t* h_iters,
                                 int32_t* h_status) {
  clear_error();
  XT_REQUIRE(b != nullptr, TRON_EINVAL, "tron_batch_solve_host: null handle");
  XT_REQUIRE(b->host_ready, TRON_EINVAL,
             "tron_batch_solve_host: call tron_batch_host_enable first");
  if (b->nprob == 0) return TRON_OK;
  XT_REQUIRE(h_lower && h_upper && h_x0 && h_delta0 && h_x && h_delta && h_f && h_pgnorm &&
                 h_iters && h_status,
             TRON_EINVAL, "tron_batch_solve_host: null host array");
  XT_REQUIRE(h_params || b->params_len == 0, TRON_EINVAL,
             "tron_batch_solve_host: h_params is NULL");
  const int hi = b->host_next;
  auto& h = b->hs[hi];
  cudaStream_t run = b->s_run[hi];
  b->host_next ^= 1;
  const size_t np = (size_t)b->nprob, nv = (size_t)b->total_n;
  const cudaMemcpyKind up = cudaMemcpyHostToDevice, down = cudaMemcpyDeviceToHost;
  // inputs, once the previous use of this buffer set has been copied out
  XT_CUDA(cudaStreamWaitEvent(b->s_in, h.out_done, 0));
  if (b->params_len > 0)
    XT_CUDA(cudaMemcpyAsync(h.params, h_params, (size_t)b->params_len * sizeof(double), up,
                            b->s_in));
  XT_CUDA(cudaMemcpyAsync(h.lo, h_lower, nv * sizeof(double), up, b->s_in));
  XT_CUDA(cudaMemcpyAsync(h.hi, h_upper, nv * sizeof(double), up, b->s_in));
  XT_CUDA(cudaMemcpyAsync(h.x, h_x0, nv * sizeof(double), up, b->s_in));
  XT_CUDA(cudaMemcpyAsync(h.delta, h_delta0, np * sizeof(double), up, b->s_in));
  XT_CUDA(cudaEventRecord(h.in_done, b->s_in));
  // the solve, on this set's stream: the previous call's solve (other set) may still be
  // finishing its last wave
  XT_CUDA(cudaStreamWaitEvent(run, h.in_done, 0));
  tron_err_t e = tron_batch_solve(b, b->params_len > 0 ? h.params : nullptr, h.lo, h.hi, h.x,
                                  h.delta, h.f, h.pg, h.iters, h.status, run);
  if (e != TRON_OK) return e;
  XT_CUDA(cudaEventRecord(h.solved, run));
  // results
  XT_CUDA(cudaStreamWaitEvent(b->s_out, h.solved, 0));
  XT_CUDA(cudaMemcpyAsync(h_x, h.x, nv * sizeof(double), down, b->s_out));
  XT_CUDA(cudaMemcpyAsync(h_delta, h.delta, np * sizeof(double), down, b->s_out));
  XT_CUDA(cudaMemcpyAsync(h_f, h.f, np * sizeof(double), down, b->s_out));
  XT_CUDA(cudaMemcpyAsync(h_pgnorm, h.pg, np * sizeof(double), down, b->s_out));
  XT_CUDA(cudaMemcpyAsync(h_iters, h.iters, np * sizeof(int32_t), down, b->s_out));
  XT_CUDA(cudaMemcpyAsync(h_status, h.status, np * sizeof(int32_t), down, b->s_out));
  XT_CUDA(cudaEventRecord(h.out_done, b->s_out));
  return TRON_OK;
}

tron_err_t tron_batch_host_sync(tron_batch_t* b) {
  clear_error();
  XT_REQUIRE(b != nullptr, TRON_EINVAL, "tron_batch_host_sync: null handle");
  if (!b->host_ready) return TRON_OK;
  XT_CUDA(cudaStreamSynchronize(b->s_in));
  XT_CUDA(cudaStreamSynchronize(b->s_run[0]));
  XT_CUDA(cudaStreamSynchronize(b->s_run[1]));
  XT_CUDA(cudaStreamSynchronize(b->s_out));
  return TRON_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------------------
// Entry point that allocates nothing on the device.
//
// Some callers must not allocate device memory from a library call: hosts whose device
// memory is all handed to their own pool allocator (a cudaMalloc beside the pool fails
// or fragments it) and processes run under a fixed device-memory budget.
// tron_solve_mixed_noalloc serves them: it solves a batch of mixed sizes with the
// persistent kernel, keeping the per-problem size/offset tables, the per-class problem
// lists and the work counters in the fixed array below instead of in memory it would
// otherwise allocate.  The array is reserved on every GPU that loads this library and
// stays there until the process exits.  The size classes run one after another on the
// caller's stream.
// --------------------------------------------------------------------------------------
namespace xt {

constexpr int64_t kNoAllocMaxProblems = TRON_NOALLOC_MAX_PROBLEMS;
constexpr size_t kNaCounters = 0;                                   // 8 x uint64 (<= 8 classes)
constexpr size_t kNaN = 256;                                        // int32 [max]
constexpr size_t kNaPoff = kNaN + 4 * kNoAllocMaxProblems;          // int64 [max]
constexpr size_t kNaVoff = kNaPoff + 8 * kNoAllocMaxProblems;       // int64 [max]
constexpr size_t kNaList = kNaVoff + 8 * kNoAllocMaxProblems;       // int32 [max]
constexpr size_t kNaBytes = kNaList + 4 * kNoAllocMaxProblems;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

static std::mutex g_na_mu;
static void* g_na_addr[256];  // device address of the array, per device ordinal

// Device address of the array for the current device, looked up once per device (a
// cudaDeviceReset of that device invalidates the kept address).
static tron_err_t noalloc_scratch(unsigned char** out) {
  int dev = 0;
  XT_CUDA(cudaGetDevice(&dev));
  XT_REQUIRE(dev >= 0 && dev < 256, TRON_EUNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (g_na_addr[dev] == nullptr) {
    void* p = nullptr;
    XT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_na_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_na_addr[dev]);
  return TRON_OK;
}

}  // namespace xt

extern "C" tron_err_t tron_solve_mixed_noalloc(
    tron_obj_t kind, int64_t nprob, const int32_t* n_host, const tron_options_t* opt,
    const double* d_params, const double* d_lower, const double* d_upper, double* d_x,
    double* d_delta, double* d_f, double* d_pgnorm, int32_t* d_iters, int32_t* d_status,
    void* stream) {
  clear_error();
  XT_REQUIRE(kind == TRON_OBJ_ACOPF_BRANCH || kind == TRON_OBJ_DENSE_QUARTIC ||
                 kind == TRON_OBJ_HS45 || kind == TRON_OBJ_GEN_RAMP,
             TRON_EINVAL, "tron_solve_mixed_noalloc: unknown objective kind %d", (int)kind);
  XT_REQUIRE(nprob >= 0 && nprob <= kNoAllocMaxProblems, TRON_EINVAL,
             "tron_solve_mixed_noalloc: nprob = %lld exceeds the fixed scratch capacity of "
             "%lld problems (TRON_NOALLOC_MAX_PROBLEMS); use tron_batch_create/solve",
             (long long)nprob, (long long)kNoAllocMaxProblems);
  if (nprob == 0) return TRON_OK;
  XT_REQUIRE(n_host != nullptr, TRON_EINVAL, "tron_solve_mixed_noalloc: n_host is NULL");
  XT_REQUIRE(d_lower && d_upper && d_x && d_delta && d_f && d_pgnorm && d_iters && d_status,
             TRON_EINVAL, "tron_solve_mixed_noalloc: null device array");
  XT_REQUIRE(d_params || kind == TRON_OBJ_HS45, TRON_EINVAL,
             "tron_solve_mixed_noalloc: d_params is NULL");
  tron_options_t o;
  if (opt) o = *opt;
  else tron_options_default(&o);
  tron_err_t e = check_options(&o);
  if (e != TRON_OK) return e;
  o.schedule = TRON_SCHED_PERSISTENT;
  const int sms = device_sm_count();
  XT_REQUIRE(sms > 0, TRON_ECUDA, "tron_solve_mixed_noalloc: no CUDA device");
  unsigned char* base = nullptr;
  e = noalloc_scratch(&base);
  if (e != TRON_OK) return e;

  // host-side tables (host memory only), then one upload of each into the array
  std::vector<int64_t> poff(nprob), voff(nprob);
  std::vector<int32_t> lists;
  lists.reserve(nprob);
  int64_t start[kNumClasses] = {0}, count[kNumClasses] = {0};
  {
    int64_t pa = 0, va = 0;
    for (int64_t p = 0; p < nprob; ++p) {
      const int c = size_class(kind, n_host[p]);
      XT_REQUIRE(c > 0, TRON_EUNSUPPORTED,
                 "tron_solve_mixed_noalloc: problem %lld has unsupported size %d",
                 (long long)p, n_host[p]);
      poff[p] = pa;
      voff[p] = va;
      pa += record_size(kind, n_host[p]);
      va += n_host[p];
      count[class_slot(c)]++;
    }
    int64_t at = 0;
    for (int s = kNumClasses - 1; s >= 0; --s) {  // largest class first
      start[s] = at;
      at += count[s];
    }
    lists.resize(nprob);
    int64_t fill[kNumClasses] = {0};
    for (int64_t p = 0; p < nprob; ++p) {
      const int s = class_slot(size_class(kind, n_host[p]));
      lists[start[s] + fill[s]++] = (int32_t)p;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* na_n = reinterpret_cast<int32_t*>(base + kNaN);
  int64_t* na_poff = reinterpret_cast<int64_t*>(base + kNaPoff);
  int64_t* na_voff = reinterpret_cast<int64_t*>(base + kNaVoff);
  int32_t* na_list = reinterpret_cast<int32_t*>(base + kNaList);
  unsigned long long* na_ctr = reinterpret_cast<unsigned long long*>(base + kNaCounters);
  // the counters must start at zero on every call; the tables are overwritten in full
  XT_CUDA(cudaMemsetAsync(na_ctr, 0, 8 * sizeof(unsigned long long), st));
  XT_CUDA(cudaMemcpyAsync(na_n, n_host, sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));
  XT_CUDA(cudaMemcpyAsync(na_poff, poff.data(), sizeof(int64_t) * nprob,
                          cudaMemcpyHostToDevice, st));
  XT_CUDA(cudaMemcpyAsync(na_voff, voff.data(), sizeof(int64_t) * nprob,
                          cudaMemcpyHostToDevice, st));
  XT_CUDA(cudaMemcpyAsync(na_list, lists.data(), sizeof(int32_t) * nprob,
                          cudaMemcpyHostToDevice, st));

  const int wpb0 = o.warps_per_block ? o.warps_per_block : 4;
  const int optin = device_smem_optin();
  for (int s = kNumClasses - 1; s >= 0; --s) {
    if (count[s] == 0) continue;
    const int N = kClasses[s];
    const int G = o.group ? o.group : default_group(kind, N, count[s], sms);
    KernelEntry* ke = find_entry(kind, N, G, o.layout);
    XT_REQUIRE(ke, TRON_EUNSUPPORTED, "no kernel for kind %d, size class %d, group %d",
               (int)kind, N, G);
    const Geometry geo = geometry(*ke, fit_wpb(wpb0, ke->warp_doubles, optin));
    const int wpb = geo.wpb;
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.params = d_params;
    a.lo = d_lower;
    a.hi = d_upper;
    a.x = d_x;
    a.delta = d_delta;
    a.f = d_f;
    a.pg = d_pgnorm;
    a.iters = d_iters;
    a.status = d_status;
    a.nvec = na_n;
    a.poff = na_poff;
    a.voff = na_voff;
    a.plist = na_list + start[s];
    a.count = count[s];
    a.n_uniform = 0;
    a.pstride = 0;
    a.counter = na_ctr + s;
    a.opt = o;
    const size_t smem = geo.smem;
    int occ = 0;
    {
      std::lock_guard<std::mutex> lk(g_table_mu);
      XT_CUDA(cudaFuncSetAttribute(ke->persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      occ = ke->occupancy[wpb];
      if (occ == 0) {
        XT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ke->persistent, geo.threads,
                                                              smem));
        ke->occupancy[wpb] = occ;
      }
    }
    XT_REQUIRE(occ > 0, TRON_EUNSUPPORTED, "kernel does not fit on an SM (smem %zu)", smem);
    if (o.ctas_per_sm > 0) occ = std::min(occ, (int)o.ctas_per_sm);
    const int64_t grid =
        std::min<int64_t>((int64_t)occ * sms, (count[s] + geo.per_cta - 1) / geo.per_cta);
    void* args[] = {&a};
    XT_CUDA(cudaLaunchKernel(ke->persistent, dim3((unsigned)grid), dim3(geo.threads), args, smem,
                             st));
  }
  return TRON_OK;
}
