// Device side of the tensor-train Fourier pricer (arXiv 2203.02804), sm_103a.
//
// One persistent CTA runs one whole TT-cross job (one train: the min-call, or
// one term of the max-call) at a time, taking jobs from a queue sorted by cost.
// Every step of a core update is fused in the CTA and the fiber matrix never
// leaves shared memory:
//   (a) integrand evaluation on the fibers (Eq. main / Eq. discr integrand,
//       written as exp(E) * unit phase * rational factor, with the quadratic
//       form u^T Cov u split into per-index-set partial sums so that one point
//       costs a few FMAs, one exp2 and one reciprocal);
//   (b) cross-interpolation linear algebra (Section IV.B): GEPP tournament over
//       row blocks for the initial rows, then cyclic block maxvol with block
//       GEMMs B = A M and warp-shuffle argmax reductions;
//   (c) the contraction with the quadrature weights (Section IV.A): the row sums
//       of each core's fiber are accumulated while it streams through, and the
//       running product v <- v S P^{-1} is an FP64 solve.
// No wait in this file spins: every loop has a fixed or counted bound.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ttp {

// Optional per-phase cycle counters (profiling builds only: -DTTP_PHASE_TIMERS).
// Thread 0 of each CTA adds the clock64() span of each phase; the totals show
// where a CTA's time goes, waits at barriers included.
// Slots 16..23 count events instead (TTP_COUNT).
#ifdef TTP_PHASE_TIMERS
__device__ unsigned long long g_phase_cycles[24];
#define TTP_COUNT(slot, n)                                                               \
  do {                                                                                   \
    if (threadIdx.x == 0) atomicAdd(&g_phase_cycles[slot], (unsigned long long)(n));     \
  } while (0)
#define TTP_TIC(v) const long long v = clock64()
#define TTP_TOC(v, slot)                                                            \
  do {                                                                              \
    if (threadIdx.x == 0) atomicAdd(&g_phase_cycles[slot], (unsigned long long)(clock64() - (v))); \
  } while (0)
#else
#define TTP_COUNT(slot, n) \
  do {                     \
  } while (0)
#define TTP_TIC(v) \
  do {             \
  } while (0)
#define TTP_TOC(v, slot) \
  do {                   \
  } while (0)
#endif

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum : int { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_NUMERIC = -6, ST_INVALID = -1 };

// aligned as a pair, so that one complex moves in one 8-byte (FP32) or 16-byte
// (FP64) load or store; every cpx array starts on such a boundary
template <typename R>
struct alignas(2 * sizeof(R)) cpx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ void cfma(cpx<R>& acc, cpx<R> a, cpx<R> b) {  // acc += a*b
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
template <typename R>
__device__ __forceinline__ void cfms(cpx<R>& acc, cpx<R> a, cpx<R> b) {  // acc -= a*b
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
template <typename R>
__device__ __forceinline__ R cabs2(cpx<R> a) {
  return fma(a.re, a.re, a.im * a.im);  // one fixed rounding sequence at every call site
}
// 1/a by Smith's method (Smith 1962): no squares of the operands, so it stays
// finite for any nonzero a in range.  FP32 uses the fast reciprocal (its error
// is a few ulp, far below the path's 1e-4 target).
template <typename R>
__device__ __forceinline__ R fast_rcp(R v) {
  if constexpr (sizeof(R) == 4) {
    return __fdividef(R(1), v);
  } else {
    return R(1) / v;
  }
}
template <typename R>
__device__ __forceinline__ cpx<R> crecip(cpx<R> a) {
  if (fabs(a.re) >= fabs(a.im)) {
    const R r = a.im * fast_rcp(a.re), inv = fast_rcp(a.re + a.im * r);
    return {inv, -r * inv};
  }
  const R r = a.re * fast_rcp(a.im), inv = fast_rcp(a.re * r + a.im);
  return {r * inv, -inv};
}

// exp of the log-magnitude: FP32 tables hold E in log2 units, FP64 in natural units.
template <typename R> struct Num;
// Both paths scale every fiber column so that its largest entry is about one
// (kScaleColumns): fibers through far tails reach magnitudes whose squares and
// whose pivot-block inverses leave the floating-point range (~1e-20 in FP32,
// ~1e-200 in FP64 for the call on the maximum).  `unscale` undoes a shift.
template <> struct Num<float> {
  static constexpr double kLogScale = 1.4426950408889634;  // log2(e)
  static constexpr bool kScaleColumns = true;  // power-of-two shifts
  static constexpr float kHuge = 3.0e38f;
  __device__ static __forceinline__ float ex(float e) { return exp2f(e); }
  __device__ static __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  __device__ static __forceinline__ double unscale(double shift) { return exp2(shift); }
  __device__ static __forceinline__ double log_unscale(double shift) { return shift * 0.6931471805599453; }
  __device__ static __forceinline__ float ceil_(float v) { return ceilf(v); }
  __device__ static __forceinline__ float logu(float v) { return __log2f(v); }
};
template <> struct Num<double> {
  static constexpr double kLogScale = 1.0;
  static constexpr bool kScaleColumns = true;  // power-of-two shifts, as k ln 2
  static constexpr double kHuge = 1.0e300;
  __device__ static __forceinline__ double ex(double e) { return exp(e); }
  __device__ static __forceinline__ double div(double a, double b) { return a / b; }
  __device__ static __forceinline__ double unscale(double shift) { return exp(shift); }
  __device__ static __forceinline__ double log_unscale(double shift) { return shift; }
  __device__ static __forceinline__ double ceil_(double v) {
    return ceil(v * 1.4426950408889634) * 0.6931471805599453;
  }
  __device__ static __forceinline__ double logu(double v) { return log(v); }
};

// ---------------------------------------------------------------------------
// descriptors shared with the host
// ---------------------------------------------------------------------------
// What a job's train approximates: the pricing integrand, or (two-train form,
// Eq. braket) one of its two factors.
enum : int { FACTOR_PRODUCT = 0, FACTOR_VHAT = 1, FACTOR_PHI = 2 };

struct JobDesc {
  int d, n, rmax, instance;
  int cauchy;     // 1: min-call, has the 1/(D0 + i sum u) factor
  int term;       // max-call term (0 for the min-call): selects the pivot stream
  int param_off;  // doubles: cov[d*d] row-major, delta[d], pcoef[d], kind[d]
  int factor;     // FACTOR_*
  unsigned long long seed;
  double T, D0, L;
  double Tq;      // time factor of the Gaussian exponent -Tq/2 u^T Cov u (0: no Gaussian)
  double logscale, sign, weight;  // true integrand = sign*exp(logscale + sum norms)*value
  double cap;  // no-arbitrage bound on the train's share of the price: the sum of the spots
  double theta;    // rank threshold of this job (its class's, else the options')
  int block_rows;  // rows per elimination/maxvol block of this job
  int warm_off;    // offset of this job's warm-start record in the warm buffer (-1: none)
};

// Pivot records (warm starts and the final right sets): for k = 1..d-1 a count
// c_k, then c_k multi-indices over axes k..d-1.  Entries of the largest record.
__host__ __device__ inline size_t pivot_record_entries(int dmax, int rmax) {
  return (size_t)(dmax > 0 ? dmax - 1 : 0) + (size_t)rmax * dmax * (dmax > 0 ? dmax - 1 : 0) / 2;
}

// Skeleton of a factor train's core k (two-train form), written by the cross at
// each left-to-right core: rank rho, the selected fiber rows W[t] = o N + i (o
// the outer index), the kept columns' multi-indices K[t][pos] over axes
// k+1..d-1, t in pivot-row order.  One record of emit_core_bytes per core.
__host__ __device__ inline size_t emit_core_bytes(int rall, int dmax) {
  return ((size_t)4 + 4 * (size_t)rall + 2 * (size_t)rall * dmax + 15) / 16 * 16;
}

struct JobResult {
  double est_re, est_im;  // TT sum of the normalised integrand
  double norm_sum;        // sum over axes of the per-axis log normalisation
  double flops;
  long long evaluations, swaps, visits;
  int status, half_sweeps, max_rank, fail_step, rollbacks;
};

struct InstanceResult {
  double price, imag, flops;
  long long evaluations, swaps, visits;
  int status, half_sweeps, max_rank, terms, fail_step, rollbacks;
};

struct Knobs {
  double theta;    // rank threshold
  double tau;      // maxvol tolerance
  double sweep_tol;
  int max_half_sweeps;
  int block_rows;
};

// per-CTA global scratch, byte offsets (pair: PairE<R> entries)
struct Layout {
  size_t u, lam, om, lset, rset, lstate, rstate, lvec, rvec, pair, P, sacc, chain, cb, stride;
  int dmax, nmax, rmax;
};

// maxvol's per-block, per-column bounds on |B| (floats per CTA): a core whose
// blocks x rank exceed it revisits every block
constexpr int kBoundCap = 8192;

// shared-memory carve, byte offsets (sizes depend on R)
struct SmemLayout {
  int sw, m, wvals, stage, tab, colmax, cshift, cref, wrow, wnew, jp, selr, selc, scand, scnt, redv, redi, redk, swcol,
      swrow, mcol, lsz, rsz, misc, total;
  int sw_elems;
};

// ---------------------------------------------------------------------------
// block-wide argmax of (value, index): larger value wins, then lower index.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void am_merge(R& v, int& i, R v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}
// Values are magnitudes (>= 0) or -1 for "no candidate"; NaN never wins.
template <typename R>
__device__ __forceinline__ void warp_argmax(R& v, int& i) {
  if constexpr (sizeof(R) == 4) {
    // non-negative floats order like their bit patterns: two warp reductions
    const unsigned key = (v >= R(0)) ? __float_as_uint(v) + 1u : 0u;
    const unsigned mk = __reduce_max_sync(0xffffffffu, key);
    const unsigned mi = __reduce_min_sync(0xffffffffu, key == mk ? (unsigned)i : 0xffffffffu);
    v = mk == 0u ? R(-1) : __uint_as_float(mk - 1u);
    i = (int)mi;
  } else {
    if (!(v >= R(0))) v = R(-1);  // NaN would make lanes disagree
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      R v2 = __shfl_xor_sync(0xffffffffu, v, off);
      int i2 = __shfl_xor_sync(0xffffffffu, i, off);
      am_merge(v, i, v2, i2);
    }
  }
}
// Writes the warp partial into buffer `buf`, syncs, and returns the block result
// in every thread.  Callers alternate `buf` so that the next write cannot race
// with slower warps still reading.
template <typename R>
__device__ __forceinline__ void block_argmax(R& v, int& i, R* redv, int* redi, int buf) {
  warp_argmax(v, i);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    redv[buf * kWarps + warp] = v;
    redi[buf * kWarps + warp] = i;
  }
  __syncthreads();
  v = redv[buf * kWarps];
  i = redi[buf * kWarps];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) am_merge(v, i, redv[buf * kWarps + w], redi[buf * kWarps + w]);
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based hash
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long pivot_key(unsigned long long seed, int term, int k,
                                                        int t, int b, int j) {
  return seed ^ ((unsigned long long)term << 52) ^ ((unsigned long long)k << 40) ^
         ((unsigned long long)t << 24) ^ ((unsigned long long)b << 12) ^ (unsigned long long)j;
}
// min(n^e, cap) without overflow
__device__ __forceinline__ long long ipow_cap(long long n, int e, long long cap) {
  long long v = 1;
  for (int q = 0; q < e; ++q) {
    v *= n;
    if (v >= cap) return cap;
  }
  return v;
}

// ---------------------------------------------------------------------------
// per-CTA context
// ---------------------------------------------------------------------------
// Pair entry of core k for (outer index o, column c): everything about the
// integrand at fiber point (o, i, c) that does not depend on the grid index i.
template <typename R>
struct alignas(8 * sizeof(R)) PairE {
  R e0;   // log-magnitude part (scaled units)
  R h;    // coefficient of u_i in the log-magnitude
  R s0;   // sum of the other coordinates (for 1/(D0 + i sum u))
  R ore, oim;  // unit phase of the other coordinates
  R pad0, pad1, pad2;
};

constexpr int kStageO = 4;  // outer indices whose pair entries a block stages in shared memory

template <typename R>
struct Ctx {
  // job
  int d, n, rmax;
  int cauchy;
  R D0;
  double T;
  const double* cov;  // [d*d]
  // global scratch
  double* u;          // [n]
  double* lam;        // [d][nmax]
  double2* om;        // [d][nmax]
  uint16_t* lset;     // [(dmax+1)][rmax_all][dmax]
  uint16_t* rset;
  double* lstate;     // [rmax_all][8]
  double* rstate;
  double* lvec;       // [rmax_all][dmax]
  double* rvec;
  PairE<R>* pair;     // [rmax_all][rmax_all]
  cpx<R>* P;          // [rmax_all][rmax_all] pivot rows A[W, Jp], then the saved copy
  double2* sacc;      // [rmax_all][rmax_all]
  double2* vchain;    // [rmax_all]
  double2* ychain;    // [rmax_all]
  float* cb;          // [kBoundCap] maxvol revisit bounds
  int dmax, nmax, rall;
  // shared
  cpx<R>* sw;
  cpx<R>* M;
  cpx<R>* wvals;      // [rmax_all cols][rmax_all rows] original values of the current winners
  PairE<R>* stage;    // [kStageO][rmax_all]
  int stage_lo, stage_n;
  R* tl;  // [nmax] lam' of the active axis (scaled)
  R* tu;  // [nmax] u
  R* tor;
  R* toi;
  R* colmax;
  R* cshift;  // per-column shift of the log-magnitude (a power of two of the value)
  R* cref;    // per-column largest |entry|^2 over the fiber, shifted units (in (1/4, 1])
  int* wrow;
  int* wnew;
  int* jp;
  int* selr;
  int* selc;
  int* scand;  // screened candidate rows [kWarps * 16]
  int* scnt;   // per-warp kept counts [kWarps]
  R* redv;
  int* redi;
  unsigned* redk;
  cpx<R>* swcol;
  cpx<R>* swrow;
  cpx<R>* mcol;
  int* lsz;
  int* rsz;
  int* misc;
  // bookkeeping (thread 0 only)
  double flops;
  long long evals, swaps, visits;
  int rollbacks;
  // FP32 path: tensor-core block product (completion barrier, TMEM accumulators)
  uint64_t* mbar;  // two completion barriers, one per operand buffer
  uint32_t tmem, tmem_cols, mma_phase;  // mma_phase: bit k = next parity of barrier k
  int tc_pending;  // a completion wait gave up: wait again before releasing TMEM
  int fail_step;
  char* emit;      // two-train form: this job's skeleton records (NULL: none)
  const uint16_t* warm;  // this job's warm-start record (NULL: draw every initial pivot)
};

// Index sets: left set at bond k holds multi-indices over axes 0..k-1,
// right set at bond k over axes k..d-1 (stored from position 0).
template <typename R>
__device__ __forceinline__ uint16_t* lset_at(const Ctx<R>& x, int k, int a) {
  return x.lset + ((size_t)k * x.rall + a) * x.dmax;
}
template <typename R>
__device__ __forceinline__ uint16_t* rset_at(const Ctx<R>& x, int k, int b) {
  return x.rset + ((size_t)k * x.rall + b) * x.dmax;
}

template <typename R>
__device__ __forceinline__ const PairE<R>& pair_at(const Ctx<R>& x, int o, int col) {
  const int so = o - x.stage_lo;
  if (so >= 0 && so < x.stage_n) return x.stage[so * x.rall + col];
  return x.pair[o * x.rall + col];
}

// log-magnitude (scaled units) of the integrand at one fiber point, before
// shifts; the phase factors have unit modulus, the min-call's Cauchy factor
// 1/(D0 + i s) has modulus (s^2 + D0^2)^(-1/2)
template <typename R>
__device__ __forceinline__ R eval_logmag(const Ctx<R>& x, int o, int i, int col) {
  const PairE<R>& q = pair_at(x, o, col);
  const R ui = x.tu[i];
  R e = q.e0 + x.tl[i] + q.h * ui;
  if (x.cauchy) {
    const R s = q.s0 + ui;
    e -= R(0.5) * Num<R>::logu(fma(s, s, x.D0 * x.D0));
  }
  return e;
}

// ---------------------------------------------------------------------------
// integrand at one fiber point (Scaled: with the FP32 column shift)
// ---------------------------------------------------------------------------
template <typename R, bool Scaled = true>
__device__ __forceinline__ cpx<R> eval_point(const Ctx<R>& x, int o, int i, int col) {
  const PairE<R> q = pair_at(x, o, col);
  const R ui = x.tu[i];
  R e = q.e0 + x.tl[i] + q.h * ui;
  if constexpr (Num<R>::kScaleColumns && Scaled) e -= x.cshift[col];
  cpx<R> w = cmul(cpx<R>{q.ore, q.oim}, cpx<R>{x.tor[i], x.toi[i]});
  R f = Num<R>::ex(e);
  if (x.cauchy) {
    const R s = q.s0 + ui;
    const R den = fma(s, s, x.D0 * x.D0);
    f = Num<R>::div(f, den);
    w = cmul(w, cpx<R>{x.D0, -s});
  }
  return {w.re * f, w.im * f};
}

// the grid-index part of a fiber point, loaded once per row
template <typename R>
struct RowTab {
  R l, u, re, im;
};
template <typename R>
__device__ __forceinline__ RowTab<R> row_tab(const Ctx<R>& x, int i) {
  return {x.tl[i], x.tu[i], x.tor[i], x.toi[i]};
}
template <typename R>
__device__ __forceinline__ cpx<R> eval_row_point(const Ctx<R>& x, const RowTab<R>& rt, int o, int col) {
  const PairE<R> q = pair_at(x, o, col);
  R e = q.e0 + rt.l + q.h * rt.u;
  if constexpr (Num<R>::kScaleColumns) e -= x.cshift[col];
  cpx<R> w = cmul(cpx<R>{q.ore, q.oim}, cpx<R>{rt.re, rt.im});
  R f = Num<R>::ex(e);
  if (x.cauchy) {
    const R s = q.s0 + rt.u;
    const R den = fma(s, s, x.D0 * x.D0);
    f = Num<R>::div(f, den);
    w = cmul(w, cpx<R>{x.D0, -s});
  }
  return {w.re * f, w.im * f};
}

}  // namespace ttp
