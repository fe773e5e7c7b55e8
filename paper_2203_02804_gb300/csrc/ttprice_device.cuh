// Device steps of one TT-cross job.  See ttprice_kernels.cuh for the overview.
#pragma once

#include <climits>

#include "ttprice_kernels.cuh"
#include "ttprice_tc.cuh"

namespace ttp {

enum : int { MISC_JOB = 0, MISC_PIV = 1, MISC_FAIL = 2, MISC_DRAW = 3, MISC_SING = 4, MISC_OLDW = 5, MISC_MBAR = 8,
             MISC_TMEM = 12 };  // MISC_MBAR: two 8-byte barriers (ints 8..11)

// Functions templated on <R, bool TC>: TC selects the maxvol block-product engine,
// tensor cores (FP32 only: P^{-1} kept as hi/lo TF32 planes) or CUDA cores.
enum : int { DIR_LR = 0, DIR_RL = 1 };

// block sum of a complex double held by every thread; result valid in all threads
__device__ __forceinline__ double2 block_sum_d2(double2 v, double* dscr) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    dscr[2 * warp] = v.x;
    dscr[2 * warp + 1] = v.y;
  }
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  for (int w = 0; w < kWarps; ++w) {
    s.x += dscr[2 * w];
    s.y += dscr[2 * w + 1];
  }
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// job set-up: per-axis tables (FP64), their normalisation, initial right sets
// ---------------------------------------------------------------------------
// Random initial pivots (the paper starts TT-cross from random column sets):
// the first kPeakAttempts attempts of a slot draw each coordinate around the
// grid centre where the integrand's Gaussian factor lives, later ones uniformly.
constexpr int kPeakAttempts = 64;

// For axis j and grid point u the separable factor is
//   kind 0:  1/(i u - delta_j)                       * e^{-i p_j u}
//   kind 1:  1/((i u - delta_j)(1 - delta_j + i u))  * e^{-i p_j u}
//   kind 2:  e^{-i p_j u}  (the characteristic function alone, two-train form)
// stored as log|.| (minus its maximum over the grid) and a unit phase.
// `draw` = false builds the tables only (no initial right sets).
template <typename R>
__device__ void job_setup(Ctx<R>& x, const JobDesc& jd, const double* prm, double* dscr,
                          double& norm_sum, bool draw = true) {
  const int d = jd.d, n = jd.n, tid = threadIdx.x;
  const double* delta = prm + d * d;
  const double* pcoef = delta + d;
  const double* kind = pcoef + d;
  const double eta = 2.0 * jd.L / n;
  for (int i = tid; i < n; i += kThreads) x.u[i] = -jd.L + (i + 0.5) * eta;
  for (int idx = tid; idx < d * n; idx += kThreads) {
    const int j = idx / n, i = idx % n;
    const double u = -jd.L + (i + 0.5) * eta;
    const double dl = delta[j];
    double lr, c, s;
    if constexpr (sizeof(R) == 4) {
      // Mixed path: the linear phase p_j u (tens of radians) is formed and reduced
      // modulo 2 pi in FP64; the bounded parts (log-magnitudes, the arguments of
      // the rational factors, the sine/cosine of the reduced angle) in FP32.
      const float uf = (float)u, df = (float)dl;
      float lrf = 0.0f, pr = 0.0f;
      if (kind[j] != 2.0) {
        lrf = -0.5f * logf(uf * uf + df * df);
        pr = -atan2f(uf, -df);
      }
      if (kind[j] == 1.0) {
        const float ef = 1.0f - df;
        lrf += -0.5f * logf(uf * uf + ef * ef);
        pr -= atan2f(uf, ef);
      }
      const double lin = -pcoef[j] * u;
      const double turns = rint(lin * 0.15915494309189535);  // 1/(2 pi)
      const float red = (float)fma(-turns, 6.283185307179586, lin) + pr;
      float sf, cf;
      sincosf(red, &sf, &cf);
      lr = lrf;
      c = cf;
      s = sf;
    } else {
      lr = 0.0;
      double ph = -pcoef[j] * u;
      if (kind[j] != 2.0) {
        lr = -0.5 * log(u * u + dl * dl);
        ph -= atan2(u, -dl);
      }
      if (kind[j] == 1.0) {
        const double e = 1.0 - dl;
        lr += -0.5 * log(u * u + e * e);
        ph -= atan2(u, e);
      }
      sincos(ph, &s, &c);
    }
    x.lam[(size_t)j * x.nmax + i] = lr;
    x.om[(size_t)j * x.nmax + i] = make_double2(c, s);
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  double part = 0.0;
  for (int j = warp; j < d; j += kWarps) {
    double mx = -1e300;
    for (int i = lane; i < n; i += 32) mx = fmax(mx, x.lam[(size_t)j * x.nmax + i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    for (int i = lane; i < n; i += 32) x.lam[(size_t)j * x.nmax + i] -= mx;
    part += mx;  // identical in every lane
  }
  if (lane == 0) dscr[16 + warp] = part;
  // initial right index sets, one thread per bond
  // one warp per core k; lanes draw slots (first attempts) or coordinates (redraws) in
  // parallel, duplicates are resolved slot by slot in order, so the accepted sets
  // are those of a plain sequential draw
  for (int k = 1 + warp; draw && k < d; k += kWarps) {
    const int width = d - k;
    const long long cap = jd.rmax;
    long long rk = ipow_cap(n, k, cap + 1);
    rk = rk < cap ? rk : cap;
    const long long nw = ipow_cap(n, width, cap + 1);
    if (nw < rk) rk = nw;
    if (lane == 0) x.rsz[k] = (int)rk;
    if (nw == rk) {  // every right multi-index, lexicographic
      for (int bb = lane; bb < rk; bb += 32) {
        uint16_t* dst = rset_at(x, k, bb);
        int rem = bb;
        for (int pos = width - 1; pos >= 0; --pos) {
          dst[pos] = (uint16_t)(rem % n);
          rem /= n;
        }
      }
    } else {
      // coordinate pos of slot bb at attempt t (around the centre for the first
      // kPeakAttempts attempts, uniform after); every FP64 operation rounded
      // separately (no contraction) so the draw is reproducible
      auto coord = [&](int bb, int t, int pos) -> uint16_t {
        const int j = k + pos;
        if (t < kPeakAttempts) {
          const double w = __ddiv_rn(1.5, __dmul_rn(__dsqrt_rn(__dmul_rn(prm[j * d + j], jd.T)), eta));
          double sum = 0.0;
          for (int qq = 0; qq < 4; ++qq) {
            const unsigned long long h = splitmix64(pivot_key(jd.seed, jd.term, k, t, bb, 4 * j + qq));
            sum = __dadd_rn(sum, __dmul_rn((double)(h >> 11), 0x1p-53));
          }
          const double z = __dmul_rn(__dsub_rn(sum, 2.0), 1.7320508075688772);
          long long idx = n / 2 + (long long)floor(__dadd_rn(__dmul_rn(w, z), 0.5));
          idx = idx < 0 ? 0 : (idx > n - 1 ? n - 1 : idx);
          return (uint16_t)idx;
        }
        return (uint16_t)(splitmix64(pivot_key(jd.seed, jd.term, k, t, bb, j)) % n);
      };
      // a warm start fills the first slots from its record; otherwise slot 0 is
      // the grid centre; the remaining slots are drawn
      int first = 0;
      if (x.warm) {
        const uint16_t* w = x.warm;
        for (int kk = 1; kk < k; ++kk) w += 1 + (int)w[0] * (d - kk);  // this bond's part
        first = min((int)w[0], (int)rk);
        for (int idx = lane; idx < first * width; idx += 32)
          rset_at(x, k, idx / width)[idx % width] = w[1 + idx];
      }
      if (first == 0) {
        uint16_t* c0 = rset_at(x, k, 0);
        for (int pos = lane; pos < width; pos += 32) c0[pos] = (uint16_t)(n / 2);
        first = 1;
      }
      for (int bb = first + lane; bb < rk; bb += 32) {
        uint16_t* dst = rset_at(x, k, bb);
        for (int pos = 0; pos < width; ++pos) dst[pos] = coord(bb, 0, pos);
      }
      __syncwarp();
      for (int bb = first; bb < rk; ++bb) {
        uint16_t* dst = rset_at(x, k, bb);
        bool fresh = false;
        for (int t = 0; t < 65536 && !fresh; ++t) {
          if (t > 0) {
            for (int pos = lane; pos < width; pos += 32) dst[pos] = coord(bb, t, pos);
            __syncwarp();
          }
          bool dup = false;
          for (int q = lane; q < bb && !dup; q += 32) {
            const uint16_t* o = rset_at(x, k, q);
            bool same = true;
            for (int pos = 0; pos < width && same; ++pos) same = (o[pos] == dst[pos]);
            dup = same;
          }
          fresh = !__any_sync(0xffffffffu, dup);
        }
        if (!fresh && lane == 0) x.misc[MISC_DRAW] = 1;
        __syncwarp();
      }
    }
  }
  if (tid == 0) {
    x.lsz[0] = 1;
    x.rsz[d] = 1;
  }
  __syncthreads();
  norm_sum = 0.0;
  for (int w = 0; w < kWarps; ++w) norm_sum += dscr[16 + w];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// per-core states and the pair table (FP64, stored in R)
// ---------------------------------------------------------------------------
// Left entry a (axes 0..k-1) and right entry b (axes k+1..d-1) of core k:
//   E0(a,b) = lam_L + lam_R - T/2 (q_L + q_R + 2 u_L^T Cov_LR u_R)
//   H(a,b)  = -T (Cov_kL u_L + Cov_kR u_R)      (coefficient of u at axis k)
//   S0(a,b) = sum u_L + sum u_R,   Om(a,b) = phase_L * phase_R
// so that at grid point u of axis k the log-magnitude is
//   E0 + lam_k(u) - T/2 Cov_kk u^2 + H u.
template <typename R>
__device__ void core_states(Ctx<R>& x, int k, int dir) {
  const int d = x.d, tid = threadIdx.x;
  const int nl = x.lsz[k], nr = x.rsz[k + 1];
  const int wr = d - k - 1;
  const double* C = x.cov;
  for (int a = tid; a < nl; a += kThreads) {
    const uint16_t* ix = lset_at(x, k, a);
    double q = 0.0, s = 0.0, lm = 0.0, y = 0.0;
    double2 om = make_double2(1.0, 0.0);
    for (int j = 0; j < k; ++j) {
      const double uj = x.u[ix[j]];
      double t = 0.0;
      for (int l = 0; l < k; ++l) t += C[j * d + l] * x.u[ix[l]];
      q += uj * t;
      s += uj;
      lm += x.lam[(size_t)j * x.nmax + ix[j]];
      const double2 w = x.om[(size_t)j * x.nmax + ix[j]];
      om = make_double2(om.x * w.x - om.y * w.y, om.x * w.y + om.y * w.x);
      y += C[k * d + j] * uj;
    }
    for (int l = 0; l < wr; ++l) {
      double v = 0.0;
      for (int j = 0; j < k; ++j) v += C[(k + 1 + l) * d + j] * x.u[ix[j]];
      x.lvec[(size_t)a * x.dmax + l] = v;
    }
    double* st = x.lstate + 8 * a;
    st[0] = q; st[1] = s; st[2] = lm; st[3] = y; st[4] = om.x; st[5] = om.y;
  }
  for (int b = tid; b < nr; b += kThreads) {
    const uint16_t* ix = rset_at(x, k + 1, b);
    double q = 0.0, s = 0.0, lm = 0.0, z = 0.0;
    double2 om = make_double2(1.0, 0.0);
    for (int l = 0; l < wr; ++l) {
      const int ax = k + 1 + l;
      const double ul = x.u[ix[l]];
      double t = 0.0;
      for (int mm = 0; mm < wr; ++mm) t += C[ax * d + k + 1 + mm] * x.u[ix[mm]];
      q += ul * t;
      s += ul;
      lm += x.lam[(size_t)ax * x.nmax + ix[l]];
      const double2 w = x.om[(size_t)ax * x.nmax + ix[l]];
      om = make_double2(om.x * w.x - om.y * w.y, om.x * w.y + om.y * w.x);
      z += C[k * d + ax] * ul;
      x.rvec[(size_t)b * x.dmax + l] = ul;
    }
    double* st = x.rstate + 8 * b;
    st[0] = q; st[1] = s; st[2] = lm; st[3] = z; st[4] = om.x; st[5] = om.y;
  }
  __syncthreads();
  const double T = x.T, ls = Num<R>::kLogScale;
  for (int p = tid; p < nl * nr; p += kThreads) {
    const int a = p % nl, b = p / nl;
    const double* sl = x.lstate + 8 * a;
    const double* sr = x.rstate + 8 * b;
    double xab = 0.0;
    for (int l = 0; l < wr; ++l) xab += x.lvec[(size_t)a * x.dmax + l] * x.rvec[(size_t)b * x.dmax + l];
    const double e0 = sl[2] + sr[2] - 0.5 * T * (sl[0] + sr[0] + 2.0 * xab);
    const double h = -T * (sl[3] + sr[3]);
    const double s0 = sl[1] + sr[1];
    const double ore = sl[4] * sr[4] - sl[5] * sr[5];
    const double oim = sl[4] * sr[5] + sl[5] * sr[4];
    const int o = dir == DIR_LR ? a : b, c = dir == DIR_LR ? b : a;
    PairE<R> q;
    q.e0 = (R)(e0 * ls);
    q.h = (R)(h * ls);
    q.s0 = (R)s0;
    q.ore = (R)ore;
    q.oim = (R)oim;
    q.pad0 = q.pad1 = q.pad2 = R(0);
    x.pair[o * x.rall + c] = q;
  }
  if (tid == 0) x.stage_n = 0;
  __syncthreads();
}

// Copy the pair entries of outer indices olo..ohi (all nc columns) to shared
// memory when they fit; eval_point then reads them from there.
template <typename R>
__device__ void stage_pairs(Ctx<R>& x, int olo, int ohi, int nc) {
  const int cnt = ohi - olo + 1;
  __syncthreads();  // nobody may still read the previous stage
  if (cnt <= kStageO) {
    for (int idx = threadIdx.x; idx < cnt * nc; idx += kThreads) {
      const int so = idx / nc, c = idx % nc;
      x.stage[so * x.rall + c] = x.pair[(olo + so) * x.rall + c];
    }
  }
  if (threadIdx.x == 0) {
    x.stage_lo = olo;
    x.stage_n = cnt <= kStageO ? cnt : 0;
  }
  __syncthreads();
}

// the active axis' table in shared memory (R precision, exponent pre-scaled)
template <typename R>
__device__ void load_axis_table(Ctx<R>& x, int k) {
  const double ckk = x.cov[k * x.d + k], T = x.T, ls = Num<R>::kLogScale;
  for (int i = threadIdx.x; i < x.n; i += kThreads) {
    const double u = x.u[i];
    x.tl[i] = (R)((x.lam[(size_t)k * x.nmax + i] - 0.5 * T * ckk * u * u) * ls);
    x.tu[i] = (R)u;
    const double2 w = x.om[(size_t)k * x.nmax + i];
    x.tor[i] = (R)w.x;
    x.toi[i] = (R)w.y;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Shift every fiber column by a power of two so that its largest entry has
// magnitude in (1/2, 1], and record that largest |entry|^2 (shifted units) for
// the rank reveal.  Elimination pivots and maxvol's B = A P^{-1} are invariant
// under column scaling, and the contraction step v S P^{-1} sees the same
// scale in S and P, so the shift changes no exact result; it keeps |a|^2 and
// the pivot-block inverse inside the floating-point range for columns through
// far tails.
// ---------------------------------------------------------------------------
template <typename R>
__device__ void column_shifts(Ctx<R>& x, int no, int nc) {
  if constexpr (Num<R>::kScaleColumns) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, N = x.n, m = no * N;
    for (int c = warp; c < nc; c += kWarps) {
      // four independent maxima per lane (a max does not depend on its order), rows
      // walked as (outer index, grid index): no integer division
      R m0 = R(-3.0e38), m1 = R(-3.0e38), m2 = R(-3.0e38), m3 = R(-3.0e38);
      for (int o = 0; o < no; ++o) {
        int i = lane;
        for (; i + 96 < N; i += 128) {
          m0 = fmax(m0, eval_logmag(x, o, i, c));
          m1 = fmax(m1, eval_logmag(x, o, i + 32, c));
          m2 = fmax(m2, eval_logmag(x, o, i + 64, c));
          m3 = fmax(m3, eval_logmag(x, o, i + 96, c));
        }
        for (; i < N; i += 32) m0 = fmax(m0, eval_logmag(x, o, i, c));
      }
      R mx = fmax(fmax(m0, m1), fmax(m2, m3));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0) {
        const R sh = Num<R>::ceil_(mx);
        x.cshift[c] = sh;
        x.cref[c] = Num<R>::ex(R(2) * (mx - sh));
      }
    }
    if (threadIdx.x == 0) x.flops += 4.0 * (double)m * nc;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// GEPP on the candidate matrix sw (q rows x ncol, column-major, leading dim ld)
// Returns the number of pivots; selr/selc hold (candidate row, column) pairs.
// Each thread owns one candidate row (q <= kThreads).
// ---------------------------------------------------------------------------
template <typename R>
__device__ int gepp_select(Ctx<R>& x, int q, int ncol, int ld, R thr2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  cpx<R>* __restrict__ S = x.sw;
  for (int c = warp; c < ncol; c += kWarps) {
    R mx = 0;
    for (int r = lane; r < q; r += 32) mx = fmax(mx, cabs2(S[c * ld + r]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) x.colmax[c] = mx;
  }
  __syncthreads();
  // up to 128 candidates: two threads per row, the row's columns split by parity
  // (the half holding column c + 1 offers the row for the next pivot); more: one
  // thread per row
  static_assert(kThreads == 256, "two threads per row: tid >> 7 picks the half");
  const bool split = q <= kThreads / 2;
  const int row = split ? (tid & (kThreads / 2 - 1)) : tid;
  const int half = split ? (tid >> 7) : 0;
  const int js = split ? 2 : 1;
  const bool own = row < q;
  bool mine_used = false;
  R v = (own && half == 0) ? cabs2(S[row]) : R(-1);
  int vi = (own && half == 0) ? row : INT_MAX;
  int buf = 0;
  block_argmax(v, vi, x.redv, x.redi, buf);
  int nsel = 0;
  long long fl = 0;  // complex multiply-adds (thread 0's count is used)
  for (int c = 0; c < ncol; ++c) {
    const int p = vi;
    const bool take = (v > thr2 * x.colmax[c]) && (v > R(0));
    if (take) {
      if (tid == 0) {
        x.selr[nsel] = p;
        x.selc[nsel] = c;
      }
      const bool active = own && !mine_used && row != p;
      if (row == p) mine_used = true;
      if (active && c + 1 < ncol) {
        const cpx<R> l = cmul(S[c * ld + row], crecip(S[c * ld + p]));
        // this thread's columns: c + 1 onwards with its parity (split) or all;
        // four at a time, loads first, then the updates
        int j = c + 1;
        if (split && ((j & 1) != half)) ++j;
        for (; j + 3 * js < ncol; j += 4 * js) {
          cpx<R> a0 = S[j * ld + row], a1 = S[(j + js) * ld + row];
          cpx<R> a2 = S[(j + 2 * js) * ld + row], a3 = S[(j + 3 * js) * ld + row];
          const cpx<R> p0 = S[j * ld + p], p1 = S[(j + js) * ld + p];
          const cpx<R> p2 = S[(j + 2 * js) * ld + p], p3 = S[(j + 3 * js) * ld + p];
          cfms(a0, l, p0);
          cfms(a1, l, p1);
          cfms(a2, l, p2);
          cfms(a3, l, p3);
          S[j * ld + row] = a0;
          S[(j + js) * ld + row] = a1;
          S[(j + 2 * js) * ld + row] = a2;
          S[(j + 3 * js) * ld + row] = a3;
        }
        for (; j < ncol; j += js) cfms(S[j * ld + row], l, S[j * ld + p]);
      }
      ++nsel;
      if (tid == 0) fl += (long long)(q - nsel) * (ncol - c - 1);
    }
    if (c + 1 < ncol) {
      const bool offer = own && !mine_used && (!split || (((c + 1) & 1) == half));
      v = offer ? cabs2(S[(c + 1) * ld + row]) : R(-1);
      vi = offer ? row : INT_MAX;
      buf ^= 1;
      block_argmax(v, vi, x.redv, x.redi, buf);
    }
  }
  if (tid == 0) x.flops += 8.0 * (double)fl;
  __syncthreads();
  return nsel;
}

// ---------------------------------------------------------------------------
// P^{-1} of the FP32 path: hi and lo TF32 parts in K-major tensor-core planes
// (hi in M, lo in the winner-value buffer, free during maxvol)
// ---------------------------------------------------------------------------
constexpr int kTcChunk = 16;               // kept columns per evaluation/MMA chunk (two K steps)
constexpr int kTcBufs = 16 / kTcChunk;     // operand buffers in the 32 KB (1: chunk 16, 2: chunk 8)

__device__ __forceinline__ float tf32_hi(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// P^{-1}[t][s] from / to its hi and lo planes (row s, k t of the B operand)
template <typename R>
__device__ __forceinline__ cpx<R> minv_get(const Ctx<R>& x, int kp, int t, int s) {
  const int sbo = kp * 32, off = tc::kmaj(s, t, sbo), plane = (kp / 8) * sbo;
  const unsigned char* hi = reinterpret_cast<const unsigned char*>(x.M);
  const unsigned char* lo = reinterpret_cast<const unsigned char*>(x.wvals);
  return {*reinterpret_cast<const R*>(hi + off) + *reinterpret_cast<const R*>(lo + off),
          *reinterpret_cast<const R*>(hi + plane + off) + *reinterpret_cast<const R*>(lo + plane + off)};
}
template <typename R>
__device__ __forceinline__ void minv_set(Ctx<R>& x, int kp, int t, int s, cpx<R> v) {
  const int sbo = kp * 32, off = tc::kmaj(s, t, sbo), plane = (kp / 8) * sbo;
  unsigned char* hi = reinterpret_cast<unsigned char*>(x.M);
  unsigned char* lo = reinterpret_cast<unsigned char*>(x.wvals);
  const R hr = tf32_hi(v.re), hm = tf32_hi(v.im);
  *reinterpret_cast<R*>(hi + off) = hr;
  *reinterpret_cast<R*>(lo + off) = v.re - hr;
  *reinterpret_cast<R*>(hi + plane + off) = hm;
  *reinterpret_cast<R*>(lo + plane + off) = v.im - hm;
}

// ---------------------------------------------------------------------------
// M = P^{-1} by Gauss-Jordan with partial pivoting on [P | I], in R, scratch in
// sw.  Rows are never moved: the pivot of column c is the unused row with the
// largest |entry|^2 (order[c]); every other row subtracts its multiple of the
// pivot row at the columns right of c, and the threads holding column c + 1
// collect its argmax, so a step costs one block barrier.  At the end row c of
// P^{-1} is the right half of row order[c] over its pivot.
// Returns false (M not written) when a pivot is zero or not finite.
// ---------------------------------------------------------------------------
template <typename R, bool TC>
__device__ bool invert_pivots(Ctx<R>& x, int rho) {
  const int tid = threadIdx.x;
  const int w2 = 2 * rho, ld = w2 + 1;  // odd row stride: column accesses are conflict-free
  cpx<R>* G = x.sw;
  int* order = x.selr;
  const int lane = tid & 31, warp = tid >> 5;
  for (int c = lane; c < rho; c += 32)  // column per lane, rows per warp
    for (int r = warp; r < rho; r += kWarps) {
      G[r * ld + c] = x.P[r * x.rall + c];
      G[r * ld + rho + c] = cpx<R>{R(r == c), R(0)};
    }
  __syncthreads();
  const int tpr = rho <= 32 ? 8 : 4;  // threads per row (rho <= 64)
  const int myr = tid / tpr, part = tid % tpr;
  R v = R(-1);
  int vi = INT_MAX;
  if (myr < rho && part == 0) am_merge(v, vi, cabs2(G[myr * ld]), myr);
  int buf = 0;
  block_argmax(v, vi, x.redv, x.redi, buf);
  unsigned long long used = 0ull;
  bool ok = true;
  for (int c = 0; c < rho; ++c) {  // v, vi, used: block-uniform
    if (!(v > R(0)) || !(v < R(INFINITY))) {
      ok = false;
      break;
    }
    const int p = vi;
    if (tid == 0) order[c] = p;
    used |= 1ull << p;
    v = R(-1);
    vi = INT_MAX;
    if (myr < rho && myr != p) {
      // column c and row p are only read in this step
      const cpx<R> f = cmul(G[myr * ld + c], crecip(G[p * ld + c]));
      for (int j = c + 1 + part; j < w2; j += tpr) {
        cpx<R> a = G[myr * ld + j];
        cfms(a, f, G[p * ld + j]);
        G[myr * ld + j] = a;
        if (j == c + 1 && j < rho && !((used >> myr) & 1ull)) am_merge(v, vi, cabs2(a), myr);
      }
    }
    buf ^= 1;
    block_argmax(v, vi, x.redv, x.redi, buf);  // its barrier also publishes the updates
  }
  if (ok) {
    if constexpr (TC) {
      // the tensor-core operand: hi and lo K-major planes, zero outside rho x rho
      const int kp = tc::pad16(rho);
      for (int c = lane; c < kp; c += 32)
        for (int r = warp; r < kp; r += kWarps) {
          cpx<R> m = {R(0), R(0)};
          if (r < rho && c < rho) {
            const int pr = order[r];
            m = cmul(G[pr * ld + rho + c], crecip(G[pr * ld + r]));
          }
          minv_set(x, kp, r, c, m);
        }
    } else {
      for (int c = lane; c < rho; c += 32)
        for (int r = warp; r < rho; r += kWarps) {
          const int pr = order[r];
          x.M[r * x.rall + c] = cmul(G[pr * ld + rho + c], crecip(G[pr * ld + r]));
        }
    }
  }
  if (tid == 0) x.flops += 8.0 * (double)rho * rho * (2.0 * rho);
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------
// evaluate pivot row j of P (fiber row g at the kept columns)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void eval_prow(Ctx<R>& x, int j, int g, int rho) {
  const int o = g / x.n, i = g % x.n;
  for (int t = threadIdx.x; t < rho; t += kThreads) x.P[j * x.rall + t] = eval_point(x, o, i, x.jp[t]);
}

// ---------------------------------------------------------------------------
// GEPP tournament over row blocks: initial rows W and kept columns Jp.
// The winners' original rows are cached in wvals (column-major, ld rall), so a
// merge evaluates only its block and the block rows that win.
// ---------------------------------------------------------------------------
// Fibers of more than kScreenMinRows rows are screened: every kScreenBlock rows
// form one merge, whose candidates are, from each kScreenSub-row sub-block, the
// kScreenKeep rows with the largest max_c log|a_rc| (the log-magnitude in the
// working precision, which needs no complex evaluation; ties to the lower row),
// in ascending row order.  One warp screens one sub-block.
constexpr int kScreenMinRows = 512;  // larger fibers offer >= 4 full sub-blocks: 64 candidates
constexpr int kScreenBlock = 1024;
constexpr int kScreenSub = 128;
constexpr int kScreenKeep = 16;
constexpr int kScreenRpl = kScreenSub / 32;  // rows per lane
static_assert(kScreenBlock == kWarps * kScreenSub, "one warp per sub-block");

// Warp argmax of a key of either sign (larger wins, then lower index); a lane
// with no candidate passes valid = false; i = INT_MAX when no lane has one.
template <typename R>
__device__ __forceinline__ void warp_argmax_key(R v, int& i, bool valid) {
  if constexpr (sizeof(R) == 4) {
    // order-preserving map of the float's bits to unsigned; 0 = no candidate
    const unsigned u = __float_as_uint(v);
    const unsigned key = valid ? max(1u, (u & 0x80000000u) ? ~u : (u | 0x80000000u)) : 0u;
    const unsigned mk = __reduce_max_sync(0xffffffffu, key);
    const unsigned mi = __reduce_min_sync(0xffffffffu, (key == mk) ? (unsigned)i : 0xffffffffu);
    i = mk == 0u ? INT_MAX : (int)mi;
  } else {
    int bi = valid ? i : INT_MAX;
    R bv = v;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, bv, off);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, off);
      if (i2 != INT_MAX && (bi == INT_MAX || v2 > bv || (v2 == bv && i2 < bi))) {
        bv = v2;
        bi = i2;
      }
    }
    i = bi;
  }
}

template <typename R>
__device__ int screen_block(Ctx<R>& x, int ss, int se, int nc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = x.n;
  const int base = ss + warp * kScreenSub;
  R key[kScreenRpl];
  bool valid[kScreenRpl];
#pragma unroll
  for (int h = 0; h < kScreenRpl; ++h) {
    const int r = base + lane + 32 * h;
    valid[h] = r < se;
    key[h] = R(0);
    if (valid[h]) {
      R mx = -Num<R>::kHuge;
      for (int c = 0; c < nc; ++c) mx = fmax(mx, eval_logmag(x, r / N, r % N, c));
      key[h] = mx;
      valid[h] = mx == mx;  // a NaN log-magnitude never screens in
    }
  }
  // warp top-kScreenKeep: repeated argmax; the kept set is a row mask, 32 rows per word
  unsigned kept[kScreenRpl];
  bool taken[kScreenRpl];
#pragma unroll
  for (int h = 0; h < kScreenRpl; ++h) {
    kept[h] = 0u;
    taken[h] = false;
  }
  for (int t = 0; t < kScreenKeep; ++t) {
    R v = R(0);
    int vi = INT_MAX;
    bool any = false;
#pragma unroll
    for (int h = 0; h < kScreenRpl; ++h)
      if (valid[h] && !taken[h] && (!any || key[h] > v)) {  // rows ascend with h: ties keep the lower
        v = key[h];
        vi = lane + 32 * h;
        any = true;
      }
    warp_argmax_key(v, vi, any);
    if (vi == INT_MAX) break;
#pragma unroll
    for (int h = 0; h < kScreenRpl; ++h)
      if ((vi >> 5) == h) {
        kept[h] |= 1u << (vi & 31);
        if ((vi & 31) == lane) taken[h] = true;
      }
  }
  // write the kept rows of this sub-block in ascending order: lane q takes the q-th set bit
  int cnt = 0;
#pragma unroll
  for (int h = 0; h < kScreenRpl; ++h) {
    const int c = __popc(kept[h]);
    if (lane >= cnt && lane < cnt + c) {
      unsigned msk = kept[h];
      for (int q = 0; q < lane - cnt; ++q) msk &= msk - 1u;  // drop the lowest set bits
      x.scand[warp * kScreenKeep + lane] = base + 32 * h + __ffs((int)msk) - 1;
    }
    cnt += c;
  }
  if (lane == 0) x.scnt[warp] = cnt;
  __syncthreads();
  // compact the per-warp lists (warp order = row order)
  int tot = 0;
  for (int w = 0; w < kWarps; ++w) tot += x.scnt[w];
  int out = 0, sel = -1;
  for (int w = 0; w < kWarps; ++w) {
    if (tid >= out && tid < out + x.scnt[w]) sel = x.scand[w * kScreenKeep + (tid - out)];
    out += x.scnt[w];
  }
  __syncthreads();
  if (sel >= 0) x.scand[tid] = sel;
  if (tid == 0) x.flops += 4.0 * (double)(se - ss) * nc;
  __syncthreads();
  return tot;
}

template <typename R>
__device__ int tournament(Ctx<R>& x, int m, int nc, int b, R thr2) {
  const int tid = threadIdx.x, N = x.n;
  const bool screened = m > kScreenMinRows;
  const int step = screened ? kScreenBlock : b;
  const int nb = (m + step - 1) / step;
  const int ldq = x.rall + max(b, kWarps * kScreenKeep);
  int rho = 0;
  for (int beta = 0; beta < nb; ++beta) {
    const int rs = beta * step;
    const int bs0 = min(step, m - rs);
    TTP_TIC(t_ev);
    int bs = bs0;
    if (screened) {
      stage_pairs(x, 0, -1, nc);  // screening reads pair entries from global memory
      bs = screen_block(x, rs, rs + bs0, nc);
    } else {
      stage_pairs(x, rs / N, (rs + bs0 - 1) / N, nc);
    }
    const int q = rho + bs;
    for (int idx = tid; idx < rho * nc; idx += kThreads) {
      const int t = idx % rho, c = idx / rho;
      x.sw[c * ldq + t] = x.wvals[c * x.rall + t];
    }
    if (bs <= kThreads / 2) {
      // two threads per candidate row, each every other column: the row's indices and
      // grid-index table once, four independent points at a time (loads before stores)
      const int r = tid & (kThreads / 2 - 1);
      if (r < bs) {
        const int g = screened ? x.scand[r] : rs + r;
        const int o = g / N;
        const RowTab<R> rt = row_tab(x, g - o * N);
        cpx<R>* dst = x.sw + rho + r;
        int c = tid / (kThreads / 2);
        for (; c + 6 < nc; c += 8) {
          const cpx<R> v0 = eval_row_point(x, rt, o, c);
          const cpx<R> v1 = eval_row_point(x, rt, o, c + 2);
          const cpx<R> v2 = eval_row_point(x, rt, o, c + 4);
          const cpx<R> v3 = eval_row_point(x, rt, o, c + 6);
          dst[c * ldq] = v0;
          dst[(c + 2) * ldq] = v1;
          dst[(c + 4) * ldq] = v2;
          dst[(c + 6) * ldq] = v3;
        }
        for (; c < nc; c += 2) dst[c * ldq] = eval_row_point(x, rt, o, c);
      }
    } else {
      // four independent evaluations per thread and iteration (loads before stores)
      const int tot = bs * nc;
      for (int base = tid; base < tot; base += 4 * kThreads) {
        cpx<R> v[4];
        int dst[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = base + u * kThreads;
          dst[u] = -1;
          if (idx < tot) {
            const int r = idx % bs, c = idx / bs;
            const int g = screened ? x.scand[r] : rs + r;
            v[u] = eval_point(x, g / N, g % N, c);
            dst[u] = c * ldq + rho + r;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (dst[u] >= 0) x.sw[dst[u]] = v[u];
      }
    }
    if (tid == 0) x.flops += 24.0 * bs * nc;
    __syncthreads();
    TTP_TOC(t_ev, 2);
    TTP_TIC(t_ge);
    const int nsel = gepp_select(x, q, nc, ldq, thr2);
    TTP_TOC(t_ge, 3);
    TTP_TIC(t_ga);
    // new winners' original rows, gathered into sw (free now), then copied
    for (int idx = tid; idx < nsel * nc; idx += kThreads) {
      const int t = idx % nsel, c = idx / nsel;
      const int cr = x.selr[t];
      cpx<R> v;
      if (cr < rho) {
        v = x.wvals[c * x.rall + cr];
      } else {
        const int g = screened ? x.scand[cr - rho] : rs + cr - rho;
        v = eval_point(x, g / N, g % N, c);
      }
      x.sw[c * x.rall + t] = v;
    }
    for (int t = tid; t < nsel; t += kThreads) {
      const int cr = x.selr[t];
      x.wnew[t] = cr < rho ? x.wrow[cr] : (screened ? x.scand[cr - rho] : rs + cr - rho);
    }
    __syncthreads();
    for (int idx = tid; idx < nsel * nc; idx += kThreads) {
      const int t = idx % nsel, c = idx / nsel;
      x.wvals[c * x.rall + t] = x.sw[c * x.rall + t];
    }
    for (int t = tid; t < nsel; t += kThreads) {
      x.wrow[t] = x.wnew[t];
      x.jp[t] = x.selc[t];
    }
    rho = nsel;
    __syncthreads();
    TTP_TOC(t_ga, 4);
  }
  return rho;
}

// ---------------------------------------------------------------------------
// Rank-revealing reduction of the winners' pivot block A[W, Jp] (rho x rho):
//  1. a column whose largest |entry|^2 in the block is at most theta^2 times
//     its largest over the whole fiber is numerically absent and is dropped;
//  2. complete pivoting on the column-equilibrated block: each entry's |.|^2
//     over its column's largest in the block; the next pivot is the largest
//     such value of the remaining block (lowest row-major index on ties), and
//     the reduction stops once it is at most theta^2.
// Both rules are invariant under column scaling.  The kept rows and columns,
// in pivot order, form a block of condition number about 1/theta after column
// equilibration (the tournament's partial pivoting alone leaves some far
// worse).  W and Jp are reordered and P = A[W, Jp] is built; returns the rank.
// ---------------------------------------------------------------------------
template <typename R>
__device__ int rank_reveal(Ctx<R>& x, int rho, R thr2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ld = rho + 1, tot = rho * rho;
  cpx<R>* __restrict__ G = x.sw;  // odd row stride: row and column reads are conflict-free
  for (int t = lane; t < rho; t += 32) {  // column per lane, rows per warp
    const int src = x.jp[t] * x.rall;
    for (int j = warp; j < rho; j += kWarps) G[j * ld + t] = x.wvals[src + j];
  }
  __syncthreads();
  R* cm = x.colmax;  // equilibration: the column's largest |entry|^2 in the block (inf: dropped)
  for (int t = warp; t < rho; t += kWarps) {
    R mx = 0;
    for (int j = lane; j < rho; j += 32) mx = fmax(mx, cabs2(G[j * ld + t]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) cm[t] = (mx > R(0) && mx > thr2 * x.cref[x.jp[t]]) ? mx : R(INFINITY);
  }
  __syncthreads();
  // entry (j, t) carries index 64 j + t (rho <= 64): row-major order for ties, and
  // decoded by shifts
  R v = R(-1);
  int vi = INT_MAX;
  for (int t = lane; t < rho; t += 32)
    for (int j = warp; j < rho; j += kWarps) am_merge(v, vi, cabs2(G[j * ld + t]) / cm[t], (j << 6) | t);
  int buf = 0;
  block_argmax(v, vi, x.redv, x.redi, buf);
  unsigned long long free_r = ~0ull, free_c = ~0ull;  // rho <= 64
  int k = 0;
  long long fl = 0;
  // v, vi and the masks are block-uniform: every thread runs the same steps
  while (k < rho && v > thr2) {
    const int p = vi >> 6, c = vi & 63;
    if (tid == 0) {
      x.selr[k] = p;
      x.selc[k] = c;
    }
    free_r &= ~(1ull << p);
    free_c &= ~(1ull << c);
    ++k;
    fl += (long long)(rho - k) * (rho - k);
    // eliminate with the pivot (row p and column c are only read in this step)
    const cpx<R> ip = crecip(G[p * ld + c]);
    v = R(-1);
    vi = INT_MAX;
    for (int j = lane; j < rho; j += 32) {  // column per lane, rows per warp
      if (!(free_c >> j & 1ull)) continue;
      const cpx<R> pj = G[p * ld + j];
      for (int r = warp; r < rho; r += kWarps) {
        if (free_r >> r & 1ull) {
          cpx<R> a = G[r * ld + j];
          cfms(a, cmul(G[r * ld + c], ip), pj);
          G[r * ld + j] = a;
          am_merge(v, vi, cabs2(a) / cm[j], (r << 6) | j);
        }
      }
    }
    buf ^= 1;
    block_argmax(v, vi, x.redv, x.redi, buf);  // its barrier also publishes the updates
  }
  for (int idx = tid; idx < k * k; idx += kThreads) {
    const int s = idx / k, t = idx % k;
    x.P[s * x.rall + t] = x.wvals[x.jp[x.selc[t]] * x.rall + x.selr[s]];
  }
  for (int s = tid; s < k; s += kThreads) {
    x.wnew[s] = x.wrow[x.selr[s]];
    x.scand[s] = x.jp[x.selc[s]];
  }
  __syncthreads();
  for (int s = tid; s < k; s += kThreads) {
    x.wrow[s] = x.wnew[s];
    x.jp[s] = x.scand[s];
  }
  if (tid == 0) x.flops += 8.0 * (double)fl + 4.0 * (double)tot;
  __syncthreads();
  return k;
}

// ---------------------------------------------------------------------------
// cyclic block maxvol on the kept columns (rows W start from the tournament)
// P holds A[W, Jp]; M = P^{-1} is kept current by rank-one (Sherman-Morrison)
// updates at each swap and recomputed after kRefreshSwaps of them.
// The first cycle also accumulates the row sums S[o, t] = sum_i A[(o,i), Jp[t]].
// Every successful recomputation saves (W, P).  If a recomputation finds P
// singular in working precision (swaps chosen from a drifted FP32 inverse),
// W and P return to the saved pair and the core's maxvol ends there: no more
// swaps, only the row sums of the blocks the first cycle has not reached.
// ---------------------------------------------------------------------------
constexpr int kRefreshSwaps = 16;

// ---------------------------------------------------------------------------
// Skipping provably swap-free revisits (bound_prepare / bound_apply at each
// swap, bound_store after each visit).  After a visit of block q, cb[q][t]
// holds the largest |B_rt| of the block's non-pivot rows.  A swap of row i into
// slot j updates every row by B'_r = B_r - B_rj (B_i - e_j) / B_ij, so
// |B'_rt| <= |B_rt| + |B_rj| v_t with v_t = |B_it - [t = j]| / |B_ij|, and the
// bounds of the other blocks follow as cb[q][t] += cb[q][j] v_t; the pivot row
// the swap releases (B = e_j before) gets at most [t = j] + v_t.  A revisit of a
// block whose bounds are all within 1 + tau finds no entry to swap, so it is
// skipped: the rows and the prices are those of the full revisit.
// ---------------------------------------------------------------------------
// block-uniform: true when block beta's bounds allow no swap
__device__ __forceinline__ bool bound_allows_skip(const float* cb, int beta, int rho, float lim) {
  bool over = false;
  for (int t = threadIdx.x; t < rho; t += kThreads) over |= !(cb[beta * rho + t] <= lim);
  return !__syncthreads_or(over);
}

// after a visit: block beta's column maxima over its non-pivot rows (B column-major,
// leading dimension b); rounding slack keeps the bound above the stored values
template <typename R>
__device__ void bound_store(float* cb, int beta, const cpx<R>* B, int b, int bs, int rho,
                            const unsigned char* inw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < rho; t += kWarps) {
    R mx = R(0);
    for (int r = lane; r < bs; r += 32)
      if (!inw[r]) mx = fmax(mx, cabs2(B[t * b + r]));
    if constexpr (sizeof(R) == 4) {
      // non-negative floats order like their bits (a NaN above all: no skip then)
      mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
    } else {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) cb[beta * rho + t] = (mx == mx) ? sqrtf((float)mx) * 1.0001f : INFINITY;
  }
}

// A swap of row i into slot j of block beta, in two phases around the swap's
// barrier.  Before it: v_t from B's row i (still unchanged) and a snapshot of
// every block's column-j bound, after the bounds (kept in the bound buffer past
// the nb x rho bounds).  After it: every bound of every other block, one FMA
// each; the block of the pivot row the swap releases (`oldb`) also takes
// [t = j] + v_t.
template <typename R>
__device__ void bound_prepare(float* cb, int nb, int rho, int j, const cpx<R>* B, int b, int i) {
  float* cj = cb + nb * rho;
  float* v = cj + nb;
  const float piv = sqrtf((float)cabs2(B[j * b + i]));
  for (int t = threadIdx.x; t < rho; t += kThreads) {
    cpx<R> e = B[t * b + i];
    if (t == j) e.re -= R(1);
    v[t] = sqrtf((float)cabs2(e)) / piv;
  }
  for (int q = threadIdx.x; q < nb; q += kThreads) cj[q] = cb[q * rho + j];
}

__device__ __forceinline__ void bound_apply(float* cb, int nb, int rho, int beta, int j, int oldb) {
  const float* cj = cb + nb * rho;
  const float* v = cj + nb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = lane; t < rho; t += 32) {  // column per lane, blocks per warp: no integer division
    const float vt = v[t];
    for (int q = warp; q < nb; q += kWarps) {
      if (q == beta) continue;
      const int idx = q * rho + t;
      float nv = fmaf(cj[q], vt, cb[idx]);
      if (q == oldb) nv = fmaxf(nv, (t == j ? 1.0f : 0.0f) + vt);
      cb[idx] = nv == nv ? nv : INFINITY;
    }
  }
}

// The rank-one update of a maxvol swap on a block of B (bs rows, column-major,
// leading dimension b): B_rt -= B_rj (B_it - [t = j]) / B_ij, with the argmax of
// |B_rt|^2 over the non-pivot rows.  With bs <= 128 two threads share a row (tid
// & 127), each every other column, so no index needs an integer division; the
// arithmetic per entry is the same either way.
template <typename R>
__device__ __forceinline__ void swap_update(cpx<R>* B, int b, int bs, int rho, int j, cpx<R> ipiv,
                                            const cpx<R>* swrow, const cpx<R>* swcol, const unsigned char* inw,
                                            R& bv, int& bi) {
  const int tid = threadIdx.x;
  if (bs <= kThreads / 2) {
    const int r = tid & (kThreads / 2 - 1);
    if (r < bs) {
      const cpx<R> sc = swcol[r];
      const bool cand = !inw[r];
      for (int t = tid / (kThreads / 2); t < rho; t += 2) {
        cpx<R> rv = swrow[t];
        if (t == j) rv.re -= R(1);
        cpx<R> bb = B[t * b + r];
        cfms(bb, sc, cmul(rv, ipiv));
        B[t * b + r] = bb;
        if (cand) am_merge(bv, bi, cabs2(bb), (r << 6) | t);
      }
    }
  } else {
    for (int idx = tid; idx < bs * rho; idx += kThreads) {
      const int r = idx % bs, t = idx / bs;
      cpx<R> rv = swrow[t];
      if (t == j) rv.re -= R(1);
      cpx<R> bb = B[t * b + r];
      cfms(bb, swcol[r], cmul(rv, ipiv));
      B[t * b + r] = bb;
      if (!inw[r]) am_merge(bv, bi, cabs2(bb), (r << 6) | t);
    }
  }
}

template <typename R>
__device__ void maxvol_refine(Ctx<R>& x, int m, int no, int rho, int b, R thr) {
  const int tid = threadIdx.x, N = x.n;
  const int nb = (m + b - 1) / b;
  for (int idx = tid; idx < no * rho; idx += kThreads) {
    const int o = idx / rho, t = idx % rho;
    x.sacc[o * x.rall + t] = make_double2(0.0, 0.0);
  }
  int quiet = 0, visits = 0, beta = 0, since_inv = kRefreshSwaps;
  int buf = 0;
  long long nswaps = 0;
  const int nct = (rho + 3) / 4;
  const int rtiles = kThreads / nct;  // row tiles per round: thread (rt, ct) owns rows rt + a*rtiles
  const int rpr = 4 * rtiles;
  int ncs = 0;  // pair columns to stage: up to the largest kept column (Jp is in pivot order)
  for (int t = 0; t < rho; ++t) ncs = max(ncs, x.jp[t] + 1);
  cpx<R>* Psave = x.P + x.rall * x.rall;
  bool saved = false, frozen = false;
  // revisit bounds (see bound_prepare); blocks not yet visited have none
  const bool cbon = nb * (rho + 1) + rho <= kBoundCap;  // bounds, column-j snapshot, v
  const float blim = sqrtf((float)thr);
  if (cbon)
    for (int idx = tid; idx < nb * rho; idx += kThreads) x.cb[idx] = INFINITY;
  int skipped = 0;
  while (quiet < nb && visits < 4 * nb) {
    if (since_inv >= kRefreshSwaps && !frozen) {
      TTP_TIC(t_inv);
      if (invert_pivots<R, false>(x, rho)) {
        for (int idx = tid; idx < rho * rho; idx += kThreads) {
          const int j = idx / rho, t = idx % rho;
          Psave[j * x.rall + t] = x.P[j * x.rall + t];
        }
        for (int t = tid; t < rho; t += kThreads) x.wnew[t] = x.wrow[t];
        saved = true;
      } else if (saved) {
        for (int idx = tid; idx < rho * rho; idx += kThreads) {
          const int j = idx / rho, t = idx % rho;
          x.P[j * x.rall + t] = Psave[j * x.rall + t];
        }
        for (int t = tid; t < rho; t += kThreads) x.wrow[t] = x.wnew[t];
        __syncthreads();
        invert_pivots<R, false>(x, rho);  // the saved P inverted before
        frozen = true;
        if (tid == 0) x.rollbacks += 1;
      } else {
        if (tid == 0) {
          x.misc[MISC_FAIL] = 1;
          x.fail_step = 2;
        }
        break;
      }
      since_inv = 0;
      __syncthreads();
      TTP_TOC(t_inv, 5);
    }
    if (frozen && visits >= nb) break;
    if (cbon && !frozen && visits >= nb && bound_allows_skip(x.cb, beta, rho, blim)) {
      ++quiet;  // a swap-free revisit, known without the block product
      ++visits;
      ++skipped;
      beta = (beta + 1) % nb;
      continue;
    }
    TTP_TIC(t_rev);
    const int rs = beta * b;
    const int bs = min(b, m - rs);
    cpx<R>* A = x.sw;  // bs x rho, column-major, leading dimension b
    stage_pairs(x, rs / N, (rs + bs - 1) / N, ncs);
    // rows of this block that are pivots already: their B rows are unit vectors,
    // never maxvol candidates (excluding them only guards against FP32 drift)
    unsigned char* inw = reinterpret_cast<unsigned char*>(x.scand);
    for (int r = tid; r < bs; r += kThreads) inw[r] = 0;
    // two threads per row (128 rows per pass), each the row's every other kept
    // column, four independent points at a time (loads before stores)
    for (int rr = tid & 127; rr < bs; rr += 128) {
      const int g = rs + rr;
      const RowTab<R> rt = row_tab(x, g % N);
      const int o = g / N;
      int t = tid >> 7;
      for (; t + 6 < rho; t += 8) {
        const cpx<R> v0 = eval_row_point(x, rt, o, x.jp[t]);
        const cpx<R> v1 = eval_row_point(x, rt, o, x.jp[t + 2]);
        const cpx<R> v2 = eval_row_point(x, rt, o, x.jp[t + 4]);
        const cpx<R> v3 = eval_row_point(x, rt, o, x.jp[t + 6]);
        A[t * b + rr] = v0;
        A[(t + 2) * b + rr] = v1;
        A[(t + 4) * b + rr] = v2;
        A[(t + 6) * b + rr] = v3;
      }
      for (; t < rho; t += 2) A[t * b + rr] = eval_row_point(x, rt, o, x.jp[t]);
    }
    if (tid == 0) x.flops += 24.0 * bs * rho + (frozen ? 0.0 : 8.0 * (double)bs * rho * rho);
    __syncthreads();
    TTP_TOC(t_rev, 6);
    TTP_TIC(t_gemm);
    for (int t = tid; t < rho; t += kThreads) {
      const int g = x.wrow[t] - rs;
      if (g >= 0 && g < bs) inw[g] = 1;
    }
    if (visits < nb) {  // first cycle: row sums over i per outer index
      // one warp per (outer index, kept column); lanes take consecutive rows
      // (conflict-free), compensated (Kahan) partial sums, then a fixed-order
      // warp reduction, added to the FP64 accumulator
      const int lane = tid & 31, warp = tid >> 5;
      const int olo = rs / N, ohi = (rs + bs - 1) / N;
      const int nol = ohi - olo + 1;
      for (int pr = warp; pr < nol * rho; pr += kWarps) {
        const int ol = pr % nol, t = pr / nol;
        const int o = olo + ol;
        const int r0 = max(o * N, rs) - rs, r1 = min(o * N + N, rs + bs) - rs;
        R sr = 0, si = 0, cr = 0, ci = 0;
        for (int r = r0 + lane; r < r1; r += 32) {
          const cpx<R> a = A[t * b + r];
          R y = a.re - cr; R s2 = sr + y; cr = (s2 - sr) - y; sr = s2;
          y = a.im - ci; s2 = si + y; ci = (s2 - si) - y; si = s2;
        }
        R vr = sr - cr, vi = si - ci;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          vr += __shfl_xor_sync(0xffffffffu, vr, off);
          vi += __shfl_xor_sync(0xffffffffu, vi, off);
        }
        if (lane == 0) {  // one add per accumulator and visit: the visits' barriers fix the order
          double2* acc = &x.sacc[o * x.rall + t];
          atomicAdd(&acc->x, (double)vr);
          atomicAdd(&acc->y, (double)vi);
        }
      }
    }
    // B = A M in row strips; each strip is read completely before it is overwritten
    TTP_TIC(t_prod);
    R bv = R(-1);
    int bi = INT_MAX;
    for (int r0 = 0; r0 < (frozen ? 0 : bs); r0 += rpr) {
      const int rt = tid % rtiles, ct = tid / rtiles;
      const int col0 = 4 * ct;
      const bool act = ct < nct && r0 + rt < bs;
      cpx<R> acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = cpx<R>{R(0), R(0)};
      if (act) {
        for (int t = 0; t < rho; ++t) {
          cpx<R> av[4], mv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int r = r0 + rt + a * rtiles;
            av[a] = r < bs ? A[t * b + r] : cpx<R>{R(0), R(0)};
          }
#pragma unroll
          for (int c = 0; c < 4; ++c)
            mv[c] = (col0 + c < rho) ? x.M[t * x.rall + col0 + c] : cpx<R>{R(0), R(0)};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) cfma(acc[a][c], av[a], mv[c]);
        }
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int r = r0 + rt + a * rtiles, cc = col0 + c;
            if (r < bs && cc < rho) {
              A[cc * b + r] = acc[a][c];
              if (!inw[r]) am_merge(bv, bi, cabs2(acc[a][c]), (r << 6) | cc);
            }
          }
      }
    }
    TTP_COUNT(21, clock64() - t_prod);  // the block product and its stores (cycles)
    if (!frozen) {  // block-uniform
      buf ^= 1;
      block_argmax(bv, bi, x.redv, x.redi, buf);
    }
    TTP_TOC(t_gemm, 8);
    TTP_TIC(t_sw);
    bool swapped = false;
    for (int it = 0; it < rho; ++it) {
      if (!(bv > thr)) break;
      const int i = bi >> 6, j = bi & 63;  // entry (r, t) carries 64 r + t (rho <= 64)
      for (int r = tid; r < bs; r += kThreads) x.swcol[r] = A[j * b + r];
      for (int t = tid; t < rho; t += kThreads) {
        x.swrow[t] = A[t * b + i];
        x.mcol[t] = x.M[t * x.rall + j];
      }
      if (tid == 0) {
        const int old = x.wrow[j] - rs;
        x.misc[MISC_OLDW] = x.wrow[j];
        if (old >= 0 && old < bs) inw[old] = 0;
        inw[i] = 1;
        x.wrow[j] = rs + i;
      }
      if (cbon) bound_prepare(x.cb, nb, rho, j, A, b, i);
      __syncthreads();
      eval_prow(x, j, rs + i, rho);
      if (cbon) bound_apply(x.cb, nb, rho, beta, j, x.misc[MISC_OLDW] / b);
      const cpx<R> ipiv = crecip(x.swrow[j]);
      bv = R(-1);
      bi = INT_MAX;
      swap_update(A, b, bs, rho, j, ipiv, x.swrow, x.swcol, inw, bv, bi);
      // P^{-1} update, column t per lane, rows per warp (no integer division)
      {
        const int lane = tid & 31, warp = tid >> 5;
        for (int t = lane; t < rho; t += 32) {
          cpx<R> rv = x.swrow[t];
          if (t == j) rv.re -= R(1);
          const cpx<R> f = cmul(rv, ipiv);
          for (int r = warp; r < rho; r += kWarps) cfms(x.M[r * x.rall + t], x.mcol[r], f);
        }
      }
      if (tid == 0) x.flops += 8.0 * (bs + rho) * rho + 24.0 * rho;
      buf ^= 1;
      block_argmax(bv, bi, x.redv, x.redi, buf);
      swapped = true;
      ++since_inv;
      ++nswaps;
      TTP_COUNT(20, 1);
    }
    TTP_COUNT(19, clock64() - t_sw);  // the visit's swaps (cycles)
    if (cbon && !frozen) bound_store(x.cb, beta, A, b, bs, rho, inw);
    quiet = swapped ? 0 : quiet + 1;
    ++visits;
    beta = (beta + 1) % nb;
    __syncthreads();
    TTP_TOC(t_sw, 9);
  }
  if (tid == 0) {
    x.swaps += nswaps;
    x.visits += visits - skipped;  // block products made
  }
}

// ---------------------------------------------------------------------------
// FP32 maxvol with the block product on the tensor cores.  Same visits, swaps,
// rollback and row sums as maxvol_refine.  Per visit the block's fiber rows at
// the kept columns are evaluated in chunks of kTcChunk columns into four K-major
// planes (hi and lo TF32 parts of Re A and Im A, 128 rows zero-padded; with
// chunks of 8, two buffers let one chunk's products run while the next is
// evaluated) and multiplied into TMEM with 3xTF32 products
//   A P^{-1} ~ A_hi M_hi + A_hi M_lo + A_lo M_hi,
// as two real products of N = 2 kp, D = Re A [Re M | Im M] and
// E = Im A [Re M | Im M]; the read-back combines them, B = (D_re - E_im) +
// i (D_im + E_re), and stores complex B[t*b + r] for the swaps.
// P^{-1} is kept as its own hi and lo planes (M_hi in M, M_lo in the winner-
// value buffer, free during maxvol); their sum is the FP32 inverse.  One TF32
// product (2^-11) is not enough: B = A P^{-1} cancels by up to the condition
// number of P (up to 1/theta), and 3xTF32 brings the rounding to ~2^-21, about
// an FP32 product's, so the swapped-in row of B updates P^{-1} directly.
// ---------------------------------------------------------------------------
template <typename R>
__device__ void maxvol_refine_tc(Ctx<R>& x, int m, int no, int rho, int b, R thr) {
  static_assert(sizeof(R) == 4, "the tensor-core maxvol is the FP32 path");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = x.n;
  const int nb = (m + b - 1) / b;
  const int kp = tc::pad16(rho);
  // A chunk planes: 128 rows x kTcChunk columns, 32 kTcChunk bytes per 8-row group;
  // a buffer holds four (hi and lo of Re A and Im A); kTcBufs buffers
  constexpr int kSboA = kTcChunk * 32, kPlaneA = (tc::kRows / 8) * kSboA, kBufA = 4 * kPlaneA;
  unsigned char* a_pl = reinterpret_cast<unsigned char*>(x.sw);
  const int sbo_m = kp * 32;
  // P^{-1} operands (hi in M, lo in wvals): the re plane, then the im plane
  const unsigned char* m_hi = reinterpret_cast<const unsigned char*>(x.M);
  const unsigned char* m_lo = reinterpret_cast<const unsigned char*>(x.wvals);
  cpx<R>* B = x.sw;  // after the product: bs x rho, column-major, leading dimension b
  for (int idx = tid; idx < no * rho; idx += kThreads) {
    const int o = idx / rho, t = idx % rho;
    x.sacc[o * x.rall + t] = make_double2(0.0, 0.0);
  }
  if (x.tc_pending) {  // an earlier product never completed: no more tensor-core work in this CTA
    if (tid == 0) {
      x.misc[MISC_FAIL] = 1;
      x.fail_step = 6;
    }
    __syncthreads();
    return;
  }
  uint32_t phase[2] = {x.mma_phase & 1u, (x.mma_phase >> 1) & 1u};  // per buffer barrier; block-uniform
  int quiet = 0, visits = 0, beta = 0, since_inv = kRefreshSwaps;
  int buf = 0;
  long long nswaps = 0;
  int ncs = 0;  // pair columns to stage: up to the largest kept column (Jp is in pivot order)
  for (int t = 0; t < rho; ++t) ncs = max(ncs, x.jp[t] + 1);
  cpx<R>* Psave = x.P + x.rall * x.rall;
  bool saved = false, frozen = false;
  // revisit bounds (see bound_prepare); blocks not yet visited have none
  const bool cbon = nb * (rho + 1) + rho <= kBoundCap;  // bounds, column-j snapshot, v
  const float blim = sqrtf((float)thr);
  if (cbon)
    for (int idx = tid; idx < nb * rho; idx += kThreads) x.cb[idx] = INFINITY;
  int skipped = 0;
  while (quiet < nb && visits < 4 * nb) {
    if (since_inv >= kRefreshSwaps && !frozen) {
      TTP_TIC(t_inv);
      if (invert_pivots<R, true>(x, rho)) {
        for (int idx = tid; idx < rho * rho; idx += kThreads) {
          const int j = idx / rho, t = idx % rho;
          Psave[j * x.rall + t] = x.P[j * x.rall + t];
        }
        for (int t = tid; t < rho; t += kThreads) x.wnew[t] = x.wrow[t];
        saved = true;
      } else if (saved) {
        for (int idx = tid; idx < rho * rho; idx += kThreads) {
          const int j = idx / rho, t = idx % rho;
          x.P[j * x.rall + t] = Psave[j * x.rall + t];
        }
        for (int t = tid; t < rho; t += kThreads) x.wrow[t] = x.wnew[t];
        __syncthreads();
        invert_pivots<R, true>(x, rho);  // the saved P inverted before
        frozen = true;
        if (tid == 0) x.rollbacks += 1;
      } else {
        if (tid == 0) {
          x.misc[MISC_FAIL] = 1;
          x.fail_step = 2;
        }
        break;
      }
      since_inv = 0;
      __syncthreads();
      TTP_TOC(t_inv, 5);
    }
    if (frozen && visits >= nb) break;
    if (cbon && !frozen && visits >= nb && bound_allows_skip(x.cb, beta, rho, blim)) {
      ++quiet;  // a swap-free revisit, known without the block product
      ++visits;
      ++skipped;
      beta = (beta + 1) % nb;
      continue;
    }
    TTP_TIC(t_rev);
    const int rs = beta * b;
    const int bs = min(b, m - rs);
    stage_pairs(x, rs / N, (rs + bs - 1) / N, ncs);
    // rows of this block that are pivots already: their B rows are unit vectors,
    // never maxvol candidates (excluding them guards against rounding)
    unsigned char* inw = reinterpret_cast<unsigned char*>(x.scand);
    for (int r = tid; r < bs; r += kThreads) inw[r] = 0;
    __syncthreads();
    for (int t = tid; t < rho; t += kThreads) {
      const int g = x.wrow[t] - rs;
      if (g >= 0 && g < bs) inw[g] = 1;
    }
    bool failed = false;
    // chunk c of 8 kept columns goes to buffer c & 1; its 12 MMAs run while chunk
    // c + 1 is evaluated into the other buffer.  Buffer k's products complete on
    // barrier k, so each barrier has at most one phase outstanding.
    const int nch = kp / kTcChunk;
    for (int c = 0; c < nch && !failed; ++c) {
      // chunk c uses buffer c % kTcBufs and completes on barrier c & 1
      const int bufk = c & 1, c0 = c * kTcChunk;
      unsigned char* const pb = a_pl + (c % kTcBufs) * kBufA;
      bool ok = true;
      if (!frozen && c >= kTcBufs) {  // the products that last read this buffer (checked at the next barrier)
        const int pk = (c - kTcBufs) & 1;
        ok = tc::mbar_wait(x.mbar + pk, phase[pk], tc::kLoopWaitLimit);
        if (ok) phase[pk] ^= 1u;  // a phase that timed out stays the outstanding one
      }
      // evaluation: lane -> rows 8g + lane/4 (two row groups per warp), columns
      // lane%4 + 4jj; a warp's store is 8 rows x 4 columns = 128 bytes
      TTP_TIC(t_ev8);
#pragma unroll
      for (int gg = 0; gg < 2; ++gg) {
        const int r = 8 * (2 * warp + gg) + (lane >> 2);
        const bool live = r < bs;
        const int g = rs + (live ? r : 0);
        const RowTab<R> rt = row_tab(x, g % N);
        // the row's points first, then the stores (loads before stores: independent)
        cpx<R> v[kTcChunk / 4];
#pragma unroll
        for (int jj = 0; jj < kTcChunk / 4; ++jj) {
          const int t = c0 + (lane & 3) + 4 * jj;
          v[jj] = (live && t < rho) ? eval_row_point(x, rt, g / N, x.jp[t]) : cpx<R>{R(0), R(0)};
        }
#pragma unroll
        for (int jj = 0; jj < kTcChunk / 4; ++jj) {
          const int tl = (lane & 3) + 4 * jj;
          const int off = tc::kmaj(r, tl, kSboA);
          const R hr = tf32_hi(v[jj].re), hm = tf32_hi(v[jj].im);
          *reinterpret_cast<R*>(pb + off) = hr;
          *reinterpret_cast<R*>(pb + kPlaneA + off) = hm;
          *reinterpret_cast<R*>(pb + 2 * kPlaneA + off) = v[jj].re - hr;
          *reinterpret_cast<R*>(pb + 3 * kPlaneA + off) = v[jj].im - hm;
        }
      }
      TTP_TOC(t_ev8, 14);
      tc::fence_async_smem();  // the planes (and P^{-1} after swaps) were written by the generic proxy
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      // two issuing threads in different warps, one per accumulator chain (the MMA
      // queue is short, so one thread issuing all six would stall its warp)
      if (!frozen && (tid & 127) == 0) {
        TTP_TIC(t_mma);
        tc::fence_after_sync();
        // D = Re A [M_re | M_im] and E = Im A [M_re | M_im] (N = 2 kp: the re and im
        // planes of P^{-1} are adjacent), each as hi*hi + hi*lo + lo*hi; a plane
        // further on is (byte offset >> 4) further in the start-address field
        const uint64_t a0 = tc::smem_desc(tc::smem_u32(pb), (uint32_t)kSboA), ap = kPlaneA >> 4;
        const uint32_t id = tc::instr_desc(2 * kp, false);
        // thread 0: D = Re A [M] into columns [0, 2kp); thread 128: E = Im A [M] into [2kp, 4kp)
        const int part = tid >> 7;
        const uint32_t dst = x.tmem + (uint32_t)(part * 2 * kp);
        for (int ks = 0; ks < kTcChunk / 8; ++ks) {  // K = 8 per instruction: 256 bytes along K
          const uint32_t km = (uint32_t)(c0 / 4 + 2 * ks) * 128u;
          const uint64_t mh = tc::smem_desc(tc::smem_u32(m_hi) + km, (uint32_t)sbo_m);
          const uint64_t ml = tc::smem_desc(tc::smem_u32(m_lo) + km, (uint32_t)sbo_m);
          const uint64_t ko = (uint64_t)ks * (256 >> 4);
          const uint64_t ahi = a0 + (uint64_t)part * ap + ko, alo = a0 + (uint64_t)(2 + part) * ap + ko;
          const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
          tc::mma_tf32(dst, ahi, mh, id, acc);  // A hi * M hi
          tc::mma_tf32(dst, ahi, ml, id, 1u);   // A hi * M lo
          tc::mma_tf32(dst, alo, mh, id, 1u);   // A lo * M hi
        }
        tc::commit(x.mbar + bufk);            // the barrier expects both issuing threads
        TTP_TOC(t_mma, 11);
      }
      TTP_TIC(t_rsum);
      if (visits < nb) {  // first cycle: row sums of this chunk's columns (the MMAs only read)
        // one warp per (outer index, kept column); lanes take rows, compensated
        // (Kahan) partial sums, a fixed-order warp reduction, FP64 accumulator
        const int olo = rs / N, ohi = (rs + bs - 1) / N;
        const int nol = ohi - olo + 1, ncol = min(kTcChunk, rho - c0);
        for (int pr = warp; pr < nol * ncol; pr += kWarps) {
          const int ol = pr % nol, tl = pr / nol;
          const int o = olo + ol;
          const int r0 = max(o * N, rs) - rs, r1 = min(o * N + N, rs + bs) - rs;
          R sr = 0, si = 0, cr = 0, ci = 0;
          for (int r = r0 + lane; r < r1; r += 32) {
            const int off = tc::kmaj(r, tl, kSboA);
            const R are = *reinterpret_cast<const R*>(pb + off) + *reinterpret_cast<const R*>(pb + 2 * kPlaneA + off);
            const R aim = *reinterpret_cast<const R*>(pb + kPlaneA + off) +
                          *reinterpret_cast<const R*>(pb + 3 * kPlaneA + off);
            R y = are - cr; R s2 = sr + y; cr = (s2 - sr) - y; sr = s2;
            y = aim - ci; s2 = si + y; ci = (s2 - si) - y; si = s2;
          }
          R vr = sr - cr, vi = si - ci;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, off);
            vi += __shfl_xor_sync(0xffffffffu, vi, off);
          }
          if (lane == 0) {  // one add per accumulator and chunk: the barriers fix the order
            double2* acc = &x.sacc[o * x.rall + c0 + tl];
            atomicAdd(&acc->x, (double)vr);
            atomicAdd(&acc->y, (double)vi);
          }
        }
      }
      TTP_TOC(t_rsum, 15);
      // the next chunk overwrites what the row sums read (with one buffer, or no products)
      if (frozen || kTcBufs == 1) __syncthreads();
    }
    // the products of the last two chunks
    if (!frozen && !failed) {
      bool ok = true;
      for (int c = max(0, nch - kTcBufs); c < nch; ++c) {
        const int bufk = c & 1;
        const bool done = tc::mbar_wait(x.mbar + bufk, phase[bufk], tc::kLoopWaitLimit);
        if (done) phase[bufk] ^= 1u;
        ok = ok && done;
      }
      failed = __syncthreads_or(!ok);
    }
    if (failed) {
      if (tid == 0) {
        x.misc[MISC_FAIL] = 1;
        x.fail_step = 6;
        x.tc_pending = 1;
        x.mma_phase = phase[0] | (phase[1] << 1);  // the phases still outstanding
      }
      __syncthreads();
      break;
    }
    // algorithmic work: 24 per evaluation, 8 per complex multiply-add of the block
    // product (the 3xTF32 split triples the tensor-core work, not the algorithm's)
    if (tid == 0) x.flops += 24.0 * bs * rho + (frozen ? 0.0 : 8.0 * (double)bs * rho * rho);
    TTP_TOC(t_rev, 6);
    TTP_TIC(t_gemm);
    R bv = R(-1);
    int bi = INT_MAX;
    if (!frozen) {
      tc::fence_after_sync();
      // warp quarter q reads TMEM lanes (block rows) 32q..32q+31; warp half h the
      // columns [h kp/2, (h+1) kp/2) of both accumulators
      const int q = warp & 3, h = warp >> 2, row = 32 * q + lane;
      for (int cc = h * (kp / 2); cc < (h + 1) * (kp / 2); cc += 8) {
        float dr[8], di[8], er[8], ei[8];
        const uint32_t ta = x.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cc;
        tc::tmem_ld8(ta, dr);
        tc::tmem_ld8(ta + (uint32_t)kp, di);
        tc::tmem_ld8(ta + (uint32_t)(2 * kp), er);
        tc::tmem_ld8(ta + (uint32_t)(3 * kp), ei);
        tc::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int s = cc + c;
          if (row < bs && s < rho) {
            const cpx<R> v = {dr[c] - ei[c], di[c] + er[c]};  // Re A M + i Im A M
            B[s * b + row] = v;
            if (!inw[row]) am_merge(bv, bi, cabs2(v), (row << 6) | s);
          }
        }
      }
      tc::fence_before_sync();
      buf ^= 1;
      block_argmax(bv, bi, x.redv, x.redi, buf);  // its barrier also publishes B
    }
    TTP_TOC(t_gemm, 8);
    TTP_TIC(t_sw);
    bool swapped = false;
    for (int it = 0; it < rho; ++it) {
      if (!(bv > thr)) break;
      const int i = bi >> 6, j = bi & 63;  // entry (r, t) carries 64 r + t (rho <= 64)
      for (int r = tid; r < bs; r += kThreads) x.swcol[r] = B[j * b + r];
      for (int t = tid; t < rho; t += kThreads) {
        x.swrow[t] = B[t * b + i];
        x.mcol[t] = minv_get(x, kp, t, j);
      }
      if (tid == 0) {
        const int old = x.wrow[j] - rs;
        x.misc[MISC_OLDW] = x.wrow[j];
        if (old >= 0 && old < bs) inw[old] = 0;
        inw[i] = 1;
        x.wrow[j] = rs + i;
      }
      if (cbon) bound_prepare(x.cb, nb, rho, j, B, b, i);
      __syncthreads();
      eval_prow(x, j, rs + i, rho);  // P[j][t] = A(i, t), FP32
      if (cbon) bound_apply(x.cb, nb, rho, beta, j, x.misc[MISC_OLDW] / b);
      const cpx<R> ipiv = crecip(x.swrow[j]);
      bv = R(-1);
      bi = INT_MAX;
      swap_update(B, b, bs, rho, j, ipiv, x.swrow, x.swcol, inw, bv, bi);
      // P^{-1} update, column t per lane, rows per warp (no integer division)
      for (int t = lane; t < rho; t += 32) {
        cpx<R> rv = x.swrow[t];
        if (t == j) rv.re -= R(1);
        const cpx<R> f = cmul(rv, ipiv);
        for (int r = warp; r < rho; r += kWarps) {
          cpx<R> mv = minv_get(x, kp, r, t);
          cfms(mv, x.mcol[r], f);
          minv_set(x, kp, r, t, mv);
        }
      }
      if (tid == 0) x.flops += 8.0 * (bs + 2 * rho) * rho + 24.0 * rho;
      buf ^= 1;
      block_argmax(bv, bi, x.redv, x.redi, buf);
      swapped = true;
      ++since_inv;
      ++nswaps;
    }
    if (cbon && !frozen) bound_store(x.cb, beta, B, b, bs, rho, inw);
    quiet = swapped ? 0 : quiet + 1;
    ++visits;
    beta = (beta + 1) % nb;
    __syncthreads();
    TTP_TOC(t_sw, 9);
  }
  if (tid == 0) {
    x.swaps += nswaps;
    x.visits += visits - skipped;  // block products made
    if (!x.tc_pending) x.mma_phase = phase[0] | (phase[1] << 1);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// contraction step: v <- (v S) P^{-1}, FP64 (Gaussian elimination on P^T)
// ---------------------------------------------------------------------------
// block argmax of an FP64 magnitude (larger wins, then lower index); 2 kWarps
// doubles and ints of scratch per buffer pair
__device__ __forceinline__ void block_argmax_f64(double& v, int& i, double* rv, int* ri, int buf) {
  warp_argmax(v, i);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    rv[buf * kWarps + warp] = v;
    ri[buf * kWarps + warp] = i;
  }
  __syncthreads();
  v = rv[buf * kWarps];
  i = ri[buf * kWarps];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) am_merge(v, i, rv[buf * kWarps + w], ri[buf * kWarps + w]);
}

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// sum over aligned groups of g consecutive lanes (g a power of two <= 32)
template <typename T>
__device__ __forceinline__ T group_sum(T v, int g) {
  for (int off = g >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// P^{-1}[t][s] as maxvol leaves it: R-precision, updated through its swaps
template <typename R, bool TC>
__device__ __forceinline__ cpx<R> minv_at(const Ctx<R>& x, int kp, int t, int s) {
  if constexpr (TC) {
    return minv_get(x, kp, t, s);
  } else {
    return x.M[t * x.rall + s];
  }
}

#ifndef TTP_REFINE_ITERS
#define TTP_REFINE_ITERS 12
#endif
constexpr int kRefineIters = TTP_REFINE_ITERS;  // a build with 0 solves every system by elimination

// y P = w (w = v S, the contraction's row vector) by iterative refinement on
// maxvol's running inverse M ~ P^{-1}: y_0 = 0, r_0 = w; then d = r M in R,
// y += d and r = w - y P in FP64, until |d|max <= tol |y|max.  The residual
// is formed in FP64 from P's exact entries, so the iterates converge to the
// FP64 solution of the same system as long as |I - M P| < 1 (Wilkinson's
// mixed-precision refinement); each step gains about -log10 |I - M P| digits.
// The right-hand side is scaled by a power of two before rounding to R, so an
// FP64 chain vector far outside R's range keeps its relative precision.
// Returns false (nothing written) when the corrections stop shrinking by at
// least half per step before reaching tol, or do not reach it within
// kRefineIters steps: the caller then eliminates instead.  Scratch: r(r+3)
// complex doubles and 3 kWarps doubles in sw.
template <typename R, bool TC>
__device__ bool chain_refine(Ctx<R>& x, int no, int rho) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tpc = rho <= 32 ? 8 : 4;  // threads per output (rho <= 64)
  const int out = tid / tpc, part = tid % tpc;
  // every lane of a warp reaches each shuffle below (the loop counts are
  // block-uniform); lanes without an output carry zeros through the sums
  const bool own = out < rho;
  const int kp = tc::pad16(rho);
  double2* Pd = reinterpret_cast<double2*>(x.sw);  // [rho][rho], P's entries in FP64
  double2* w = Pd + rho * rho;
  double2* y = w + rho;
  double2* r = y + rho;
  double* red = reinterpret_cast<double*>(r + rho);  // 3 kWarps: |d|, |y|, then |w| apart
  // stop at |d|max <= 1e-9 |y|max with an R = FP32 inverse (two orders below the
  // FP32 rounding of the fiber entries P and w come from), 1e-12 with an FP64 one
  const double tol2 = sizeof(R) == 4 ? 1e-18 : 1e-24;
  // w = v S over the outer indices, FP64
  double2 s = make_double2(0.0, 0.0);
  if (own) {
    for (int o = part; o < no; o += tpc) {
      const double2 v = x.vchain[o], a = x.sacc[o * x.rall + out];
      s.x += v.x * a.x - v.y * a.y;
      s.y += v.x * a.y + v.y * a.x;
    }
  }
  s.x = group_sum(s.x, tpc);
  s.y = group_sum(s.y, tpc);
  double wn = 0.0;
  if (own && part == 0) {
    w[out] = s;
    r[out] = s;
    y[out] = make_double2(0.0, 0.0);
    wn = s.x * s.x + s.y * s.y;
  }
  for (int c = lane; c < rho; c += 32)  // column per lane, rows per warp
    for (int r = warp; r < rho; r += kWarps) {
      const cpx<R> p = x.P[r * x.rall + c];
      Pd[r * rho + c] = make_double2((double)p.re, (double)p.im);
    }
  for (int off = 16; off > 0; off >>= 1) wn = fmax(wn, __shfl_xor_sync(0xffffffffu, wn, off));
  if (lane == 0) red[2 * kWarps + warp] = wn;
  __syncthreads();
  wn = red[2 * kWarps];
#pragma unroll
  for (int q = 1; q < kWarps; ++q) wn = fmax(wn, red[2 * kWarps + q]);
  if (!(wn > 0.0) || !(wn < INFINITY)) return false;  // block-uniform
  // r is rounded to R after scaling by 2^-e, |w|max in [2^(e-1), 2^e)
  int e;
  frexp(sqrt(wn), &e);
  const double sc = ldexp(1.0, -e), isc = ldexp(1.0, e);
  double prev = INFINITY;
  bool done = false;
  int it_used = 0;
  for (int it = 0; it < kRefineIters; ++it) {
    it_used = it + 1;
    // d = r M (R precision), output s = out, sum over t
    R dr = R(0), di = R(0);
    if (own) {
      for (int t = part; t < rho; t += tpc) {
        const double2 rt = r[t];
        const R ar = (R)(rt.x * sc), ai = (R)(rt.y * sc);
        const cpx<R> m = minv_at<R, TC>(x, kp, t, out);
        dr += ar * m.re - ai * m.im;
        di += ar * m.im + ai * m.re;
      }
    }
    dr = group_sum(dr, tpc);
    di = group_sum(di, tpc);
    double dn = 0.0, yn = 0.0;
    if (own && part == 0) {
      const double ddr = (double)dr * isc, ddi = (double)di * isc;
      double2 yv = y[out];
      yv.x += ddr;
      yv.y += ddi;
      y[out] = yv;
      dn = ddr * ddr + ddi * ddi;
      yn = yv.x * yv.x + yv.y * yv.y;
    }
    for (int off = 16; off > 0; off >>= 1) {
      dn = fmax(dn, __shfl_xor_sync(0xffffffffu, dn, off));
      yn = fmax(yn, __shfl_xor_sync(0xffffffffu, yn, off));
    }
    if (lane == 0) {
      red[warp] = dn;
      red[kWarps + warp] = yn;
    }
    __syncthreads();  // also publishes y
    dn = red[0];
    yn = red[kWarps];
#pragma unroll
    for (int q = 1; q < kWarps; ++q) {
      dn = fmax(dn, red[q]);
      yn = fmax(yn, red[kWarps + q]);
    }
    if (!(dn < INFINITY) || !(yn < INFINITY)) break;  // block-uniform
    if (dn <= tol2 * yn) {
      done = true;
      break;
    }
    if (!(dn <= 0.25 * prev)) break;
    prev = dn;
    // r = w - y P (FP64), output t = out, sum over j
    double2 q2 = make_double2(0.0, 0.0);
    if (own) {
      for (int j = part; j < rho; j += tpc) {
        const double2 yv = y[j], p = Pd[j * rho + out];
        q2.x += yv.x * p.x - yv.y * p.y;
        q2.y += yv.x * p.y + yv.y * p.x;
      }
    }
    q2.x = group_sum(q2.x, tpc);
    q2.y = group_sum(q2.y, tpc);
    if (own && part == 0) r[out] = make_double2(w[out].x - q2.x, w[out].y - q2.y);
    __syncthreads();
  }
  if (done)
    for (int t = tid; t < rho; t += kThreads) x.vchain[t] = y[t];
  (void)it_used;
  TTP_COUNT(16, 1);
  TTP_COUNT(17, done ? 0 : 1);
  TTP_COUNT(18, it_used);
  __syncthreads();
  return done;
}

// y P = w by Gaussian elimination with partial pivoting on [P^T | w^T], FP64.
// Rows stay in place: the pivot of column c is the unused row with the largest
// |entry|^2 (order[c]); the other unused rows subtract their multiple of it at
// the columns right of c, tpr threads per row (the row's first thread forms the
// multiplier and passes it on by shuffle), and the threads holding column c + 1
// collect its argmax, so an elimination step costs one block barrier.  The pivot
// row's first thread forms 1/pivot meanwhile, and warp 0 back-substitutes by
// shuffles alone.
template <typename R, bool TC>
__device__ void chain_solve(Ctx<R>& x, int no, int rho) {
  __syncthreads();  // maxvol's last reads of sw are done; its failure flag is visible
  if (!x.misc[MISC_FAIL] && chain_refine<R, TC>(x, no, rho)) {
    // the solve's algorithmic count is elimination's, however it is reached
    if (threadIdx.x == 0) x.flops += 8.0 * (double)no * rho + 8.0 * (double)rho * rho * rho / 3.0;
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < rho; t += kThreads) {
    double2 y = make_double2(0.0, 0.0);
    for (int o = 0; o < no; ++o) {
      const double2 v = x.vchain[o], s = x.sacc[o * x.rall + t];
      y.x += v.x * s.x - v.y * s.y;
      y.y += v.x * s.y + v.y * s.x;
    }
    x.ychain[t] = y;
  }
  __syncthreads();
  double2* G = reinterpret_cast<double2*>(x.sw);  // rho x (rho+1), row-major: [P^T | y^T]
  const int lg = rho + 1;
  double* rv = reinterpret_cast<double*>(G + rho * lg);  // 2 kWarps doubles, then 2 kWarps ints
  int* ri = reinterpret_cast<int*>(rv + 2 * kWarps);
  double2* ipiv = reinterpret_cast<double2*>(x.swcol);  // 1/pivot of step c
  int* order = x.selr;
  for (int idx = tid; idx < rho * lg; idx += kThreads) {
    const int r = idx / lg, c = idx % lg;
    if (c < rho) {
      const cpx<R> pv = x.P[c * x.rall + r];
      G[idx] = make_double2((double)pv.re, (double)pv.im);
    } else {
      G[idx] = x.ychain[r];
    }
  }
  __syncthreads();
  const int tpr = rho <= 32 ? 8 : 4;  // threads per row (rho <= 64)
  const int myr = tid / tpr, part = tid % tpr;
  double v = -1.0;
  int vi = INT_MAX;
  if (myr < rho && part == 0) {
    const double2 g = G[myr * lg];
    am_merge(v, vi, g.x * g.x + g.y * g.y, myr);
  }
  int buf = 0;
  block_argmax_f64(v, vi, rv, ri, buf);
  unsigned long long used = 0ull;
  bool ok = true;
  for (int c = 0; c < rho; ++c) {  // v, vi, used: block-uniform
    if (!(v > 0.0) || !(v < INFINITY)) {
      ok = false;
      break;
    }
    const int p = vi;
    if (tid == 0) order[c] = p;
    used |= 1ull << p;
    v = -1.0;
    vi = INT_MAX;
    const bool active = myr < rho && !((used >> myr) & 1ull);  // unused after this step (p excluded)
    double2 f = make_double2(0.0, 0.0);
    if (part == 0 && myr < rho && (active || myr == p)) {
      // one division on the step's critical path: conj(pivot) / |pivot|^2
      const double2 pv = G[p * lg + c];
      const double rd = 1.0 / (pv.x * pv.x + pv.y * pv.y);
      const double2 ip = make_double2(pv.x * rd, -pv.y * rd);
      if (active) {
        f = cmul_d(G[myr * lg + c], ip);
      } else {
        ipiv[c] = ip;
      }
    }
    // the row's first thread hands its multiplier to the row's other threads
    f.x = __shfl_sync(0xffffffffu, f.x, lane & ~(tpr - 1));
    f.y = __shfl_sync(0xffffffffu, f.y, lane & ~(tpr - 1));
    if (active) {
      for (int j = c + 1 + part; j <= rho; j += tpr) {
        double2 a = G[myr * lg + j];
        const double2 g = G[p * lg + j];
        a.x -= f.x * g.x - f.y * g.y;
        a.y -= f.x * g.y + f.y * g.x;
        G[myr * lg + j] = a;
        if (j == c + 1 && j < rho) am_merge(v, vi, a.x * a.x + a.y * a.y, myr);
      }
    }
    buf ^= 1;
    block_argmax_f64(v, vi, rv, ri, buf);  // its barrier also publishes the updates
  }
  if (!ok) {
    if (tid == 0) {
      x.misc[MISC_FAIL] = 1;
      x.fail_step = 3;
    }
  } else if (warp == 0) {
    // back substitution, lane l holding the right-hand side of step l (and l + 32)
    double2 r0 = lane < rho ? G[order[lane] * lg + rho] : make_double2(0.0, 0.0);
    double2 r1 = lane + 32 < rho ? G[order[lane + 32] * lg + rho] : make_double2(0.0, 0.0);
    for (int c = rho - 1; c >= 0; --c) {
      const bool hi = c >= 32;
      const int owner = c & 31;
      double2 xc = make_double2(0.0, 0.0);
      if (lane == owner) xc = cmul_d(hi ? r1 : r0, ipiv[c]);
      xc.x = __shfl_sync(0xffffffffu, xc.x, owner);
      xc.y = __shfl_sync(0xffffffffu, xc.y, owner);
      if (lane == owner) {
        if (hi) r1 = xc;
        else r0 = xc;
      }
      // steps before c subtract their coefficient of x_c
      if (lane < c) {
        const double2 g = G[order[lane] * lg + c];
        r0.x -= g.x * xc.x - g.y * xc.y;
        r0.y -= g.x * xc.y + g.y * xc.x;
      }
      if (lane + 32 < c) {
        const double2 g = G[order[lane + 32] * lg + c];
        r1.x -= g.x * xc.x - g.y * xc.y;
        r1.y -= g.x * xc.y + g.y * xc.x;
      }
    }
    if (lane < rho) x.vchain[lane] = r0;
    if (lane + 32 < rho) x.vchain[lane + 32] = r1;
  }
  if (tid == 0) x.flops += 8.0 * (double)no * rho + 8.0 * (double)rho * rho * rho / 3.0;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// one core of a half-sweep: tournament, maxvol, interpolation solve, new index set
// ---------------------------------------------------------------------------
template <typename R, bool TC>
__device__ int core_select(Ctx<R>& x, const Knobs& kn, int k, int dir) {
  const int tid = threadIdx.x;
  const int N = x.n;
  TTP_TIC(t_st);
  core_states(x, k, dir);
  load_axis_table(x, k);
  TTP_TOC(t_st, 0);
  const int no = dir == DIR_LR ? x.lsz[k] : x.rsz[k + 1];
  const int nc = dir == DIR_LR ? x.rsz[k + 1] : x.lsz[k];
  const int m = no * N;
  const int b = kn.block_rows;
  if (tid == 0) x.evals += (long long)m * nc;
  TTP_TIC(t_cs);
  column_shifts(x, no, nc);
  TTP_TOC(t_cs, 1);
  const R thr2 = (R)(kn.theta * kn.theta);
  const int rho0 = tournament(x, m, nc, b, thr2);
  if (rho0 == 0) {
    if (tid == 0) {
      x.misc[MISC_FAIL] = 1;
      x.fail_step = 1;
    }
    __syncthreads();
    return 0;
  }
  TTP_TIC(t_rr);
  const int rho = rank_reveal(x, rho0, thr2);
  TTP_TOC(t_rr, 7);
  if (rho == 0) {  // every column negligible in its fiber
    if (tid == 0) {
      x.misc[MISC_FAIL] = 1;
      x.fail_step = 1;
    }
    __syncthreads();
    return 0;
  }
  if constexpr (TC) {
    maxvol_refine_tc(x, m, no, rho, b, (R)((1.0 + kn.tau) * (1.0 + kn.tau)));
  } else {
    maxvol_refine(x, m, no, rho, b, (R)((1.0 + kn.tau) * (1.0 + kn.tau)));
  }
  TTP_TIC(t_ch);
  chain_solve<R, TC>(x, no, rho);
  TTP_TOC(t_ch, 10);
  // new index set
  if (dir == DIR_LR) {
    const int w = k + 1;
    for (int idx = tid; idx < rho * w; idx += kThreads) {
      const int t = idx / w, pos = idx % w;
      const int g = x.wrow[t];
      lset_at(x, k + 1, t)[pos] = pos < k ? lset_at(x, k, g / N)[pos] : (uint16_t)(g % N);
    }
    if (tid == 0) x.lsz[k + 1] = rho;
    if (x.emit) {  // two-train form: this core's skeleton (the latest left-to-right one stays)
      int* er = reinterpret_cast<int*>(x.emit + (size_t)k * emit_core_bytes(x.rall, x.dmax));
      int* ew = er + 1;
      uint16_t* ek = reinterpret_cast<uint16_t*>(ew + x.rall);
      const int wr = x.d - k - 1;
      if (tid == 0) er[0] = rho;
      for (int t = tid; t < rho; t += kThreads) ew[t] = x.wrow[t];
      for (int idx = tid; idx < rho * wr; idx += kThreads) {
        const int t = idx / wr, pos = idx % wr;
        ek[t * x.dmax + pos] = rset_at(x, k + 1, x.jp[t])[pos];
      }
    }
  } else {
    const int w = x.d - k;
    for (int idx = tid; idx < rho * w; idx += kThreads) {
      const int t = idx / w, pos = idx % w;
      const int g = x.wrow[t];
      rset_at(x, k, t)[pos] = pos == 0 ? (uint16_t)(g % N) : rset_at(x, k + 1, g / N)[pos - 1];
    }
    if (tid == 0) x.rsz[k] = rho;
  }
  __syncthreads();
  return rho;
}


// end core of a half-sweep: est = sum_o v[o] * sum_i A[(o,i)]
template <typename R>
__device__ double2 core_sum(Ctx<R>& x, int k, int dir, double* dscr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = x.n;
  core_states(x, k, dir);
  load_axis_table(x, k);
  const int no = dir == DIR_LR ? x.lsz[k] : x.rsz[k + 1];
  column_shifts(x, no, 1);
  // one warp per outer index: lanes over the grid index, a warp sum, the
  // contraction weight; one block sum at the end (lane 0 carries its warp's part)
  double2 est = make_double2(0.0, 0.0);
  for (int o = warp; o < no; o += kWarps) {  // warp-uniform
    double sx = 0.0, sy = 0.0;
    for (int i = lane; i < N; i += 32) {
      const cpx<R> a = eval_point(x, o, i, 0);
      sx += (double)a.re;
      sy += (double)a.im;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, off);
      sy += __shfl_xor_sync(0xffffffffu, sy, off);
    }
    const double2 v = x.vchain[o];
    est.x += v.x * sx - v.y * sy;
    est.y += v.x * sy + v.y * sx;
  }
  if (lane != 0) est = make_double2(0.0, 0.0);
  est = block_sum_d2(est, dscr);
  if (tid == 0) {
    x.evals += (long long)no * N;
    x.flops += 24.0 * (double)no * N;
  }
  if constexpr (Num<R>::kScaleColumns) {
    const double sc = Num<R>::unscale((double)x.cshift[0]);
    est.x *= sc;
    est.y *= sc;
  }
  return est;
}

}  // namespace ttp
