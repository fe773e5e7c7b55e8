// Tensor-train Fourier pricer (arXiv 2203.02804) for GB300 / sm_103a:
// the C ABI declared in include/ttprice.h, the host-side preparation and the
// persistent TT-cross kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "ttprice.h"
#include "ttprice_device.cuh"

namespace ttp {

// ---------------------------------------------------------------------------
// the persistent kernel: one CTA = one TT-cross job at a time
// ---------------------------------------------------------------------------
template <typename R>
struct MinBlocks {
#ifndef TTP_MIN_BLOCKS_F32
#define TTP_MIN_BLOCKS_F32 3
#endif
  static constexpr int value = sizeof(R) == 4 ? TTP_MIN_BLOCKS_F32 : 1;  // FP32: several CTAs per SM
};

constexpr double kBlowup = 100.0;  // FP32 half-sweep growth guard (see the sweep loop)
constexpr double kImagTrust = 0.25;  // FP32: largest |Im| / |Re| of a reportable estimate

// one job's half-sweep state (see the sweep loop)
struct SweepState {
  double sign, bound;  // the train's sign; cap / (weight exp(logscale + norm_sum))
  double norm_sum;
  double2 est;         // the estimate to report
  double2 trusted;     // FP32: the latest plausible estimate
  double2 hist[2];     // the last two half-sweeps' estimates, by parity
  int have_trusted, ok_hist[2];
};

// an FP32 half-sweep estimate that can be reported: |Im| <= kImagTrust |Re| and the
// train's share of the price, sign weight exp(logscale + norm_sum) Re, in (0, cap]
__device__ __forceinline__ bool plausible(const SweepState& ss, double2 est) {
  const double re = ss.sign * est.x;
  return re > 0.0 && fabs(est.y) <= kImagTrust * re && re <= ss.bound;
}

template <typename R, bool TC>
__global__ void __launch_bounds__(kThreads, MinBlocks<R>::value) tt_cross_kernel(const JobDesc* __restrict__ jobs,
                                                            const double* __restrict__ params,
                                                            const int* __restrict__ order, int njobs,
                                                            int* counter, JobResult* results,
                                                            char* scratch, Layout lay, SmemLayout sl,
                                                            Knobs kn, char* emit, size_t emit_stride,
                                                            const uint16_t* __restrict__ warm_buf,
                                                            uint16_t* piv_out, int pstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double dscr[32];
  __shared__ SweepState ss;
  // The context is uniform across the CTA: keeping it in shared memory (written
  // by thread 0) keeps its ~40 pointers out of every thread's registers.
  __shared__ Ctx<R> x;
  const int tid = threadIdx.x;
  char* base = scratch + (size_t)blockIdx.x * lay.stride;
  if (tid == 0) {
  x.dmax = lay.dmax;
  x.nmax = lay.nmax;
  x.rall = lay.rmax;
  x.u = reinterpret_cast<double*>(base + lay.u);
  x.lam = reinterpret_cast<double*>(base + lay.lam);
  x.om = reinterpret_cast<double2*>(base + lay.om);
  x.lset = reinterpret_cast<uint16_t*>(base + lay.lset);
  x.rset = reinterpret_cast<uint16_t*>(base + lay.rset);
  x.lstate = reinterpret_cast<double*>(base + lay.lstate);
  x.rstate = reinterpret_cast<double*>(base + lay.rstate);
  x.lvec = reinterpret_cast<double*>(base + lay.lvec);
  x.rvec = reinterpret_cast<double*>(base + lay.rvec);
  x.pair = reinterpret_cast<PairE<R>*>(base + lay.pair);
  x.P = reinterpret_cast<cpx<R>*>(base + lay.P);
  x.sacc = reinterpret_cast<double2*>(base + lay.sacc);
  x.vchain = reinterpret_cast<double2*>(base + lay.chain);
  x.ychain = x.vchain + lay.rmax;
  x.cb = reinterpret_cast<float*>(base + lay.cb);
  x.sw = reinterpret_cast<cpx<R>*>(smem + sl.sw);
  x.M = reinterpret_cast<cpx<R>*>(smem + sl.m);
  x.wvals = reinterpret_cast<cpx<R>*>(smem + sl.wvals);
  x.stage = reinterpret_cast<PairE<R>*>(smem + sl.stage);
  x.stage_lo = 0;
  x.stage_n = 0;
  {
    R* tb = reinterpret_cast<R*>(smem + sl.tab);
    x.tl = tb;
    x.tu = tb + lay.nmax;
    x.tor = tb + 2 * lay.nmax;
    x.toi = tb + 3 * lay.nmax;
  }
  x.colmax = reinterpret_cast<R*>(smem + sl.colmax);
  x.cshift = reinterpret_cast<R*>(smem + sl.cshift);
  x.cref = reinterpret_cast<R*>(smem + sl.cref);
  x.wrow = reinterpret_cast<int*>(smem + sl.wrow);
  x.wnew = reinterpret_cast<int*>(smem + sl.wnew);
  x.jp = reinterpret_cast<int*>(smem + sl.jp);
  x.selr = reinterpret_cast<int*>(smem + sl.selr);
  x.selc = reinterpret_cast<int*>(smem + sl.selc);
  x.scand = reinterpret_cast<int*>(smem + sl.scand);
  x.scnt = reinterpret_cast<int*>(smem + sl.scnt);
  x.redv = reinterpret_cast<R*>(smem + sl.redv);
  x.redi = reinterpret_cast<int*>(smem + sl.redi);
  x.swcol = reinterpret_cast<cpx<R>*>(smem + sl.swcol);
  x.swrow = reinterpret_cast<cpx<R>*>(smem + sl.swrow);
  x.mcol = reinterpret_cast<cpx<R>*>(smem + sl.mcol);
  x.redk = reinterpret_cast<unsigned*>(smem + sl.redk);
  x.lsz = reinterpret_cast<int*>(smem + sl.lsz);
  x.rsz = reinterpret_cast<int*>(smem + sl.rsz);
  x.misc = reinterpret_cast<int*>(smem + sl.misc);
  x.mbar = reinterpret_cast<uint64_t*>(x.misc + MISC_MBAR);
  x.tmem_cols = tc::tmem_cols(lay.rmax);
  x.mma_phase = 0;
  x.tc_pending = 0;
  }
  __syncthreads();
  if constexpr (TC) {
    if (tid == 0) {  // two arrivals per phase: the two issuing threads' commits
      tc::mbar_init(x.mbar, 2);
      tc::mbar_init(x.mbar + 1, 2);
    }
    if (tid < 32) tc::tmem_alloc(reinterpret_cast<uint32_t*>(x.misc + MISC_TMEM), x.tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) x.tmem = *reinterpret_cast<uint32_t*>(x.misc + MISC_TMEM);
    __syncthreads();
  }

  for (int guard = 0; guard < njobs + 1; ++guard) {  // at most njobs jobs per CTA
    if (tid == 0) x.misc[MISC_JOB] = atomicAdd(counter, 1);
    __syncthreads();
    const int slot = x.misc[MISC_JOB];
    if (slot >= njobs) break;
    const int jid = order[slot];
    const JobDesc jd = jobs[jid];
    const double* prm = params + jd.param_off;
    if (tid == 0) {
      x.d = jd.d;
      x.n = jd.n;
      x.rmax = jd.rmax;
      x.cauchy = jd.cauchy;
      x.D0 = (R)jd.D0;
      x.T = jd.Tq;
      x.emit = jd.factor != FACTOR_PRODUCT ? emit + (size_t)jid * emit_stride : nullptr;
      x.warm = (warm_buf && jd.warm_off >= 0) ? warm_buf + jd.warm_off : nullptr;
      x.cov = prm;
      x.flops = 0.0;
      x.evals = 0;
      x.swaps = 0;
      x.visits = 0;
      x.rollbacks = 0;
      x.fail_step = 0;
      x.misc[MISC_FAIL] = 0;
      x.misc[MISC_DRAW] = 0;
    }
    __syncthreads();
    double norm_sum = 0.0;
    TTP_TIC(t_js);
    job_setup(x, jd, prm, dscr, norm_sum);
    TTP_TOC(t_js, 13);

    // The job's sweep state is uniform across the CTA; it sits in shared memory
    // (thread 0 writes it, the barriers of the next half-sweep publish it) rather
    // than in registers that would stay live through the cores' loops.
    if (tid == 0) {
      ss.sign = jd.sign;
      ss.bound = exp(fmin(log(jd.cap / jd.weight) - jd.logscale - norm_sum, 700.0));
      ss.norm_sum = norm_sum;
      ss.est = ss.trusted = ss.hist[0] = ss.hist[1] = make_double2(0.0, 0.0);
      ss.have_trusted = 0;
      ss.ok_hist[0] = ss.ok_hist[1] = 0;
    }
    // the job's own rank threshold and block height (its class's, else the options')
    Knobs jk = kn;
    jk.theta = jd.theta;
    jk.block_rows = jd.block_rows;
    int status = x.misc[MISC_DRAW] ? ST_INVALID : ST_NOT_CONVERGED;
    int hs = 0, maxrank = 1;
    const int d = jd.d;
    for (int s = 0; s < kn.max_half_sweeps && status == ST_NOT_CONVERGED; ++s) {
      if (tid == 0) x.vchain[0] = make_double2(1.0, 0.0);
      __syncthreads();
      double2 est = make_double2(0.0, 0.0);
      if ((s & 1) == 0) {
        for (int k = 0; k + 1 < d; ++k) {
          const int rho = core_select<R, TC>(x, jk, k, DIR_LR);
          maxrank = max(maxrank, rho);
          if (x.misc[MISC_FAIL]) break;
        }
        TTP_TIC(t_cs);
        if (!x.misc[MISC_FAIL]) est = core_sum(x, d - 1, DIR_LR, dscr);
        TTP_TOC(t_cs, 12);
      } else {
        for (int k = d - 1; k >= 1; --k) {
          const int rho = core_select<R, TC>(x, jk, k, DIR_RL);
          maxrank = max(maxrank, rho);
          if (x.misc[MISC_FAIL]) break;
        }
        TTP_TIC(t_cs);
        if (!x.misc[MISC_FAIL]) est = core_sum(x, 0, DIR_RL, dscr);
        TTP_TOC(t_cs, 12);
      }
      hs = s + 1;
      if (x.misc[MISC_FAIL] || !isfinite(est.x) || !isfinite(est.y)) {
        if (tid == 0 && x.fail_step == 0) x.fail_step = 4;
        status = ST_NUMERIC;
        break;
      }
      // A factor train of the two-train form runs a fixed count of half-sweeps: its
      // own grid sum (the payoff transform's cancels to ~1e-10 of its entries) is no
      // stop criterion and no share of the price.
      if (x.emit) {
        if (tid == 0) ss.est = est;
        if (d == 1 || s + 1 == kn.max_half_sweeps) status = ST_OK;
        continue;
      }
      // The midpoint grid is symmetric and the payoff real, so the exact grid sum
      // is real and |Im est| is a lower bound on the estimate's error; the train's
      // share of the price lies in (0, sum of spots].  In FP32 a half-sweep built on
      // poor index sets (the first one, from random pivots, or a rank-limited one)
      // can amplify the integrand's rounding past both; such an estimate neither
      // converges nor is reported, and the sweeps go on from its index sets.
      bool est_ok = true;
      if constexpr (sizeof(R) == 4) est_ok = plausible(ss, est);
      if (tid == 0) {
        ss.est = est;
        if (est_ok) {
          ss.trusted = est;
          ss.have_trusted = 1;
        }
      }
      if (d == 1) {
        status = ST_OK;
        break;
      }
      // the previous estimate: written at s - 1 into slot (s - 1) & 1; slot s & 1 is
      // written below, while other threads may still read this one
      const double2 prev = ss.hist[(s + 1) & 1];
      const bool prev_ok = ss.ok_hist[(s + 1) & 1];
      if (s >= 1) {
        const double dx = est.x - prev.x, dy = est.y - prev.y;
        const double change = sqrt(dx * dx + dy * dy);
        if (est_ok && change <= kn.sweep_tol * sqrt(est.x * est.x + est.y * est.y)) {
          status = ST_OK;
          break;
        }
        // FP32 guard: a half-sweep whose estimate moves away from a plausible one by
        // more than kBlowup times that one has followed a drifted P^{-1} into an
        // ill-conditioned pivot block; keep the previous estimate and stop
        if constexpr (sizeof(R) == 4) {
          if (prev_ok && change > kBlowup * sqrt(prev.x * prev.x + prev.y * prev.y)) {
            if (tid == 0) {
              ss.est = prev;
              x.fail_step = 7;
            }
            break;
          }
        }
      }
      if (tid == 0) {
        ss.hist[s & 1] = est;
        ss.ok_hist[s & 1] = est_ok;
      }
    }
    if (tid == 0) {
      double2 est = ss.est;
      if constexpr (sizeof(R) == 4) {
        if ((status == ST_OK || status == ST_NOT_CONVERGED) && !x.emit && !plausible(ss, est)) {
          if (ss.have_trusted) {  // the latest plausible estimate
            est = ss.trusted;
            status = ST_NOT_CONVERGED;
            x.fail_step = 7;
          } else if (hypot(est.x, est.y) > ss.bound) {  // nothing reportable
            status = ST_NUMERIC;
            x.fail_step = 8;
          }
        }
      }
      JobResult r;
      r.est_re = est.x;
      r.est_im = est.y;
      r.norm_sum = ss.norm_sum;
      r.flops = x.flops;
      r.evaluations = x.evals;
      r.swaps = x.swaps;
      r.visits = x.visits;
      r.rollbacks = x.rollbacks;
      r.status = status;
      r.half_sweeps = hs;
      r.max_rank = maxrank;
      r.fail_step = status == ST_INVALID ? 5 : x.fail_step;
      results[jid] = r;
    }
    if (piv_out && tid < 32) {  // the final right sets (latest right-to-left half-sweep)
      uint16_t* rec = piv_out + (size_t)jid * pstride;
      int off = 0;
      for (int k = 1; k < d; ++k) {
        const int c = x.rsz[k], w = d - k;
        if (tid == 0) rec[off] = (uint16_t)c;
        for (int idx = tid; idx < c * w; idx += 32) rec[off + 1 + idx] = rset_at(x, k, idx / w)[idx % w];
        off += 1 + c * w;
      }
    }
    __syncthreads();
  }
  if constexpr (TC) {
    // a block product whose completion wait gave up may still be running: wait
    // (bounded) before the accumulator columns are released
    if (x.tc_pending) {
      tc::mbar_wait(x.mbar, x.mma_phase & 1u);
      tc::mbar_wait(x.mbar + 1, (x.mma_phase >> 1) & 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(x.tmem, x.tmem_cols);
  }
}

// per-instance combination of the trains: price = sum Re(weight sign e^{logscale+norms} est)
__global__ void finalize_kernel(const JobDesc* __restrict__ jobs, const JobResult* __restrict__ jres,
                                const int* __restrict__ first, const int* __restrict__ count,
                                const int* __restrict__ hstatus, int ninst, InstanceResult* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  InstanceResult r;
  r.price = 0.0;
  r.imag = 0.0;
  r.flops = 0.0;
  r.evaluations = 0;
  r.swaps = 0;
  r.visits = 0;
  r.fail_step = 0;
  r.rollbacks = 0;
  r.half_sweeps = 0;
  r.max_rank = 0;
  r.terms = count[i];
  int worst_err = 0, worst_warn = 0, err_step = 0;
  if (hstatus[i] < 0) worst_err = hstatus[i];
  for (int t = 0; t < count[i]; ++t) {
    const int j = first[i] + t;
    const JobDesc& jd = jobs[j];
    const JobResult& q = jres[j];
    if (jd.factor != FACTOR_PHI) {  // a payoff-transform train carries its bracket's value
      const double sc = jd.weight * jd.sign * exp(jd.logscale + q.norm_sum);
      r.price += sc * q.est_re;
      r.imag += sc * q.est_im;
    }
    r.flops += q.flops;
    r.evaluations += q.evaluations;
    r.swaps += q.swaps;
    r.visits += q.visits;
    r.rollbacks += q.rollbacks;
    if (q.fail_step != 0 && r.fail_step == 0) r.fail_step = q.fail_step;
    r.half_sweeps = max(r.half_sweeps, q.half_sweeps);
    r.max_rank = max(r.max_rank, q.max_rank);
    if (q.status < 0 && (worst_err == 0 || q.status < worst_err)) {
      worst_err = q.status;
      err_step = q.fail_step;
    }
    if (q.status > worst_warn) worst_warn = q.status;
  }
  r.status = worst_err != 0 ? worst_err : worst_warn;
  if (worst_err != 0 && err_step != 0) r.fail_step = err_step;  // the failing train's step
  if (r.status < 0 || !isfinite(r.price)) {
    if (r.status >= 0) r.status = ST_NUMERIC;
    r.price = nan("");
  }
  out[i] = r;
}

// ---------------------------------------------------------------------------
// Two-train form (Section IV, Eq. braket): the bracket <vhat | phi> of the two
// factor trains of one term, contracted site by site, one CTA per bracket.
// Each factor's cores are rebuilt from its skeleton (selected rows W_k, kept
// columns K_k) with the cross's own integrand evaluation and column shifts:
//   A_k(i) = F(I_{k-1}, i, K_k),  P_k = A_k[W_k],  G_k(i) = A_k(i) P_k^{-1}
// (the shifts cancel in G), the end core G(i) = F(I_{d-2}, i); then
//   E <- sum_i G^v_k(i)^T E G^phi_k(i),  E_0 = [1].
// Regrouped, E <- (P^v_k)^{-T} [sum_i A^v_k(i)^T E A^phi_k(i)] (P^phi_k)^{-1}, so
// the inverses (FP64 Gauss-Jordan with partial pivoting) apply once per core.
// The bracket, in the v train's normalised units, goes to that train's result;
// the phi train's carries no price.
// ---------------------------------------------------------------------------
struct BrSmem {
  int tab[2], cshift[2], cref[2], lsz[2], rsz[2], W[2];
  int E, X, Av, Af, Gv, Gf, Mv, Mf, red, total;
};

// FP64 [P | I] -> P^{-1} (n x n, rows of length ld >= 2n in G), written to M in R
// (leading dimension n); false when a pivot is zero or not finite.
template <typename R>
__device__ bool gj_inverse_f64(double2* G, int n, int ld, cpx<R>* M, double* redv, int* redi) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = 0; c < n; ++c) {
    if (warp == 0) {
      double v = -1.0;
      int vi = INT_MAX;
      for (int r = c + lane; r < n; r += 32) {
        const double2 g = G[r * ld + c];
        am_merge(v, vi, g.x * g.x + g.y * g.y, r);
      }
      warp_argmax(v, vi);
      if (lane == 0) {
        redv[0] = v;
        redi[0] = vi;
      }
    }
    __syncthreads();
    const double pv = redv[0];
    const int p = redi[0];
    if (!(pv > 0.0) || !(pv < 1e300)) return false;  // block-uniform
    if (p != c)
      for (int j = tid; j < 2 * n; j += kThreads) {
        const double2 a = G[c * ld + j];
        G[c * ld + j] = G[p * ld + j];
        G[p * ld + j] = a;
      }
    __syncthreads();
    const double2 g = G[c * ld + c];
    const double2 inv = make_double2(g.x / pv, -g.y / pv);
    __syncthreads();  // every thread has read the pivot before row c is scaled
    for (int j = c + tid; j < 2 * n; j += kThreads) {
      const double2 a = G[c * ld + j];
      G[c * ld + j] = make_double2(a.x * inv.x - a.y * inv.y, a.x * inv.y + a.y * inv.x);
    }
    __syncthreads();
    const int w = 2 * n - c - 1;  // columns right of c
    for (int idx = tid; idx < n * w; idx += kThreads) {
      const int r = idx / w, j = c + 1 + idx % w;
      if (r == c) continue;
      const double2 f = G[r * ld + c], b = G[c * ld + j];
      double2 a = G[r * ld + j];
      a.x -= f.x * b.x - f.y * b.y;
      a.y -= f.x * b.y + f.y * b.x;
      G[r * ld + j] = a;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < n * n; idx += kThreads) {
    const int r = idx / n, c = idx % n;
    const double2 a = G[r * ld + n + c];
    M[idx] = cpx<R>{(R)a.x, (R)a.y};
  }
  __syncthreads();
  return true;
}

template <typename R>
__device__ void bracket_ctx(Ctx<R>& x, const JobDesc& jd, const double* params, char* base, const Layout& lay,
                            unsigned char* smem, const BrSmem& S, int f, int* misc) {
  x.dmax = lay.dmax;
  x.nmax = lay.nmax;
  x.rall = lay.rmax;
  x.d = jd.d;
  x.n = jd.n;
  x.rmax = jd.rmax;
  x.cauchy = jd.cauchy;
  x.D0 = (R)jd.D0;
  x.T = jd.Tq;
  x.cov = params + jd.param_off;
  x.u = reinterpret_cast<double*>(base + lay.u);
  x.lam = reinterpret_cast<double*>(base + lay.lam);
  x.om = reinterpret_cast<double2*>(base + lay.om);
  x.lset = reinterpret_cast<uint16_t*>(base + lay.lset);
  x.rset = reinterpret_cast<uint16_t*>(base + lay.rset);
  x.lstate = reinterpret_cast<double*>(base + lay.lstate);
  x.rstate = reinterpret_cast<double*>(base + lay.rstate);
  x.lvec = reinterpret_cast<double*>(base + lay.lvec);
  x.rvec = reinterpret_cast<double*>(base + lay.rvec);
  x.pair = reinterpret_cast<PairE<R>*>(base + lay.pair);
  R* tab = reinterpret_cast<R*>(smem + S.tab[f]);
  x.tl = tab;
  x.tu = tab + lay.nmax;
  x.tor = tab + 2 * lay.nmax;
  x.toi = tab + 3 * lay.nmax;
  x.cshift = reinterpret_cast<R*>(smem + S.cshift[f]);
  x.cref = reinterpret_cast<R*>(smem + S.cref[f]);
  x.lsz = reinterpret_cast<int*>(smem + S.lsz[f]);
  x.rsz = reinterpret_cast<int*>(smem + S.rsz[f]);
  x.stage = nullptr;
  x.stage_lo = 0;
  x.stage_n = 0;
  x.misc = misc;
  x.flops = 0.0;
  x.evals = 0;
  x.emit = nullptr;
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 2) bracket_kernel(const JobDesc* __restrict__ jobs,
                                                              const double* __restrict__ params,
                                                              const int2* __restrict__ pairs, int npairs,
                                                              const char* __restrict__ emit, size_t emit_stride,
                                                              int* counter, JobResult* results, char* scratch,
                                                              Layout lay, BrSmem S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double dscr[32];
  __shared__ Ctx<R> xs[2];
  __shared__ int misc[16];
  __shared__ int slot;
  const int tid = threadIdx.x;
  const size_t ecb = emit_core_bytes(lay.rmax, lay.dmax);
  cpx<R>* E = reinterpret_cast<cpx<R>*>(smem + S.E);
  cpx<R>* X = reinterpret_cast<cpx<R>*>(smem + S.X);
  cpx<R>* Av = reinterpret_cast<cpx<R>*>(smem + S.Av);
  cpx<R>* Af = reinterpret_cast<cpx<R>*>(smem + S.Af);
  cpx<R>* Gv = reinterpret_cast<cpx<R>*>(smem + S.Gv);
  cpx<R>* Gf = reinterpret_cast<cpx<R>*>(smem + S.Gf);
  double* redv = reinterpret_cast<double*>(smem + S.red);
  int* redi = reinterpret_cast<int*>(redv + 2);
  constexpr int kAcc = 4;  // accumulator entries per thread: r_v r_phi <= 1024 (the host checks)
  for (;;) {  // brackets from a queue: a CTA that shares its SM takes fewer
    __syncthreads();  // every thread has read the previous slot
    if (tid == 0) slot = atomicAdd(counter, 1);
    __syncthreads();
    const int pr = slot;
    if (pr >= npairs) break;
    const int2 jp = pairs[pr];
    const JobDesc jv = jobs[jp.x], jf = jobs[jp.y];
    if (results[jp.x].status < 0 || results[jp.y].status < 0) continue;  // a train failed: the price is NaN
    if (tid == 0) {
      for (int f = 0; f < 2; ++f)
        bracket_ctx(xs[f], f ? jf : jv, params, scratch + (2 * (size_t)blockIdx.x + f) * lay.stride, lay, smem, S,
                    f, misc);
    }
    __syncthreads();
    double ns[2];
    for (int f = 0; f < 2; ++f) job_setup(xs[f], f ? jf : jv, params + (f ? jf : jv).param_off, dscr, ns[f], false);
    const int d = jv.d, N = jv.n;
    if (tid == 0) E[0] = cpx<R>{R(1), R(0)};
    bool ok = true;
    double lu = 0.0;
    for (int k = 0; k < d && ok; ++k) {
      const bool last = k == d - 1;
      for (int f = 0; f < 2 && ok; ++f) {
        Ctx<R>& x = xs[f];
        int* W = reinterpret_cast<int*>(smem + S.W[f]);
        const char* e = emit + (size_t)(f ? jp.y : jp.x) * emit_stride + (size_t)k * ecb;
        const int rp = x.lsz[k];
        const int rk = last ? 1 : *reinterpret_cast<const int*>(e);
        if (!last) {
          const int* ew = reinterpret_cast<const int*>(e) + 1;
          const uint16_t* ek = reinterpret_cast<const uint16_t*>(ew + lay.rmax);
          const int wr = d - k - 1;
          for (int idx = tid; idx < rk * wr; idx += kThreads) {
            const int t = idx / wr, pos = idx % wr;
            rset_at(x, k + 1, t)[pos] = ek[t * lay.dmax + pos];
          }
          for (int t = tid; t < rk; t += kThreads) W[t] = ew[t];
          if (tid == 0) x.rsz[k + 1] = rk;
        }
        __syncthreads();
        core_states(x, k, DIR_LR);
        load_axis_table(x, k);
        if (last) {
          column_shifts(x, rp, rk);
        } else {
          // shifts from the pivot rows alone: the skeleton's rows dominate (maxvol:
          // |A P^{-1}| <= 1 + tau), so a column's largest fiber entry is at most
          // (1 + tau) rk times its largest pivot-row entry, well inside the range
          const int lane = tid & 31, warp = tid >> 5;
          for (int c = warp; c < rk; c += kWarps) {
            R mx = R(-1e300);
            for (int t = lane; t < rk; t += 32) {
              const int g = W[t];
              mx = fmax(mx, eval_logmag(x, g / N, g % N, c));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
            if (lane == 0) x.cshift[c] = Num<R>::ceil_(mx);
          }
          __syncthreads();
        }
        if (!last) {
          // the pivot block A[W, :] in FP64, inverted
          double2* G = reinterpret_cast<double2*>(smem + S.X);
          const int ld = 2 * rk;
          for (int idx = tid; idx < rk * rk; idx += kThreads) {
            const int t = idx / rk, c = idx % rk, g = W[t];
            const cpx<R> a = eval_point(x, g / N, g % N, c);
            G[t * ld + c] = make_double2((double)a.re, (double)a.im);
            G[t * ld + rk + c] = make_double2(t == c ? 1.0 : 0.0, 0.0);
          }
          __syncthreads();
          ok = gj_inverse_f64(G, rk, ld, reinterpret_cast<cpx<R>*>(smem + (f ? S.Mf : S.Mv)), redv, redi);
        } else if (tid == 0) {
          lu += Num<R>::log_unscale((double)x.cshift[0]);
        }
      }
      if (!ok) break;
      const int rpv = xs[0].lsz[k], rkv = last ? 1 : xs[0].rsz[k + 1];
      const int rpf = xs[1].lsz[k], rkf = last ? 1 : xs[1].rsz[k + 1];
      const cpx<R>* Mv = reinterpret_cast<const cpx<R>*>(smem + S.Mv);
      const cpx<R>* Mf = reinterpret_cast<const cpx<R>*>(smem + S.Mf);
      cpx<R> acc[kAcc];
#pragma unroll
      for (int q = 0; q < kAcc; ++q) acc[q] = cpx<R>{R(0), R(0)};
      // Walks along the grid index: for a fixed fiber pair (a, b) the exponent is
      // e0 - shift + h u_i + tl(i) with u_i = u_0 + i eta, so exp(e0 - shift + h u_i)
      // is stepped by the factor exp(h eta) and exp(tl(i)) comes from a table; a
      // pair whose exponent range would leave FP64 is evaluated directly.  Thread
      // tid owns entries tid + q kThreads of each factor's A(i).
      R wcur[2][kAcc], wstep[2][kAcc], ws0[2][kAcc];
      cpx<R> wph[2][kAcc];
      unsigned wdir = 0;
      {
        const R eta = (R)(2.0 * jv.L / N);
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const Ctx<R>& x = xs[f];
          R* tex = reinterpret_cast<R*>(smem + S.tab[f]) + 4 * lay.nmax;
          for (int i = tid; i < N; i += kThreads) tex[i] = Num<R>::ex(x.tl[i]);
          const int rp = x.lsz[k], rk = last ? 1 : x.rsz[k + 1];
#pragma unroll
          for (int q = 0; q < kAcc; ++q) {
            const int idx = tid + q * kThreads;
            wcur[f][q] = wstep[f][q] = ws0[f][q] = R(0);
            wph[f][q] = cpx<R>{R(0), R(0)};
            if (idx < rp * rk) {
              const int a = idx / rk, b = idx % rk;
              const PairE<R> pq = x.pair[a * x.rall + b];
              const R e = pq.e0 - x.cshift[b] + pq.h * x.tu[0], he = pq.h * eta;
              if (fabs((double)e) < 600.0 && fabs((double)he) * N < 100.0) {
                wcur[f][q] = Num<R>::ex(e);
                wstep[f][q] = Num<R>::ex(he);
              } else {
                wdir |= 1u << (f * kAcc + q);
              }
              ws0[f][q] = pq.s0;
              wph[f][q] = cpx<R>{pq.ore, pq.oim};
            }
          }
        }
        __syncthreads();
      }
      // Et = sum_i A^v(i)^T E A^phi(i), then E <- (P^v)^{-T} Et (P^phi)^{-1}: the
      // inverses leave the grid loop (G(i)^T E G(i) with G = A P^{-1}, regrouped)
      for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const Ctx<R>& x = xs[f];
          const R* tex = reinterpret_cast<const R*>(smem + S.tab[f]) + 4 * lay.nmax;
          const int rp = x.lsz[k], rk = last ? 1 : x.rsz[k + 1];
          cpx<R>* A = f ? Af : Av;
          const cpx<R> tph = {x.tor[i], x.toi[i]};
          const R ui = x.tu[i], tx = tex[i];
#pragma unroll
          for (int q = 0; q < kAcc; ++q) {
            const int idx = tid + q * kThreads;
            if (idx < rp * rk) {
              if ((wdir >> (f * kAcc + q)) & 1u) {
                A[idx] = eval_point(x, idx / rk, i, idx % rk);
              } else {
                R mag = wcur[f][q] * tx;
                cpx<R> w = cmul(wph[f][q], tph);
                if (x.cauchy) {
                  const R sv = ws0[f][q] + ui;
                  mag = Num<R>::div(mag, fma(sv, sv, x.D0 * x.D0));
                  w = cmul(w, cpx<R>{x.D0, -sv});
                }
                A[idx] = cpx<R>{w.re * mag, w.im * mag};
                wcur[f][q] *= wstep[f][q];
              }
            }
          }
          // a train above rank 32 (r_{k-1} r_k > kAcc kThreads): the rest evaluated directly
          for (int idx = tid + kAcc * kThreads; idx < rp * rk; idx += kThreads)
            A[idx] = eval_point(x, idx / rk, i, idx % rk);
        }
        __syncthreads();
        // X = E A^phi(i): rpv x rkf
        for (int idx = tid; idx < rpv * rkf; idx += kThreads) {
          const int a = idx / rkf, t = idx % rkf;
          cpx<R> s2 = {R(0), R(0)};
          for (int b = 0; b < rpf; ++b) cfma(s2, E[a * rpf + b], Af[b * rkf + t]);
          X[idx] = s2;
        }
        __syncthreads();
        // acc(a', b') += sum_a A^v(i)[a][a'] X[a][b']
#pragma unroll
        for (int q = 0; q < kAcc; ++q) {
          const int idx = tid + q * kThreads;
          if (idx < rkv * rkf) {
            const int ap = idx / rkf, bp = idx % rkf;
            for (int a = 0; a < rpv; ++a) cfma(acc[q], Av[a * rkv + ap], X[a * rkf + bp]);
          }
        }
        __syncthreads();
      }
      if (last) {
        if (tid == 0) E[0] = acc[0];
      } else {
        // Y = Et (P^phi)^{-1} into Gf, then E = (P^v)^{-T} Y
#pragma unroll
        for (int q = 0; q < kAcc; ++q) {
          const int idx = tid + q * kThreads;
          if (idx < rkv * rkf) Gv[idx] = acc[q];
        }
        __syncthreads();
        for (int idx = tid; idx < rkv * rkf; idx += kThreads) {
          const int ap = idx / rkf, t = idx % rkf;
          cpx<R> s2 = {R(0), R(0)};
          for (int c = 0; c < rkf; ++c) cfma(s2, Gv[ap * rkf + c], Mf[c * rkf + t]);
          Gf[idx] = s2;
        }
        __syncthreads();
        for (int idx = tid; idx < rkv * rkf; idx += kThreads) {
          const int s3 = idx / rkf, t = idx % rkf;
          cpx<R> s2 = {R(0), R(0)};
          for (int c = 0; c < rkv; ++c) cfma(s2, Mv[c * rkv + s3], Gf[c * rkf + t]);
          E[idx] = s2;
        }
      }
      if (tid == 0) {
        const double pts = (double)N * (rpv * rkv + rpf * rkf);
        xs[0].evals += (long long)pts;
        xs[0].flops += 24.0 * pts + 8.0 * (N * ((double)rpv * rpf * rkf + (double)rpv * rkv * rkf) +
                                           (last ? 0.0 : (double)rkv * rkf * (rkf + rkv)));
      }
      // next core's left sets: I_k[t] = I_{k-1}[W[t] / N] followed by W[t] % N
      if (!last) {
        for (int f = 0; f < 2; ++f) {
          Ctx<R>& x = xs[f];
          const int* W = reinterpret_cast<const int*>(smem + S.W[f]);
          const int rk = x.rsz[k + 1], w = k + 1;
          for (int idx = tid; idx < rk * w; idx += kThreads) {
            const int t = idx / w, pos = idx % w, g = W[t];
            lset_at(x, k + 1, t)[pos] = pos < k ? lset_at(x, k, g / N)[pos] : (uint16_t)(g % N);
          }
          if (tid == 0) x.lsz[k + 1] = rk;
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      JobResult r = results[jp.x];
      const cpx<R> b = E[0];
      if (ok && isfinite((double)b.re) && isfinite((double)b.im)) {
        r.est_re = (double)b.re;
        r.est_im = (double)b.im;
        r.norm_sum = ns[0] + ns[1] + jf.logscale + lu;
      } else {
        r.status = ST_NUMERIC;
        r.fail_step = 9;
      }
      r.flops += xs[0].flops;
      r.evaluations += xs[0].evals;
      results[jp.x] = r;
    }
    __syncthreads();
  }
}

}  // namespace ttp

// ===========================================================================
// host side
// ===========================================================================
namespace {

using ttp::InstanceResult;
using ttp::JobDesc;
using ttp::JobResult;
using ttp::Knobs;
using ttp::Layout;
using ttp::SmemLayout;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Resolved {
  tt_options o;
  Knobs kn;
  int max_jobs;
  size_t max_params;
  int n_classes;
  tt_class_tuning classes[TT_MAX_CLASSES];  // copied from the options
};

bool resolve(const tt_options* in, Resolved* r) {
  if (!in) return false;
  r->o = *in;
  tt_options& o = r->o;
  if (o.max_d < 1 || o.max_d > 255) return false;
  if (o.max_n < 2 || o.max_n > 4096) return false;
  if (o.max_rank < 1 || o.max_rank > 64) return false;
  if (o.max_batch < 1 || o.max_batch > (1 << 22)) return false;
  if (o.precision != TT_FP64 && o.precision != TT_MIXED) return false;
  if (o.block_rows == 0) o.block_rows = 128;
  if (o.block_rows < o.max_rank || o.block_rows + o.max_rank > ttp::kThreads) return false;
  if (o.engine < TT_ENGINE_AUTO || o.engine > TT_ENGINE_TENSOR_CORES) return false;
  if (o.graph != 0 && o.graph != 1) return false;
  if (o.method != TT_METHOD_SINGLE_TRAIN && o.method != TT_METHOD_TWO_TRAINS) return false;
  if (o.pivot_io != 0 && o.pivot_io != 1) return false;
  const bool two = o.method == TT_METHOD_TWO_TRAINS;
  if (two && (o.max_rank > 40 || o.max_n > 1024)) return false;  // the bracket kernel's tile sizes
  if (o.precision == TT_FP64) {
    if (o.engine == TT_ENGINE_TENSOR_CORES) return false;  // no FP64 tensor-core product
    o.engine = TT_ENGINE_CUDA_CORES;
  } else if (o.engine == TT_ENGINE_AUTO) {
    o.engine = o.max_rank > 32 ? TT_ENGINE_TENSOR_CORES : TT_ENGINE_CUDA_CORES;
  }
  // the tensor-core block product is one 128-row tile
  if (o.engine == TT_ENGINE_TENSOR_CORES && o.block_rows > ttp::tc::kRows) return false;
  if (o.max_half_sweeps == 0) o.max_half_sweeps = two ? 3 : 8;
  if (o.max_half_sweeps < 1 || o.max_half_sweeps > 1000) return false;
  const bool f64 = o.precision == TT_FP64;
  if (!(o.sweep_tol > 0)) o.sweep_tol = f64 ? 1e-6 : 1e-4;
  if (!(o.rank_tol > 0)) o.rank_tol = f64 ? 1e-8 : 1e-6;
  if (!(o.maxvol_tol > 0)) o.maxvol_tol = 0.05;
  if (!std::isfinite(o.sweep_tol) || !std::isfinite(o.rank_tol) || !std::isfinite(o.maxvol_tol))
    return false;
  if (o.n_classes < 0 || o.n_classes > TT_MAX_CLASSES || (o.n_classes > 0 && !o.classes)) return false;
  r->n_classes = o.n_classes;
  for (int c = 0; c < o.n_classes; ++c) {
    tt_class_tuning t = o.classes[c];
    if (!std::isfinite(t.rank_tol)) return false;
    if (t.block_rows < 0 || t.block_rows > o.block_rows) return false;
    if (!(t.rank_tol > 0)) t.rank_tol = 0.0;
    r->classes[c] = t;
  }
  o.classes = nullptr;  // the copy above is what the handle keeps
  r->kn.theta = o.rank_tol;
  r->kn.tau = o.maxvol_tol;
  r->kn.sweep_tol = o.sweep_tol;
  r->kn.max_half_sweeps = o.max_half_sweeps;
  r->kn.block_rows = o.block_rows;
  const long long mj = (long long)o.max_batch * o.max_d * (two ? 2 : 1);
  if (mj > (1 << 24)) return false;
  r->max_jobs = (int)mj;
  r->max_params = (size_t)r->max_jobs * ((size_t)o.max_d * o.max_d + 3 * (size_t)o.max_d);
  return true;
}

Layout make_layout(const tt_options& o, bool f64) {
  Layout L;
  const size_t A = 256;
  const size_t d = o.max_d, n = o.max_n, r = o.max_rank;
  const size_t rs = f64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes, A);
    return at;
  };
  L.u = take(n * 8);
  L.lam = take(d * n * 8);
  L.om = take(d * n * 16);
  L.lset = take((d + 1) * r * d * 2);
  L.rset = take((d + 1) * r * d * 2);
  L.lstate = take(r * 8 * 8);
  L.rstate = take(r * 8 * 8);
  L.lvec = take(r * d * 8);
  L.rvec = take(r * d * 8);
  L.pair = take(8 * r * r * rs);
  L.P = take(2 * r * r * 2 * rs);  // P and the copy maxvol falls back to
  L.sacc = take(r * r * 16);
  L.chain = take(2 * r * 16);
  L.cb = take(sizeof(float) * ttp::kBoundCap);
  L.stride = align_up(off, A);
  L.dmax = (int)d;
  L.nmax = (int)n;
  L.rmax = (int)r;
  return L;
}

SmemLayout make_smem(const tt_options& o, bool f64) {
  SmemLayout S;
  const int rs = f64 ? 8 : 4, cs = 2 * rs;
  const int r = o.max_rank, b = o.block_rows, n = o.max_n, d = o.max_d;
  int sw_elems = std::max((r + std::max(b, 128)) * r, 2 * r * r);
  // the FP64 interpolation solve: [P^T | y] (r x (r+1) complex doubles) and its reduction
  // scratch; its refinement: P, w, y and the residual (r (r+3) complex doubles), 3 kWarps doubles
  sw_elems = std::max(sw_elems, (r * (r + 1) * 16 + 2 * ttp::kWarps * 12 + cs - 1) / cs);
  sw_elems = std::max(sw_elems, (r * (r + 3) * 16 + 3 * ttp::kWarps * 8 + cs - 1) / cs);
  const int kp = ttp::tc::pad16(r);
  const bool tcore = o.engine == TT_ENGINE_TENSOR_CORES;
  // tensor cores: kTcBufs buffers of four 128-row planes of one kTcChunk-column chunk
  // (hi and lo parts of Re A and Im A)
  if (tcore) sw_elems = std::max(sw_elems, ttp::kTcBufs * 4 * ttp::tc::kRows * ttp::kTcChunk * 4 / cs);
  int off = 0;
  auto take = [&](int bytes) {
    int at = off;
    off = (int)align_up(off + bytes, 16);
    return at;
  };
  S.sw_elems = sw_elems;
  S.sw = take(sw_elems * cs);
  S.m = take(tcore ? 2 * kp * kp * 4 : r * r * cs);  // tensor cores: hi planes (re, im) of P^{-1}
  S.wvals = take(tcore ? std::max(r * r * cs, 2 * kp * kp * 4) : r * r * cs);  // tensor cores: also the lo planes
  S.stage = take(ttp::kStageO * r * 8 * rs);
  S.tab = take(4 * n * rs);
  S.colmax = take(r * rs);
  S.cshift = take((r + 1) * rs);
  S.cref = take((r + 1) * rs);
  S.wrow = take(r * 4);
  S.wnew = take(r * 4);
  S.jp = take(r * 4);
  S.selr = take(r * 4);
  S.selc = take(r * 4);
  S.scand = take(ttp::kThreads * 4);
  S.scnt = take(ttp::kWarps * 4);
  S.redv = take(2 * ttp::kWarps * rs);
  S.redi = take(2 * ttp::kWarps * 4);
  S.redk = take(2 * ttp::kWarps * 4);
  S.swcol = take(std::max(b * cs, r * 16));
  S.swrow = take(2 * r * cs);
  S.mcol = take(r * cs);
  S.lsz = take((d + 1) * 4);
  S.rsz = take((d + 1) * 4);
  S.misc = take(16 * 4);
  S.total = off;
  return S;
}

// the bracket kernel's shared memory (two-train form)
ttp::BrSmem make_brsmem(const tt_options& o, bool f64) {
  ttp::BrSmem S;
  const int rs = f64 ? 8 : 4, cs = 2 * rs;
  const int r = o.max_rank, n = o.max_n, d = o.max_d;
  int off = 0;
  auto take = [&](int bytes) {
    int at = off;
    off = (int)align_up(off + bytes, 16);
    return at;
  };
  for (int f = 0; f < 2; ++f) {
    S.tab[f] = take(5 * n * rs);  // tl, tu, tor, toi, exp(tl)
    S.cshift[f] = take((r + 1) * rs);
    S.cref[f] = take((r + 1) * rs);
    S.lsz[f] = take((d + 1) * 4);
    S.rsz[f] = take((d + 1) * 4);
    S.W[f] = take(r * 4);
  }
  const int rr = std::min(r * r, 1024);  // E and its products: r_v r_phi <= 1024
  S.E = take(rr * cs);
  // X .. Gf are contiguous: the FP64 Gauss-Jordan buffer [P | I] (r x 2r) aliases them
  S.X = take(rr * cs);
  S.Av = take(r * r * cs);
  S.Af = take(r * r * cs);
  S.Gv = take(rr * cs);
  S.Gf = take(std::max(rr * cs, 2 * r * r * 16 - (off - S.X)));
  S.Mv = take(r * r * cs);
  S.Mf = take(r * r * cs);
  S.red = take(32);
  S.total = off;
  return S;
}

struct DevLayout {  // offsets inside the device workspace
  size_t stage, stage_bytes, jres, ires, counter, scratch, emit, emit_stride, total;
  size_t o_jobs, o_params, o_order, o_first, o_count, o_hstatus, o_pairs;  // inside the stage block
  size_t o_host;  // host-only scratch of the preparation (never copied to the device)
  size_t o_disc;  // host-only: per-problem relative discretisation-error factor
  size_t o_warm;  // warm-start records, pstride entries per job (pivot_io)
  size_t pivots, pstride;  // device: final right sets, pstride entries per job (pivot_io)
};

// doubles of host scratch the preparation of one problem needs (d <= max_d):
// a Cholesky factor and the derived per-axis vectors
constexpr size_t host_scratch_doubles(size_t max_d) { return max_d * max_d + 8 * max_d; }

DevLayout make_dev_layout(const Resolved& R, const Layout& L, int grid) {
  DevLayout D;
  const size_t A = 256;
  size_t s = 0;
  auto take = [&](size_t bytes) {
    size_t at = s;
    s = align_up(s + bytes, A);
    return at;
  };
  D.o_jobs = take(sizeof(JobDesc) * R.max_jobs);
  D.o_params = take(sizeof(double) * R.max_params);
  D.o_order = take(sizeof(int) * R.max_jobs);
  D.o_first = take(sizeof(int) * R.o.max_batch);
  D.o_count = take(sizeof(int) * R.o.max_batch);
  D.o_hstatus = take(sizeof(int) * R.o.max_batch);
  const bool two = R.o.method == TT_METHOD_TWO_TRAINS;
  D.o_pairs = take(two ? sizeof(int2) * (size_t)R.max_jobs / 2 : 0);
  D.o_host = take(sizeof(double) * host_scratch_doubles((size_t)R.o.max_d));
  D.o_disc = take(sizeof(double) * R.o.max_batch);
  D.pstride = ttp::pivot_record_entries(R.o.max_d, R.o.max_rank);
  D.o_warm = take(R.o.pivot_io ? sizeof(uint16_t) * D.pstride * (size_t)R.max_jobs : 0);
  D.stage_bytes = s;
  size_t off = 0;
  auto take2 = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes, A);
    return at;
  };
  D.stage = take2(D.stage_bytes);
  D.jres = take2(sizeof(JobResult) * R.max_jobs);
  D.ires = take2(sizeof(InstanceResult) * R.o.max_batch);
  D.counter = take2(sizeof(int) * 4);
  D.scratch = take2(L.stride * (size_t)grid);
  // two-train form: every factor train's skeleton records, one per core
  D.emit_stride = two ? align_up(ttp::emit_core_bytes(L.rmax, L.dmax) * L.dmax, A) : 0;
  D.emit = take2(D.emit_stride * (two ? (size_t)R.max_jobs : 0));
  D.pivots = take2(R.o.pivot_io ? sizeof(uint16_t) * D.pstride * (size_t)R.max_jobs : 0);
  D.total = off;
  return D;
}

// Dynamic shared memory above 48 KB needs a per-kernel opt-in, which is a
// process-wide setting of the current device, shared by every pricer (and the
// allocation-free entry point) that launches that kernel.  Pricers of different
// sizes need different amounts, so the opt-in only ever rises: each launch path
// raises it to at least its own need before it launches or replays a graph, and
// a smaller pricer created later never lowers it under a larger one.
constexpr int kMaxDevices = 64;
std::mutex g_smem_mutex;

template <typename K>
cudaError_t raise_smem_optin(K* kernel, int* high, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_smem_mutex);
  if (bytes <= high[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) high[dev] = bytes;
  return e;
}

template <typename R, bool TC>
cudaError_t cross_smem_optin(int bytes) {
  static int high[kMaxDevices];
  return raise_smem_optin(ttp::tt_cross_kernel<R, TC>, high, bytes);
}

cudaError_t bracket_smem_optin(int bytes) {
  static int high[kMaxDevices];
  return raise_smem_optin(ttp::bracket_kernel<double>, high, bytes);
}

// shared-memory opt-in and blocks per SM for one instantiation of the kernel
template <typename R, bool TC>
cudaError_t kernel_occupancy(const SmemLayout& S, int* per_sm, cudaFuncAttributes* fa) {
  cudaError_t e = cross_smem_optin<R, TC>(S.total);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ttp::tt_cross_kernel<R, TC>, ttp::kThreads, S.total);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(fa, ttp::tt_cross_kernel<R, TC>);
  return e;
}

int grid_for(const tt_options& o, const SmemLayout& S, int* grid_out) {
  int dev_sms = 0;
  if (cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess)
    return TT_ERR_CUDA;
  int per_sm = 0;
  cudaFuncAttributes fa;
  const bool tcore = o.engine == TT_ENGINE_TENSOR_CORES;
  cudaError_t e = o.precision == TT_FP64 ? kernel_occupancy<double, false>(S, &per_sm, &fa)
                  : tcore                ? kernel_occupancy<float, true>(S, &per_sm, &fa)
                                         : kernel_occupancy<float, false>(S, &per_sm, &fa);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  if (tcore) {
    // The occupancy query answers 1 block per SM for this kernel once it holds
    // tensor memory, although 3 x 128 of the SM's 512 TMEM columns are free for
    // it; residency here is set by registers, shared memory and TMEM columns,
    // counted directly.  (A CTA that finds no free slot starts when one ends and
    // finds the job queue empty, so an over-count costs nothing.)
    int smem_sm = 0, regs_sm = 0;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, o.device) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, o.device) == cudaSuccess) {
      const int by_smem = smem_sm / (S.total + (int)fa.sharedSizeBytes + 1024);
      const int by_regs = regs_sm / std::max(1, fa.numRegs * ttp::kThreads);
      const int by_tmem = 512 / (int)ttp::tc::tmem_cols(o.max_rank);
      per_sm = std::max(per_sm, std::min(std::min(by_smem, by_regs), by_tmem));
    } else {
      cudaGetLastError();
    }
  }
  if (per_sm < 1) return TT_ERR_CAPACITY;
  *grid_out = dev_sms * per_sm;
  return TT_OK;
}

// ---- per-problem validation and derivation (FP64, host) ----
bool finite_all(const double* p, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// FP64 Cholesky test of a symmetric matrix (the paper assumes a positive
// definite covariance, Section II.A); l: d*d doubles of scratch
bool cholesky_ok(const double* c, int d, double* l) {
  for (int i = 0; i < d * d; ++i) l[i] = 0.0;
  double scale = 0.0;
  for (int i = 0; i < d * d; ++i) scale = std::max(scale, std::fabs(c[i]));
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(c[i * d + j] - c[j * d + i]) > 1e-12 * scale) return false;
  for (int j = 0; j < d; ++j) {
    double s = c[j * d + j];
    for (int k = 0; k < j; ++k) s -= l[j * d + k] * l[j * d + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    l[j * d + j] = ljj;
    for (int i = j + 1; i < d; ++i) {
      double t = c[i * d + j];
      for (int k = 0; k < j; ++k) t -= l[i * d + k] * l[j * d + k];
      l[i * d + j] = t / ljj;
    }
  }
  return true;
}

}  // namespace

struct tt_pricer {
  Resolved R;
  Layout lay;
  SmemLayout sml;
  DevLayout dl;
  int grid;
  cudaStream_t stream;
  bool own_ws;
  char* ws;
  char* h_stage;           // pinned, capacity layout, filled by validation
  char* h_pack;            // pinned, packed copy that is sent to the device
  InstanceResult* h_ires;  // pinned
  int count, njobs, npairs;
  size_t p_jobs, p_params, p_order, p_first, p_count, p_hstatus, p_pairs, p_warm, p_bytes;  // packed offsets
  ttp::BrSmem bsm;  // two-train form: the bracket kernel's shared-memory carve
  int bgrid;
  size_t last_h2d, last_d2h;
  // graph replay (options.graph): the capture stream, ordering events, the
  // instantiated graph and the batch layout it was captured for
  cudaStream_t cap;
  cudaEvent_t ev_in, ev_out;
  cudaGraphExec_t gexec;
  size_t gkey[8];
};

namespace {

// Validation of one problem (FP64, host); `scr` holds d*d doubles.  Returns
// TT_OK or the problem's status.
// Entries of a warm-start record for d assets and `terms` trains, or -1 when it
// is malformed: counts above the rank cap, indices outside the grid, repeated
// multi-indices within a bond.
long long warm_record_entries(const unsigned short* w, int d, int terms, int rank, int n) {
  long long off = 0;
  for (int t = 0; t < terms; ++t)
    for (int k = 1; k < d; ++k) {
      const int c = w[off], wd = d - k;
      if (c > rank) return -1;
      const unsigned short* e = w + off + 1;
      for (int i = 0; i < c * wd; ++i)
        if (e[i] >= n) return -1;
      for (int a = 0; a < c; ++a)
        for (int b = 0; b < a; ++b)
          if (std::memcmp(e + a * wd, e + b * wd, sizeof(unsigned short) * wd) == 0) return -1;
      off += 1 + (long long)c * wd;
    }
  return off;
}

int validate_problem(const tt_problem& p, const tt_options& o, double* scr) {
  const int d = p.d;
  if (o.method == TT_METHOD_TWO_TRAINS) {  // the phi train's bond dimension, and the bracket's E
    const int rphi = p.max_rank_phi > 0 ? p.max_rank_phi : p.max_rank;
    if (p.max_rank_phi < 0) return TT_ERR_INVALID;
    if (rphi > o.max_rank || (long long)p.max_rank * rphi > 1024) return TT_ERR_CAPACITY;
  }
  if (d < 1 || d > o.max_d || p.n_grid < 2 || p.n_grid > o.max_n || p.max_rank < 1 || p.max_rank > o.max_rank ||
      !p.spot || !p.cov || !p.damping || (p.payoff != TT_MIN_CALL && p.payoff != TT_MAX_CALL))
    return (d > o.max_d || p.n_grid > o.max_n || p.max_rank > o.max_rank) ? TT_ERR_CAPACITY : TT_ERR_INVALID;
  if (!(p.trunc_L > 0) || !std::isfinite(p.trunc_L) || !(p.maturity > 0) || !std::isfinite(p.maturity) ||
      !(p.strike > 0) || !std::isfinite(p.strike) || !std::isfinite(p.rate) || !finite_all(p.spot, d) ||
      !finite_all(p.cov, d * d) || !finite_all(p.damping, d))
    return TT_ERR_INVALID;
  for (int j = 0; j < d; ++j)
    if (!(p.spot[j] > 0)) return TT_ERR_INVALID;
  if (!cholesky_ok(p.cov, d, scr)) return TT_ERR_NOT_PD;
  if (p.warm_sets) {  // warm starts: single-train form with pivot_io, a well-formed record
    if (!o.pivot_io || o.method != TT_METHOD_SINGLE_TRAIN) return TT_ERR_INVALID;
    if (warm_record_entries(p.warm_sets, d, p.payoff == TT_MIN_CALL ? 1 : d, p.max_rank, p.n_grid) < 0)
      return TT_ERR_INVALID;
  }
  if (p.payoff == TT_MIN_CALL) {
    double sd = 0.0;
    int stv = TT_OK;
    for (int j = 0; j < d; ++j) {
      if (!(-p.damping[j] > 0)) stv = TT_ERR_STRIP;
      sd += -p.damping[j];
    }
    if (!(sd > 1.0)) stv = TT_ERR_STRIP;
    return stv;
  }
  for (int j = 0; j < d; ++j)
    if (!(std::fabs(p.damping[j]) > 0)) return TT_ERR_STRIP;
  return TT_OK;
}

// Per-train derivation (Section III.C): covariance of the train's variables,
// shifts delta, linear phase coefficients, log prefactor, sign and weight.
// Writes the problem's jobs at jobs[nj..] and their parameter blocks at
// params[poff..]; `scr` holds 8 d doubles.  No heap memory.
// The rank threshold and block height of a problem: its class's (first match),
// else the options'.
void problem_knobs(const Resolved& R, const tt_problem& p, double* theta, int* block_rows) {
  *theta = R.o.rank_tol;
  *block_rows = R.o.block_rows;
  for (int c = 0; c < R.n_classes; ++c) {
    const tt_class_tuning& t = R.classes[c];
    if (p.d < t.d_min || p.d > t.d_max || (t.n_grid && t.n_grid != p.n_grid) ||
        (t.max_rank && t.max_rank != p.max_rank) || (t.payoff >= 0 && t.payoff != p.payoff))
      continue;
    if (t.rank_tol > 0) *theta = t.rank_tol;
    if (t.block_rows >= p.max_rank && t.block_rows > 0) *block_rows = t.block_rows;
    return;
  }
}

void derive_trains(const Resolved& R, const tt_problem& p, int i, bool two, JobDesc* jobs, double* params,
                   int2* pairs, int& nj, int& np, size_t& poff, int* cnt, double* scr) {
  const int d = p.d;
  double theta = 0.0;
  int brows = 0;
  problem_knobs(R, p, &theta, &brows);
  const double T = p.maturity, K = p.strike, lk = std::log(K);
  const int N = p.n_grid;
  const double eta = 2.0 * p.trunc_L / N;
  const double weight = std::exp(-p.rate * T) * std::pow(eta / (2.0 * M_PI), d);
  double cap = 0.0;  // a call on the minimum or maximum is worth less than the sum of the spots
  for (int j = 0; j < d; ++j) cap += p.spot[j];
  double* m = scr;
  for (int j = 0; j < d; ++j) m[j] = std::log(p.spot[j] / K) + (p.rate - 0.5 * p.cov[j * d + j]) * T;
  const int terms = p.payoff == TT_MIN_CALL ? 1 : d;
  auto base_job = [&](int term) {
    JobDesc jd;
    std::memset(&jd, 0, sizeof(jd));
    jd.d = d;
    jd.n = N;
    jd.rmax = p.max_rank;
    jd.instance = i;
    jd.term = term;
    jd.param_off = (int)poff;
    jd.seed = p.seed;
    jd.T = T;
    jd.Tq = T;
    jd.L = p.trunc_L;
    jd.weight = weight;
    jd.cap = cap;
    jd.theta = theta;
    jd.block_rows = brows;
    return jd;
  };
  // covariance of max-call term j0's variables y_j0 = x_j0, y_l = x_l - x_j0: A Cov A^T
  auto term_cov = [&](int j0, double* cv) {
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double v = p.cov[a * d + b];
        if (a != j0) v -= p.cov[j0 * d + b];
        if (b != j0) v -= p.cov[a * d + j0];
        if (a != j0 && b != j0) v += p.cov[j0 * d + j0];
        cv[a * d + b] = v;
      }
  };
  if (two) {
    // Two-train form (Eq. braket): per term a payoff-transform train and a
    // characteristic-function train, in the term's variables.  With mu_t the
    // term's mean log-price vector, s the strike's direction (all ones for the
    // min-call, e_j for max-call term j), delta the shift and C the covariance:
    //   phi_T(-z) = exp(delta.mu_t + T/2 delta^T C delta) exp(-T/2 u^T C u)
    //               * exp(-i u.(mu_t + T C delta)),
    //   vhat(z)   = K^(1 - s.delta) e^{i ln K s.u} * (rational factors: 1/(i z_l),
    //               1/((i z_j)(1 + i z_j)), and the min-call's 1/(1 + i sum z)).
    const bool mn = p.payoff == TT_MIN_CALL;
    double* dlv = m + d;
    double* kdv = dlv + d;
    double* mut = kdv + d;
    double* sv = mut + d;
    double* cd = sv + d;
    for (int term = 0; term < terms; ++term) {
      const int j0 = term;
      // the term's covariance goes straight into the first factor's block
      double* cv0 = params + poff;
      if (mn) {
        std::memcpy(cv0, p.cov, sizeof(double) * d * d);
      } else {
        term_cov(j0, cv0);
      }
      for (int l = 0; l < d; ++l) {
        if (mn) {
          dlv[l] = -p.damping[l];
          kdv[l] = 0.0;
          mut[l] = m[l] + lk;
          sv[l] = 1.0;
        } else {
          dlv[l] = l == j0 ? 1.0 + std::fabs(p.damping[l]) : -std::fabs(p.damping[l]);
          kdv[l] = l == j0 ? 1.0 : 0.0;
          mut[l] = l == j0 ? m[j0] + lk : m[l] - m[j0];
          sv[l] = l == j0 ? 1.0 : 0.0;
        }
      }
      double quad = 0.0, sdl = 0.0, dmu = 0.0;
      for (int l = 0; l < d; ++l) {
        double c = 0.0;
        for (int q = 0; q < d; ++q) c += cv0[(size_t)l * d + q] * dlv[q];
        cd[l] = c;
        quad += dlv[l] * c;
        sdl += dlv[l] * sv[l];
        dmu += dlv[l] * mut[l];
      }
      pairs[np].x = nj;
      pairs[np].y = nj + 1;
      ++np;
      for (int fi = 0; fi < 2; ++fi) {
        const bool vh = fi == 0;
        JobDesc jd = base_job(term);
        jd.factor = vh ? ttp::FACTOR_VHAT : ttp::FACTOR_PHI;
        if (!vh && p.max_rank_phi > 0) jd.rmax = p.max_rank_phi;  // D_phi
        jd.Tq = vh ? 0.0 : T;
        double* cv = params + poff;
        double* dl = cv + (size_t)d * d;
        double* pc = dl + d;
        double* kd = pc + d;
        poff += (size_t)d * d + 3 * (size_t)d;
        if (cv != cv0) std::memcpy(cv, cv0, sizeof(double) * d * d);
        for (int l = 0; l < d; ++l) {
          dl[l] = dlv[l];
          pc[l] = vh ? -lk * sv[l] : mut[l] + T * cd[l];
          kd[l] = vh ? kdv[l] : 2.0;
        }
        jd.cauchy = vh && mn ? 1 : 0;
        jd.D0 = vh && mn ? 1.0 - sdl : 0.0;
        jd.logscale = vh ? lk * (1.0 - sdl) : dmu + 0.5 * T * quad;
        jd.sign = vh && mn && d % 2 == 0 ? -1.0 : 1.0;  // (-1)^(d+1) on the min-call's transform
        jobs[nj++] = jd;
        ++cnt[i];
      }
    }
    return;
  }
  for (int term = 0; term < terms; ++term) {
    JobDesc jd = base_job(term);
    double* cv = params + poff;
    double* dl = cv + (size_t)d * d;
    double* pc = dl + d;
    double* kd = pc + d;
    poff += (size_t)d * d + 3 * (size_t)d;
    if (p.payoff == TT_MIN_CALL) {
      std::memcpy(cv, p.cov, sizeof(double) * d * d);
      double sd = 0.0, dm = 0.0, quad = 0.0;
      for (int j = 0; j < d; ++j) {
        dl[j] = -p.damping[j];
        sd += dl[j];
        dm += dl[j] * m[j];
        kd[j] = 0.0;
      }
      for (int j = 0; j < d; ++j) {
        double c = 0.0;
        for (int l = 0; l < d; ++l) c += p.cov[j * d + l] * dl[l];
        pc[j] = m[j] + T * c;
        quad += dl[j] * c;
      }
      jd.cauchy = 1;
      jd.D0 = 1.0 - sd;
      jd.logscale = lk + dm + 0.5 * T * quad;
      jd.sign = (d % 2 == 1) ? 1.0 : -1.0;  // (-1)^(d+1)
    } else {
      // term `term`: y_term = x_term, y_l = x_l - x_term; C' = A Cov A^T
      const int j0 = term;
      term_cov(j0, cv);
      double lsc = lk, quad = 0.0;
      for (int l = 0; l < d; ++l) {
        dl[l] = l == j0 ? 1.0 + std::fabs(p.damping[l]) : -std::fabs(p.damping[l]);
        kd[l] = l == j0 ? 1.0 : 0.0;
      }
      for (int l = 0; l < d; ++l) {
        const double mp = l == j0 ? m[j0] : m[l] - m[j0];
        double c = 0.0;
        for (int q = 0; q < d; ++q) c += cv[l * d + q] * dl[q];
        pc[l] = mp + T * c;
        lsc += dl[l] * mp;
        quad += dl[l] * c;
      }
      jd.cauchy = 0;
      jd.D0 = 0.0;
      jd.logscale = lsc + 0.5 * T * quad;
      jd.sign = 1.0;
    }
    jobs[nj++] = jd;
    ++cnt[i];
  }
}

// Relative discretisation error of the midpoint grid (Eq. discr) by the
// Poisson-summation model: axis j aliases at rate a_j (delta_j for the call on
// the minimum; |alpha_j| for the maximum, on its maximum's axis delta - 1) with
// a relative term exp(-2 pi a_j / eta), and the cut Gaussian tail adds
// exp(-T sigma_j^2 L^2 / 2).  Multiplied by the price at the end.
double disc_factor(const tt_problem& p) {
  const double eta = 2.0 * p.trunc_L / p.n_grid;
  double f = 0.0;
  for (int j = 0; j < p.d; ++j) {
    const double a = p.payoff == TT_MIN_CALL ? -p.damping[j] : std::fabs(p.damping[j]);
    f += std::exp(-2.0 * M_PI * a / eta);
    f += std::exp(-0.5 * p.maturity * p.cov[j * p.d + j] * p.trunc_L * p.trunc_L);
  }
  return f;
}

// Queue cost of a job (largest first): its fiber work d N r^2.
double job_cost(const JobDesc& q) {
  return (double)std::max(q.d - 1, 1) * q.n * (double)q.rmax * q.rmax * (q.d > 1 ? 1.0 : 0.01);
}

// A1 of the hot path: validate every problem, derive its trains into the
// handle's host stage, order the jobs by cost, pack the used parts and make one
// host-to-device copy.  Heap-free (the allocation-free entry point runs it on
// its fixed arrays too).
int prepare_impl(tt_pricer* h, const tt_problem* probs, int count) {
  const tt_options& o = h->R.o;
  if (count < 0 || count > o.max_batch || (count > 0 && !probs)) return TT_ERR_INVALID;
  char* st = h->h_stage;
  JobDesc* jobs = reinterpret_cast<JobDesc*>(st + h->dl.o_jobs);
  double* params = reinterpret_cast<double*>(st + h->dl.o_params);
  int* order = reinterpret_cast<int*>(st + h->dl.o_order);
  int* first = reinterpret_cast<int*>(st + h->dl.o_first);
  int* cnt = reinterpret_cast<int*>(st + h->dl.o_count);
  int* hstat = reinterpret_cast<int*>(st + h->dl.o_hstatus);
  int2* pairs = reinterpret_cast<int2*>(st + h->dl.o_pairs);
  double* scr = reinterpret_cast<double*>(st + h->dl.o_host);
  double* disc = reinterpret_cast<double*>(st + h->dl.o_disc);
  uint16_t* warm = reinterpret_cast<uint16_t*>(st + h->dl.o_warm);
  size_t wused = 0;
  const bool two = o.method == TT_METHOD_TWO_TRAINS;
  int nj = 0, np = 0;
  size_t poff = 0;
  for (int i = 0; i < count; ++i) {
    first[i] = nj;
    cnt[i] = 0;
    hstat[i] = validate_problem(probs[i], o, scr);
    disc[i] = std::nan("");
    if (hstat[i] == TT_OK) {
      const int j0 = nj;
      derive_trains(h->R, probs[i], i, two, jobs, params, pairs, nj, np, poff, cnt, scr);
      disc[i] = disc_factor(probs[i]);
      for (int j = j0; j < nj; ++j) jobs[j].warm_off = -1;
      if (probs[i].warm_sets) {  // validated: one record per train, each job its own copy
        const tt_problem& p = probs[i];
        const unsigned short* w = p.warm_sets;
        for (int j = j0; j < nj; ++j) {
          const long long len = warm_record_entries(w, p.d, 1, p.max_rank, p.n_grid);
          std::memcpy(warm + (size_t)wused, w, sizeof(uint16_t) * len);
          jobs[j].warm_off = (int)wused;
          wused += len;
          w += len;
        }
      }
    }
  }
  // largest jobs first, ties by job number (std::sort works in place)
  for (int j = 0; j < nj; ++j) order[j] = j;
  std::sort(order, order + nj, [&](int a, int b) {
    const double ca = job_cost(jobs[a]), cb = job_cost(jobs[b]);
    return ca != cb ? ca > cb : a < b;
  });
  h->count = count;
  h->njobs = nj;
  h->npairs = np;
  // pack the used parts into one contiguous block: one host-to-device copy
  size_t off = 0;
  auto put = [&](size_t src_off, size_t bytes) {
    const size_t at = off;
    if (bytes) std::memcpy(h->h_pack + at, h->h_stage + src_off, bytes);
    off = align_up(off + bytes, 16);
    return at;
  };
  h->p_jobs = put(h->dl.o_jobs, sizeof(JobDesc) * nj);
  h->p_params = put(h->dl.o_params, sizeof(double) * poff);
  h->p_order = put(h->dl.o_order, sizeof(int) * nj);
  h->p_first = put(h->dl.o_first, sizeof(int) * count);
  h->p_count = put(h->dl.o_count, sizeof(int) * count);
  h->p_hstatus = put(h->dl.o_hstatus, sizeof(int) * count);
  h->p_pairs = put(h->dl.o_pairs, sizeof(int2) * np);
  h->p_warm = put(h->dl.o_warm, sizeof(uint16_t) * wused);
  h->p_bytes = off;
  h->last_h2d = off;
  if (off && cudaMemcpyAsync(h->ws + h->dl.stage, h->h_pack, off, cudaMemcpyHostToDevice,
                             h->stream) != cudaSuccess)
    return TT_ERR_CUDA;
  return TT_OK;
}

int launch_all(tt_pricer* h, cudaStream_t stream) {
  char* st = h->ws + h->dl.stage;
  const JobDesc* jobs = reinterpret_cast<const JobDesc*>(st + h->p_jobs);
  const double* params = reinterpret_cast<const double*>(st + h->p_params);
  const int* order = reinterpret_cast<const int*>(st + h->p_order);
  const int* first = reinterpret_cast<const int*>(st + h->p_first);
  const int* cnt = reinterpret_cast<const int*>(st + h->p_count);
  const int* hstat = reinterpret_cast<const int*>(st + h->p_hstatus);
  int* counter = reinterpret_cast<int*>(h->ws + h->dl.counter);
  JobResult* jres = reinterpret_cast<JobResult*>(h->ws + h->dl.jres);
  InstanceResult* ires = reinterpret_cast<InstanceResult*>(h->ws + h->dl.ires);
  char* scratch = h->ws + h->dl.scratch;
  if (cudaMemsetAsync(counter, 0, 2 * sizeof(int), stream) != cudaSuccess) return TT_ERR_CUDA;
  char* emit = h->ws + h->dl.emit;
  const size_t es = h->dl.emit_stride;
  // pivot records (tt_options.pivot_io): warm starts in, final right sets out
  const uint16_t* warm = h->R.o.pivot_io ? reinterpret_cast<const uint16_t*>(st + h->p_warm) : nullptr;
  uint16_t* pout = h->R.o.pivot_io ? reinterpret_cast<uint16_t*>(h->ws + h->dl.pivots) : nullptr;
  if (h->njobs > 0) {
    const int grid = std::min(h->grid, h->njobs);
    if (h->R.o.precision == TT_FP64)
      ttp::tt_cross_kernel<double, false><<<grid, ttp::kThreads, h->sml.total, stream>>>(
          jobs, params, order, h->njobs, counter, jres, scratch, h->lay, h->sml, h->R.kn, emit, es, warm, pout,
          (int)h->dl.pstride);
    else if (h->R.o.engine == TT_ENGINE_TENSOR_CORES)
      ttp::tt_cross_kernel<float, true><<<grid, ttp::kThreads, h->sml.total, stream>>>(
          jobs, params, order, h->njobs, counter, jres, scratch, h->lay, h->sml, h->R.kn, emit, es, warm, pout,
          (int)h->dl.pstride);
    else
      ttp::tt_cross_kernel<float, false><<<grid, ttp::kThreads, h->sml.total, stream>>>(
          jobs, params, order, h->njobs, counter, jres, scratch, h->lay, h->sml, h->R.kn, emit, es, warm, pout,
          (int)h->dl.pstride);
    if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  }
  if (h->npairs > 0) {  // two-train form: the brackets, two scratch blocks per CTA
    const int2* pairs = reinterpret_cast<const int2*>(st + h->p_pairs);
    const int bg = std::min(h->bgrid, h->npairs);
    // FP64 in both paths: in the mixed path the FP32 crosses choose the index sets,
    // and the cores G = A P^{-1} are formed from FP64 integrand values (P can be
    // conditioned up to 1/rank_tol, which FP32 values would turn into 1e-3 errors)
    ttp::bracket_kernel<double><<<bg, ttp::kThreads, h->bsm.total, stream>>>(
        jobs, params, pairs, h->npairs, emit, es, counter + 1, jres, scratch, h->lay, h->bsm);
    if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  }
  if (h->count > 0) {
    ttp::finalize_kernel<<<(h->count + 127) / 128, 128, 0, stream>>>(jobs, jres, first, cnt, hstat,
                                                                          h->count, ires);
    if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  }
  return TT_OK;
}

// the shared-memory opt-in of every kernel this pricer launches (see raise_smem_optin)
int ensure_smem_optin(const tt_pricer* h) {
  cudaError_t e = h->R.o.precision == TT_FP64 ? cross_smem_optin<double, false>(h->sml.total)
                  : h->R.o.engine == TT_ENGINE_TENSOR_CORES ? cross_smem_optin<float, true>(h->sml.total)
                                                            : cross_smem_optin<float, false>(h->sml.total);
  if (e == cudaSuccess && h->R.o.method == TT_METHOD_TWO_TRAINS) e = bracket_smem_optin(h->bsm.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  return TT_OK;
}

// graph replay: re-captured whenever the batch layout (job and problem counts,
// packed offsets) differs from the captured one
int run_impl(tt_pricer* h) {
  // before any launch, capture or replay (no attribute call inside a capture)
  const int orc = ensure_smem_optin(h);
  if (orc != TT_OK) return orc;
  if (!h->R.o.graph) return launch_all(h, h->stream);
  const size_t key[8] = {(size_t)h->njobs, (size_t)h->count, h->p_jobs, h->p_params,
                         h->p_order, h->p_first, h->p_count, h->p_hstatus ^ (h->p_pairs << 32) ^ (size_t)h->npairs};
  if (!h->gexec || std::memcmp(key, h->gkey, sizeof(key)) != 0) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TT_ERR_CUDA;
    const int rc = launch_all(h, h->cap);
    const cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (rc != TT_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return TT_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->gexec = nullptr;
      cudaGetLastError();
      return TT_ERR_CUDA;
    }
    std::memcpy(h->gkey, key, sizeof(key));
  }
  if (cudaEventRecord(h->ev_in, h->stream) != cudaSuccess || cudaStreamWaitEvent(h->cap, h->ev_in, 0) != cudaSuccess ||
      cudaGraphLaunch(h->gexec, h->cap) != cudaSuccess || cudaEventRecord(h->ev_out, h->cap) != cudaSuccess ||
      cudaStreamWaitEvent(h->stream, h->ev_out, 0) != cudaSuccess)
    return TT_ERR_CUDA;
  return TT_OK;
}

int results_impl(tt_pricer* h, double* prices, tt_diag* diag) {
  if (h->count > 0 && !prices) return TT_ERR_INVALID;
  h->last_d2h = sizeof(InstanceResult) * (size_t)h->count;
  if (h->count > 0) {
    if (cudaMemcpyAsync(h->h_ires, h->ws + h->dl.ires, h->last_d2h, cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
      return TT_ERR_CUDA;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return TT_ERR_CUDA;
  int worst_err = 0, worst_warn = 0;
  for (int i = 0; i < h->count; ++i) {
    const InstanceResult& r = h->h_ires[i];
    prices[i] = r.price;
    if (diag) {
      diag[i].status = r.status;
      diag[i].half_sweeps = r.half_sweeps;
      diag[i].final_rank_max = r.max_rank;
      diag[i].terms = r.terms;
      diag[i].evaluations = r.evaluations;
      diag[i].maxvol_swaps = r.swaps;
      diag[i].block_visits = r.visits;
      diag[i].fail_step = r.fail_step;
      diag[i].maxvol_rollbacks = r.rollbacks;
      diag[i].imag_part = r.imag;
      diag[i].flops = r.flops;
      diag[i].est_discretization_err =
          std::fabs(r.price) * reinterpret_cast<const double*>(h->h_stage + h->dl.o_disc)[i];
    }
    if (r.status < 0 && (worst_err == 0 || r.status < worst_err)) worst_err = r.status;
    if (r.status > worst_warn) worst_warn = r.status;
  }
  return worst_err != 0 ? worst_err : worst_warn;
}

}  // namespace

extern "C" {

size_t tt_workspace_bytes(const tt_options* opt) {
  Resolved R;
  if (!resolve(opt, &R)) return 0;
  const bool f64 = R.o.precision == TT_FP64;
  SmemLayout S = make_smem(R.o, f64);
  if (S.total > 227 * 1024) return 0;
  int grid = 0;
  if (cudaSetDevice(R.o.device) != cudaSuccess) return 0;
  if (grid_for(R.o, S, &grid) != TT_OK) return 0;
  Layout L = make_layout(R.o, f64 || R.o.method == TT_METHOD_TWO_TRAINS);
  return make_dev_layout(R, L, grid).total;
}

int tt_price_create(const tt_options* opt, tt_pricer** out) {
  if (!out) return TT_ERR_INVALID;
  *out = nullptr;
  Resolved R;
  if (!resolve(opt, &R)) return TT_ERR_INVALID;
  const bool f64 = R.o.precision == TT_FP64;
  SmemLayout S = make_smem(R.o, f64);
  if (S.total > 227 * 1024) return TT_ERR_CAPACITY;
  if (cudaSetDevice(R.o.device) != cudaSuccess) return TT_ERR_CUDA;
  int grid = 0;
  int rc = grid_for(R.o, S, &grid);
  if (rc != TT_OK) return rc;
  tt_pricer* h = new (std::nothrow) tt_pricer();
  if (!h) return TT_ERR_INVALID;
  h->R = R;
  h->lay = make_layout(R.o, f64 || R.o.method == TT_METHOD_TWO_TRAINS);  // the bracket runs in FP64
  h->sml = S;
  h->grid = grid;
  h->npairs = 0;
  h->bgrid = 0;
  h->bsm = ttp::BrSmem{};
  if (R.o.method == TT_METHOD_TWO_TRAINS) {
    h->bsm = make_brsmem(R.o, true);
    const cudaError_t e = bracket_smem_optin(h->bsm.total);
    if (h->bsm.total > 227 * 1024 || e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return TT_ERR_CAPACITY;
    }
    // every CTA resident (they share the queue); two scratch blocks each
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ttp::bracket_kernel<double>, ttp::kThreads,
                                                      h->bsm.total) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, R.o.device) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
      sms = grid / 2;
    }
    h->bgrid = std::max(1, std::min(grid / 2, std::max(1, per_sm) * sms));
  }
  h->dl = make_dev_layout(R, h->lay, grid);
  h->stream = reinterpret_cast<cudaStream_t>(R.o.cuda_stream);
  h->count = 0;
  h->njobs = 0;
  if (R.o.workspace) {
    if (R.o.workspace_bytes < h->dl.total || (reinterpret_cast<uintptr_t>(R.o.workspace) & 255u)) {
      delete h;
      return TT_ERR_CAPACITY;
    }
    h->ws = reinterpret_cast<char*>(R.o.workspace);
    h->own_ws = false;
  } else {
    if (cudaMalloc(&h->ws, h->dl.total) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return TT_ERR_CUDA;
    }
    h->own_ws = true;
  }
  h->h_stage = nullptr;
  h->h_pack = nullptr;
  h->h_ires = nullptr;
  h->p_jobs = h->p_params = h->p_order = h->p_first = h->p_count = h->p_hstatus = h->p_pairs = h->p_warm =
      h->p_bytes = 0;
  h->last_h2d = h->last_d2h = 0;
  h->cap = nullptr;
  h->ev_in = h->ev_out = nullptr;
  h->gexec = nullptr;
  std::memset(h->gkey, 0, sizeof(h->gkey));
  if (R.o.graph && (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    tt_price_destroy(h);
    return TT_ERR_CUDA;
  }
  if (cudaMallocHost(&h->h_stage, h->dl.stage_bytes) != cudaSuccess ||
      cudaMallocHost(&h->h_pack, h->dl.stage_bytes) != cudaSuccess ||
      cudaMallocHost(&h->h_ires, sizeof(InstanceResult) * R.o.max_batch) != cudaSuccess) {
    cudaGetLastError();
    tt_price_destroy(h);
    return TT_ERR_CUDA;
  }
  std::memset(h->h_stage, 0, h->dl.stage_bytes);
  *out = h;
  return TT_OK;
}

int tt_price_prepare(tt_pricer* h, const tt_problem* probs, int count) {
  if (!h) return TT_ERR_INVALID;
  if (cudaSetDevice(h->R.o.device) != cudaSuccess) return TT_ERR_CUDA;
  return prepare_impl(h, probs, count);
}

int tt_price_run(tt_pricer* h) {
  if (!h) return TT_ERR_INVALID;
  if (cudaSetDevice(h->R.o.device) != cudaSuccess) return TT_ERR_CUDA;
  return run_impl(h);
}

int tt_price_results(tt_pricer* h, double* prices, tt_diag* diag) {
  if (!h) return TT_ERR_INVALID;
  if (cudaSetDevice(h->R.o.device) != cudaSuccess) return TT_ERR_CUDA;
  return results_impl(h, prices, diag);
}

int tt_price_evaluate(tt_pricer* h, const tt_problem* probs, int count, double* prices,
                      tt_diag* diag) {
  if (!h) return TT_ERR_INVALID;
  int rc = tt_price_prepare(h, probs, count);
  if (rc != TT_OK) return rc;
  rc = tt_price_run(h);
  if (rc != TT_OK) return rc;
  return tt_price_results(h, prices, diag);
}

void tt_price_destroy(tt_pricer* h) {
  if (!h) return;
  cudaSetDevice(h->R.o.device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->cap) cudaStreamSynchronize(h->cap);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  if (h->h_pack) cudaFreeHost(h->h_pack);
  if (h->h_ires) cudaFreeHost(h->h_ires);
  delete h;
}

int tt_price_transfer_bytes(const tt_pricer* h, size_t* h2d, size_t* d2h) {
  if (!h) return TT_ERR_INVALID;
  if (h2d) *h2d = h->last_h2d;
  if (d2h) *d2h = h->last_d2h;
  return TT_OK;
}

size_t tt_pivot_record_entries(int max_d, int max_rank) {
  if (max_d < 1 || max_rank < 1) return 0;
  return ttp::pivot_record_entries(max_d, max_rank);
}

int tt_price_pivots(tt_pricer* h, int problem, unsigned short* out, size_t cap) {
  if (!h || !out || problem < 0 || problem >= h->count) return TT_ERR_INVALID;
  if (!h->R.o.pivot_io) return TT_ERR_INVALID;
  if (cudaSetDevice(h->R.o.device) != cudaSuccess) return TT_ERR_CUDA;
  const char* st = h->h_stage;
  const int first = reinterpret_cast<const int*>(st + h->dl.o_first)[problem];
  const int cnt = reinterpret_cast<const int*>(st + h->dl.o_count)[problem];
  const JobDesc* jobs = reinterpret_cast<const JobDesc*>(st + h->dl.o_jobs);
  size_t used = 0;
  for (int j = first; j < first + cnt; ++j) {
    // the record's length follows from its counts; fetch the whole stride
    const size_t stride = h->dl.pstride;
    if (used + stride > cap && used + 1 > cap) return TT_ERR_CAPACITY;
    uint16_t* dst = reinterpret_cast<uint16_t*>(out + used);
    const size_t n = std::min(stride, cap - used);
    if (cudaMemcpyAsync(dst, h->ws + h->dl.pivots + sizeof(uint16_t) * stride * (size_t)j, sizeof(uint16_t) * n,
                        cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return TT_ERR_CUDA;
    size_t len = 0;
    const int d = jobs[j].d;
    for (int k = 1; k < d; ++k) {
      if (len >= n) return TT_ERR_CAPACITY;
      len += 1 + (size_t)dst[len] * (d - k);
    }
    if (len > n) return TT_ERR_CAPACITY;
    used += len;
  }
  return (int)used;
}

const char* tt_status_string(int status) {
  switch (status) {
    case TT_OK: return "ok";
    case TT_WARN_NOT_CONVERGED: return "sweep cap reached before the price settled";
    case TT_ERR_INVALID: return "invalid argument";
    case TT_ERR_NOT_PD: return "covariance is not positive definite";
    case TT_ERR_STRIP: return "damping outside the payoff transform's strip";
    case TT_ERR_CAPACITY: return "exceeds the pricer's capacity";
    case TT_ERR_CUDA: return "CUDA error";
    case TT_ERR_NUMERIC: return "numerical failure (rank collapse or non-finite price)";
    default: return "unknown status";
  }
}

}  // extern "C"

// ===========================================================================
// Allocation-free entry point (tt_price_evaluate_static): for callers that may
// not allocate device or host memory.  Its scratch is one file-scope device
// array; its host staging is file-scope host arrays.  It shares the kernels and
// the launch/result code above, and has its own fixed-size preparation.
// ===========================================================================
namespace {

constexpr int kStaticJobs = TT_STATIC_MAX_BATCH * TT_STATIC_MAX_D;
constexpr size_t kStaticParams = (size_t)kStaticJobs * (TT_STATIC_MAX_D * TT_STATIC_MAX_D + 3 * TT_STATIC_MAX_D);
constexpr size_t kStaticStageBytes =
    (sizeof(JobDesc) * kStaticJobs + 255) / 256 * 256 + (sizeof(double) * kStaticParams + 255) / 256 * 256 +
    (sizeof(int) * kStaticJobs + 255) / 256 * 256 + 3 * ((sizeof(int) * TT_STATIC_MAX_BATCH + 255) / 256 * 256) +
    (sizeof(double) * host_scratch_doubles(TT_STATIC_MAX_D) + 255) / 256 * 256 +
    (sizeof(double) * TT_STATIC_MAX_BATCH + 255) / 256 * 256;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[TT_STATIC_SCRATCH_BYTES];

alignas(256) static unsigned char g_static_stage[kStaticStageBytes];
alignas(256) static unsigned char g_static_pack[kStaticStageBytes];
alignas(256) static InstanceResult g_static_ires[TT_STATIC_MAX_BATCH];

struct StaticDevice {
  bool ready;
  char* scratch;  // device address of g_static_scratch on this device
  int grid[2];    // CTAs per precision that fit in the array and on the GPU
};
static StaticDevice g_static_dev[kStaticMaxDevices];

tt_options static_options(int precision, int device, void* stream) {
  tt_options o;
  std::memset(&o, 0, sizeof(o));
  o.max_d = TT_STATIC_MAX_D;
  o.max_n = TT_STATIC_MAX_N;
  o.max_rank = TT_STATIC_MAX_RANK;
  o.max_batch = TT_STATIC_MAX_BATCH;
  o.precision = precision == TT_MIXED ? TT_MIXED : TT_FP64;
  o.device = device;
  o.cuda_stream = stream;
  return o;
}

// One-time set-up per device (with that device current): the array's device
// address and the launch width that fits in it.
int static_setup(int dev) {
  StaticDevice& sd = g_static_dev[dev];
  if (sd.ready) return TT_OK;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  for (int prec = 0; prec < 2; ++prec) {
    Resolved R;
    tt_options o = static_options(prec, dev, nullptr);
    if (!resolve(&o, &R)) return TT_ERR_INVALID;
    const bool f64 = R.o.precision == TT_FP64;
    SmemLayout S = make_smem(R.o, f64);
    int grid = 0;
    const int rc = grid_for(R.o, S, &grid);
    if (rc != TT_OK) return rc;
    Layout L = make_layout(R.o, f64);
    const DevLayout D0 = make_dev_layout(R, L, 0);
    if (D0.total > TT_STATIC_SCRATCH_BYTES || D0.stage_bytes > kStaticStageBytes) return TT_ERR_CAPACITY;
    const long long fit = (long long)(TT_STATIC_SCRATCH_BYTES - D0.total) / (long long)L.stride;
    if (fit < 1) return TT_ERR_CAPACITY;
    sd.grid[prec] = (int)std::min<long long>(grid, fit);
  }
  sd.scratch = reinterpret_cast<char*>(ptr);
  sd.ready = true;
  return TT_OK;
}

}  // namespace

extern "C" int tt_price_evaluate_static(const tt_problem* probs, int count, int precision,
                                        void* cuda_stream, double* prices, tt_diag* diag) {
  if (count < 0 || (count > 0 && (!probs || !prices))) return TT_ERR_INVALID;
  if (count > TT_STATIC_MAX_BATCH) return TT_ERR_CAPACITY;
  if (precision != TT_FP64 && precision != TT_MIXED) return TT_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TT_ERR_CUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return TT_ERR_CAPACITY;
  int rc = static_setup(dev);
  if (rc != TT_OK) return rc;
  const StaticDevice& sd = g_static_dev[dev];
  tt_pricer h;  // on the stack: views of the static arrays, nothing allocated
  tt_options o = static_options(precision, dev, cuda_stream);
  if (!resolve(&o, &h.R)) return TT_ERR_INVALID;
  const bool f64 = h.R.o.precision == TT_FP64;
  h.lay = make_layout(h.R.o, f64);
  h.sml = make_smem(h.R.o, f64);
  h.grid = sd.grid[f64 ? 0 : 1];
  h.dl = make_dev_layout(h.R, h.lay, h.grid);
  if (h.dl.total > TT_STATIC_SCRATCH_BYTES || h.dl.stage_bytes > kStaticStageBytes) return TT_ERR_CAPACITY;
  h.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  h.own_ws = false;
  h.ws = sd.scratch;
  h.h_stage = reinterpret_cast<char*>(g_static_stage);
  h.h_pack = reinterpret_cast<char*>(g_static_pack);
  h.h_ires = g_static_ires;
  h.count = 0;
  h.njobs = 0;
  h.npairs = 0;
  h.p_pairs = 0;
  h.p_warm = 0;
  h.last_h2d = h.last_d2h = 0;
  rc = prepare_impl(&h, probs, count);
  if (rc != TT_OK) return rc;
  rc = run_impl(&h);
  if (rc != TT_OK) return rc;
  return results_impl(&h, prices, diag);
}

#ifdef TTP_PHASE_TIMERS
// Profiling builds only (not part of the ABI in include/ttprice.h): read and
// optionally clear the per-phase cycle counters of the current device.
extern "C" int tt_phase_cycles(unsigned long long* out24, int reset) {
  if (out24 && cudaMemcpyFromSymbol(out24, ttp::g_phase_cycles, 24 * sizeof(unsigned long long)) != cudaSuccess)
    return TT_ERR_CUDA;
  if (reset) {
    const unsigned long long z[24] = {0};
    if (cudaMemcpyToSymbol(ttp::g_phase_cycles, z, sizeof(z)) != cudaSuccess) return TT_ERR_CUDA;
  }
  return TT_OK;
}
#endif
