"""Seeded synthetic pricing problems (the only module shared by tests, bench and oracle users).

This module draws option parameters; it holds none of the pricing method's
arithmetic.  The paper uses synthetic parameters only (Section V: r, sigma,
T, S0 = K and the equicorrelation family Sigma(beta) of Eq. covmat); the
workloads below follow the same recipe with the distributions listed in each
generator, seeded with ``numpy.random.default_rng(220302804 + index)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

SEED_BASE = 220302804


@dataclass
class Problem:
    """One option: GBM assets with covariance ``cov`` (annualised, SPD)."""
    spot: np.ndarray
    cov: np.ndarray
    rate: float
    maturity: float
    strike: float
    payoff: str                 # "min" or "max"
    damping: np.ndarray         # alpha per axis; Im z_j = -damping_j for the min-call
    n_grid: int
    trunc_L: float
    max_rank: int
    seed: int = 0
    meta: dict = field(default_factory=dict)
    max_rank_phi: int = 0       # two-train form: D_phi (0: max_rank, which is D_v)
    warm_sets: object = None    # warm-start record (uint16 array, include/ttprice.h format) or None

    @property
    def d(self) -> int:
        return int(len(self.spot))

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def cov_from(sigma, corr):
    sigma = np.asarray(sigma, dtype=np.float64)
    return np.asarray(corr, dtype=np.float64) * np.outer(sigma, sigma)


def equicorrelation(d, rho):
    return (1.0 - rho) * np.eye(d) + rho * np.ones((d, d))


def paper_beta_correlation(d, beta):
    """Sigma(beta) = (beta |+><+| + 1)/(1 + beta)  (Eq. covmat): rho = beta/(1+beta) off-diagonal."""
    return (beta * np.ones((d, d)) + np.eye(d)) / (1.0 + beta)


def two_asset_min_call(n_grid=64, trunc_L=40.0, max_rank=8, seed=1, payoff="min"):
    """d=2 call on the minimum: S0=(100,100), K=100, sigma=(0.2,0.3), rho=0.5,
    r=0.01, T=1, alpha=-1.5 per axis, N=64 on [-40,40], rank 8."""
    return Problem(spot=np.array([100.0, 100.0]),
                   cov=cov_from([0.2, 0.3], equicorrelation(2, 0.5)),
                   rate=0.01, maturity=1.0, strike=100.0, payoff=payoff,
                   damping=np.array([-1.5, -1.5]), n_grid=n_grid, trunc_L=trunc_L,
                   max_rank=max_rank, seed=seed,
                   meta={"workload": "d2-min-call", "rho": 0.5, "sigma": [0.2, 0.3]})


def five_asset_batch(count, n_grid=128, trunc_L=40.0, max_rank=32, index=1, rho=0.3):
    """d=5 calls on the minimum: S0_j~U[90,110], sigma_j~U[0.15,0.35],
    C=(1-rho)I + rho 11^T with rho=0.3, K=100, r=0.02, T=1, alpha=-1.5,
    N=128 on [-40,40], rank 32.  One problem per draw; draws in that order."""
    rng = np.random.default_rng(SEED_BASE + index)
    out = []
    for n in range(count):
        spot = rng.uniform(90.0, 110.0, 5)
        sigma = rng.uniform(0.15, 0.35, 5)
        out.append(Problem(spot=spot, cov=cov_from(sigma, equicorrelation(5, rho)),
                           rate=0.02, maturity=1.0, strike=100.0, payoff="min",
                           damping=np.full(5, -1.5), n_grid=n_grid, trunc_L=trunc_L,
                           max_rank=max_rank, seed=SEED_BASE + 1000 * index + n,
                           meta={"workload": "d5-min-call", "rho": rho, "sigma": sigma}))
    return out


def mixed_batch(count, index=2, d_range=(3, 10), grids=(64, 128, 256), ranks=(8, 16, 32)):
    """Heterogeneous batch: d~U{3..10}, N~U{64,128,256}, rank~U{8,16,32},
    K~U[80,120], T~U[0.25,2], sigma_j~U[0.1,0.4], rho~U[0,0.6] (equicorrelated),
    payoff min/max with probability 1/2, S0_j=100, r=0.02, alpha=-1.5.

    Truncation L balances the two errors of the midpoint rule for the drawn N:
    the cut tail, about exp(-s^2 T L^2 / 2) for the slowest-decaying axis (s the
    smallest per-axis spread the payoff's integrand sees: sigma_j for the
    min-call, for the max-call also the spread volatilities
    sqrt(sigma_j^2 + sigma_l^2 - 2 rho sigma_j sigma_l)), and the aliasing of
    the log-price function at period 2 pi / eta = pi N / L, about
    exp(-(1/2) pi N / L) for damping 1.5 (the damped payoff decays as e^{-x/2}).
    Equal exponents give L = (pi N / (s^2 T))^(1/3).  A fixed L = 8/(s sqrt T)
    would leave eta = 2L/N too coarse for N = 64 on slow axes."""
    rng = np.random.default_rng(SEED_BASE + index)
    out = []
    for n in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        n_grid = int(rng.choice(grids))
        rank = int(rng.choice(ranks))
        strike = float(rng.uniform(80.0, 120.0))
        maturity = float(rng.uniform(0.25, 2.0))
        sigma = rng.uniform(0.1, 0.4, d)
        rho = float(rng.uniform(0.0, 0.6))
        payoff = "min" if rng.random() < 0.5 else "max"
        vol = sigma.copy()
        if payoff == "max":
            spread = np.sqrt(np.maximum(sigma[:, None] ** 2 + sigma[None, :] ** 2
                                        - 2.0 * rho * np.outer(sigma, sigma), 0.0))
            spread[np.eye(d, dtype=bool)] = np.inf
            vol = np.minimum(vol, spread.min(axis=1))
        s2t = float(vol.min()) ** 2 * maturity
        trunc = float(np.cbrt(np.pi * n_grid / s2t))
        out.append(Problem(spot=np.full(d, 100.0), cov=cov_from(sigma, equicorrelation(d, rho)),
                           rate=0.02, maturity=maturity, strike=strike, payoff=payoff,
                           damping=np.full(d, -1.5), n_grid=n_grid, trunc_L=trunc,
                           max_rank=rank, seed=SEED_BASE + 1000 * index + n,
                           meta={"workload": "mixed-batch", "rho": rho, "sigma": sigma}))
    return out


def surrogate_batch(count, index=5, n_grid=128, trunc_L=40.0, max_rank=32):
    """d=5 calls on the minimum spread over a parameter box, for the learned
    surrogate: S0_j~U[90,110], sigma_j~U[0.15,0.35], equicorrelation rho~U[0,0.6],
    K~U[90,110], T~U[0.5,1.5], r~U[0,0.05], alpha~U[-2,-1.2] (same on every axis),
    N=128 on [-40,40], rank 32."""
    rng = np.random.default_rng(SEED_BASE + index)
    out = []
    for n in range(count):
        spot = rng.uniform(90.0, 110.0, 5)
        sigma = rng.uniform(0.15, 0.35, 5)
        rho = float(rng.uniform(0.0, 0.6))
        strike = float(rng.uniform(90.0, 110.0))
        maturity = float(rng.uniform(0.5, 1.5))
        rate = float(rng.uniform(0.0, 0.05))
        alpha = float(rng.uniform(-2.0, -1.2))
        out.append(Problem(spot=spot, cov=cov_from(sigma, equicorrelation(5, rho)), rate=rate,
                           maturity=maturity, strike=strike, payoff="min", damping=np.full(5, alpha),
                           n_grid=n_grid, trunc_L=trunc_L, max_rank=max_rank,
                           seed=SEED_BASE + 1000 * index + n, meta={"workload": "surrogate"}))
    return out


def tuning_batch(count, d, n_grid, max_rank, payoff="min", index=4):
    """Synthetic batch of one workload shape for the autotuner: S0_j~U[90,110],
    sigma_j~U[0.15,0.35], equicorrelation 0.3, K=100, r=0.02, T=1, L=40,
    alpha_j = -1.5 up to d = 10 and -5/d above (as the high-d workload)."""
    rng = np.random.default_rng(SEED_BASE + 1000 * index + 17 * d + n_grid + max_rank)
    alpha = -1.5 if d <= 10 else -5.0 / d
    out = []
    for n in range(count):
        spot = rng.uniform(90.0, 110.0, d)
        sigma = rng.uniform(0.15, 0.35, d)
        out.append(Problem(spot=spot, cov=cov_from(sigma, equicorrelation(d, 0.3)), rate=0.02,
                           maturity=1.0, strike=100.0, payoff=payoff, damping=np.full(d, alpha),
                           n_grid=n_grid, trunc_L=40.0, max_rank=max_rank,
                           seed=SEED_BASE + 1000 * index + n, meta={"workload": "tuning"}))
    return out


def random_correlation(d, rng):
    """C = D^{-1/2} A D^{-1/2} with A = W W^T / d + 0.5 I, W Gaussian d x d."""
    w = rng.standard_normal((d, d))
    a = w @ w.T / d + 0.5 * np.eye(d)
    s = 1.0 / np.sqrt(np.diag(a))
    return a * np.outer(s, s)


def balanced_truncation(n_grid, rate_axis, d, s2t):
    """L balancing the midpoint rule's two errors on a d-axis grid of N points:
    aliasing, about d exp(-pi a N / L) for damping rate a per axis, and the cut
    Gaussian tail exp(-s^2 T L^2 / 2) of the slowest axis (solved by bisection)."""
    lo, hi = 1e-3, 1e4
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = np.pi * rate_axis * n_grid / mid - np.log(d) - 0.5 * s2t * mid * mid
        lo, hi = (mid, hi) if f > 0 else (lo, mid)
    return 0.5 * (lo + hi)


def high_dim_problem(d, payoff="min", n_grid=256, trunc_L=None, max_rank=64, index=3, damping=None):
    """d in {20, 50, 100}: sigma_j~U[0.15,0.35], random correlation as above,
    K=100, S0=100, r=0.02, T=1.

    Damping: for the call on the maximum, |alpha_j| = 10/d.  Term j's integrand
    carries exp(T/2 (1 + d|alpha|)^2 sigma_j^2 + ...) through the maximum's axis, so
    a fixed |alpha| makes its scale e^{T delta' Cov delta / 2} reach ~e^180 at d = 50
    (alpha = -1.5), and FP32 sums lose everything to cancellation; at 10/d the
    coefficient stays 11.  The call on the minimum keeps alpha_j = -1.5 (its scale
    grows only like alpha^2 sigma^2 d).  L balances aliasing at the damping rate
    against the cut tail of the slowest axis (``balanced_truncation``), unless
    given: with N = 256 that predicts ~5e-5 of discretisation error at d = 20,
    ~1e-2 at d = 50 and ~2e-1 at d = 100 for the call on the maximum."""
    rng = np.random.default_rng(SEED_BASE + index * 1000 + d)
    sigma = rng.uniform(0.15, 0.35, d)
    corr = random_correlation(d, rng)
    if damping is None:
        damping = -10.0 / d if payoff == "max" else -1.5
    if trunc_L is None:
        rate = abs(damping)
        trunc_L = float(balanced_truncation(n_grid, rate, d, float(sigma.min()) ** 2))
    return Problem(spot=np.full(d, 100.0), cov=cov_from(sigma, corr), rate=0.02, maturity=1.0,
                   strike=100.0, payoff=payoff, damping=np.full(d, float(damping)), n_grid=n_grid,
                   trunc_L=trunc_L, max_rank=max_rank, seed=SEED_BASE + index * 1000 + d,
                   meta={"workload": f"d{d}-{payoff}-call"})


def paper_table_problem(d, n_grid=50, trunc_L=None, max_rank=15, beta=0.5):
    """The paper's own setting (Section V): r=0.3, sigma=0.5, T=1, S0=K=100,
    Sigma(beta=0.5), alpha=5/d, N=50; eta from its table (0.5 at d=2 ... 0.2 at d>=6)."""
    eta = {2: 0.5, 3: 0.4, 4: 0.3, 5: 0.3}.get(d, 0.2)
    if trunc_L is None:
        trunc_L = 0.5 * eta * n_grid
    sigma = np.full(d, 0.5)
    return Problem(spot=np.full(d, 100.0), cov=cov_from(sigma, paper_beta_correlation(d, beta)),
                   rate=0.3, maturity=1.0, strike=100.0, payoff="min",
                   damping=np.full(d, -5.0 / d), n_grid=n_grid, trunc_L=trunc_L,
                   max_rank=max_rank, seed=SEED_BASE + 7000 + d, meta={"workload": f"paper-d{d}"})
