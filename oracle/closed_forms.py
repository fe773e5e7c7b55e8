"""Reference prices that pin the Fourier integrand and the TT-cross oracle.

Test infrastructure only (see the package docstring).

  * ``bs_call``             -- Black-Scholes, Eq. (BSexact).
  * ``bvn_cdf``             -- bivariate normal CDF by Sheppard's one-dimensional
                               integral over the correlation angle (textbook; no
                               paper counterpart).
  * ``stulz_min_call``      -- the two-asset call on the minimum (Stulz 1982,
                               derived by a change of numeraire); max-call by
                               (max-K)^+ = (S1-K)^+ + (S2-K)^+ - (min-K)^+.
  * ``one_factor_price``    -- equicorrelated d-asset min/max call: conditional on
                               the common factor the assets are independent, so
                               P(min S > s) = E_Z0[prod_j P(S_j > s | Z0)] and the
                               price is e^{-rT} int_K^inf P(.) ds.
  * ``mc_price``            -- Monte Carlo, Eq. (mc) steps (a)-(c), sampling the
                               exact GBM terminal law instead of time stepping.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special


def norm_cdf(x):
    return special.ndtr(x)


def bs_call(spot, strike, rate, maturity, sigma):
    """S0 Phi(d1) - K e^{-rT} Phi(d2), d_{1,2} = (ln(S0/K) + (r +- sigma^2/2)T)/(sigma sqrt T)."""
    st = sigma * math.sqrt(maturity)
    d1 = (math.log(spot / strike) + (rate + 0.5 * sigma * sigma) * maturity) / st
    d2 = d1 - st
    return spot * norm_cdf(d1) - strike * math.exp(-rate * maturity) * norm_cdf(d2)


def bvn_cdf(h, k, rho):
    """P(X <= h, Y <= k) for standard normals with correlation rho.

    Sheppard: M = Phi(h)Phi(k) + 1/(2 pi) int_0^{asin rho}
                  exp(-(h^2 + k^2 - 2 h k sin t) / (2 cos^2 t)) dt.
    """
    base = norm_cdf(h) * norm_cdf(k)
    if rho == 0.0:
        return float(base)
    top = math.asin(rho)

    def f(t):
        c2 = math.cos(t) ** 2
        return math.exp(-(h * h + k * k - 2.0 * h * k * math.sin(t)) / (2.0 * c2))

    val, _ = integrate.quad(f, 0.0, top, epsabs=1e-16, epsrel=1e-14, limit=200)
    return float(base + val / (2.0 * math.pi))


def stulz_min_call(s1, s2, strike, rate, maturity, sig1, sig2, rho):
    """Two-asset call on the minimum (Stulz 1982)."""
    sq = math.sqrt(maturity)
    sbar = math.sqrt(sig1 * sig1 + sig2 * sig2 - 2.0 * rho * sig1 * sig2)
    d1 = (math.log(s1 / strike) + (rate + 0.5 * sig1 * sig1) * maturity) / (sig1 * sq)
    d2 = (math.log(s2 / strike) + (rate + 0.5 * sig2 * sig2) * maturity) / (sig2 * sq)
    e = (math.log(s1 / s2) + 0.5 * sbar * sbar * maturity) / (sbar * sq)
    rho1 = (rho * sig2 - sig1) / sbar
    rho2 = (rho * sig1 - sig2) / sbar
    return (s1 * bvn_cdf(d1, -e, rho1)
            + s2 * bvn_cdf(d2, e - sbar * sq, rho2)
            - strike * math.exp(-rate * maturity) * bvn_cdf(d1 - sig1 * sq, d2 - sig2 * sq, rho))


def stulz_max_call(s1, s2, strike, rate, maturity, sig1, sig2, rho):
    """Two-asset call on the maximum from the pointwise identity with the min-call."""
    return (bs_call(s1, strike, rate, maturity, sig1) + bs_call(s2, strike, rate, maturity, sig2)
            - stulz_min_call(s1, s2, strike, rate, maturity, sig1, sig2, rho))


def one_factor_price(spot, sigma, rho, strike, rate, maturity, payoff, n_hermite=160):
    """Equicorrelated (rho >= 0) d-asset call on the min or max.

    ln S_j(T) = mu_j + sigma_j sqrt(T) (sqrt(rho) Z0 + sqrt(1-rho) Z_j).
    min: e^{-rT} int_K^inf E_Z0[prod_j Phibar(a_j(s, Z0))] ds
    max: e^{-rT} int_K^inf (1 - E_Z0[prod_j Phi(a_j(s, Z0))]) ds
    with a_j = (ln s - mu_j - sigma_j sqrt(T rho) Z0) / (sigma_j sqrt(T (1-rho))).
    The s-integral is taken in x = ln s (ds = e^x dx); Z0 by Gauss-Hermite.
    """
    spot = np.asarray(spot, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    mu = np.log(spot) + (rate - 0.5 * sigma * sigma) * maturity
    xg, wg = np.polynomial.hermite.hermgauss(n_hermite)
    z0 = math.sqrt(2.0) * xg
    wz = wg / math.sqrt(math.pi)
    common = sigma * math.sqrt(maturity * rho)
    idio = sigma * math.sqrt(maturity * (1.0 - rho))

    def prob(x):
        a = (x - mu[None, :] - common[None, :] * z0[:, None]) / idio[None, :]
        if payoff == "min":
            return float(wz @ np.prod(special.ndtr(-a), axis=1))
        return float(1.0 - wz @ np.prod(special.ndtr(a), axis=1))

    lo = math.log(strike)
    hi = float(np.max(mu + 14.0 * sigma * math.sqrt(maturity)))
    if hi <= lo:
        return 0.0
    # split the range so quad resolves the bulk of every asset's density
    pts = sorted({lo, *[float(m) for m in mu if lo < m < hi], hi})
    total = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        val, _ = integrate.quad(lambda x: math.exp(x) * prob(x), a, b,
                                epsabs=0.0, epsrel=1e-13, limit=400)
        total += val
    return math.exp(-rate * maturity) * total


def mc_price(spot, cov, strike, rate, maturity, payoff, n_paths, seed, batch=1 << 20):
    """Monte Carlo with exact terminal sampling X = mu + sqrt(T) L Z (L L^T = Cov).

    Returns (mean, standard error).  Numbers are drawn from NumPy's PCG64 stream
    seeded with ``seed``.
    """
    spot = np.asarray(spot, dtype=np.float64)
    cov = np.asarray(cov, dtype=np.float64)
    d = spot.size
    mu = np.log(spot) + (rate - 0.5 * np.diag(cov)) * maturity
    chol = np.linalg.cholesky(cov)
    rng = np.random.default_rng(seed)
    s1 = 0.0
    s2 = 0.0
    done = 0
    while done < n_paths:
        m = min(batch, n_paths - done)
        z = rng.standard_normal((m, d))
        x = mu + math.sqrt(maturity) * (z @ chol.T)
        s = np.exp(x)
        agg = s.min(axis=1) if payoff == "min" else s.max(axis=1)
        pay = np.maximum(agg - strike, 0.0)
        s1 += float(pay.sum())
        s2 += float((pay * pay).sum())
        done += m
    disc = math.exp(-rate * maturity)
    mean = s1 / n_paths
    var = max(s2 / n_paths - mean * mean, 0.0)
    return disc * mean, disc * math.sqrt(var / n_paths)
