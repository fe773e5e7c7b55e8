"""Pins for the oracle's integrand (characteristic function, payoff transforms, grid sum).

Every pin is something the paper or textbook mathematics fixes independently of
the oracle's own formulas: phi(0) = 1, the martingale identity, direct
numerical Fourier transforms of the damped payoffs, Black-Scholes (Eq.
BSexact), the Stulz two-asset formulas and the one-factor semi-analytic price.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import closed_forms, integrand
from paper_2203_02804_gb300 import inputs


def _random_cov(d, rng):
    a = rng.standard_normal((d, d))
    corr = a @ a.T + d * np.eye(d)
    s = 1.0 / np.sqrt(np.diag(corr))
    corr = corr * np.outer(s, s)
    sigma = rng.uniform(0.1, 0.5, d)
    return corr * np.outer(sigma, sigma)


def test_char_fn_at_zero_is_one():
    rng = np.random.default_rng(0)
    cov = _random_cov(4, rng)
    mu = rng.standard_normal(4)
    assert abs(integrand.char_fn(np.zeros(4), mu, cov, 1.7) - 1.0) < 1e-15


@pytest.mark.parametrize("maturity", [0.25, 1.0, 2.5])
def test_martingale_identity(maturity):
    """phi(-i e_j) = E[S_j(T)] = S0_j e^{rT}; fails if the T on the quadratic term is dropped."""
    rng = np.random.default_rng(1)
    d = 3
    cov = _random_cov(d, rng)
    spot = rng.uniform(50, 150, d)
    rate = 0.04
    mu = integrand.drift_mean(spot, cov, rate, maturity)
    for j in range(d):
        w = np.zeros(d, dtype=complex)
        w[j] = -1j
        got = integrand.char_fn(w, mu, cov, maturity)
        assert abs(got - spot[j] * math.exp(rate * maturity)) < 1e-10 * spot[j]


def _cquad(f, a, b):
    re = integrate.quad(lambda x: f(x).real, a, b, epsabs=1e-13, epsrel=1e-12, limit=4000)[0]
    im = integrate.quad(lambda x: f(x).imag, a, b, epsabs=1e-13, epsrel=1e-12, limit=4000)[0]
    return re + 1j * im


@pytest.mark.parametrize("z", [0.7 + 1.8j, -2.3 + 1.3j, 0.0 + 2.5j])
def test_call_transform_matches_direct_quadrature(z):
    """d=1: int e^{izx} (e^x - K)^+ dx on Im z > 1 equals the closed transform."""
    k = 95.0
    f = lambda x: np.exp(1j * z * x) * (math.exp(x) - k)
    upper = math.log(k) + 40.0 / (z.imag - 1.0)   # the damped payoff decays like e^{(1 - Im z) x}
    direct = _cquad(f, math.log(k), upper)
    got = integrand.payoff_transform_min(np.array([z]), k)
    assert abs(got - direct) < 1e-9 * abs(direct)


def _dbl(f, x0lo, x0hi, x1lo, x1hi):
    opts = dict(epsabs=1e-12, epsrel=1e-10)
    re = integrate.dblquad(lambda y, x: f(x, y).real, x0lo, x0hi, x1lo, x1hi, **opts)[0]
    im = integrate.dblquad(lambda y, x: f(x, y).imag, x0lo, x0hi, x1lo, x1hi, **opts)[0]
    return re + 1j * im


def test_min_transform_d2_matches_direct_quadrature():
    """d=2: the corrected constant (-1)^(d+1)/prod(i z_j); the printed one is off by i^d (-1)."""
    k = 100.0
    z = np.array([0.4 + 0.9j, -0.6 + 0.8j])
    lk = math.log(k)

    def f(x0, x1):
        return np.exp(1j * (z[0] * x0 + z[1] * x1)) * (min(math.exp(x0), math.exp(x1)) - k)

    # split at the kink x0 = x1 so that each piece is smooth
    up = lk + 60.0
    direct = (_dbl(f, lk, up, lambda x: lk, lambda x: x)
              + _dbl(f, lk, up, lambda x: x, lambda x: up))
    got = integrand.payoff_transform_min(z, k)
    assert abs(got - direct) < 1e-8 * abs(direct)


def test_printed_min_transform_constant_reading():
    """The printed K^(1+i sum z)/((-1)^d (1+i sum z) prod z_j) agrees with the
    derived transform at d=2 but is off by a factor -i at d=1 (so it would not
    reduce to the single-asset call transform, which the paper says it does)."""
    k = 100.0
    for d, ratio in ((1, -1j), (2, 1.0), (3, 1j)):
        z = np.array([0.3 + 1.7j, -0.2 + 0.6j, 0.5 + 0.4j][:d])
        printed = k ** (1 + 1j * z.sum()) / ((-1) ** d * (1 + 1j * z.sum()) * np.prod(z))
        assert abs(printed / integrand.payoff_transform_min(z, k) - ratio) < 1e-12


def test_max_term_transform_d2_matches_direct_quadrature():
    """Term 0 of the max-call: (e^{y0} - K)^+ 1{y1 <= 0} on Im z0 > 1, Im z1 < 0."""
    k = 100.0
    z = np.array([0.3 + 2.2j, -0.5 - 1.1j])
    lk = math.log(k)

    def f(y0, y1):
        return np.exp(1j * (z[0] * y0 + z[1] * y1)) * (math.exp(y0) - k)

    direct = _dbl(f, lk, lk + 40.0, lambda x: -40.0, lambda x: 0.0)
    got = integrand.payoff_transform_max_term(z, k, 0)
    assert abs(got - direct) < 1e-7 * abs(direct)


def test_single_asset_grid_sum_matches_black_scholes():
    """d=1 (Eq. maincont discretised): exponential convergence to Eq. BSexact.

    At d=1 the aliasing rate is (delta - 1) 2 pi / eta, so delta = 3 here."""
    spot, k, r, t, s = 105.0, 100.0, 0.03, 0.8, 0.25
    p = inputs.Problem(spot=np.array([spot]), cov=np.array([[s * s]]), rate=r, maturity=t,
                       strike=k, payoff="min", damping=np.array([-3.0]), n_grid=512,
                       trunc_L=80.0, max_rank=1)
    price, imag = integrand.full_grid_price(p)
    bs = closed_forms.bs_call(spot, k, r, t, s)
    assert abs(price - bs) < 1e-10 * bs
    assert abs(imag) < 1e-12 * bs


def test_two_asset_min_call_grid_sum_matches_stulz():
    p = inputs.two_asset_min_call(n_grid=256)
    price, imag = integrand.full_grid_price(p)
    ref = closed_forms.stulz_min_call(100, 100, 100, 0.01, 1.0, 0.2, 0.3, 0.5)
    assert abs(price - ref) < 1e-11 * ref
    assert abs(imag) < 1e-13 * ref


def test_two_asset_min_call_discretisation_error_at_n64():
    """N=64, L=40: eta=1.25, so the aliasing term e^{-delta 2pi/eta} leaves ~1e-3."""
    p = inputs.two_asset_min_call(n_grid=64)
    price, _ = integrand.full_grid_price(p)
    ref = closed_forms.stulz_min_call(100, 100, 100, 0.01, 1.0, 0.2, 0.3, 0.5)
    assert 1e-4 < abs(price / ref - 1) < 5e-3


def test_two_asset_max_call_grid_sum_matches_stulz():
    p = inputs.two_asset_min_call(n_grid=256, payoff="max")
    price, imag = integrand.full_grid_price(p)
    ref = closed_forms.stulz_max_call(100, 100, 100, 0.01, 1.0, 0.2, 0.3, 0.5)
    assert abs(price - ref) < 1e-9 * ref
    assert abs(imag) < 1e-12 * ref


@pytest.mark.parametrize("payoff", ["min", "max"])
def test_three_asset_grid_sum_matches_one_factor(payoff):
    spot = np.array([95.0, 100.0, 108.0])
    sigma = np.array([0.2, 0.25, 0.3])
    rho = 0.35
    p = inputs.Problem(spot=spot, cov=inputs.cov_from(sigma, inputs.equicorrelation(3, rho)),
                       rate=0.02, maturity=1.0, strike=100.0, payoff=payoff,
                       damping=np.full(3, -1.5), n_grid=128, trunc_L=40.0, max_rank=1)
    price, imag = integrand.full_grid_price(p)
    ref = closed_forms.one_factor_price(spot, sigma, rho, 100.0, 0.02, 1.0, payoff)
    assert abs(price / ref - 1) < 2e-5
    assert abs(imag) < 1e-12 * ref


def test_grid_is_symmetric_midpoint():
    u, eta = integrand.grid(8, 4.0)
    assert eta == 1.0
    assert np.allclose(u, -u[::-1])
    assert u[0] == -3.5 and u[-1] == 3.5
