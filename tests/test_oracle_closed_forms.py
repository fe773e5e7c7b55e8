"""Pins for the closed-form references (they pin the Fourier oracle in turn)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import closed_forms


def test_bvn_special_cases():
    for h, k in [(0.3, -0.7), (1.2, 0.4), (-2.0, -0.5)]:
        assert abs(closed_forms.bvn_cdf(h, k, 0.0) - stats.norm.cdf(h) * stats.norm.cdf(k)) < 1e-15
    for rho in (-0.6, 0.2, 0.9):
        # orthant probability: P(X<=0, Y<=0) = 1/4 + asin(rho)/(2 pi)
        assert abs(closed_forms.bvn_cdf(0.0, 0.0, rho) - (0.25 + math.asin(rho) / (2 * math.pi))) < 1e-14


@pytest.mark.parametrize("h,k,rho", [(0.5, -0.3, 0.4), (-1.1, 0.8, -0.7), (2.0, 1.5, 0.85)])
def test_bvn_matches_library(h, k, rho):
    lib = stats.multivariate_normal(mean=[0, 0], cov=[[1, rho], [rho, 1]]).cdf([h, k])
    assert abs(closed_forms.bvn_cdf(h, k, rho) - lib) < 1e-7


def test_one_factor_reduces_to_black_scholes():
    for rho in (0.0, 0.5):
        got = closed_forms.one_factor_price([103.0], [0.3], rho, 100.0, 0.02, 1.3, "min")
        assert abs(got - closed_forms.bs_call(103.0, 100.0, 0.02, 1.3, 0.3)) < 1e-11
        got = closed_forms.one_factor_price([103.0], [0.3], rho, 100.0, 0.02, 1.3, "max")
        assert abs(got - closed_forms.bs_call(103.0, 100.0, 0.02, 1.3, 0.3)) < 1e-11


@pytest.mark.parametrize("payoff", ["min", "max"])
def test_stulz_equals_one_factor(payoff):
    s1, s2, k, r, t, v1, v2, rho = 100.0, 96.0, 100.0, 0.01, 1.0, 0.2, 0.3, 0.5
    f = closed_forms.stulz_min_call if payoff == "min" else closed_forms.stulz_max_call
    a = f(s1, s2, k, r, t, v1, v2, rho)
    b = closed_forms.one_factor_price([s1, s2], [v1, v2], rho, k, r, t, payoff)
    assert abs(a - b) < 1e-11 * a


def test_max_min_inclusion_exclusion_d3():
    """(max - K)^+ = sum over nonempty S of (-1)^{|S|+1} (min_S - K)^+ (pointwise identity)."""
    spot = np.array([97.0, 101.0, 110.0])
    sigma = np.array([0.15, 0.3, 0.22])
    rho, k, r, t = 0.3, 100.0, 0.02, 0.75
    total = 0.0
    for mask in range(1, 8):
        idx = [j for j in range(3) if mask >> j & 1]
        sign = 1.0 if len(idx) % 2 else -1.0
        total += sign * closed_forms.one_factor_price(spot[idx], sigma[idx], rho, k, r, t, "min")
    direct = closed_forms.one_factor_price(spot, sigma, rho, k, r, t, "max")
    assert abs(total - direct) < 1e-10 * direct


@pytest.mark.parametrize("payoff", ["min", "max"])
def test_monte_carlo_brackets_one_factor(payoff):
    spot = np.array([95.0, 102.0, 100.0, 99.0, 104.0])
    sigma = np.array([0.2, 0.3, 0.25, 0.18, 0.33])
    rho = 0.3
    corr = (1 - rho) * np.eye(5) + rho
    cov = corr * np.outer(sigma, sigma)
    mean, se = closed_forms.mc_price(spot, cov, 100.0, 0.02, 1.0, payoff, 400_000, seed=7)
    ref = closed_forms.one_factor_price(spot, sigma, rho, 100.0, 0.02, 1.0, payoff)
    assert abs(mean - ref) < 4.5 * se
