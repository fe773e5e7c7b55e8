"""Pins for the oracle's two-train (bra-ket) form of the price (Section IV,
Eq. braket): the site-by-site contraction against brute force, the factor split
against the single-train integrand, full-rank exactness against the full grid
sum, a separable case against its closed form, and Stulz at d=2."""
import itertools

import numpy as np
import pytest

from oracle import closed_forms, integrand, ttcross, twomps
from paper_2203_02804_gb300 import inputs


def _random_train(rng, n, ranks):
    return [rng.standard_normal((ranks[k], n, ranks[k + 1])) + 1j * rng.standard_normal((ranks[k], n, ranks[k + 1]))
            for k in range(len(ranks) - 1)]


def test_bracket_matches_dense_sum():
    """Two random trains of different bond dimensions (d=3, N=4): the site-by-site
    contraction equals the sum over all 64 entries of the brute-force product."""
    rng = np.random.default_rng(5)
    a = _random_train(rng, 4, [1, 2, 3, 1])
    b = _random_train(rng, 4, [1, 3, 2, 1])
    dense = np.sum(ttcross.dense_from_cores(a) * ttcross.dense_from_cores(b))
    got = twomps.mps_bracket(a, b)
    assert abs(got - dense) <= 1e-12 * abs(dense)
    # no conjugation: swapping the trains gives the same number, conjugating one does not
    assert abs(twomps.mps_bracket(b, a) - dense) <= 1e-12 * abs(dense)
    assert abs(twomps.mps_bracket([c.conj() for c in a], b) - dense) > 1e-3 * abs(dense)


@pytest.mark.parametrize("payoff", ["min", "max"])
def test_factors_multiply_to_the_integrand(payoff):
    """phi_T(-z) times vhat(z) is the single-train integrand at every point
    (min-call; max-call terms in their own variables)."""
    p = inputs.paper_table_problem(3).with_(payoff=payoff)
    rng = np.random.default_rng(2)
    idx = rng.integers(0, p.n_grid, size=(50, 3))
    terms = [None] if payoff == "min" else [0, 1, 2]
    for term in terms:
        prod = integrand.FourierTensor(p, term)(idx)
        f = twomps.FactorTensor(p, "phi", term)(idx) * twomps.FactorTensor(p, "vhat", term)(idx)
        np.testing.assert_allclose(f, prod, rtol=1e-13, atol=0)


@pytest.mark.parametrize("payoff", ["min", "max"])
def test_full_rank_bracket_is_the_grid_sum(payoff):
    """d=2 with the rank cap at N: the initial right sets list every grid point,
    the cross interpolates each factor exactly, and the bracket equals the full
    grid sum of the product integrand."""
    p = inputs.paper_table_problem(2).with_(n_grid=8, max_rank=8, payoff=payoff)
    price, imag, _ = twomps.two_train_price(p)
    ref, _ = integrand.full_grid_price(p)
    assert abs(price - ref) <= 1e-10 * abs(ref)
    assert abs(imag) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("d", [3, 4])
def test_paper_setting_matches_the_grid_sum(d):
    """The paper's own setting (r=0.3, sigma=0.5, beta=0.5, N=50, bond dimension
    15): the bracket is within 1e-6 of the full N^d grid sum."""
    p = inputs.paper_table_problem(d)
    price, imag, diags = twomps.two_train_price(p)
    ref, _ = integrand.full_grid_price(p)
    assert abs(price / ref - 1) < 1e-6
    assert abs(imag) < 1e-6 * ref
    for dv, dp in diags:
        assert dv.half_sweeps == dp.half_sweeps == twomps.HALF_SWEEPS


def test_separable_phi_train_has_rank_one():
    """Without correlation phi_T(-z) factorises over the axes: a rank-1 cross
    reproduces it, and its bracket with the all-ones train is the product of the
    one-dimensional sums."""
    d = 4
    p = inputs.paper_table_problem(d).with_(cov=np.diag(np.full(d, 0.25)), max_rank=1, n_grid=32)
    t = twomps.FactorTensor(p, "phi")
    _, dg = ttcross.tt_cross_sum(t, 1, int(p.seed), keep_train=True)
    ones = [np.ones((1, p.n_grid, 1), dtype=np.complex128) for _ in range(d)]
    got = twomps.mps_bracket(dg.train, ones)
    ref = twomps.separable_phi_sum(p)
    assert abs(got - ref) <= 1e-9 * abs(ref)  # the sum cancels to ~1e-3 of its terms
    # and the train is the function itself at sampled points
    rng = np.random.default_rng(4)
    idx = rng.integers(0, p.n_grid, size=(20, d))
    dense = ttcross.dense_from_cores(dg.train)
    np.testing.assert_allclose(dense[tuple(idx.T)], t(idx), rtol=1e-11)


def test_two_asset_price_against_stulz():
    """d=2 call on the minimum (N=64): the bracket is within the grid's
    discretisation error (3e-3 here) of Stulz's closed form, and its error against
    the full grid sum falls with the bond dimension (2e-6 at rank 24, 1e-7 at 32),
    agreeing with the single-train cross."""
    p = inputs.two_asset_min_call(max_rank=24)
    price, imag, diags = twomps.two_train_price(p)
    sig = p.meta["sigma"]
    exact = closed_forms.stulz_min_call(100.0, 100.0, p.strike, p.rate, p.maturity, sig[0], sig[1], p.meta["rho"])
    assert abs(price / exact - 1) < 3e-3
    ref, _ = integrand.full_grid_price(p)
    assert abs(price / ref - 1) < 5e-6  # rank 24 of 64
    price32, _, _ = twomps.two_train_price(p.with_(max_rank=32))
    assert abs(price32 / ref - 1) < 5e-7
    single, _, _ = ttcross.tt_price(p.with_(max_rank=32))  # stops at a 1e-6 relative change
    assert abs(price32 / single - 1) < 1e-6
    for dv, dp in diags:
        assert dv.train is not None and dp.train is not None


def test_two_asset_max_call_against_stulz():
    """d=2 call on the maximum (two brackets, one per asset that can be the
    maximum) at N=128 and rank 128: within 1e-8 of the full grid sum, and within
    the grid's error (2.3e-6 here) of Stulz's max-call closed form."""
    p = inputs.two_asset_min_call(n_grid=128, max_rank=128, payoff="max")
    price, imag, diags = twomps.two_train_price(p)
    assert len(diags) == 2
    grid, _ = integrand.full_grid_price(p)
    assert abs(price / grid - 1) < 1e-8
    sig = p.meta["sigma"]
    exact = closed_forms.stulz_max_call(100.0, 100.0, p.strike, p.rate, p.maturity, sig[0], sig[1], p.meta["rho"])
    assert abs(price / exact - 1) < 1e-5
    assert abs(imag) < 1e-8 * exact
