"""Pins for the one-factor grid sum (oracle/grid_sum.py): the exact N^d midpoint-grid
price of the call on the minimum for equicorrelated assets, at any d.

It must equal the brute-force full grid sum where that is feasible (d <= 4),
be insensitive to its own quadrature steps, and approach the exact one-factor
integral as the grid is refined (Eq. main is what Eq. discr discretises)."""
import numpy as np
import pytest

from oracle import closed_forms, grid_sum, integrand
from paper_2203_02804_gb300 import inputs


def _problem(d, n, rho, trunc, seed, sigma_lo=0.15, sigma_hi=0.35, maturity=1.0, alpha=-1.5):
    rng = np.random.default_rng(seed)
    sig = rng.uniform(sigma_lo, sigma_hi, d)
    return inputs.Problem(spot=rng.uniform(90, 110, d),
                          cov=inputs.cov_from(sig, inputs.equicorrelation(d, rho)),
                          rate=0.02, maturity=maturity, strike=100.0, payoff="min",
                          damping=np.full(d, alpha), n_grid=n, trunc_L=trunc, max_rank=8)


@pytest.mark.parametrize("d,n,rho,trunc", [(1, 64, 0.0, 40.0), (2, 64, 0.5, 40.0), (2, 37, 0.0, 25.0),
                                           (3, 32, 0.3, 20.0), (3, 29, 0.6, 12.0), (4, 16, 0.3, 20.0)])
def test_equals_brute_force_full_grid(d, n, rho, trunc):
    p = _problem(d, n, rho, trunc, seed=d * 100 + n)
    got, imag = grid_sum.grid_sum_for(p)
    ref, _ = integrand.full_grid_price(p)
    assert abs(got / ref - 1) < 1e-12
    assert abs(imag) < 1e-12 * abs(got)


def test_paper_setting_and_heterogeneous_shapes_equal_brute_force():
    """The paper's own setting (Sigma(beta), alpha = 5/d, eta per its table) and a
    short-maturity, low-volatility shape like the heterogeneous batch's."""
    p = inputs.paper_table_problem(3, n_grid=40)
    assert abs(grid_sum.grid_sum_for(p)[0] / integrand.full_grid_price(p)[0] - 1) < 1e-12
    q = _problem(3, 40, 0.6, 30.0, seed=7, sigma_lo=0.1, sigma_hi=0.12, maturity=0.25)
    assert abs(grid_sum.grid_sum_for(q)[0] / integrand.full_grid_price(q)[0] - 1) < 1e-12


def test_quadrature_steps_do_not_move_the_value():
    for p in (inputs.five_asset_batch(1)[0], _problem(8, 256, 0.6, 30.0, seed=9, sigma_lo=0.1, sigma_hi=0.4)):
        a = grid_sum.grid_sum_for(p)[0]
        b = grid_sum.grid_sum_for(p, refine=1.7)[0]
        assert abs(a / b - 1) < 1e-12


def test_converges_to_the_one_factor_integral():
    """d = 5: the midpoint grid's error (aliasing at rate delta per axis, Poisson
    summation) falls as eta shrinks; at N = 512 it is below 1e-9."""
    p = inputs.five_asset_batch(1)[0]
    sig = np.sqrt(np.diag(p.cov))
    exact = closed_forms.one_factor_price(p.spot, sig, 0.3, 100.0, 0.02, 1.0, "min")
    errs = [abs(grid_sum.grid_sum_for(p.with_(n_grid=n))[0] / exact - 1) for n in (64, 128, 512)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9


def test_rejects_what_it_does_not_cover():
    p = _problem(3, 16, 0.3, 20.0, seed=1)
    with pytest.raises(ValueError):
        grid_sum.grid_sum_for(p.with_(payoff="max"))
    c = np.array(p.cov)
    c[0, 1] = c[1, 0] = 0.9 * c[0, 1]
    with pytest.raises(ValueError):
        grid_sum.grid_sum_for(p.with_(cov=c))
