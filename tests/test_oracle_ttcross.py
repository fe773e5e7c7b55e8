"""Pins for the oracle's TT-cross: GEPP vs LAPACK, maxvol vs brute force,
exact reproduction of low-rank tensors, full-rank exactness, and convergence
to the exact grid sum (Section IV of the paper): the brute-force full grid
for d <= 4, the one-factor grid sum (oracle/grid_sum.py) at d = 5."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import integrand, ttcross
from oracle.splitmix import pivot_key, splitmix64
from paper_2203_02804_gb300 import inputs


class TableTensor:
    """Tensor given by a callable on integer multi-indices."""

    def __init__(self, d, n, fn):
        self.d, self.n, self.fn = d, n, fn

    def __call__(self, idx):
        return self.fn(np.asarray(idx))


def test_splitmix64_published_sequence():
    """First outputs of SplitMix64 from state 0 (the published reference generator)."""
    gamma = 0x9E3779B97F4A7C15
    mask = (1 << 64) - 1
    assert splitmix64(0) == 0xE220A8397B1DCDAF
    assert splitmix64(gamma) == 0x6E789E6AA1B965F4
    assert splitmix64((2 * gamma) & mask) == 0x06C45D188009454F


def test_pivot_key_fields_are_disjoint():
    keys = {pivot_key(0, t, k, a, b, j) for t in range(2) for k in range(2) for a in range(2)
            for b in range(2) for j in range(2)}
    assert len(keys) == 32


def test_initial_right_sets():
    s = ttcross.initial_right_set(5, 16, 2, 20, seed=3, term=0)
    assert len(s) == 20 and len(set(s)) == 20
    assert s[0] == (8, 8, 8)
    assert all(len(x) == 3 and all(0 <= v < 16 for v in x) for x in s)
    full = ttcross.initial_right_set(3, 4, 2, 4, seed=3, term=0)
    assert full == [(0,), (1,), (2,), (3,)]
    assert ttcross.bond_ranks(4, 3, 5) == [1, 3, 5, 3, 1]


def test_gepp_select_matches_lapack_partial_pivoting():
    rng = np.random.default_rng(5)
    for m, n in [(9, 3), (40, 8), (17, 17)]:
        a = rng.standard_normal((m, n))
        rows, cols = ttcross.gepp_select(a, 1e-12)
        p, _, _ = scipy.linalg.lu(a)
        perm = p.argmax(axis=0)
        assert cols == list(range(n))
        assert rows == list(perm[:n])


def test_gepp_select_skips_dependent_columns():
    rng = np.random.default_rng(6)
    x = rng.standard_normal((12, 2)) + 1j * rng.standard_normal((12, 2))
    a = np.column_stack([x[:, 0], 2.0 * x[:, 0] - 1j * x[:, 1], x[:, 1], x[:, 0] + x[:, 1]])
    rows, cols = ttcross.gepp_select(a, 1e-10)
    assert cols == [0, 1]
    assert len(set(rows)) == 2


@pytest.mark.parametrize("seed", range(6))
def test_maxvol_is_dominant_and_near_max_volume(seed):
    rng = np.random.default_rng(100 + seed)
    m, n, tau = 9, 3, 0.05
    a = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    rows, _ = ttcross.gepp_select(a, 1e-12)
    rows, _, ok = ttcross.maxvol(a, rows, tau, 100 * n)
    assert ok
    b = a @ np.linalg.inv(a[rows, :])
    assert np.abs(b).max() <= 1.0 + tau + 1e-12
    vol = abs(np.linalg.det(a[rows, :]))
    best = max(abs(np.linalg.det(a[list(s), :])) for s in itertools.combinations(range(m), n))
    # a dominant submatrix: det(B[best rows]) = vol_best / vol and |B| <= 1 + tau (Hadamard)
    assert vol >= best / (math.sqrt(n) * (1 + tau)) ** n
    assert vol <= best * (1 + 1e-12)


def test_maxvol_on_a_tall_fiber_bounds_b_everywhere():
    """A 4096 x 24 complex matrix (the size of a d=5 core's fiber): maxvol ends with
    |B| <= 1 + tau on every row, and every swap raised the volume."""
    rng = np.random.default_rng(41)
    a = (rng.standard_normal((4096, 24)) + 1j * rng.standard_normal((4096, 24))) * rng.uniform(0.1, 10, 4096)[:, None]
    rows0, cols = ttcross.gepp_select(a, 1e-8)
    assert cols == list(range(24))
    rows, swaps, ok = ttcross.maxvol(a, rows0, 0.05, 2400)
    assert ok and swaps > 0
    assert np.abs(a @ np.linalg.inv(a[rows, :])).max() <= 1.05 + 1e-9
    assert abs(np.linalg.det(a[rows, :])) > abs(np.linalg.det(a[rows0, :]))


def test_rank_one_tensor_is_reproduced_exactly():
    rng = np.random.default_rng(7)
    d, n = 4, 9
    g = rng.standard_normal((d, n)) + 1j * rng.standard_normal((d, n))
    t = TableTensor(d, n, lambda idx: np.prod(g[np.arange(d), idx], axis=-1))
    exact = np.prod(g.sum(axis=1))
    for r in (1, 3):
        est, dg = ttcross.tt_cross_sum(t, r, seed=11)
        assert abs(est - exact) < 1e-12 * abs(exact)
        assert dg.max_rank == 1 and dg.converged


def test_rank_two_additive_tensor_is_reproduced_exactly():
    rng = np.random.default_rng(8)
    d, n = 5, 7
    h = rng.standard_normal((d, n)) + 1j * rng.standard_normal((d, n))
    t = TableTensor(d, n, lambda idx: h[np.arange(d), idx].sum(axis=-1))
    exact = h.sum() * n ** (d - 1)
    est, dg = ttcross.tt_cross_sum(t, 4, seed=12)
    assert abs(est - exact) < 1e-11 * abs(exact)
    assert dg.max_rank == 2


def test_full_rank_cross_reproduces_full_grid_sum():
    """Rank 16 on a 16 x 16 grid: the cross keeps every direction above the rank
    threshold (1e-8 of the first pivot), so the train is the grid sum to ~1e-10."""
    p = inputs.two_asset_min_call(n_grid=16, max_rank=16)
    t = integrand.tensors_for(p)[0]
    est, dg = ttcross.tt_cross_sum(t, 16, seed=1)
    exact = integrand.full_grid_sum(t)
    assert abs(est - exact) < 1e-9 * abs(exact)


def test_single_axis_sum_is_plain_sum():
    rng = np.random.default_rng(9)
    g = rng.standard_normal(13) + 1j * rng.standard_normal(13)
    t = TableTensor(1, 13, lambda idx: g[idx[..., 0]])
    est, dg = ttcross.tt_cross_sum(t, 4, seed=1)
    assert abs(est - g.sum()) < 1e-14 * abs(g.sum())
    assert dg.half_sweeps == 1


def _three_asset(n_grid=64, payoff="min"):
    spot = np.array([96.0, 103.0, 99.0])
    sigma = np.array([0.2, 0.3, 0.25])
    return inputs.Problem(spot=spot, cov=inputs.cov_from(sigma, inputs.equicorrelation(3, 0.3)),
                          rate=0.02, maturity=1.0, strike=100.0, payoff=payoff,
                          damping=np.full(3, -1.5), n_grid=n_grid, trunc_L=40.0,
                          max_rank=8, seed=5)


def test_tt_error_decreases_with_rank_against_full_grid():
    """The paper's bond-dimension claim (Section V.C): error falls quickly with D."""
    p = _three_asset()
    exact, _ = integrand.full_grid_price(p)
    errs = []
    for r in (8, 16, 32):
        price, imag, _ = ttcross.tt_price(p.with_(max_rank=r))
        errs.append(abs(price / exact - 1))
    assert errs[0] > errs[2]
    assert errs[2] < 1e-6


def test_tt_max_call_against_full_grid():
    p = _three_asset(payoff="max").with_(max_rank=24)
    exact, _ = integrand.full_grid_price(p)
    price, imag, diags = ttcross.tt_price(p)
    assert len(diags) == 3
    assert abs(price / exact - 1) < 1e-6
    assert abs(imag) < 1e-6 * exact


def test_paper_setting_three_assets():
    """The paper's own parameters (r=0.3, sigma=0.5, beta=0.5, N=50, alpha=5/d):
    Table I reports a truncation error ~4e-6 at d=3; a rank-20 train gets there."""
    p = inputs.paper_table_problem(3, max_rank=20)
    exact, _ = integrand.full_grid_price(p)
    price, _, _ = ttcross.tt_price(p)
    assert abs(price / exact - 1) < 2e-5


def _equicorrelated(d, n, r, trunc, seed):
    rng = np.random.default_rng(1000 + 17 * d + n + r)
    spot = rng.uniform(90, 110, d)
    sigma = rng.uniform(0.15, 0.35, d)
    return inputs.Problem(spot=spot, cov=inputs.cov_from(sigma, inputs.equicorrelation(d, 0.3)),
                          rate=0.02, maturity=1.0, strike=100.0, payoff="min",
                          damping=np.full(d, -1.5), n_grid=n, trunc_L=trunc, max_rank=r, seed=seed)


@pytest.mark.parametrize("d,n,r,trunc", [(3, 37, 24, 20.0), (4, 32, 40, 20.0), (5, 24, 32, 10.0)])
def test_converged_trains_match_the_exact_grid_sum(d, n, r, trunc):
    """At ranks above the integrand's numerical rank the cross reproduces the N^d
    grid sum it approximates: within 5e-7 of the exact sum (the one-factor grid
    sum, itself equal to the brute-force grid where that is feasible).  Measured
    1.3e-8 .. 3.6e-7."""
    from oracle import grid_sum

    p = _equicorrelated(d, n, r, trunc, seed=3)
    exact, _ = grid_sum.grid_sum_for(p)
    price, imag, diags = ttcross.tt_price(p, ttcross.CrossOptions(sweep_tol=1e-10))
    assert abs(price / exact - 1) < 5e-7
    assert abs(imag) < 1e-6 * abs(price)
    assert all(dg.maxvol_unconverged == 0 for dg in diags)


def test_benchmark_workload_tt_error_is_small():
    """The d=5, N=128, rank-32 workload: the train's error against the exact grid
    sum is the method's TT error at that rank, a few 1e-6 at most."""
    from oracle import grid_sum

    p = inputs.five_asset_batch(2)[1]
    exact, _ = grid_sum.grid_sum_for(p)
    price, _, _ = ttcross.tt_price(p)
    assert abs(price / exact - 1) < 5e-6
