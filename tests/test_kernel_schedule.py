"""The kernel-schedule replay (tests/kernel_schedule.py), the debugging aid that
runs the CUDA kernel's own pivot schedule in FP64: its rank reveal keeps a
well-conditioned block, is invariant under column scaling, and its block maxvol
ends dominant.  It is not the oracle; these tests only keep it honest."""
import itertools
import math

import numpy as np

import kernel_schedule as ks  # tests/ is on sys.path (conftest)
from oracle import integrand, ttcross
from paper_2203_02804_gb300 import inputs


def test_block_maxvol_is_dominant_and_near_max_volume():
    rng = np.random.default_rng(100)
    m, n, tau = 9, 3, 0.05
    a = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    rows, _ = ks.tournament_select(a, 4, 1e-12)
    rows, _, ok = ks.maxvol_refine(a, rows, 4, tau)
    assert ok
    b = a @ np.linalg.inv(a[rows, :])
    assert np.abs(b).max() <= 1.0 + tau + 1e-12
    vol = abs(np.linalg.det(a[rows, :]))
    best = max(abs(np.linalg.det(a[list(s), :])) for s in itertools.combinations(range(m), n))
    assert vol >= best / (math.sqrt(n) * (1 + tau)) ** n


def test_rank_reveal_keeps_a_well_conditioned_block():
    """Complete pivoting on a block whose last columns are nearly dependent:
    it stops at the numerical rank, and the kept sub-block has condition ~1/theta."""
    rng = np.random.default_rng(31)
    base = rng.standard_normal((8, 5)) + 1j * rng.standard_normal((8, 5))
    mix = rng.standard_normal((5, 8))
    block = base @ mix + 1e-12 * rng.standard_normal((8, 8))  # rank 5 up to 1e-12
    rows, cols = ks.rank_reveal(block, 1e-8)
    assert len(rows) == len(cols) == 5
    assert np.linalg.cond(block[np.ix_(rows, cols)]) < 1e8
    full_rows, _ = ks.rank_reveal(rng.standard_normal((6, 6)), 1e-8)
    assert len(full_rows) == 6


def test_rank_reveal_is_invariant_under_column_scaling():
    """Columns scaled by 1e-150 .. 1e+150 (with their reference sizes): the same
    pivots as unscaled, and a rank-1 block keeps one pivot."""
    rng = np.random.default_rng(32)
    block = rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))
    scale = 10.0 ** rng.uniform(-150, 150, 7)
    ref = rng.uniform(1.0, 3.0, 7) * (np.abs(block) ** 2).max(axis=0)
    assert ks.rank_reveal(block, 1e-8) == ks.rank_reveal(block * scale, 1e-8)
    assert ks.rank_reveal(block, 1e-8, ref) == ks.rank_reveal(block * scale, 1e-8, ref * scale ** 2)
    # equilibrated: every column's largest entry scores exactly 1, so the first
    # pivot is the one of them that comes first in row-major order
    rows, cols = ks.rank_reveal(block * scale, 1e-8)
    col_argmax = np.abs(block).argmax(axis=0)
    assert (rows[0], cols[0]) == min((int(col_argmax[c]), c) for c in range(7))
    x = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    rows, cols = ks.rank_reveal(np.outer(x, x * scale), 1e-8)
    assert len(rows) == 1 and rows[0] == int(np.argmax(np.abs(x)))


def test_rank_reveal_drops_a_column_negligible_in_its_fiber():
    """A column whose block entries are 1e-10 of its fiber-wide size is numerically
    absent from the block (below theta = 1e-8 once measured against its fiber)."""
    rng = np.random.default_rng(33)
    block = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    ref = (np.abs(block) ** 2).max(axis=0)
    ref[2] *= 1e20
    rows, cols = ks.rank_reveal(block, 1e-8, ref)
    assert len(cols) == 4 and 2 not in cols


def test_schedule_and_oracle_reach_the_same_grid_sum():
    """Different pivot schedules, one tensor: at full rank both reproduce the grid sum."""
    p = inputs.two_asset_min_call(n_grid=16, max_rank=16)
    exact, _ = integrand.full_grid_price(p)
    assert abs(ks.replay_price(p)[0] / exact - 1) < 1e-9
    assert abs(ttcross.tt_price(p)[0] / exact - 1) < 1e-9
